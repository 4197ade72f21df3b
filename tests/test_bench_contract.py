"""The benchmark's reference arm (the CPU oracle on a bounded sample) prints
the one JSON line the harness reads, with the same metric and config as the
GPU arm; ranks other than 0 print nothing and exit 0."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(env_extra):
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, env=env, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return [l for l in r.stdout.splitlines() if l.startswith("{")]


def test_reference_arm_line():
    sys.path.insert(0, ROOT)
    import bench
    lines = run({})
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "rows/s"
    assert d["higher_is_better"] is True and d["value"] > 0
    assert d["config"] == bench.workload_config(16, 41, 55, 3, 257, 3, 128, bench.N_CT, 32)
    cb = d["cpu_baseline"]
    import oracle as O
    assert cb["kind"] == "oracle" and cb["cores"] == O.threads() and cb["value"] == d["value"] and cb["sample"]
    # the line's rate is the measured one: rows per step over the measured time per step
    assert abs(d["rows_per_step"] / (d["ms_per_step"] / 1e3) - d["value"]) < 1e-6 * d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_are_silent():
    assert run({"RANK": "1", "WORLD_SIZE": "2"}) == []
