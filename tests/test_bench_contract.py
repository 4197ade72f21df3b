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


def test_short_served_and_batched_runs_are_summarised(monkeypatch):
    """The default run adds `served` and `batched` objects from child runs of
    `--serve` and `--batched`; a child that fails leaves an error string in
    place of the object instead of breaking the line (children faked here)."""
    sys.path.insert(0, ROOT)
    import bench

    serve_out = {"config": {"workload": "mixed"}, "capacity_qps": 9.0, "verified_against_plaintext": True,
                 "runs": [{"form": "plain", "queries": 100, "arrival_qps": 18.0, "qps": 9.1, "p50_ms": 3200.0,
                           "p99_ms": 5400.0},
                          {"form": "served", "queries": 100, "arrival_qps": 18.0, "qps": 12.9, "p50_ms": 2400.0,
                           "p99_ms": 3700.0}]}
    batch_out = {"metric": "batched", "plain_pairs_per_s": 214.1, "batched_pairs_per_s": 423.1, "speedup": 1.976,
                 "tuned": {"chunk": 32, "streams": 3, "ntt_tile_words": 2048},
                 "merged_lanes_graph_ms": {"chunk 8": 204.0}, "verified_against_plaintext": True}
    calls = []

    class R:
        def __init__(self, rc, out, err=""):
            self.returncode, self.stdout, self.stderr = rc, out, err

    def fake_run(cmd, **kw):
        calls.append(cmd)
        if "--serve" in cmd:
            assert "--no-serve-burst" in cmd and cmd[cmd.index("--serve-rates") + 1] == "2c"
            return R(0, "log line\n" + json.dumps(serve_out) + "\n")
        return R(1, "", "boom: no device")

    monkeypatch.setattr(bench.subprocess, "run", fake_run)
    out = bench.run_extras()
    assert len(calls) == 2
    sv = out["served"]
    assert sv["plain"] == {"qps": 9.1, "p50_ms": 3200.0, "p99_ms": 5400.0}
    assert sv["served"]["qps"] == 12.9 and sv["arrivals"] == 100 and sv["verified_against_plaintext"] is True
    assert "error" in out["batched"] and "boom" in out["batched"]["error"]
    monkeypatch.setattr(bench.subprocess, "run", lambda cmd, **kw: R(0, json.dumps(batch_out) + "\n"))
    bt = bench.run_extras()["batched"]
    assert bt["speedup"] == 1.976 and bt["batched_pairs_per_s"] == 423.1 and bt["tuned"]["streams"] == 3
