"""The benchmark's multi-rank path on CPU: two gloo ranks (127.0.0.1) run the
rendezvous, the barrier and the max-over-ranks reduction that bench.py uses
to time replicas (one independent query per rank, weak scaling)."""
import os
import socket
import subprocess
import sys
import textwrap

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_gloo_ranks_barrier_and_max():
    port = free_port()
    code = textwrap.dedent("""
        import os, sys
        sys.path.insert(0, %r)
        import bench
        rank, world = bench.dist_init()
        bench.barrier(world)
        m = bench.max_over_ranks(float(rank * 10 + 3), world)
        print("RESULT", rank, world, m)
        import torch.distributed as dist
        dist.destroy_process_group()
    """ % ROOT)
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), SS_BENCH_BACKEND="gloo")
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=120) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e
    res = sorted(l.split()[1:] for o, _ in outs for l in o.splitlines() if l.startswith("RESULT"))
    assert res == [["0", "2", "13.0"], ["1", "2", "13.0"]]


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference"], env=env,
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
