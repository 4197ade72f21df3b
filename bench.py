"""Benchmark: encrypted compare-then-SUM query throughput on one GB300.

Workload: N = 2^16, 41 data primes of 55 bits + 3 special primes,
p^r = 257^3, 128 slots per ciphertext; four encrypted columns a, b, c1, c2
of 32 ciphertexts each (4096 rows, uniform in [0, 257^3)); one step is the
query SUM(a*b) WHERE c1 < c2 (3-digit comparison, Algorithm 4) over the
whole table with every input resident in HBM. The inputs (5.5 GB) exceed L2.

Prints one JSON line. `--impl reference` times the plain CPU reference on a
bounded sample of the same workload instead.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "encrypted compare+SUM rows/s at N=2^16; NTT/keyswitch HBM GB/s; p99 latency"
PRESET = 2
N_CT = 32
SEED = 0x5EED0002
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM = 6800.0
# Integer-multiply issue ceiling of one GB300: 152 SMs x 4 sub-partitions x
# 16-lane fmaheavy pipe = 64 multiply issue slots per SM per clock, at the
# 2070 MHz maximum SM clock.
IMAD_PEAK = 152 * 64 * 2.07e9
# 32-bit multiplies in one 64-bit Shoup butterfly product (schoolbook minimum):
# the high 64 bits of a*w' need the high half of aL*wL and the full products
# aL*wH, aH*wL, aH*wH; the low 64 bits of a*w and of qhat*q each need one full
# product and two low halves. 5 of the 10 are widening (32 x 32 -> 64) products;
# their cost in issue slots is the measured ratio of the 32-bit and widening
# multiply-add rates (probe kinds 0 and 2).
IMAD_PER_BUTTERFLY = 10
WIDE_PER_BUTTERFLY = 5
# DRAM bytes per limb transform (forward and inverse, both phases each) from one
# ncu capture of the transform kernels (dram__bytes_read.sum +
# dram__bytes_write.sum per limb), over the 1 MB (16 N) it must move.
NTT_TRAFFIC_PER_ALGO_BYTE = 1.860


def hbm_peak():
    try:
        with open(PEAKS) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


class Clocks:
    """Samples nvidia-smi clocks during the timed region."""

    def __init__(self):
        self.samples, self.proc, self.thr = [], None, None

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", os.environ.get("LOCAL_RANK", "0"),
                                          "--query-gpu=" + q, "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return

        def read():
            for line in self.proc.stdout:
                self.samples.append([x.strip() for x in line.split(",")])
        self.thr = threading.Thread(target=read, daemon=True)
        self.thr.start()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.thr.join(timeout=2)
        sm = sorted(float(s[0]) for s in self.samples if len(s) >= 7 and s[0].replace(".", "").isdigit())
        mx = [float(s[1]) for s in self.samples if len(s) >= 7 and s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples if len(s) >= 7 for i in range(4)
                          if s[3 + i].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("SS_BENCH_BACKEND") != "gloo" else "gloo")
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def plain_query(A, B, C1, C2, t):
    """Plaintext meaning of the query: sum of a*b over rows whose centred
    difference c1 - c2 (mod t) is negative (Algorithm 4), mod t."""
    d = (C1.astype(object) - C2.astype(object)) % t
    keep = d > t // 2
    return int((A.astype(object) * B.astype(object))[keep].sum()) % t


# ------------------------------------------------------------------ CPU reference sample
def cpu_reference_sample(seconds, one_thread=False):
    """The plain CPU reference timed on this host's cores on the benchmark's
    workload: the parameter set, seeds and nonces of the GPU run, the first
    ciphertext of columns c1 and c2, d = c1 - c2, then multiplications at the
    top of the chain (the query's leading operations: the powers of the first
    G_{p,3} evaluation), repeated until `seconds` have passed. The query's rows
    per second follow from the reference's own count of limb transforms: the
    sample's transforms over the transforms the whole query runs per ciphertext
    of a column (counted on a 256-point ring with the same chain, where the
    count is the same). With one_thread, one more multiplication at the top
    level runs on a single thread (the paper's setting, Section 5.1)."""
    import numpy as np
    import oracle as O
    from paper_2604_19890_gb300 import synth
    prm = dict(logN=16, L=41, alpha=3, bits=55, p=257, r=3, h=120, seed=SEED)
    slope, fixed = query_ntt_count()
    per_ct = slope + fixed / N_CT
    o = O.Oracle(**prm)
    o.keygen([])
    cols = synth.table(SEED, N_CT, o.slots, o.t, columns=("a", "b", "c1", "c2"))
    c1 = o.encrypt(o.encode(cols["c1"][0]), 3000)
    c2 = o.encrypt(o.encode(cols["c2"][0]), 4000)
    d = o.sub(c1, c2)
    threads = O.threads()
    O.ntt_count(True)
    t0 = time.perf_counter()
    x, n_mul = d, 0
    while n_mul == 0 or (time.perf_counter() - t0 < seconds and x.level > 2):
        x = o.mul(x, x)
        n_mul += 1
    dt = time.perf_counter() - t0
    ntts = O.ntt_count()
    res = {"rows_per_s": 128.0 * ntts / per_ct / dt, "seconds": dt, "transforms": ntts, "multiplications": n_mul,
           "query_transforms_per_ct": per_ct, "threads": threads, "rows": 128.0 * ntts / per_ct}
    if one_thread:
        O.set_threads(1)
        O.ntt_count(True)
        t0 = time.perf_counter()
        o.mul(d, d)
        dt1 = time.perf_counter() - t0
        n1 = O.ntt_count()
        O.set_threads(threads)
        res["one_thread"] = {"rows_per_s": 128.0 * n1 / per_ct / dt1, "seconds": dt1, "transforms": n1}
    return res


def cpu_baseline_entry(r):
    return {"value": r["rows_per_s"], "unit": "rows/s", "cores": r["threads"], "kind": "oracle",
            "host_cpus": os.cpu_count(),
            "sample": "the reference on all %d host threads: %d multiplications at the top of the N=2^16, "
                      "L=41 chain on the query's first c1 - c2 ciphertext, %.1f s, %d limb transforms = %.4f "
                      "of the %.0f transforms the query runs per ciphertext of a column"
                      % (r["threads"], r["multiplications"], r["seconds"], r["transforms"],
                         r["transforms"] / r["query_transforms_per_ct"], r["query_transforms_per_ct"]),
            "one_thread": ({"value": r["one_thread"]["rows_per_s"], "unit": "rows/s", "cores": 1,
                            "sample": "one multiplication at level 41 on one thread, %.1f s"
                                      % r["one_thread"]["seconds"]} if "one_thread" in r else None)}


def run_cpu_full(args):
    """The whole query on the CPU reference for one ciphertext per column (128
    rows), all host threads, timed end to end, next to the sample-based rate
    (validation of the sample's scaling)."""
    import numpy as np
    import oracle as O
    from paper_2604_19890_gb300 import synth
    prm = dict(logN=16, L=41, alpha=3, bits=55, p=257, r=3, h=120, seed=SEED)
    o = O.Oracle(**prm)
    o.keygen(o.rotate_sum_elements())
    cols = synth.table(SEED, N_CT, o.slots, o.t, columns=("a", "b", "c1", "c2"))
    cols = {k: v[:1] for k, v in cols.items()}
    enc = {k: [o.encrypt(o.encode(cols[k][0]), 1000 * (i + 1))] for i, k in enumerate(("a", "b", "c1", "c2"))}
    O.ntt_count(True)
    t0 = time.perf_counter()
    res = o.query(enc["a"], enc["b"], enc["c1"], enc["c2"])
    dt = time.perf_counter() - t0
    ntts = O.ntt_count()
    ok = int(o.decrypt_slots(res)[0]) == plain_query(cols["a"], cols["b"], cols["c1"], cols["c2"], o.t)
    sample = cpu_reference_sample(args.cpu_seconds)
    print(json.dumps({"cpu_full_query": True, "threads": O.threads(), "host_cpus": os.cpu_count(), "rows": 128,
                      "seconds": dt, "rows_per_s": 128 / dt, "transforms": ntts,
                      "sample_rows_per_s": sample["rows_per_s"], "sample_over_full": sample["rows_per_s"] * dt / 128,
                      "verified_against_plaintext": bool(ok)}))
    return 0 if ok else 1


def query_ntt_count(n_ct_small=(1, 2)):
    """Limb transforms the reference runs for the query, per ciphertext of a
    column (slope) plus the fixed rotate-and-sum part, on a 256-point ring with
    the same chain and slot count (the count does not depend on N)."""
    import numpy as np
    import oracle as O
    o = O.Oracle(logN=8, L=41, alpha=3, bits=55, p=257, r=3, h=120, seed=SEED)
    o.keygen()
    counts = []
    for n in n_ct_small:
        cs = [o.encrypt_slots(np.arange(o.slots, dtype=np.uint64), 100 + i) for i in range(n)]
        O.ntt_count(True)
        o.query(cs, cs, cs, cs)
        counts.append(O.ntt_count())
    slope = counts[1] - counts[0]
    return slope, counts[0] - slope


def workload_config(logN, L, bits, alpha, p, r, slots, n_ct, batch, m_odd=1):
    """The `config` object both arms print for one workload."""
    rows = n_ct * slots
    ring = {3: "m=3N ring X^N-X^(N/2)+1", 5: "m=5N/2 ring Phi_10(X^(N/4))"}.get(m_odd, "ring X^N+1")
    wl = ("compare-then-SUM query, N=2^%d, %s, L=%d x %d-bit + %d special primes, p^r=%d^%d, %d slots, "
          "%d ciphertexts per column (%d rows) per GPU" % (logN, ring, L, bits, alpha, p, r, slots, n_ct, rows))
    return {"workload": wl, "batch": batch,
            "l2": "inputs (%.1f GB) larger than L2" % (4 * n_ct * 2 * L * (1 << logN) * 8 / 1e9)}


def run_reference(args):
    rank, world = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return 0
    times, rows_done, last = [], 0.0, None
    for i in range(args.warmup + args.steps):
        r = cpu_reference_sample(args.cpu_seconds)
        if i >= args.warmup:
            times.append(r["seconds"])
            rows_done += r["rows"]
            last = r
    v = rows_done / sum(times)
    base = cpu_baseline_entry(last)
    base["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "rows/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sum(times) / len(times) * 1e3,
            "rows_per_step": rows_done / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": workload_config(16, 41, 55, 3, 257, 3, 128, N_CT, args.batch),
            "cpu_baseline": base,
            "e2e": {"value": v, "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ kernel micro mode
def run_kernel(args):
    """Times one kernel family alone on the benchmark's parameter set (for
    profiling): `ntt` runs forward then inverse transforms over `--limbs` limbs
    of the N = 2^16 chain; `relin` runs tensor + relinearisation + modulus
    switch on a batch of `--n-ct` ciphertexts at the top level; `mul` runs the
    query's multiplication (tensor, then relinearise-and-drop in one ModDown)
    on such a batch."""
    import numpy as np
    import torch

    import paper_2604_19890_gb300 as ssg
    from paper_2604_19890_gb300 import build as ssbuild

    ssbuild.build()
    prm = ssg.preset(args.preset)
    g = ssg.Context(params=prm)
    peak, kind = hbm_peak()
    out = {"kernel": args.kernel, "preset": args.preset}
    if args.kernel == "ntt":
        L = g.L
        n = args.limbs - args.limbs % L
        rng = np.random.default_rng(0)
        data = torch.from_numpy(np.stack([rng.integers(0, int(g.primes[i % L]), g.N, dtype=np.uint64)
                                          for i in range(L)]).view(np.int64)).cuda().repeat(n // L, 1)
        for _ in range(args.warmup):
            g.ntt_forward(data, 0, L)
            g.ntt_inverse(data, 0, L)
        g.kernel_timing(True)
        for _ in range(args.steps):
            g.ntt_forward(data, 0, L)
            g.ntt_inverse(data, 0, L)
        st = g.kernel_stats()["ntt"]
        g.kernel_timing(False)
        out.update({"limbs": n, "launches": st[0], "avg_launch_ms": st[1] / st[0],
                    "GB/s": st[2] / (st[1] / 1e3) / 1e9, "us_per_limb": st[1] * 1e3 / (st[0] * n)})
    else:
        g.keygen([])
        rng = np.random.default_rng(0)
        a = g.encrypt(np.stack([g.encode(rng.integers(0, g.t, g.slots)) for _ in range(args.n_ct)]), 1)
        b = g.encrypt(np.stack([g.encode(rng.integers(0, g.t, g.slots)) for _ in range(args.n_ct)]), 100)
        op = (lambda: g.modswitch(g.relin(g.mul(a, b)), 1)) if args.kernel == "relin" else (lambda: g.mul_relin(a, b))
        for _ in range(args.warmup):
            op()
        g.kernel_timing(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            op()
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / args.steps
        ks = g.kernel_stats()
        g.kernel_timing(False)
        out.update({"n_ct": args.n_ct, "level": g.L, "ms_per_mul": dt * 1e3,
                    "classes": {k: {"launches": v[0], "ms": v[1], "GB/s": v[2] / (v[1] / 1e3) / 1e9 if v[1] else 0}
                                for k, v in ks.items() if v[0]}})
    out["peak_hbm_gbs"] = peak
    print(json.dumps(out))
    return 0


# ------------------------------------------------------------------ served form
def run_serve(args):
    """Poisson-arriving compare-then-SUM queries against device-resident tables
    of two parameter sets: N = 2^16 with 257^3 (SUM(a*b) WHERE c1 < c2) and
    N = 2^15 with 257^2 (SUM(a*b) WHERE c < t, t encrypted), `--serve-ct`
    ciphertexts per column each, keys of both resident, queries drawn from both
    at random. Compares the plain form (one worker, one query per pass) with
    the served form (continuous batching: several workers, compatible queries
    of one context merged per pass, one HBM budget) at arrival rates relative
    to the measured capacity and at 10 q/s, `--serve-queries` arrivals per
    point. A last run submits queries over tables of 2^15 rows (256
    ciphertexts per column at N = 2^15) mixed with small ones under an HBM
    budget of two large queries, to show admission by memory."""
    import numpy as np
    import torch

    import paper_2604_19890_gb300 as ssg
    from paper_2604_19890_gb300 import build as ssbuild
    from paper_2604_19890_gb300 import synth

    ssbuild.build()
    gs = []
    for pid in (2, 1):
        g = ssg.Context(params=ssg.preset(pid))
        g.keygen()
        g.set_batch(args.batch)
        gs.append(g)
    n_tables = 4

    def make_table(ci, i, n_ct):
        g = gs[ci]
        cols = synth.table(SEED + 100 + 10 * ci + i, n_ct, g.slots, g.t)
        if ci == 1:
            cols["c2"] = synth.threshold(SEED + 200 + i, g.slots, g.t)
        enc = [g.encrypt(np.stack([g.encode(x) for x in cols[k]]), 10000 * (i + 1) + 100 * j + 50000 * ci)
               for j, k in enumerate(("a", "b", "c1", "c2"))]
        return ci, enc, plain_query(cols["a"], cols["b"], cols["c1"], cols["c2"], g.t)

    tables = [make_table(ci, i, args.serve_ct) for i in range(n_tables) for ci in (0, 1)]
    # single-query service time over the mix
    for ci, enc, _ in tables[:2]:
        gs[ci].query(*enc)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for ci, enc, _ in tables:
        gs[ci].query(*enc)
    torch.cuda.synchronize()
    t1 = (time.perf_counter() - t0) / len(tables)
    cap = 1.0 / t1
    rng = np.random.default_rng(7)
    out = {"metric": "served compare-then-SUM queries/s and latency", "unit": "queries/s",
           "config": {"workload": "mixed: N=2^16/L=41/257^3 and N=2^15/L=30/257^2, %d ciphertexts (%d rows) per "
                                  "column per query, %d device-resident tables per parameter set"
                                  % (args.serve_ct, args.serve_ct * 128, n_tables)},
           "single_query_ms": t1 * 1e3, "capacity_qps": cap, "runs": []}
    ok = True

    def run(arrivals, picks, workers, merge, budget=0, check=2):
        nonlocal ok
        srv = ssg.Server(gs, workers=workers, max_merge=merge, hbm_budget=budget)
        tickets = []
        start = time.perf_counter()
        for i, at in enumerate(arrivals):
            now = time.perf_counter() - start
            if at > now:
                time.sleep(at - now)
            ci, enc, exp = picks[i]
            tickets.append((srv.submit(*enc, ctx_index=ci), time.perf_counter(), i))
        lat, last = [], 0.0
        for tk, t_sub, i in tickets:
            res, q_ms, r_ms = srv.wait(tk, timeout_ms=900000)
            lat.append(q_ms + r_ms)
            last = max(last, t_sub - start + (q_ms + r_ms) / 1e3)
            if i < check:
                ci, _, exp = picks[i]
                ok &= bool((gs[ci].decrypt_slots(res) == exp).all())
        st = srv.stats()
        srv.close()
        lat.sort()
        return {"queries": len(lat), "qps": len(lat) / last, "p50_ms": lat[len(lat) // 2],
                "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))], "passes": st["batches"],
                "peak_inflight_bytes": st["peak_inflight_bytes"]}

    rates = []
    for tok in args.serve_rates.split(","):  # "2c": twice the measured capacity; "10": 10 q/s
        rates.append(float(tok[:-1]) * cap if tok.endswith("c") else float(tok))
    for rate in rates:
        gaps = rng.exponential(1.0 / rate, args.serve_queries)
        arrivals = np.cumsum(gaps) - gaps[0]
        picks = [tables[int(k)] for k in rng.integers(0, len(tables), args.serve_queries)]
        for form, workers, merge in [("plain", 1, 1), ("served", 3, 8)]:
            r = run(arrivals, picks, workers, merge)
            r.update({"form": form, "arrival_qps": round(rate, 3)})
            out["runs"].append(r)
    if not args.no_serve_burst:
        # tables of 2^15 rows at N = 2^15 (256 ciphertexts per column) among small queries
        big = [make_table(1, 10 + i, 256) for i in range(2)]
        est = gs[1].query_bytes(256)
        picks = [big[0]] + tables[:6] + [big[1]] + tables[6:]
        r = run([0.0] * len(picks), picks, 3, 8, budget=int(2.5 * est), check=len(picks))
        r.update({"form": "served", "arrival": "burst", "large_queries": 2, "large_rows": 256 * 128,
                  "hbm_budget": int(2.5 * est)})
        out["runs"].append(r)
    out["verified_against_plaintext"] = ok
    print(json.dumps(out))
    return 0 if ok else 1


# ------------------------------------------------------------------ batched form
def run_batched(args):
    """64 ciphertext pairs of mixed N in {2^14, 2^15, 2^16} and levels 4..28 from
    the 17^2 / 36-bit and 257^2 / 55-bit parameter sets: multiply + relinearise
    and, where the levels allow, reduce to digits (Algorithm 3). Plain form:
    one pair at a time on one stream; batched form: autotuned chunks over
    streams or merged lanes, captured once as a CUDA graph and replayed.
    `--batched-mix small`: 64 pairs at N = 2^14 and levels 8..12 of the 17^2
    set only (many small items, where launches rather than arithmetic
    dominate)."""
    import numpy as np
    import torch

    import paper_2604_19890_gb300 as ssg
    from paper_2604_19890_gb300 import build as ssbuild

    ssbuild.build()
    sets = []
    small = args.batched_mix == "small"
    for logN in ((14,) if small else (14, 15, 16)):
        sets.append(dict(logN=logN, L=28, alpha=2, bits=36, p=17, r=2, h=120, nmax=1 << 16, seed=SEED + logN))
        if not small:
            sets.append(dict(logN=logN, L=28, alpha=2, bits=55, p=257, r=2, h=120, nmax=1 << 16,
                             seed=SEED + 100 + logN))
    gs = []
    for s in sets:
        g = ssg.Context(**s)
        g.keygen([])
        gs.append(g)
    rng = np.random.default_rng(3)
    pairs, plain_vals = [], []
    for i in range(64):
        ci = int(rng.integers(0, len(gs)))
        g = gs[ci]
        lvl = int(rng.integers(8, 13)) if small else int(rng.integers(4, 29))
        va, vb = rng.integers(0, g.t, g.slots), rng.integers(0, g.t, g.slots)
        ga = g.encrypt(g.encode(va), 10 + 2 * i)
        gb = g.encrypt(g.encode(vb), 11 + 2 * i)
        if lvl < g.L:
            ga, gb = g.modswitch(ga, g.L - lvl), g.modswitch(gb, g.L - lvl)
        pairs.append((ci, ga, gb, True))
        plain_vals.append((va, vb))
    st = torch.cuda.Stream()
    b = ssg.Batch(gs, pairs)
    info = b.get_config()
    # plain form: one pair per pass, one stream, no graph
    singles = [ssg.Batch(gs, [p]) for p in pairs]
    for sb in singles:
        sb.config(1, 1, 12)
    for sb in singles:
        sb.run(st)
    st.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for sb in singles:
        sb.run(st)
    e1.record(st)
    st.synchronize()
    plain_ms = e0.elapsed_time(e1)
    def graph_time():
        b.capture(st)
        b.run(st)
        st.synchronize()
        times = []
        for _ in range(max(3, args.steps)):
            e0.record(st)
            b.run(st)
            e1.record(st)
            st.synchronize()
            times.append(e0.elapsed_time(e1))
        return sorted(times)[len(times) // 2]

    # merged lanes (persistent transforms and inner products over all pairs), best chunk
    merged = {}
    for c in (8, 64):
        b.config(c, 0, 11)
        merged[c] = graph_time()
    best = b.tune(st)
    graph_ms = graph_time()
    # decrypted semantics of every product and digit
    ok = True
    for (ci, _, _, _), (va, vb), (prod, digs) in zip(pairs, plain_vals, b.results()):
        g = gs[ci]
        exp = (va.astype(object) * vb.astype(object)) % g.t
        ok &= bool((g.decrypt_slots(prod)[0] == exp).all())
        for k, d in enumerate(digs):
            if d.level >= 1 and d.t_exp == 1:
                vals = g.decrypt_slots(d)[0]
                want = []
                for x in exp:
                    v = int(x)
                    for _ in range(k):
                        z = v % g.p
                        z = z - g.p if z > g.p // 2 else z
                        v = (v - z) // g.p
                    z = v % g.p
                    want.append(z % g.p)
                ok &= bool((vals == np.array(want)).all())
    for sb in singles:
        sb.close()
    b.close()
    out = {"metric": "batched multiply+relinearise+reduce, 64 %s pairs" % ("small N=2^14" if small else "mixed-N"),
           "unit": "pairs/s",
           "plain_ms": plain_ms, "batched_graph_ms": graph_ms, "plain_pairs_per_s": 64 / (plain_ms / 1e3),
           "batched_pairs_per_s": 64 / (graph_ms / 1e3), "speedup": plain_ms / graph_ms,
           "tuned": {"chunk": best[0], "streams": best[1], "ntt_tile_words": 1 << best[2]},
           "merged_lanes_graph_ms": {"chunk %d" % c: v for c, v in merged.items()},
           "groups": info["groups"], "reductions_skipped": info["skipped"], "verified_against_plaintext": ok}
    print(json.dumps(out))
    return 0 if ok else 1


# ------------------------------------------------------------------ short served and batched runs
def _sub_json(argv, timeout):
    """Runs this script with `argv` in a child process (its own CUDA context,
    so nothing it allocates stays behind) and returns its JSON line."""
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__)] + argv, capture_output=True, text=True,
                           timeout=timeout, cwd=ROOT)
    except subprocess.TimeoutExpired:
        return None, "timed out after %d s" % timeout
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    if r.returncode != 0 or not lines:
        return None, "exit %d: %s" % (r.returncode, (r.stderr or r.stdout).strip().splitlines()[-1:] or "")
    try:
        return json.loads(lines[-1]), None
    except ValueError as e:
        return None, "unreadable output: %r" % (e,)


def run_extras():
    """The served and batched forms in short runs beside the headline number
    (before it, in child processes): the served form at twice the measured
    capacity with 100 Poisson arrivals over both parameter sets, plain and
    served; the batched form of 64 mixed-N pairs, one at a time against the
    tuned, graph-replayed batch. The full sweeps are `--serve` and `--batched`."""
    out = {}
    t0 = time.perf_counter()

    def served(sv):
        runs = {r["form"]: {k: round(r[k], 2) for k in ("qps", "p50_ms", "p99_ms")} for r in sv["runs"]}
        return {"workload": sv["config"]["workload"], "unit": "queries/s",
                "capacity_qps": round(sv["capacity_qps"], 2), "arrivals": sv["runs"][0]["queries"],
                "arrival_qps": sv["runs"][0]["arrival_qps"], "plain": runs.get("plain"),
                "served": runs.get("served"), "verified_against_plaintext": sv["verified_against_plaintext"]}

    def batched(bt):
        return {"workload": bt["metric"], "unit": "pairs/s",
                "plain_pairs_per_s": round(bt["plain_pairs_per_s"], 1),
                "batched_pairs_per_s": round(bt["batched_pairs_per_s"], 1),
                "speedup": round(bt["speedup"], 3), "tuned": bt["tuned"],
                "merged_lanes_graph_ms": bt["merged_lanes_graph_ms"],
                "verified_against_plaintext": bt["verified_against_plaintext"]}

    for key, argv, summary in (
            ("served", ["--serve", "--serve-queries", "100", "--serve-rates", "2c", "--no-serve-burst"], served),
            ("batched", ["--batched", "--steps", "3"], batched)):
        res, err = _sub_json(argv, 600)
        try:
            out[key] = {"error": err} if res is None else summary(res)
        except (KeyError, IndexError, TypeError, ValueError) as e:  # unexpected child output
            out[key] = {"error": "unexpected output: %r" % (e,)}
    out["extras_s"] = round(time.perf_counter() - t0, 1)
    return out


# ------------------------------------------------------------------ GPU arm
def run_ours(args):
    import numpy as np
    import torch

    import paper_2604_19890_gb300 as ssg
    from paper_2604_19890_gb300 import build as ssbuild
    from paper_2604_19890_gb300 import synth

    ssbuild.build()
    extras = {}
    if (int(os.environ.get("WORLD_SIZE", "1")) == 1 and not args.no_extras and args.preset == PRESET
            and args.n_ct == N_CT and args.batch == 32):
        extras = run_extras()
    rank, world = dist_init()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    prm = ssg.preset(args.preset)
    prm.seed = SEED + 1000 * rank
    g = ssg.Context(params=prm)
    g.keygen()
    g.set_batch(args.batch)
    t = g.t
    n_ct = args.n_ct
    cols = synth.table(SEED + rank, n_ct, g.slots, t, columns=("a", "b", "c1", "c2"))
    if args.preset == 0:  # SUM(a*a) WHERE c < 150, threshold encrypted
        cols["b"] = cols["a"]
        cols["c2"] = synth.threshold(SEED, g.slots, t, value=150)
    elif args.preset == 1:  # SUM(a*b) WHERE c < t, t uniform and encrypted
        cols["c2"] = synth.threshold(SEED, g.slots, t)
    enc = {}
    for i, (k, v) in enumerate(cols.items()):
        enc[k] = g.encrypt(np.stack([g.encode(x) for x in v]), 1000 * (i + 1))
    rows = n_ct * g.slots
    stream = torch.cuda.current_stream()

    def step():
        return g.query(enc["a"], enc["b"], enc["c1"], enc["c2"])

    # correctness of the benchmarked configuration (not timed)
    res = step()
    exp = plain_query(cols["a"], cols["b"], cols["c1"], cols["c2"], t)
    got = g.decrypt_slots(res)
    verified = bool((got == exp).all())

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    clocks = Clocks()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lat = []
    l0 = g.launches()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        lat.append((e0, e1))
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = (g.launches() - l0) // max(1, args.steps)
    clk = clocks.stop()
    barrier(world)
    ms_total = max_over_ranks(ev0.elapsed_time(ev1), world)
    lat_ms = sorted(a.elapsed_time(b) for a, b in lat)
    ms_step = ms_total / args.steps
    value = rows * world * args.steps / (ms_total / 1e3)

    # end to end through the host-memory entry point: H2D of the four columns,
    # the query, D2H of the result ciphertext, every step; measured right after
    # the device-resident steps, in the same state as the headline number, with
    # SM clocks sampled during the calls
    e2e = None
    if not args.no_e2e:
        host = {k: torch.empty(tuple(v.buf.shape), dtype=torch.int64, pin_memory=True) for k, v in enc.items()}
        for k, v in enc.items():
            host[k].copy_(v.buf)
        arrs = {k: host[k].numpy().view(np.uint64) for k in host}
        L = enc["a"].level
        h2d = sum(a.nbytes for a in arrs.values())
        ol = None
        # one untimed call first: the pool grows once for the four uploaded columns
        g.query_host(arrs["a"], arrs["b"], arrs["c1"], arrs["c2"], L)
        torch.cuda.synchronize()
        e_steps = max(1, min(args.steps, args.e2e_steps))
        e_clocks = Clocks()
        e_clocks.start()
        t0 = time.perf_counter()
        for _ in range(e_steps):
            out, ol, ot = g.query_host(arrs["a"], arrs["b"], arrs["c1"], arrs["c2"], L)
        dt = (time.perf_counter() - t0) / e_steps
        e_clk = e_clocks.stop()
        e2e_ok = bool((g.decrypt_slots(g.from_words(out[None], ot)) == exp).all())
        e2e = {"value": rows / dt, "unit": "rows/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(2 * ol * g.N * 8), "ms_per_step": dt * 1e3, "verified": e2e_ok,
               "clocks": e_clk}

    # kernel classes over one instrumented step (events on the launching stream)
    g.kernel_timing(True)
    step()
    torch.cuda.synchronize()
    ks = g.kernel_stats()
    ntt_products = g.ntt_products()
    stages = {k: round(v[1], 3) for k, v in g.stage_stats().items()}
    g.kernel_timing(False)
    # measured integer-pipe ceilings (register-only loops, no memory traffic)
    imad_rate = ssg.alu_probe(0, 65536)
    bfly_rate = ssg.alu_probe(1, 16384)
    wide_rate = ssg.alu_probe(2, 65536)
    wide_slots = imad_rate / wide_rate  # issue slots of one widening multiply
    slots_per_bfly = (IMAD_PER_BUTTERFLY - WIDE_PER_BUTTERFLY) + WIDE_PER_BUTTERFLY * wide_slots
    total_k = sum(v[1] for v in ks.values())
    dom = max(ks, key=lambda k: ks[k][1])
    peak, peak_kind = hbm_peak()

    def gbs(k):
        n, ms, b = ks[k]
        return b / (ms / 1e3) / 1e9 if ms > 0 else 0.0

    n_l, ms_l, b_l = ks[dom]
    if dom == "ntt":
        # integer-multiply roofline of the transform: the Shoup products its
        # launches performed (N/2 per stage and limb; fewer where the ModUp base
        # conversion applied the first twiddle), counted by the library
        bfly = ntt_products
        achieved = bfly * slots_per_bfly / (ms_l / 1e3) / 1e12
        peak_alu = IMAD_PEAK / 1e12
        roof = {"kernel": "ntt", "bound": "alu", "achieved": achieved, "peak": peak_alu,
                "unit": "T multiply issue slots/s", "frac": achieved / peak_alu,
                "traffic": (NTT_TRAFFIC_PER_ALGO_BYTE * b_l / n_l) if NTT_TRAFFIC_PER_ALGO_BYTE else None,
                "peak_source": "derived: 152 SMs x 64 multiply issue slots/clk x 2070 MHz; per Shoup product "
                               "10 multiplies = 5 single-slot + 5 widening at the measured slot ratio "
                               "(%.2f slots each), %.2f slots" % (wide_slots, slots_per_bfly),
                "shoup_products": bfly,
                "frac_at_one_slot_per_multiply": bfly * IMAD_PER_BUTTERFLY / (ms_l / 1e3) / IMAD_PEAK,
                "measured_imad_per_s": imad_rate, "measured_wide_imad_per_s": wide_rate,
                "measured_butterflies_per_s": bfly_rate,
                "achieved_butterflies_per_s": bfly / (ms_l / 1e3),
                "frac_of_measured_butterfly_ceiling": bfly / (ms_l / 1e3) / bfly_rate,
                "hbm_achieved_gbs": gbs(dom), "hbm_peak_gbs": peak, "hbm_frac": gbs(dom) / peak,
                "hbm_peak_source": peak_kind, "avg_launch_ms": ms_l / max(1, n_l),
                "algorithmic_bytes_per_launch": b_l / max(1, n_l),
                "share_of_kernel_time": ms_l / total_k if total_k else None}
    else:
        roof = {"kernel": dom, "bound": "hbm", "achieved": gbs(dom), "peak": peak, "unit": "GB/s",
                "frac": gbs(dom) / peak, "traffic": None, "peak_source": peak_kind,
                "avg_launch_ms": ms_l / max(1, n_l), "algorithmic_bytes_per_launch": b_l / max(1, n_l),
                "share_of_kernel_time": ms_l / total_k if total_k else None}
    classes = {k: {"launches": v[0], "ms": round(v[1], 3), "GB/s": round(gbs(k), 1),
                   "frac_of_hbm": round(gbs(k) / peak, 3)} for k, v in ks.items() if v[0]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu and args.preset == PRESET:
        cpu = cpu_baseline_entry(cpu_reference_sample(args.cpu_seconds, one_thread=True))

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u64", "data": "synthetic",
                "config": workload_config(prm.logN, prm.L, prm.bits, prm.alpha, prm.p, prm.r, g.slots, n_ct,
                                          args.batch, prm.m_odd),
                "latency_ms": {"p50": lat_ms[len(lat_ms) // 2], "p99": lat_ms[min(len(lat_ms) - 1,
                                                                                   int(0.99 * len(lat_ms)))]},
                "verified_against_plaintext": verified,
                "roofline": roof, "kernel_classes": classes, "stages_ms": stages,
                "ntt_gbs": gbs("ntt"), "keyswitch_ip_gbs": gbs("keyswitch_inner_product"),
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk}
        line.update(extras)
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0 if verified else 1


# ------------------------------------------------------------------ tensor-core rates
def run_mma_rates(args):
    """Dense matrix-multiply rates of this GPU's tensor cores for the operand
    types an exact integer contraction could use (int8 -> int32 through
    torch._int_mm, fp16 and bf16 with fp32 accumulation through torch.matmul),
    8192^3, best of 10 after warm-up, CUDA events. Context for the choice of
    the integer pipe for the transforms and the key-switch inner product."""
    import torch
    n = args.mma_n
    out = {"mma_rates": True, "n": n}
    a8 = torch.randint(-128, 127, (n, n), dtype=torch.int8, device="cuda")
    b8 = torch.randint(-128, 127, (n, n), dtype=torch.int8, device="cuda").t().contiguous().t()
    cases = {"int8_int32": lambda: torch._int_mm(a8, b8)}
    for name, dt in (("fp16_fp32acc", torch.float16), ("bf16_fp32acc", torch.bfloat16)):
        x = torch.randn(n, n, device="cuda", dtype=dt)
        y = torch.randn(n, n, device="cuda", dtype=dt)
        cases[name] = (lambda x=x, y=y: torch.matmul(x, y))
    for name, f in cases.items():
        for _ in range(3):
            f()
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            f()
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        out[name + "_tops"] = 2.0 * n ** 3 / (best / 1e3) / 1e12
    print(json.dumps(out))
    return 0


# ------------------------------------------------------------------ LT operator across (p, r)
# (bit width, p, r) from the paper's LT tables (Section 5) that power-of-two
# rings with binomial slot factors support (p = 1 mod 4).
LT_SWEEP = [(8, 5, 4), (8, 17, 2), (12, 17, 3), (16, 17, 4), (16, 41, 3), (16, 257, 2), (20, 17, 5), (20, 37, 4)]
# on the ring m = 3N also the paper's plaintext primes p = 3 mod 4 (its LT table)
LT_SWEEP_3N = LT_SWEEP + [(8, 7, 3), (12, 7, 5), (12, 11, 4), (12, 67, 2), (20, 131, 3)]


def run_lt_sweep(args):
    """LT(a, b) followed by modulus raising on a batch of ciphertexts for each
    (p, r): per-stage times (reduction, comparison, aggregation, raising) as in
    the paper's runtime breakdown, per ciphertext and amortised per slot. The
    chain is the shortest one the query schedule needs at that (p, r)."""
    import numpy as np
    import torch

    import paper_2604_19890_gb300 as ssg
    from paper_2604_19890_gb300 import build as ssbuild
    from paper_2604_19890_gb300 import synth

    ssbuild.build()
    stream = torch.cuda.current_stream()
    m_odd = {"3n": 3, "5n2": 5}.get(args.sweep_ring, 1)
    sweep = LT_SWEEP if m_odd == 1 else [x for x in LT_SWEEP_3N if not (m_odd == 5 and x[1] == 5)]
    for bw, p, r in sweep:
        base = dict(logN=args.sweep_logn, alpha=2, bits=55, p=p, r=r, h=120, nmax=0, seed=SEED + p * 10 + r,
                    m_odd=m_odd)
        probe = ssg.Context(L=64, **base)
        L = 64 - probe.query_depth(64) + 1
        del probe
        g = ssg.Context(L=L, **base)
        g.keygen([])
        vals = synth.table(SEED + bw, args.sweep_ct, g.slots, g.t, columns=("a", "b"))
        ea = g.encrypt(np.stack([g.encode(x) for x in vals["a"]]), 1)
        eb = g.encrypt(np.stack([g.encode(x) for x in vals["b"]]), 100)
        res = g.raise_modulus(g.compare("lt", ea, eb))  # warm-up and check
        exp = np.array([[1 if ((int(x) - int(y)) % g.t) > g.t // 2 else 0 for x, y in zip(ra, rb)]
                        for ra, rb in zip(vals["a"], vals["b"])])
        ok = bool((g.decrypt_slots(res) == exp).all())
        g.kernel_timing(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            g.raise_modulus(g.compare("lt", ea, eb))
        e1.record(stream)
        torch.cuda.synchronize()
        st = g.stage_stats()
        g.kernel_timing(False)
        per = args.steps * args.sweep_ct
        total = e0.elapsed_time(e1) / per
        stages = {k: st[k][1] / per for k in ("reduction", "comparison", "aggregation", "modulus_raising")}
        print(json.dumps({"lt_sweep": True, "bit_width": bw, "p": p, "r": r, "t": g.t, "N": g.N, "m": g.m, "L": L,
                          "slots": g.slots, "ciphertexts": args.sweep_ct, "ms_per_ciphertext": stages | {"total": total},
                          "amortized_ms_per_slot": total / g.slots, "verified": ok}))
        del g
        torch.cuda.empty_cache()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--kernel", choices=["ntt", "relin", "mul"], default=None,
                    help="time one kernel family alone (profiling mode)")
    ap.add_argument("--limbs", type=int, default=512)
    ap.add_argument("--n-ct", type=int, default=N_CT, help="ciphertexts per column")
    ap.add_argument("--preset", type=int, default=PRESET, choices=[0, 1, 2, 3, 4],
                    help="0: N=2^13, 17^2; 1: N=2^15, 257^2; 2: N=2^16, 257^3 (the headline workload); "
                         "3: as 2 on the ring m = 3N (256 slots); 4: on m = 5N/2 (512 slots)")
    ap.add_argument("--serve", action="store_true", help="served form: Poisson arrivals, p50/p99")
    ap.add_argument("--batched", action="store_true", help="batched form: 64 mixed-N pairs, graph replay")
    ap.add_argument("--batched-mix", choices=["mixed", "small"], default="mixed")
    ap.add_argument("--serve-ct", type=int, default=2)
    ap.add_argument("--serve-queries", type=int, default=200)
    ap.add_argument("--serve-rates", default="0.5c,1c,2c,10",
                    help="arrival rates: q/s, or a multiple of the measured capacity with a 'c' suffix")
    ap.add_argument("--no-serve-burst", action="store_true", help="skip the burst of 2^15-row tables")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline run without the short served- and batched-form measurements")
    ap.add_argument("--lt-sweep", action="store_true",
                    help="LT operator + modulus raising across (p, r) at fixed bit widths, per-stage times")
    ap.add_argument("--sweep-logn", type=int, default=15)
    ap.add_argument("--sweep-ring", choices=["2n", "3n", "5n2"], default="2n", help="LT sweep ring: m = 2N, 3N or 5N/2")
    ap.add_argument("--sweep-ct", type=int, default=8)
    ap.add_argument("--mma-rates", action="store_true", help="tensor-core int8/fp16/bf16 matmul rates")
    ap.add_argument("--cpu-seconds", type=float, default=6.0, help="length of one CPU reference sample")
    ap.add_argument("--cpu-full", action="store_true", help="whole query on the CPU reference, 1 ct per column")
    ap.add_argument("--mma-n", type=int, default=8192)
    args = ap.parse_args()
    if args.mma_rates:
        return run_mma_rates(args)
    if args.cpu_full:
        return run_cpu_full(args)
    if args.lt_sweep:
        return run_lt_sweep(args)
    if args.serve:
        return run_serve(args)
    if args.batched:
        return run_batched(args)
    if args.kernel:
        return run_kernel(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
