"""Measurement entry points on the GPU: the per-stage breakdown of the query
(Section 5's runtime breakdown of LT) and the integer-pipe probes used as the
measured ceiling beside the derived one."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_stage_breakdown_covers_the_query():
    import torch

    import paper_2604_19890_gb300 as ssg
    g = ssg.Context(logN=6, L=26, alpha=2, bits=36, p=17, r=2, h=16, nmax=0, seed=7)
    g.keygen(g.rotate_sum_elements())
    rng = np.random.default_rng(3)
    enc = [g.encrypt(np.stack([g.encode(v) for v in rng.integers(0, g.t, (3, g.slots))]), 100 * (i + 1))
           for i in range(4)]
    g.set_batch(2)  # two chunks: every stage but the final rotate-and-sum runs twice
    g.kernel_timing(True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    g.query(*enc)
    e1.record()
    torch.cuda.synchronize()
    st = g.stage_stats()
    ks = g.kernel_stats()
    g.kernel_timing(False)
    g.set_batch(8)
    assert list(st) == ssg.QUERY_STAGES
    for name in ("reduction", "comparison", "aggregation", "modulus_raising", "masked_product"):
        assert st[name][0] == 2 and st[name][1] > 0, name
    assert st["sum"][0] >= 2
    wall = e0.elapsed_time(e1)
    assert sum(v[1] for v in st.values()) <= wall * 1.05
    assert sum(v[1] for v in ks.values()) > 0
    # switching timing on again resets the stage counters
    g.kernel_timing(True)
    assert all(v == (0, 0.0) for v in g.stage_stats().values())
    g.kernel_timing(False)


def test_alu_probes_report_finite_rates():
    import paper_2604_19890_gb300 as ssg
    imad = ssg.alu_probe(0, 1024)
    bfly = ssg.alu_probe(1, 256)
    assert math.isfinite(imad) and imad > 1e11
    assert math.isfinite(bfly) and bfly > 1e9
    wide = ssg.alu_probe(2, 1024)  # widening multiply-adds: no faster than 32-bit ones
    assert math.isfinite(wide) and 1e11 < wide <= imad * 1.05
    with pytest.raises(ssg.SSError):
        ssg.alu_probe(3, 16)
    with pytest.raises(ssg.SSError):
        ssg.alu_probe(0, 0)


@pytest.mark.parametrize("logN", [6, 13])
def test_transform_product_counter(logN):
    """ss_ntt_products counts the Shoup products the timed transforms perform:
    N/2 log2 N per plain forward limb and N/2 (log2 N + 1) per plain inverse
    limb (N/2 (log2 N + 2) for the single-phase transform of N <= 4096, which
    scales every word by N^-1); inside a relinearisation on X^N + 1 with
    N >= 8192 every transform
    either gets its first stage's twiddle from the base conversion that wrote
    its input or leaves its last stage's factors to the one that reads it, so
    each of its limbs counts N/2 (log2 N - 1)."""
    import torch

    import paper_2604_19890_gb300 as ssg
    L, alpha = 5, 2
    g = ssg.Context(logN=logN, L=L, alpha=alpha, bits=36, p=17, r=2, h=16, nmax=0, seed=11)
    N = g.N
    rng = np.random.default_rng(1)
    data = torch.from_numpy(np.stack([rng.integers(0, int(g.primes[i]), N, dtype=np.uint64)
                                      for i in range(L)]).view(np.int64)).cuda()
    g.kernel_timing(True)
    g.ntt_forward(data, 0, L)
    fwd = g.ntt_products()
    g.ntt_inverse(data, 0, L)
    both = g.ntt_products()
    g.kernel_timing(False)
    inv_extra = 1 if logN >= 13 else 2
    assert fwd == L * N // 2 * logN
    assert both - fwd == L * N // 2 * (logN + inv_extra)
    g.keygen([])
    B = 3
    a = g.encrypt(np.stack([g.encode(rng.integers(0, g.t, g.slots)) for _ in range(B)]), 1)
    b = g.encrypt(np.stack([g.encode(rng.integers(0, g.t, g.slots)) for _ in range(B)]), 2)
    t = g.mul(a, b)
    g.kernel_timing(True)
    torch.cuda.synchronize()
    g.relin(t)
    torch.cuda.synchronize()
    got = g.ntt_products()
    g.kernel_timing(False)
    lvl = t.level
    dn = -(-lvl // alpha)
    # ModUp: inverse of the lvl source limbs, forward of every digit's other limbs;
    # ModDown: inverse of 2 x alpha special limbs, forward of 2 x lvl corrections
    polys_fwd = B * (dn * (lvl + alpha) - lvl) + 2 * B * lvl
    polys_inv = B * lvl + 2 * B * alpha
    if logN >= 13:
        want = (polys_fwd + polys_inv) * N // 2 * (logN - 1)
    else:  # below N = 1024 neither fold applies
        want = polys_fwd * N // 2 * logN + polys_inv * N // 2 * (logN + 2)
    assert got == want
