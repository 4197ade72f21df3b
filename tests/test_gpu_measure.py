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
