"""Parity at the sizes the benchmark runs: the CUDA path's ciphertext words
against the CPU reference's, through the C-ABI.

* Digest cases (tests/golden/fullsize_cases.py): single operations at
  N = 2^16, level 41, alpha = 3, p^r = 257^3, and the compare-then-SUM query at
  the three named parameter sets. The expected values are SHA-256 digests of
  the reference's words, written by tests/golden/make_fullsize_digests.py
  (which calls only the reference); equal digests mean equal words.
* Live cases: key switching (relinearisation, multiplication with the fused
  drop, rotations) at N = 2^13 and 2^14, and the batched form over N = 2^14
  and 2^15, compared word by word with the reference run in the test. These
  rings use the two-phase transform, including its out-of-place first inverse
  phase (ModUp reads the ciphertext in place), the digit-skipping forward
  transform of ModUp, a ragged last digit and ragged batch sizes.
All arithmetic is exact modular integer arithmetic: the tolerance is zero.
"""
import json
import os
import sys

import numpy as np
import pytest

import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import fullsize_cases as FC  # noqa: E402

pytestmark = pytest.mark.gpu

DIGESTS = json.load(open(os.path.join(HERE, "golden", "fullsize_digests.json")))


def gpu_ctx(params, galois=None):
    import paper_2604_19890_gb300 as ssg
    g = ssg.Context(nmax=0, **params)
    g.keygen(galois)
    return g


def check(name, ct, exp, b=0):
    assert (ct.ncomp, ct.level, ct.t_exp) == (exp["ncomp"], exp["level"], exp["t_exp"]), name
    assert FC.digest(ct.words()[b]) == exp["sha256"], name + ": words differ from the reference"


def test_preset_parameters_match_the_cases():
    import paper_2604_19890_gb300 as ssg
    for i, prm in FC.PRESETS.items():
        p = ssg.preset(i)
        assert {k: getattr(p, k) for k in prm} == prm


def test_ops_n65536_257cubed():
    case = FC.CASES["ops_n65536_257cubed"]
    exp = DIGESTS["ops_n65536_257cubed"]["results"]
    g = gpu_ctx(case["params"])
    va, vb = FC.ops_inputs(case, g.slots, g.t)
    a = g.encrypt(g.encode(va)[None], 1)
    b = g.encrypt(g.encode(vb)[None], 2)
    res = {"enc_a": a, "enc_b": b}
    res["tensor"] = g.mul(a, b)
    res["relin"] = g.relin(res["tensor"])
    res["mul"] = g.mul_relin(a, b)
    res["modswitch_1"] = g.modswitch(a, 1)
    res["modswitch_3"] = g.modswitch(a, 3)
    res["rotate_5"] = g.rotate(a, 5)
    res["rotate_m1"] = g.rotate(a, 2 * g.N - 1)
    res["rotate_sum"] = g.rotate_sum(res["mul"])
    for i, d in enumerate(g.reduce(a)):
        res["digit_%d" % i] = d
    assert list(res) == FC.OPS_RESULTS
    for name, ct in res.items():
        check(name, ct, exp[name])


def test_ops_n65536_257cubed_inside_a_ragged_batch():
    """The digest case's ciphertexts as element 1 of batches of three (the
    others random): every batched operation at N = 2^16, level 41 runs its
    launches over three ciphertexts (an odd count, so the inner product's last
    ciphertext pair is ragged) and element 1 must still give the reference's
    words for the case alone."""
    case = FC.CASES["ops_n65536_257cubed"]
    exp = DIGESTS["ops_n65536_257cubed"]["results"]
    g = gpu_ctx(case["params"])
    va, vb = FC.ops_inputs(case, g.slots, g.t)
    rng = np.random.default_rng(77)
    A = np.stack([rng.integers(0, g.t, g.slots), va, rng.integers(0, g.t, g.slots)])
    B = np.stack([rng.integers(0, g.t, g.slots), vb, rng.integers(0, g.t, g.slots)])
    a = g.encrypt(np.stack([g.encode(v) for v in A]), 0)  # element 1: nonce 1, as enc_a
    b = g.encrypt(np.stack([g.encode(v) for v in B]), 1)  # element 1: nonce 2, as enc_b
    check("enc_a", a, exp["enc_a"], b=1)
    check("enc_b", b, exp["enc_b"], b=1)
    t = g.mul(a, b)
    check("tensor", t, exp["tensor"], b=1)
    check("relin", g.relin(t), exp["relin"], b=1)
    m = g.mul_relin(a, b)
    check("mul", m, exp["mul"], b=1)
    check("modswitch_3", g.modswitch(a, 3), exp["modswitch_3"], b=1)
    check("rotate_5", g.rotate(a, 5), exp["rotate_5"], b=1)
    check("rotate_sum", g.rotate_sum(m), exp["rotate_sum"], b=1)
    for i, d in enumerate(g.reduce(a)):
        check("digit_%d" % i, d, exp["digit_%d" % i], b=1)
    got = g.decrypt_slots(m)
    assert (got == (A.astype(object) * B.astype(object)) % g.t).all()


@pytest.mark.parametrize("name", ["query_n8192_17sq", "query_n32768_257sq", "query_n65536_257cubed",
                                  "query_n65536_257cubed_m3n", "query_n65536_257cubed_m5n2"])
def test_query_fullsize(name):
    from oracle import plain
    case = FC.CASES[name]
    ref = DIGESTS[name]["results"]
    g = gpu_ctx(case["params"])
    cols = FC.query_inputs(case, g.slots, g.t)
    enc = {}
    for k, v in cols.items():
        if case["square"] and k == "b":
            continue
        enc[k] = g.encrypt(np.stack([g.encode(row) for row in v]), FC.NONCE[k])
        for i in range(len(v)):
            check("%s_%d" % (k, i), enc[k], ref["inputs"]["%s_%d" % (k, i)], b=i)
    if case["square"]:
        enc["b"] = enc["a"]
    res = g.query(enc["a"], enc["b"], enc["c1"], enc["c2"])
    check("query", res, ref["result"])
    assert (g.decrypt_slots(res) == plain.query(cols["a"], cols["b"], cols["c1"], cols["c2"], g.t)).all()


# ---------------------------------------------------------------------- live cases
def same(gct, oct_list):
    w = gct.words()
    assert w.shape[0] == len(oct_list)
    for b, oc in enumerate(oct_list):
        assert (gct.ncomp, gct.level, gct.t_exp) == (oc.ncomp, oc.level, oc.t_exp)
        ow = oc.words()
        diff = np.argwhere(w[b] != ow)
        assert diff.size == 0, "first differing word %s of %d" % (diff[0], len(diff))


KS_SETS = [
    # N = 2^13 at the 17^2 parameter set: 9 digits of 2 primes
    (dict(logN=13, L=18, alpha=2, bits=36, p=17, r=2, h=120, seed=501), 2),
    # N = 2^14, 55-bit primes, alpha = 3 with a ragged last digit (11 = 3+3+3+2), 3 ciphertexts
    (dict(logN=14, L=11, alpha=3, bits=55, p=257, r=2, h=120, seed=502), 3),
]


@pytest.mark.parametrize("prm,count", KS_SETS, ids=["n8192", "n16384"])
def test_keyswitch_parity_two_phase(prm, count):
    keyswitch_case(prm, count)


@pytest.mark.parametrize("prm,count", [
    (dict(logN=10, L=6, alpha=2, bits=36, p=17, r=2, h=64, seed=503), 2),
    (dict(logN=12, L=7, alpha=3, bits=55, p=257, r=2, h=120, seed=504), 3)], ids=["n1024", "n4096"])
def test_keyswitch_parity_single_phase_folded(prm, count):
    """N = 1024 and 4096: the single-phase transform with the node-1 twiddle
    folded into the base conversions that feed it (the smallest ring where a
    base-conversion block lies in one half, and the largest single-phase ring)."""
    keyswitch_case(prm, count)


def keyswitch_case(prm, count):
    import paper_2604_19890_gb300 as ssg
    g = ssg.Context(nmax=0, **prm)
    o = O.Oracle(**prm)
    gal = g.rotate_sum_elements()
    g.keygen(gal)
    o.keygen(gal)
    rng = np.random.default_rng(prm["seed"])
    A = rng.integers(0, g.t, (count, g.slots))
    B = rng.integers(0, g.t, (count, g.slots))
    ga = g.encrypt(np.stack([g.encode(v) for v in A]), 10)
    gb = g.encrypt(np.stack([g.encode(v) for v in B]), 20)
    oa = [o.encrypt(o.encode(v), 10 + i) for i, v in enumerate(A)]
    ob = [o.encrypt(o.encode(v), 20 + i) for i, v in enumerate(B)]
    same(ga, oa)
    gt = g.mul(ga, gb)
    ot = [o.tensor(x, y) for x, y in zip(oa, ob)]
    same(g.relin(gt), [o.relin(x) for x in ot])
    gm = g.mul_relin(ga, gb)
    om = [o.mul(x, y) for x, y in zip(oa, ob)]
    same(gm, om)
    same(g.mul_relin(gm, ga), [o.mul(x, y) for x, y in zip(om, oa)])  # operands at different levels
    same(g.modswitch(ga, 2), [o.modswitch(x, 2) for x in oa])
    for gel in (5, 2 * g.N - 1):
        same(g.rotate(gm, gel), [o.rotate(x, gel) for x in om])
    assert (g.decrypt_slots(gm) == (A.astype(object) * B.astype(object)) % g.t).all()


@pytest.mark.parametrize("drop", [5, 8, 17, 38, 40])
def test_modswitch_many_primes_two_phase(drop):
    """Modulus switching by many primes at once (the query aligns operands
    down by up to 39 levels): base conversion from more than four primes, to
    one up to 36 remaining primes, at N = 2^14 on the 41-prime 55-bit chain."""
    import paper_2604_19890_gb300 as ssg
    prm = dict(logN=14, L=41, alpha=3, bits=55, p=257, r=3, h=120, seed=521)
    g = ssg.Context(nmax=0, **prm)
    o = O.Oracle(**prm)
    g.keygen([])
    o.keygen([])
    rng = np.random.default_rng(drop)
    A = rng.integers(0, g.t, (2, g.slots))
    ga = g.encrypt(np.stack([g.encode(v) for v in A]), 30)
    oa = [o.encrypt(o.encode(v), 30 + i) for i, v in enumerate(A)]
    same(ga, oa)
    gs = g.modswitch(ga, drop)
    same(gs, [o.modswitch(x, drop) for x in oa])
    assert gs.level == prm["L"] - drop
    assert (g.decrypt_slots(gs) == A).all()


BATCH_SETS = [dict(logN=14, L=14, alpha=2, bits=36, p=17, r=2, h=120, seed=511),
              dict(logN=15, L=14, alpha=2, bits=55, p=257, r=2, h=120, seed=512)]


def test_batch_mixed_n_two_phase():
    """Batched form over N = 2^14 (17^2) and 2^15 (257^2): products and the
    digits of Algorithm 3, each equal to the reference word for word, eagerly
    and from the replayed graph."""
    import torch
    import paper_2604_19890_gb300 as ssg
    gs, os_ = [], []
    for s in BATCH_SETS:
        g = ssg.Context(nmax=0, **s)
        o = O.Oracle(**s)
        g.keygen([])
        o.keygen([])
        gs.append(g)
        os_.append(o)
    rng = np.random.default_rng(5)
    plan = [(0, 14, True), (1, 14, True), (0, 9, True), (1, 6, False), (0, 5, False), (1, 12, True)]
    pairs, refs = [], []
    for i, (ci, lvl, red) in enumerate(plan):
        g, o = gs[ci], os_[ci]
        va, vb = rng.integers(0, g.t, g.slots), rng.integers(0, g.t, g.slots)
        ga, gb = g.encrypt(g.encode(va), 100 + 2 * i), g.encrypt(g.encode(vb), 101 + 2 * i)
        oa, ob = o.encrypt(o.encode(va), 100 + 2 * i), o.encrypt(o.encode(vb), 101 + 2 * i)
        if lvl < g.L:
            ga, gb = g.modswitch(ga, g.L - lvl), g.modswitch(gb, g.L - lvl)
            oa, ob = o.modswitch(oa, g.L - lvl), o.modswitch(ob, g.L - lvl)
        op = o.mul(oa, ob)
        od = None
        if red:
            try:
                od = o.reduce(op)
            except O.OracleError:
                od = "skip"
        pairs.append((ci, ga, gb, red))
        refs.append((op, od))
    assert sum(1 for _, od in refs if isinstance(od, list)) >= 2

    b = ssg.Batch(gs, pairs)
    st = torch.cuda.Stream()

    def verify():
        skipped = 0
        for (prod, digs), (op, od) in zip(b.results(), refs):
            same(prod, [op])
            if od == "skip":
                skipped += 1
            elif od is not None:
                assert len(digs) == len(od)
                for d, ref in zip(digs, od):
                    same(d, [ref])
        assert b.get_config()["skipped"] == skipped

    b.config(2, 3, 11)
    b.run(st)
    st.synchronize()
    verify()
    b.config(8, 1, 12)
    b.capture(st)
    for _ in range(2):
        b.run(st)
        st.synchronize()
        verify()
    # merged lanes: the transforms of both ring dimensions in shared persistent launches
    for chunk, tile in ((1, 11), (4, 12)):
        b.config(chunk, 0, tile)
        b.run(st)
        st.synchronize()
        verify()
    b.capture(st)
    for _ in range(2):
        b.run(st)
        st.synchronize()
        verify()
    b.close()
