"""GPU path vs the CPU reference, word for word (all arithmetic is exact modular
integer arithmetic, so the tolerance is zero), through the C-ABI.

Small rings (N = 64) cover every operation and the space-switching
procedures; larger rings cover the transform and the batched kernels with
several tiles and ragged batch sizes.
"""
import numpy as np
import pytest

import oracle as O
from oracle import plain

pytestmark = pytest.mark.gpu


def gpu_ctx(**kw):
    import paper_2604_19890_gb300 as ssg
    return ssg.Context(**kw)


def make_pair(logN=6, L=26, alpha=2, bits=36, p=17, r=2, h=16, seed=7, galois=None, keys=True):
    g = gpu_ctx(logN=logN, L=L, alpha=alpha, bits=bits, p=p, r=r, h=h, nmax=0, seed=seed)
    o = O.Oracle(logN=logN, L=L, alpha=alpha, bits=bits, p=p, r=r, h=h, seed=seed)
    if keys:
        gal = g.rotate_sum_elements() if galois is None else galois
        g.keygen(gal)
        o.keygen(gal)
    return g, o


def same(gct, oct_list):
    """GPU batch words == oracle words for every ciphertext of the batch."""
    w = gct.words()
    assert w.shape[0] == len(oct_list)
    for b, oc in enumerate(oct_list):
        assert (gct.ncomp, gct.level, gct.t_exp) == (oc.ncomp, oc.level, oc.t_exp)
        ow = oc.words()
        assert w[b].shape == ow.shape
        diff = np.argwhere(w[b] != ow)
        assert diff.size == 0, "first differing word %s of %d" % (diff[0], len(diff))


@pytest.fixture(scope="module")
def tiny():
    return make_pair()


def encrypt_both(g, o, vals, nonce0):
    vals = np.atleast_2d(np.asarray(vals, dtype=np.uint64))
    gc = g.encrypt(np.stack([g.encode(v) for v in vals]), nonce0)
    oc = [o.encrypt(o.encode(v), nonce0 + i) for i, v in enumerate(vals)]
    return gc, oc


def test_context_tables_match(tiny):
    g, o = tiny
    assert (g.primes == o.primes()).all()
    assert g.slots == o.slots and g.d == o.d


@pytest.mark.parametrize("logN", [3, 6, 12, 13, 14, 15, 16])
def test_ntt_parity(logN):
    import torch
    L = 3
    g = gpu_ctx(logN=logN, L=L, alpha=1, bits=55, p=257, r=2, h=4, nmax=0, seed=1)
    o = O.Oracle(logN=logN, L=L, alpha=1, bits=55, p=257, r=2, h=4, seed=1)
    rng = np.random.default_rng(logN)
    npoly = 2 * L + 1 if logN <= 13 else L  # ragged batch: more polys than primes
    npoly -= npoly % L
    data = np.stack([rng.integers(0, int(g.primes[i % L]), g.N, dtype=np.uint64) for i in range(npoly)])
    t = torch.from_numpy(data.view(np.int64).copy()).cuda()
    g.ntt_forward(t, 0, L)
    fw = t.cpu().numpy().view(np.uint64).copy()
    for i in range(npoly):
        assert (fw[i] == o.ntt_fwd(i % L, data[i])).all(), i
    g.ntt_inverse(t, 0, L)
    assert (t.cpu().numpy().view(np.uint64) == data).all()


@pytest.mark.parametrize("logN,bits", [(13, 58), (16, 58), (16, 30)])
def test_ntt_extreme_inputs(logN, bits):
    """Largest residues (every word q - 1, alternating 0 / q - 1, a single
    q - 1) at the widest and narrowest allowed primes: the forward transform
    lets lazy residues grow through all stages before one final reduction."""
    import torch
    L = 2
    g = gpu_ctx(logN=logN, L=L, alpha=1, bits=bits, p=17, r=1, h=4, nmax=0, seed=3)
    o = O.Oracle(logN=logN, L=L, alpha=1, bits=bits, p=17, r=1, h=4, seed=3)
    rows = []
    for i in range(L):
        q = int(g.primes[i])
        full = np.full(g.N, q - 1, dtype=np.uint64)
        alt = full.copy()
        alt[::2] = 0
        one = np.zeros(g.N, dtype=np.uint64)
        one[g.N // 3] = q - 1
        rows.append((i, [full, alt, one]))
    data = np.stack([rows[i % L][1][k] for k in range(3) for i in range(L)])
    t = torch.from_numpy(data.view(np.int64).copy()).cuda()
    g.ntt_forward(t, 0, L)
    fw = t.cpu().numpy().view(np.uint64).copy()
    for j in range(data.shape[0]):
        assert (fw[j] == o.ntt_fwd(j % L, data[j])).all(), j
    g.ntt_inverse(t, 0, L)
    assert (t.cpu().numpy().view(np.uint64) == data).all()


def test_encrypt_batch_parity(tiny):
    g, o = tiny
    rng = np.random.default_rng(1)
    vals = rng.integers(0, g.t, (3, g.slots))
    gc, oc = encrypt_both(g, o, vals, 40)
    same(gc, oc)
    assert (g.decrypt_slots(gc) == vals).all()


def test_ops_parity(tiny):
    g, o = tiny
    rng = np.random.default_rng(2)
    A = rng.integers(0, g.t, (2, g.slots))
    B = rng.integers(0, g.t, (2, g.slots))
    ga, oa = encrypt_both(g, o, A, 100)
    gb, ob = encrypt_both(g, o, B, 200)
    same(g.add(ga, gb), [o.add(x, y) for x, y in zip(oa, ob)])
    same(g.sub(ga, gb), [o.sub(x, y) for x, y in zip(oa, ob)])
    same(g.mul_scalar(ga, -12345), [o.mul_scalar(x, -12345) for x in oa])
    same(g.add_scalar(ga, 77), [o.add_scalar(x, 77) for x in oa])
    gt = g.mul(ga, gb)
    ot = [o.tensor(x, y) for x, y in zip(oa, ob)]
    same(gt, ot)
    gr = g.relin(gt)
    orl = [o.relin(x) for x in ot]
    same(gr, orl)
    for drop in (1, 2, 5):
        same(g.modswitch(gr, drop), [o.modswitch(x, drop) for x in orl])
    for gel in g.rotate_sum_elements():
        same(g.rotate(ga, gel), [o.rotate(x, gel) for x in oa])
    same(g.rotate_sum(ga), [o.rotate_sum(x) for x in oa])
    # DivideByP on multiples of p
    gm, om = encrypt_both(g, o, (A * g.p) % g.t, 300)
    same(g.divide_by_p(gm), [o.divide_by_p(x) for x in om])
    # decrypted semantics of the GPU results
    assert (g.decrypt_slots(gr) == (A * B) % g.t).all()


@pytest.mark.parametrize("nterms,lim_bits", [(1, 0), (3, 0), (15, 0), (20, 0), (4, 34), (6, 31)])
def test_linear_combination_parity(tiny, nterms, lim_bits):
    g, o = tiny
    rng = np.random.default_rng(30 + nterms)
    cts = [encrypt_both(g, o, rng.integers(0, g.t, (2, g.slots)), 2000 + 10 * i) for i in range(nterms)]
    # |c| < 2^27: 64-bit accumulators of 32-bit halves; below 2^32: two 32-bit
    # products into 128-bit sums; larger: the general 64-bit product path
    lim = (1 << lim_bits) if lim_bits else g.t // 2
    coeffs = [int(c) for c in rng.integers(-lim, lim, nterms)]
    cst = int(rng.integers(-100, 100))
    got = g.linear_combination([c[0] for c in cts], coeffs, cst)
    ref = []
    for b in range(2):
        acc = None
        for (gc, oc), cf in zip(cts, coeffs):
            term = o.mul_scalar(oc[b], cf)
            acc = term if acc is None else o.add(acc, term)
        ref.append(o.add_scalar(acc, cst))
    same(got, ref)


def test_linear_combination_rejects_scalars_beyond_the_primes(tiny):
    import paper_2604_19890_gb300 as ssg
    g, o = tiny
    gc, _ = encrypt_both(g, o, np.zeros((1, g.slots)), 2900)
    for c in (1 << 35, -(1 << 40)):  # the 36-bit primes lie above 2^35
        with pytest.raises(ssg.SSError) as e:
            g.linear_combination([gc, gc], [3, c])
        assert e.value.code == ssg.SS_ERR_PARAM


def test_eval_g_reduce_compare_raise_parity(tiny):
    g, o = tiny
    rng = np.random.default_rng(3)
    A = rng.integers(0, g.t, (2, g.slots))
    B = rng.integers(0, g.t, (2, g.slots))
    ga, oa = encrypt_both(g, o, A, 400)
    gb, ob = encrypt_both(g, o, B, 500)
    same(g.eval_g(ga, 2), [o.eval_g(x, 2) for x in oa])
    gd = g.reduce(ga)
    od = [o.reduce(x) for x in oa]
    for i in range(g.r):
        same(gd[i], [d[i] for d in od])
    lt = g.compare_lt(ga, gb)
    olt = [o.compare_lt(x, y) for x, y in zip(oa, ob)]
    same(lt, olt)
    exp = np.array([[plain.lt(x, y, g.t) for x, y in zip(ra, rb)] for ra, rb in zip(A, B)])
    assert (g.decrypt_slots(lt) == exp).all()
    up = g.raise_modulus(lt)
    same(up, [o.raise_modulus(x) for x in olt])
    assert (g.decrypt_slots(up) == exp).all()


def test_compare_with_broadcast_threshold(tiny):
    g, o = tiny
    rng = np.random.default_rng(4)
    A = rng.integers(0, g.t, (3, g.slots))
    T = np.full((1, g.slots), 150)
    ga, oa = encrypt_both(g, o, A, 600)
    gt, ot = encrypt_both(g, o, T, 700)
    lt = g.compare_lt(ga, gt)
    same(lt, [o.compare_lt(x, ot[0]) for x in oa])


@pytest.mark.parametrize("n_ct,batch", [(1, 8), (3, 2), (5, 8)])
def test_query_parity(tiny, n_ct, batch):
    g, o = tiny
    rng = np.random.default_rng(10 + n_ct)
    cols = {k: rng.integers(0, g.t, (n_ct, g.slots)) for k in ("a", "b", "c1")}
    thr = np.full((1, g.slots), 150)
    gA, oA = encrypt_both(g, o, cols["a"], 1000)
    gB, oB = encrypt_both(g, o, cols["b"], 2000)
    gC, oC = encrypt_both(g, o, cols["c1"], 3000)
    gT, oT = encrypt_both(g, o, thr, 4000)
    g.set_batch(batch)
    res = g.query(gA, gB, gC, gT)
    ores = o.query(oA, oB, oC, oT)
    same(res, [ores])
    exp = plain.query(cols["a"], cols["b"], cols["c1"], thr, g.t)
    assert (g.decrypt_slots(res) == exp).all()
    assert o.noise_budget(ores) > 0
    g.set_batch(8)


@pytest.mark.parametrize("pred", ["lt", "le", "gt", "ge", "eq", "neq"])
def test_predicate_parity(tiny, pred):
    g, o = tiny
    rng = np.random.default_rng(60 + len(pred))
    A = rng.integers(0, g.t, (2, g.slots))
    B = rng.integers(0, g.t, (2, g.slots))
    B[0, :3] = A[0, :3]  # equal pairs
    B[1, 3] = (A[1, 3] + g.p) % g.t  # same low digit
    ga, oa = encrypt_both(g, o, A, 1200)
    gb, ob = encrypt_both(g, o, B, 1300)
    got = g.compare(pred, ga, gb)
    same(got, [o.compare(pred, x, y) for x, y in zip(oa, ob)])
    exp = [[plain.predicate(pred, x, y, g.t) for x, y in zip(ra, rb)] for ra, rb in zip(A, B)]
    assert (g.decrypt_slots(got) == np.array(exp)).all()


@pytest.mark.parametrize("pred", ["gt", "le", "eq"])
def test_predicate_broadcast_either_side(tiny, pred):
    g, o = tiny
    rng = np.random.default_rng(70)
    X = rng.integers(0, g.t, (2, g.slots))
    thr = np.full((1, g.slots), 150)
    X[1, :2] = 150
    gx, ox = encrypt_both(g, o, X, 1400)
    gt_, ot_ = encrypt_both(g, o, thr, 1500)
    same(g.compare(pred, gx, gt_), [o.compare(pred, x, ot_[0]) for x in ox])
    same(g.compare(pred, gt_, gx), [o.compare(pred, ot_[0], x) for x in ox])


def test_query_where_parity(tiny):
    g, o = tiny
    rng = np.random.default_rng(80)
    n = 3
    cols = {k: rng.integers(0, g.t, (n, g.slots)) for k in ("a", "b", "c1", "c2", "c3")}
    cols["c3"][:, ::3] = 7
    enc = {k: encrypt_both(g, o, v, 5000 + 100 * i) for i, (k, v) in enumerate(cols.items())}
    gk, ok = encrypt_both(g, o, np.full((1, g.slots), 7), 5900)
    g.set_batch(2)
    got = g.query_where(enc["a"][0], enc["b"][0], [("lt", enc["c1"][0], enc["c2"][0]), ("eq", enc["c3"][0], gk)])
    g.set_batch(8)
    ref = o.query_where(enc["a"][1], enc["b"][1], [("lt", enc["c1"][1], enc["c2"][1]), ("eq", enc["c3"][1], ok)])
    same(got, [ref])
    exp = plain.query_where(cols["a"], cols["b"], [("lt", cols["c1"], cols["c2"]), ("eq", cols["c3"], 7)], g.t)
    assert (g.decrypt_slots(got) == exp).all()
    # one LT condition is the LT query, word for word
    one = g.query_where(enc["a"][0], enc["b"][0], [("lt", enc["c1"][0], enc["c2"][0])])
    same(one, [o.query(enc["a"][1], enc["b"][1], enc["c1"][1], enc["c2"][1])])


@pytest.mark.parametrize("p,r", [(5, 4), (41, 3), (37, 4)])
def test_compare_raise_other_p_r(p, r):
    """LT then raising at the (p, r) of the LT sweep's other bit widths, 50-bit primes, N = 64."""
    g, o = make_pair(logN=6, L=60, alpha=2, bits=50, p=p, r=r, h=16, seed=11, galois=[])
    rng = np.random.default_rng(p * r)
    A = rng.integers(0, g.t, (2, g.slots))
    B = rng.integers(0, g.t, (2, g.slots))
    ga, oa = encrypt_both(g, o, A, 700)
    gb, ob = encrypt_both(g, o, B, 710)
    got = g.raise_modulus(g.compare("lt", ga, gb))
    same(got, [o.raise_modulus(o.compare_lt(x, y)) for x, y in zip(oa, ob)])
    exp = [[plain.lt(x, y, g.t) for x, y in zip(ra, rb)] for ra, rb in zip(A, B)]
    assert (g.decrypt_slots(got) == np.array(exp)).all()


def test_eq_schedule_trace_matches_reference(tiny):
    g, o = tiny
    rng = np.random.default_rng(9)
    ga, oa = encrypt_both(g, o, rng.integers(0, g.t, (1, g.slots)), 810)
    gb, ob = encrypt_both(g, o, rng.integers(0, g.t, (1, g.slots)), 910)
    g.trace(True)
    o.trace(True)
    g.compare("neq", ga, gb)
    o.compare("neq", oa[0], ob[0])
    gt, ot = g.trace_text(), o.trace_text()
    g.trace(False)
    o.trace(False)
    assert gt == ot and "eq digit" in gt


def test_query_from_host_memory_matches_device_query(tiny):
    """ss_query_sum_where_lt_host (columns in host memory, A and B uploaded on a
    second stream while the comparisons run) returns the device query's words."""
    g, o = tiny
    rng = np.random.default_rng(90)
    cols = [rng.integers(0, g.t, (3, g.slots)) for _ in range(4)]
    enc = [encrypt_both(g, o, v, 6000 + 100 * i)[0] for i, v in enumerate(cols)]
    ref = g.query(*enc)
    host = [e.words() for e in enc]
    out, lvl, te = g.query_host(*host, enc[0].level)
    assert (lvl, te) == (ref.level, ref.t_exp)
    assert (out == ref.words()[0]).all()


def test_schedule_trace_matches_reference(tiny):
    g, o = tiny
    rng = np.random.default_rng(5)
    ga, oa = encrypt_both(g, o, rng.integers(0, g.t, (1, g.slots)), 800)
    gb, ob = encrypt_both(g, o, rng.integers(0, g.t, (1, g.slots)), 900)
    g.trace(True)
    o.trace(True)
    g.compare_lt(ga, gb)
    o.compare_lt(oa[0], ob[0])
    gt, ot = g.trace_text(), o.trace_text()
    g.trace(False)
    o.trace(False)
    assert gt == ot and len(gt.splitlines()) > 20


def test_query_depth_matches_reference(tiny):
    g, o = tiny
    d = g.query_depth()
    rng = np.random.default_rng(6)
    ga, oa = encrypt_both(g, o, rng.integers(0, g.t, (1, g.slots)), 950)
    res = o.query(oa, oa, oa, oa)
    assert d == res.level


def test_errors_are_reported(tiny):
    import paper_2604_19890_gb300 as ssg
    g, o = tiny
    ga, _ = encrypt_both(g, o, np.zeros((1, g.slots)), 960)
    low = g.modswitch(ga, 3)
    with pytest.raises(ssg.SSError) as e:
        g.add(ga, low)
    assert e.value.code == ssg.SS_ERR_LEVEL
    with pytest.raises(ssg.SSError) as e:
        g.modswitch(ga, ga.level)
    assert e.value.code == ssg.SS_ERR_LEVEL
    d = g.divide_by_p(g.encrypt_slots(np.zeros((1, g.slots)), 970))
    with pytest.raises(ssg.SSError) as e:
        g.add(ga, d)
    assert e.value.code == ssg.SS_ERR_TMOD
    with pytest.raises(ssg.SSError) as e:
        g.rotate(ga, 3)
    assert e.value.code == ssg.SS_ERR_PARAM


def test_p257_r3_small_ring():
    g, o = make_pair(logN=5, L=44, alpha=3, bits=55, p=257, r=3, h=8, seed=21)
    rng = np.random.default_rng(7)
    A = rng.integers(0, g.t, (2, g.slots))
    B = rng.integers(0, g.t, (2, g.slots))
    ga, oa = encrypt_both(g, o, A, 10)
    gb, ob = encrypt_both(g, o, B, 20)
    lt = g.compare_lt(ga, gb)
    same(lt, [o.compare_lt(x, y) for x, y in zip(oa, ob)])
    exp = np.array([[plain.lt(x, y, g.t) for x, y in zip(ra, rb)] for ra, rb in zip(A, B)])
    assert (g.decrypt_slots(lt) == exp).all()


def test_short_chain_is_rejected_before_any_launch():
    """A chain shorter than the schedule's depth fails with SS_ERR_NOISE from
    the plan, before anything is enqueued: the library's launch count does not
    move (query, conjunctive query, host-memory query and comparison)."""
    import paper_2604_19890_gb300 as ssg
    g, _ = make_pair(L=9, seed=17)  # the 17^2 query consumes 16 levels
    rng = np.random.default_rng(18)
    cols = [g.encrypt_slots(rng.integers(0, g.t, (2, g.slots)), 100 * (i + 1)) for i in range(4)]
    calls = [lambda: g.query(*cols),
             lambda: g.query_where(cols[0], cols[1], [("lt", cols[2], cols[3]), ("eq", cols[2], cols[3])]),
             lambda: g.query_host(*[c.words() for c in cols], cols[0].level),
             lambda: g.compare_lt(cols[2], cols[3])]
    for call in calls:
        n0 = g.launches()
        with pytest.raises(ssg.SSError) as e:
            call()
        assert e.value.code == ssg.SS_ERR_NOISE
        assert g.launches() == n0
    with pytest.raises(ssg.SSError) as e:
        g.query_depth()
    assert e.value.code == ssg.SS_ERR_NOISE


def _oracle_lincomb(o, cts, coeffs, cst=0):
    acc = None
    for oc, cf in zip(cts, coeffs):
        term = o.mul_scalar(oc, cf)
        acc = term if acc is None else o.add(acc, term)
    return o.add_scalar(acc, cst) if cst else acc


def test_linear_combination_at_the_small_scalar_bound(tiny):
    """16 terms with coefficients of magnitude 2^27 - 1 and mixed signs plus a
    constant: the largest sums the 64-bit accumulators of 32-bit word halves
    must hold (the path for scalars below 2^27)."""
    g, o = tiny
    rng = np.random.default_rng(91)
    cts = [encrypt_both(g, o, rng.integers(0, g.t, (2, g.slots)), 7000 + 10 * i) for i in range(16)]
    lim = (1 << 27) - 1
    coeffs = [lim if i % 3 else -lim for i in range(16)]
    got = g.linear_combination([c[0] for c in cts], coeffs, -98765)
    same(got, [_oracle_lincomb(o, [c[1][b] for c in cts], coeffs, -98765) for b in range(2)])


@pytest.mark.parametrize("rows", [
    # every scalar below 2^27 (32-bit word halves into 64-bit sums), one row at the bound
    [[(1 << 27) - 1, -((1 << 27) - 1), 5, -7, 1], [3, 1, -1, 0, 2]],
    # one scalar at 2^27: the launch takes the path for scalars below 2^32
    [[(1 << 27) - 1, -3, 5, 1 << 27, 1], [-((1 << 31) - 5), 0, 1, 2, -(1 << 27)]],
    # one scalar at 2^33: the general path (64-bit products; the 36-bit primes lie above 2^35)
    [[1 << 33, -5, 1, 0, 7], [-((1 << 34) + 3), 2, 0, 1, 1], [1, 1, 1, 1, 1]],
])
def test_linear_combinations_parity(tiny, rows):
    """ss_linear_combinations (several outputs of one set of terms in one pass,
    the Paterson-Stockmeyer leaves) against the reference's chain of scalar
    products and additions, on each of its three scalar paths."""
    g, o = tiny
    rng = np.random.default_rng(92 + len(rows))
    n = len(rows[0])
    cts = [encrypt_both(g, o, rng.integers(0, g.t, (2, g.slots)), 7500 + 10 * i) for i in range(n)]
    got = g.linear_combinations([c[0] for c in cts], rows)
    assert len(got) == len(rows)
    for k, row in enumerate(rows):
        same(got[k], [_oracle_lincomb(o, [c[1][b] for c in cts], row) for b in range(2)])
        single = g.linear_combination([c[0] for c in cts], row)
        assert (single.words() == got[k].words()).all()


@pytest.mark.parametrize("p,r,logN,L,alpha,bits", [(17, 3, 6, 30, 2, 50), (257, 3, 5, 44, 3, 55)])
def test_reduced_g_parity(p, r, logN, L, alpha, bits):
    """The lattice-reduced G_{p,e} (Section 4.2; ss_set_g_table(ctx, 1)) on both
    sides: G evaluation, Algorithm 3, comparison and raising, word for word,
    and decrypted against the plaintext definitions."""
    g, o = make_pair(logN=logN, L=L, alpha=alpha, bits=bits, p=p, r=r, h=8, seed=23)
    g.set_g_table(1)
    o.set_reduced_g(True)
    rng = np.random.default_rng(p + r)
    A = rng.integers(0, g.t, (2, g.slots))
    B = rng.integers(0, g.t, (2, g.slots))
    ga, oa = encrypt_both(g, o, A, 30)
    gb, ob = encrypt_both(g, o, B, 40)
    red = g.eval_g(ga, r)
    same(red, [o.eval_g(x, r) for x in oa])
    gd = g.reduce(ga)
    od = [o.reduce(x) for x in oa]
    for i in range(r):
        same(gd[i], [d[i] for d in od])
    up = g.raise_modulus(g.compare_lt(ga, gb))
    same(up, [o.raise_modulus(o.compare_lt(x, y)) for x, y in zip(oa, ob)])
    exp = np.array([[plain.lt(x, y, g.t) for x, y in zip(ra, rb)] for ra, rb in zip(A, B)])
    assert (g.decrypt_slots(up) == exp).all()
    # the canonical table gives other words for the same input (the test is not vacuous)
    g.set_g_table(0)
    assert (g.eval_g(ga, r).words() != red.words()).any()


def _random_sets(n, seed):
    """Seeded parameter sets across the space the library accepts: ring 2^4..2^7,
    primes of 30..58 bits (58: the lazy-transform bound), 1..3 special primes,
    plaintext p^r in {5^2, 13^2, 17^2, 17^3, 257, 257^2}."""
    rng = np.random.default_rng(seed)
    pr = [(5, 2), (13, 2), (17, 2), (17, 3), (257, 1), (257, 2)]
    out = []
    for k in range(n):
        p, r = pr[k % len(pr)]
        out.append(dict(logN=int(rng.integers(4, 8)), L=int(rng.integers(4, 9)), alpha=int(rng.integers(1, 4)),
                        bits=int(rng.choice([30, 36, 45, 50, 55, 58])), p=p, r=r, h=8, seed=int(rng.integers(1, 1 << 30))))
    return out


@pytest.mark.parametrize("prm", _random_sets(12, 2026), ids=lambda d: "N%d_L%d_a%d_b%d_p%d_r%d" % (
    1 << d["logN"], d["L"], d["alpha"], d["bits"], d["p"], d["r"]))
def test_random_parameter_sets(prm):
    """Every BGV operation word for word against the reference on seeded random
    parameter sets: encryption, tensor, relinearisation, the evaluator's
    multiplication, modulus switching, every rotate-sum element, DivideByP,
    a linear combination, and decryption of the product."""
    import paper_2604_19890_gb300 as ssg
    try:
        g = ssg.Context(nmax=0, **prm)
    except ssg.SSError:
        pytest.skip("no prime chain of this width for this ring and plaintext modulus")
    o = O.Oracle(**prm)
    gal = g.rotate_sum_elements()
    g.keygen(gal)
    o.keygen(gal)
    rng = np.random.default_rng(prm["seed"] % 1000)
    A = rng.integers(0, g.t, (2, g.slots))
    B = rng.integers(0, g.t, (2, g.slots))
    ga, oa = encrypt_both(g, o, A, 50)
    gb, ob = encrypt_both(g, o, B, 60)
    same(ga, oa)
    gt = g.mul(ga, gb)
    ot = [o.tensor(x, y) for x, y in zip(oa, ob)]
    same(gt, ot)
    same(g.relin(gt), [o.relin(x) for x in ot])
    gm = g.mul_relin(ga, gb)
    om = [o.mul(x, y) for x, y in zip(oa, ob)]
    same(gm, om)
    if prm["L"] > 2:
        same(g.modswitch(ga, 2), [o.modswitch(x, 2) for x in oa])
    for gel in gal:
        same(g.rotate(ga, gel), [o.rotate(x, gel) for x in oa])
    same(g.linear_combination([ga, gb], [7, -3], 5), [o.add_scalar(o.add(o.mul_scalar(x, 7), o.mul_scalar(y, -3)), 5)
                                                      for x, y in zip(oa, ob)])
    if g.r >= 2:
        gp, op = encrypt_both(g, o, (A * g.p) % g.t, 70)
        same(g.divide_by_p(gp), [o.divide_by_p(x) for x in op])
    assert (g.decrypt_slots(gm) == (A.astype(object) * B.astype(object)) % g.t).all()
