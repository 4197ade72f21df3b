"""The cyclotomic ring m = 5N/2 (Phi_m = Phi_10(X^(N/4)); Section 2.1 with a
general m, Section 5.1's slot count n / Ord(m, p)) on the GPU, word for word
against the CPU reference through the C-ABI: context tables and slot algebra,
the transform at every ring size the kernels have (single-phase and the
two-phase radix-16 form with the four-way split), every BGV operation, the
space-switching procedures and the compare-then-SUM query. All arithmetic is
exact modular integer arithmetic: the tolerance is zero.
"""
import numpy as np
import pytest

import oracle as O
from oracle import plain

pytestmark = pytest.mark.gpu


def pair(logN=6, L=26, alpha=2, bits=36, p=17, r=2, h=16, seed=7, galois=None, keys=True):
    import paper_2604_19890_gb300 as ssg
    g = ssg.Context(logN=logN, L=L, alpha=alpha, bits=bits, p=p, r=r, h=h, nmax=0, seed=seed, m_odd=5)
    o = O.Oracle(logN=logN, L=L, alpha=alpha, bits=bits, p=p, r=r, h=h, seed=seed, m_odd=5)
    if keys:
        gal = g.rotate_sum_elements() if galois is None else galois
        g.keygen(gal)
        o.keygen(gal)
    return g, o


def same(gct, oct_list):
    w = gct.words()
    assert w.shape[0] == len(oct_list)
    for b, oc in enumerate(oct_list):
        assert (gct.ncomp, gct.level, gct.t_exp) == (oc.ncomp, oc.level, oc.t_exp)
        ow = oc.words()
        diff = np.argwhere(w[b] != ow)
        assert diff.size == 0, "first differing word %s of %d" % (diff[0], len(diff))


def encrypt_both(g, o, vals, nonce0):
    vals = np.atleast_2d(np.asarray(vals, dtype=np.uint64))
    gc = g.encrypt(np.stack([g.encode(v) for v in vals]), nonce0)
    oc = [o.encrypt(o.encode(v), nonce0 + i) for i, v in enumerate(vals)]
    return gc, oc


@pytest.fixture(scope="module")
def tiny():
    return pair()


@pytest.mark.parametrize("p,r,logN", [(17, 2, 6), (257, 2, 6), (13, 2, 6), (257, 3, 5), (41, 3, 7), (11, 2, 6),
                                      (257, 3, 16)])
def test_context_and_slots_match(p, r, logN):
    g, o = pair(logN=logN, L=3, alpha=2, bits=55 if p == 257 else 36, p=p, r=r, h=8, keys=False)
    assert g.m == o.m == 5 * g.N // 2
    assert (g.primes == o.primes()).all()
    assert (g.slots, g.d) == (o.slots, o.d)
    assert g.rotate_sum_elements() == o.rotate_sum_elements()
    rng = np.random.default_rng(p * r + logN)
    for te in range(1, r + 1):
        v = rng.integers(0, p ** te, o.slots)
        mg, mo = g.encode(v, te), o.encode(v, te)
        assert (mg == mo).all()
        assert (g.decode(mg, te) == v).all()
        c = rng.integers(0, p ** te, g.N).astype(np.uint64)
        assert (g.decode(c, te) == o.decode(c, te)).all()


@pytest.mark.parametrize("logN", [5, 6, 12, 13, 14, 15, 16])
def test_ntt_parity_5n2(logN):
    import torch
    import paper_2604_19890_gb300 as ssg
    L = 3
    g = ssg.Context(logN=logN, L=L, alpha=1, bits=55, p=257, r=2, h=4, nmax=0, seed=1, m_odd=5)
    o = O.Oracle(logN=logN, L=L, alpha=1, bits=55, p=257, r=2, h=4, seed=1, m_odd=5)
    rng = np.random.default_rng(logN)
    npoly = 2 * L if logN <= 13 else L
    data = np.stack([rng.integers(0, int(g.primes[i % L]), g.N, dtype=np.uint64) for i in range(npoly)])
    t = torch.from_numpy(data.view(np.int64).copy()).cuda()
    g.ntt_forward(t, 0, L)
    fw = t.cpu().numpy().view(np.uint64).copy()
    for i in range(npoly):
        assert (fw[i] == o.ntt_fwd(i % L, data[i])).all(), i
    g.ntt_inverse(t, 0, L)
    assert (t.cpu().numpy().view(np.uint64) == data).all()


@pytest.mark.parametrize("logN,bits,p", [(6, 58, 257), (13, 58, 257), (16, 58, 257), (16, 30, 13)])
def test_ntt_extreme_inputs_5n2(logN, bits, p):
    """Words q-1 and 0 everywhere, and the largest and smallest primes: the
    lazy bounds (below 38q forward) hold at the extremes."""
    import torch
    import paper_2604_19890_gb300 as ssg
    L = 2
    g = ssg.Context(logN=logN, L=L, alpha=1, bits=bits, p=p, r=2 if p == 257 else 1, h=4, nmax=0, seed=1, m_odd=5)
    o = O.Oracle(logN=logN, L=L, alpha=1, bits=bits, p=p, r=2 if p == 257 else 1, h=4, seed=1, m_odd=5)
    rows = []
    for i in range(L):
        q = int(g.primes[i])
        rows.append(np.full(g.N, q - 1, dtype=np.uint64))
        alt = np.zeros(g.N, dtype=np.uint64)
        alt[::2] = q - 1
        rows.append(alt)
    data = np.stack(rows)
    order = [0, 0, 1, 1]  # prime of each row
    t = torch.from_numpy(data.view(np.int64).copy()).cuda()
    for k, pi in enumerate(order):
        g.ntt_forward(t[k:k + 1], pi, 1)
    fw = t.cpu().numpy().view(np.uint64).copy()
    for k, pi in enumerate(order):
        assert (fw[k] == o.ntt_fwd(pi, data[k])).all(), k
    for k, pi in enumerate(order):
        g.ntt_inverse(t[k:k + 1], pi, 1)
    assert (t.cpu().numpy().view(np.uint64) == data).all()


def test_ops_parity_5n2(tiny):
    g, o = tiny
    rng = np.random.default_rng(2)
    A = rng.integers(0, g.t, (2, g.slots))
    B = rng.integers(0, g.t, (2, g.slots))
    ga, oa = encrypt_both(g, o, A, 100)
    gb, ob = encrypt_both(g, o, B, 200)
    same(ga, oa)
    assert (g.decrypt_slots(ga) == A).all()
    same(g.add(ga, gb), [o.add(x, y) for x, y in zip(oa, ob)])
    same(g.mul_scalar(ga, -12345), [o.mul_scalar(x, -12345) for x in oa])
    gt = g.mul(ga, gb)
    ot = [o.tensor(x, y) for x, y in zip(oa, ob)]
    same(gt, ot)
    gr = g.relin(gt)
    orl = [o.relin(x) for x in ot]
    same(gr, orl)
    same(g.mul_relin(ga, gb), [o.mul(x, y) for x, y in zip(oa, ob)])
    for drop in (1, 3):
        same(g.modswitch(gr, drop), [o.modswitch(x, drop) for x in orl])
    for gel in g.rotate_sum_elements():
        same(g.rotate(ga, gel), [o.rotate(x, gel) for x in oa])
    same(g.rotate_sum(ga), [o.rotate_sum(x) for x in oa])
    assert (g.decrypt_slots(g.rotate_sum(ga)) == (A.astype(object).sum(axis=1) % g.t)[:, None]).all()
    gm, om = encrypt_both(g, o, (A * g.p) % g.t, 300)
    same(g.divide_by_p(gm), [o.divide_by_p(x) for x in om])
    assert (g.decrypt_slots(gr) == (A * B) % g.t).all()


def test_reduce_compare_raise_parity_5n2(tiny):
    g, o = tiny
    rng = np.random.default_rng(3)
    A = rng.integers(0, g.t, (2, g.slots))
    B = rng.integers(0, g.t, (2, g.slots))
    ga, oa = encrypt_both(g, o, A, 400)
    gb, ob = encrypt_both(g, o, B, 500)
    gd = g.reduce(ga)
    od = [o.reduce(x) for x in oa]
    for i in range(g.r):
        same(gd[i], [d[i] for d in od])
    lt = g.compare_lt(ga, gb)
    olt = [o.compare_lt(x, y) for x, y in zip(oa, ob)]
    same(lt, olt)
    up = g.raise_modulus(lt)
    same(up, [o.raise_modulus(x) for x in olt])
    exp = np.array([[plain.lt(x, y, g.t) for x, y in zip(ra, rb)] for ra, rb in zip(A, B)])
    assert (g.decrypt_slots(up) == exp).all()


@pytest.mark.parametrize("n_ct,batch", [(1, 8), (3, 2)])
def test_query_parity_5n2(tiny, n_ct, batch):
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
    same(res, [o.query(oA, oB, oC, oT)])
    assert (g.decrypt_slots(res) == plain.query(cols["a"], cols["b"], cols["c1"], thr, g.t)).all()
    g.set_batch(8)


def test_p257_r3_query_5n2():
    """257^3 on the small ring: slots of conjugate roots over GR(257^3, 4)."""
    g, o = pair(logN=5, L=44, alpha=3, bits=55, p=257, r=3, h=16, seed=9)
    rng = np.random.default_rng(5)
    cols = {k: rng.integers(0, g.t, (1, g.slots)) for k in ("a", "b", "c1", "c2")}
    enc = {k: encrypt_both(g, o, v, 100 * (i + 1)) for i, (k, v) in enumerate(cols.items())}
    res = g.query(*(enc[k][0] for k in ("a", "b", "c1", "c2")))
    same(res, [o.query(*(enc[k][1] for k in ("a", "b", "c1", "c2")))])
    assert (g.decrypt_slots(res) == plain.query(cols["a"], cols["b"], cols["c1"], cols["c2"], g.t)).all()


@pytest.mark.parametrize("prm,count", [
    (dict(logN=13, L=18, alpha=2, bits=36, p=17, r=2, h=120, seed=601), 2),
    (dict(logN=14, L=11, alpha=3, bits=55, p=257, r=2, h=120, seed=602), 3),
], ids=["n8192", "n16384"])
def test_keyswitch_parity_two_phase_5n2(prm, count):
    """Key switching on the two-phase transform with the split stage: ModUp's
    out-of-place inverse and digit-skipping forward transforms, ModDown, the
    fused drop, and rotations by every rotate-sum element and X -> X^(m-1)."""
    g, o = pair(**prm, galois=[])
    gal = g.rotate_sum_elements() + [g.m - 1]
    g.keygen(gal)
    o.keygen(gal)
    rng = np.random.default_rng(prm["seed"])
    A = rng.integers(0, g.t, (count, g.slots))
    B = rng.integers(0, g.t, (count, g.slots))
    ga, oa = encrypt_both(g, o, A, 10)
    gb, ob = encrypt_both(g, o, B, 20)
    same(ga, oa)
    gt = g.mul(ga, gb)
    ot = [o.tensor(x, y) for x, y in zip(oa, ob)]
    same(g.relin(gt), [o.relin(x) for x in ot])
    gm = g.mul_relin(ga, gb)
    om = [o.mul(x, y) for x, y in zip(oa, ob)]
    same(gm, om)
    same(g.modswitch(ga, 2), [o.modswitch(x, 2) for x in oa])
    for gel in gal:
        same(g.rotate(gm, gel), [o.rotate(x, gel) for x in om])
    same(g.rotate_sum(gm), [o.rotate_sum(x) for x in om])
    assert (g.decrypt_slots(gm) == (A.astype(object) * B.astype(object)) % g.t).all()


def test_batch_mixed_rings_5n2():
    """Batched form over an m = 5N/2 context (N = 2^14, 17^2) and an X^N + 1
    context (N = 2^15, 257^2): products and Algorithm 3's digits equal the
    reference word for word, on streams, with merged transform lanes, and from
    the replayed graph."""
    import torch
    import paper_2604_19890_gb300 as ssg
    sets = [dict(logN=14, L=14, alpha=2, bits=36, p=17, r=2, h=120, seed=521, m_odd=5),
            dict(logN=15, L=14, alpha=2, bits=55, p=257, r=2, h=120, seed=522, m_odd=1)]
    gs, os_ = [], []
    for s in sets:
        g = ssg.Context(nmax=0, **s)
        o = O.Oracle(**s)
        g.keygen([])
        o.keygen([])
        gs.append(g)
        os_.append(o)
    rng = np.random.default_rng(6)
    plan = [(0, 14, True), (1, 14, True), (0, 9, False), (1, 6, False), (0, 12, True)]
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
    b = ssg.Batch(gs, pairs)
    st = torch.cuda.Stream()

    def verify():
        for (prod, digs), (op, od) in zip(b.results(), refs):
            same(prod, [op])
            if isinstance(od, list):
                assert len(digs) == len(od)
                for d, ref in zip(digs, od):
                    same(d, [ref])

    for chunk, nstr in ((2, 3), (1, 0), (4, 0)):
        b.config(chunk, nstr, 11)
        b.run(st)
        st.synchronize()
        verify()
    b.capture(st)
    for _ in range(2):
        b.run(st)
        st.synchronize()
        verify()
    b.close()


@pytest.mark.parametrize("p,r,L", [(7, 3, 30), (11, 4, 44)])
def test_compare_raise_p3mod4_5n2(p, r, L):
    """Plaintext primes p = 3 mod 4 (the paper's (7, 3) and (11, 4)) on m = 5N/2:
    Algorithm 3's digits, Algorithm 4 and raising word for word."""
    g, o = pair(logN=7, L=L, alpha=3, bits=55, p=p, r=r, h=16, seed=13, galois=[])
    rng = np.random.default_rng(p)
    A = rng.integers(0, g.t, (2, g.slots))
    B = rng.integers(0, g.t, (2, g.slots))
    ga, oa = encrypt_both(g, o, A, 50)
    gb, ob = encrypt_both(g, o, B, 60)
    gd = g.reduce(ga)
    od = [o.reduce(x) for x in oa]
    for i in range(r):
        same(gd[i], [d[i] for d in od])
    lt = g.compare_lt(ga, gb)
    olt = [o.compare_lt(x, y) for x, y in zip(oa, ob)]
    same(lt, olt)
    up = g.raise_modulus(lt)
    same(up, [o.raise_modulus(x) for x in olt])
    exp = np.array([[plain.lt(x, y, g.t) for x, y in zip(ra, rb)] for ra, rb in zip(A, B)])
    assert (g.decrypt_slots(up) == exp).all()


def test_served_mixed_rings_equal_alone_5n2():
    """One server over an m = 5N/2 context and an X^N + 1 context (N = 2^13,
    17^2 both): interleaved queries merge only within their context and each
    result equals the same query run alone, word for word."""
    import paper_2604_19890_gb300 as ssg
    g1 = ssg.Context(logN=13, L=18, alpha=2, bits=36, p=17, r=2, h=120, nmax=0, seed=51, m_odd=5)
    g2 = ssg.Context(logN=13, L=18, alpha=2, bits=36, p=17, r=2, h=120, nmax=0, seed=52)
    for g in (g1, g2):
        g.keygen()
    assert g1.slots == 4 * g2.slots
    rng = np.random.default_rng(8)
    qs = []
    for i, n in enumerate([1, 2, 2, 1, 1, 2]):
        ci = i % 2
        g = (g1, g2)[ci]
        cols = {k: rng.integers(0, g.t, (n, g.slots)) for k in ("a", "b", "c1")}
        c2 = np.full((1, g.slots), int(rng.integers(0, g.t)))
        enc = lambda v, nonce: g.encrypt(np.stack([g.encode(x) for x in v]), nonce)
        A, B, C1, C2 = (enc(cols["a"], 100 * i + 1), enc(cols["b"], 100 * i + 20), enc(cols["c1"], 100 * i + 40),
                        enc(c2, 100 * i + 60))
        qs.append((ci, (A, B, C1, C2), plain.query(cols["a"], cols["b"], cols["c1"], c2, g.t)))
    alone = [(g1, g2)[ci].query(*cols).words() for ci, cols, _ in qs]
    srv = ssg.Server([g1, g2], workers=2, max_merge=4)
    tickets = [srv.submit(*cols, ctx_index=ci) for ci, cols, _ in qs]
    for t, (ci, cols, exp), ref in zip(tickets, qs, alone):
        res, _, _ = srv.wait(t, timeout_ms=120000)
        assert (res.words() == ref).all()
        assert ((g1, g2)[ci].decrypt_slots(res) == exp).all()
    srv.close()
