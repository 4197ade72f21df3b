"""Served form (ss_server_*): queries submitted while others run are merged
and overlapped, and every result must equal the same query run alone, word
for word, and decrypt to the query's plaintext value."""
import threading
import time

import numpy as np
import pytest

from oracle import plain

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2604_19890_gb300 as ssg
    g = ssg.Context(logN=6, L=26, alpha=2, bits=36, p=17, r=2, h=16, nmax=0, seed=31)
    g.keygen()
    return g


def make_queries(g, seed):
    rng = np.random.default_rng(seed)
    qs = []
    for i, n in enumerate([1, 3, 2, 4, 1, 2]):
        cols = {k: rng.integers(0, g.t, (n, g.slots)) for k in ("a", "b", "c1")}
        c2 = np.full((1, g.slots), int(rng.integers(0, g.t))) if i % 2 == 0 else rng.integers(0, g.t, (n, g.slots))
        enc = lambda v, nonce: g.encrypt(np.stack([g.encode(x) for x in v]), nonce)
        A, B, C1, C2 = (enc(cols["a"], 100 * i + 1), enc(cols["b"], 100 * i + 20), enc(cols["c1"], 100 * i + 40),
                        enc(c2, 100 * i + 60))
        if i == 4:  # a query one level lower: must not merge with the others
            A, B, C1, C2 = (g.modswitch(x, 1) for x in (A, B, C1, C2))
        exp = plain.query(cols["a"], cols["b"], cols["c1"], c2, g.t)
        qs.append(((A, B, C1, C2), exp))
    return qs


def test_served_results_equal_alone(ctx):
    import paper_2604_19890_gb300 as ssg
    g = ctx
    qs = make_queries(g, 1)
    alone = [g.query(*cols).words() for cols, _ in qs]
    srv = ssg.Server(g, workers=2, max_merge=4)
    tickets = [srv.submit(*cols) for cols, _ in qs]
    for t, (cols, exp), ref in zip(tickets, qs, alone):
        res, q_ms, r_ms = srv.wait(t, timeout_ms=120000)
        assert (res.words() == ref).all()
        assert (g.decrypt_slots(res) == exp).all()
        assert q_ms >= 0 and r_ms > 0
    st = srv.stats()
    assert st["completed"] == len(qs) and st["batches"] < len(qs)  # some queries were merged
    srv.close()


def test_served_staggered_arrivals(ctx):
    import paper_2604_19890_gb300 as ssg
    g = ctx
    qs = make_queries(g, 2)
    alone = [g.query(*cols).words() for cols, _ in qs]
    srv = ssg.Server(g, workers=2, max_merge=8)
    tickets = [None] * len(qs)

    def submitter():
        for i, (cols, _) in enumerate(qs):
            tickets[i] = srv.submit(*cols)
            time.sleep(0.005 * (i % 3))

    th = threading.Thread(target=submitter)
    th.start()
    th.join()
    for t, ref in zip(tickets, alone):
        res, _, _ = srv.wait(t, timeout_ms=120000)
        assert (res.words() == ref).all()
    srv.close()


def test_server_wait_is_bounded(ctx):
    import paper_2604_19890_gb300 as ssg
    g = ctx
    (cols, exp), = make_queries(g, 3)[3:4]
    srv = ssg.Server(g, workers=1, max_merge=1)
    t = srv.submit(*cols)
    try:
        srv.wait(t, timeout_ms=0)
        finished_early = True
    except ssg.SSError as e:
        assert e.code == ssg.SS_ERR_TIMEOUT
        finished_early = False
    if not finished_early:
        res, _, _ = srv.wait(t, timeout_ms=120000)
        assert (g.decrypt_slots(res) == exp).all()
    srv.close()


def test_server_rejects_mismatched_levels(ctx):
    import paper_2604_19890_gb300 as ssg
    g = ctx
    (cols, _), = make_queries(g, 4)[1:2]
    A, B, C1, C2 = cols
    srv = ssg.Server(g, workers=1, max_merge=1)
    with pytest.raises(ssg.SSError) as e:
        srv.submit(g.modswitch(A, 1), B, C1, C2)
    assert e.value.code == ssg.SS_ERR_LEVEL
    srv.close()


def test_planning_while_the_server_runs(ctx):
    """Plan-only evaluation (ss_query_depth, and the plan every query runs
    before launching) is per thread: planning on the caller's thread while the
    server's workers evaluate on the same context changes none of their
    results."""
    import paper_2604_19890_gb300 as ssg
    g = ctx
    qs = make_queries(g, 3)
    alone = [g.query(*cols).words() for cols, _ in qs]
    depth = g.query_depth()
    srv = ssg.Server(g, workers=2, max_merge=2)
    tickets = [srv.submit(*cols) for cols, _ in qs]
    plans = 0
    while srv.stats()["completed"] < len(qs) and plans < 20000:
        assert g.query_depth() == depth
        plans += 1
    for t, ref in zip(tickets, alone):
        res, _, _ = srv.wait(t, timeout_ms=120000)
        assert (res.words() == ref).all()
    assert plans > 0
    srv.close()


def test_served_mixed_contexts_equal_alone():
    """One server over two parameter sets (N = 2^13 with 17^2, N = 2^14 with
    257^2): queries of both ring dimensions arrive interleaved, are admitted by
    one HBM budget, merge only within their context, and each result equals
    the same query run alone, word for word."""
    import paper_2604_19890_gb300 as ssg
    g1 = ssg.Context(logN=13, L=18, alpha=2, bits=36, p=17, r=2, h=120, nmax=0, seed=41)
    g2 = ssg.Context(logN=14, L=30, alpha=2, bits=55, p=257, r=2, h=120, nmax=0, seed=42)
    for g in (g1, g2):
        g.keygen()
    rng = np.random.default_rng(4)
    qs = []
    for i, n in enumerate([1, 2, 1, 2, 2, 1, 1, 2]):
        ci = i % 2
        g = (g1, g2)[ci]
        cols = {k: rng.integers(0, g.t, (n, g.slots)) for k in ("a", "b", "c1")}
        c2 = np.full((1, g.slots), int(rng.integers(0, g.t)))
        enc = lambda v, nonce: g.encrypt(np.stack([g.encode(x) for x in v]), nonce)
        A, B, C1, C2 = (enc(cols["a"], 100 * i + 1), enc(cols["b"], 100 * i + 20), enc(cols["c1"], 100 * i + 40),
                        enc(c2, 100 * i + 60))
        qs.append((ci, (A, B, C1, C2), plain.query(cols["a"], cols["b"], cols["c1"], c2, g.t)))
    alone = [(g1, g2)[ci].query(*cols).words() for ci, cols, _ in qs]
    srv = ssg.Server([g1, g2], workers=3, max_merge=4)
    tickets = [srv.submit(*cols, ctx_index=ci) for ci, cols, _ in qs]
    for t, (ci, cols, exp), ref in zip(tickets, qs, alone):
        res, _, _ = srv.wait(t, timeout_ms=120000)
        assert (res.words() == ref).all()
        assert ((g1, g2)[ci].decrypt_slots(res) == exp).all()
    assert srv.stats()["completed"] == len(qs)
    srv.close()


def test_submit_rejects_a_chain_too_short():
    """A query whose schedule needs more levels than its columns have is refused
    at submission with SS_ERR_NOISE (the plan runs before it is queued)."""
    import paper_2604_19890_gb300 as ssg
    g = ssg.Context(logN=6, L=9, alpha=2, bits=36, p=17, r=2, h=16, nmax=0, seed=33)
    g.keygen()
    rng = np.random.default_rng(5)
    cols = [g.encrypt_slots(rng.integers(0, g.t, (1, g.slots)), 10 * (i + 1)) for i in range(4)]
    srv = ssg.Server(g, workers=1, max_merge=1)
    with pytest.raises(ssg.SSError) as e:
        srv.submit(*cols)
    assert e.value.code == ssg.SS_ERR_NOISE
    assert srv.stats()["completed"] == 0
    srv.close()
