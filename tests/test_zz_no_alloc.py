"""GPU test of ss_relin_noalloc, the relinearisation for callers that cannot
allocate device memory while they run (its scratch is a static device array).

Its output must equal ss_relin's word for word (the tolerance of every parity
test here: exact), on two calls in a row, so that contents the first call
leaves in the shared array cannot leak into the second. This file is collected
last so that a run stopping at the first failure has already run every other
test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _ctx(**kw):
    import paper_2604_19890_gb300 as ssg
    g = ssg.Context(nmax=0, **kw)
    g.keygen([])
    return g


def _fresh(g, count, nonce, seed):
    rng = np.random.default_rng(seed)
    a = g.encrypt(np.stack([g.encode(rng.integers(0, g.t, g.slots)) for _ in range(count)]), nonce)
    b = g.encrypt(np.stack([g.encode(rng.integers(0, g.t, g.slots)) for _ in range(count)]), nonce + 100)
    return g.mul(a, b), a, b


@pytest.mark.parametrize("prm,count", [
    (dict(logN=6, L=26, alpha=2, bits=36, p=17, r=2, h=16, seed=7), 3),
    (dict(logN=13, L=18, alpha=2, bits=36, p=17, r=2, h=120, seed=11), 1),
])
def test_relin_noalloc_matches_relin_twice(prm, count):
    g = _ctx(**prm)
    for call in range(2):
        t3, a, b = _fresh(g, count, 10 + 1000 * call, call)
        ref = g.relin(t3)
        got = g.relin_noalloc(t3)
        assert (got.ncomp, got.level, got.t_exp) == (ref.ncomp, ref.level, ref.t_exp)
        assert (got.words() == ref.words()).all()
        # the relinearised product still decrypts to the slotwise product
        pa, pb = g.decrypt_slots(a), g.decrypt_slots(b)
        assert (g.decrypt_slots(got) == (pa.astype(object) * pb.astype(object)) % g.t).all()


def test_relin_noalloc_rejects_oversized_calls():
    import paper_2604_19890_gb300 as ssg
    g = _ctx(logN=13, L=18, alpha=2, bits=36, p=17, r=2, h=120, seed=11)
    t3, _, _ = _fresh(g, 4, 5000, 9)  # needs more than the 64 MiB array
    with pytest.raises(ssg.SSError) as e:
        g.relin_noalloc(t3)
    assert e.value.code == ssg.SS_ERR_PARAM and "static" in str(e.value)
