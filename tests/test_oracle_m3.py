"""Pins for the CPU reference on the non-power-of-two cyclotomic ring m = 3N
(Phi_3N(X) = X^N - X^(N/2) + 1, N = 2^k; Section 2.1 with a general m, the
slot count l = n / Ord(m, p) of Section 5.1). Each check is against something
other than the reference itself: direct evaluation at the roots, schoolbook
products reduced by X^N = X^(N/2) - 1, a(X^g) reduced term by term, sympy's
multiplicative orders and primitive roots, Galois-ring arithmetic written out
here, brute-force group covers and plaintext semantics.
"""
import math

import numpy as np
import pytest
import sympy

import oracle as O
from oracle import plain


def ctx(logN=5, p=17, r=2, L=3, alpha=2, bits=36, h=None, seed=11):
    N = 1 << logN
    return O.Oracle(logN=logN, L=L, alpha=alpha, bits=bits, p=p, r=r, h=h or min(8, N // 2), seed=seed, m_odd=3)


def bitrev(x, n):
    return int(format(x, "0%db" % n)[::-1], 2) if n else 0


def reduce_phi3(c, N, mod):
    """c (any length) reduced modulo X^N - X^(N/2) + 1, from the top degree down."""
    c = list(c) + [0] * max(0, N - len(c))
    for e in range(len(c) - 1, N - 1, -1):
        v, c[e] = c[e], 0
        c[e - N // 2] += v
        c[e - N] -= v
    return [x % mod for x in c[:N]]


def ring_mul(a, b, N, mod):
    out = [0] * (2 * N - 1)
    for i, x in enumerate(a):
        if x:
            for j, y in enumerate(b):
                out[i + j] += x * y
    return reduce_phi3(out, N, mod)


def substitute(a, g, N, mod):
    """a(X^g) mod Phi_3N."""
    out = [0] * (g * (N - 1) + 1)
    for i, x in enumerate(a):
        out[g * i] += x
    return reduce_phi3(out, N, mod)


def units(m):
    return [e for e in range(1, m) if math.gcd(e, m) == 1]


# ---------------------------------------------------------------- primes and roots
def test_primes_are_the_largest_admissible_for_3n():
    o = ctx(logN=5, L=5, alpha=2)
    q = [int(x) for x in o.primes()]
    M = 3 * o.N * o.t
    k = ((1 << 36) - 2) // M
    expect = []
    while len(expect) < len(q):
        c = k * M + 1
        if sympy.isprime(c):
            expect.append(c)
        k -= 1
    assert q == expect and all((1 << 35) < x < (1 << 36) for x in q)


@pytest.mark.parametrize("logN", [3, 4, 6])
def test_root_is_the_smallest_primitive_3n_th_root(logN):
    o = ctx(logN=logN, L=2, alpha=1)
    m = 3 * o.N
    for q, w in zip(o.primes(), o.psi()):
        q, w = int(q), int(w)
        c = pow(sympy.primitive_root(q), (q - 1) // m, q)
        assert min(pow(c, j, q) for j in units(m)) == w
        assert sympy.n_order(w, q) == m


# ---------------------------------------------------------------- transform
@pytest.mark.parametrize("logN", [3, 5, 6])
def test_ntt_3n_is_evaluation_at_the_roots(logN):
    o = ctx(logN=logN, L=2, alpha=1)
    N, n = o.N, o.N // 2
    exps = [(1 if i < n else 5) + 6 * bitrev(i % n, logN - 1) for i in range(N)]
    assert sorted(exps) == units(3 * N)  # every primitive 3N-th root once
    rng = np.random.default_rng(logN)
    for pi, (q, w) in enumerate(zip(o.primes(), o.psi())):
        q, w = int(q), int(w)
        a = [int(x) for x in rng.integers(0, q, N, dtype=np.uint64)]
        A = o.ntt_fwd(pi, np.array(a, dtype=np.uint64))
        for i, e in enumerate(exps):
            z = pow(w, e, q)
            assert (pow(z, N, q) - pow(z, n, q) + 1) % q == 0  # a root of Phi_3N
            assert int(A[i]) == sum(c * pow(z, k, q) for k, c in enumerate(a)) % q
        assert [int(x) for x in o.ntt_inv(pi, A)] == a


def test_ntt_3n_convolution_theorem():
    o = ctx(logN=5, L=2, alpha=1)
    rng = np.random.default_rng(3)
    q, N = int(o.primes()[0]), o.N
    a = [int(x) for x in rng.integers(0, q, N, dtype=np.uint64)]
    b = [int(x) for x in rng.integers(0, q, N, dtype=np.uint64)]
    A, B = o.ntt_fwd(0, np.array(a, np.uint64)), o.ntt_fwd(0, np.array(b, np.uint64))
    prod = np.array([(int(x) * int(y)) % q for x, y in zip(A, B)], dtype=np.uint64)
    assert [int(x) for x in o.ntt_inv(0, prod)] == ring_mul(a, b, N, q)


def test_automorphism_3n_definition():
    o = ctx(logN=4, L=2, alpha=1)
    q, N, m = int(o.primes()[0]), o.N, 3 * o.N
    rng = np.random.default_rng(5)
    a = [int(x) for x in rng.integers(0, q, N, dtype=np.uint64)]
    for g in [5, 7, 11, m - 1, 25]:
        got = [int(x) for x in o.automorph_coeff(0, g, np.array(a, np.uint64))]
        assert got == substitute(a, g, N, q)


# ---------------------------------------------------------------- slots
class GR2:
    """Z_t[u] / (u^2 - c), written out for the pins."""

    def __init__(self, c, t):
        self.c, self.t = c, t

    def mul(self, x, y):
        c, t = self.c, self.t
        return ((x[0] * y[0] + c * x[1] * y[1]) % t, (x[0] * y[1] + x[1] * y[0]) % t)

    def pow(self, x, e):
        r = (1, 0)
        while e:
            if e & 1:
                r = self.mul(r, x)
            x = self.mul(x, x)
            e >>= 1
        return r


# (p, r, logN): both slot shapes -- p = 2 mod 3 (pairs of conjugate roots per
# slot) and p = 1 mod 12 (one root per slot) -- s = 1 as well as s > 1, and
# p = 3 mod 4 (7, 11, 131), which X^N + 1 cannot split into binomial slots
SLOT_CASES = [(17, 2, 5), (257, 2, 6), (13, 2, 6), (5, 3, 7), (41, 2, 6), (37, 2, 5), (7, 3, 6), (11, 2, 5),
              (131, 2, 6)]


@pytest.mark.parametrize("p,r,logN", SLOT_CASES)
def test_slot_algebra_3n(p, r, logN):
    o = ctx(logN=logN, p=p, r=r, L=2, alpha=1)
    N, t = o.N, o.t
    assert o.m == 3 * N
    assert o.slots == N // sympy.n_order(p, 3 * N) and o.slots * o.d == N
    b = sympy.multiplicity(2, p * p - 1)
    assert o.Mp == 3 * 2 ** min(b, logN) and o.s * o.Mp == 3 * N and o.nprime * o.s == N
    assert sympy.legendre_symbol(o.gr_c, p) == -1
    G = GR2(o.gr_c, t)
    th = o.theta
    assert G.pow(th, o.Mp) == (1, 0) and G.pow(th, o.Mp // 2) != (1, 0) and G.pow(th, o.Mp // 3) != (1, 0)
    # the slots partition (Z/M')^* into orbits under multiplication by p
    orbit = lambda e: {e * pow(p, i, o.Mp) % o.Mp for i in range(o.Mp)}
    cover = [orbit(int(e)) for e in o.slot_exp]
    assert sum(len(c) for c in cover) == len(units(o.Mp)) and set().union(*cover) == set(units(o.Mp))

    rng = np.random.default_rng(p + r + logN)
    u = rng.integers(0, t, o.slots, dtype=np.uint64)
    v = rng.integers(0, t, o.slots, dtype=np.uint64)
    mu, mv = [int(x) for x in o.encode(u)], [int(x) for x in o.encode(v)]
    assert all(x == 0 for i, x in enumerate(mu) if i % o.s)  # a polynomial in X^s
    assert (o.decode(np.array(mu, np.uint64)) == u).all()
    # slotwise sum and product = ring sum and product mod t
    add = [(x + y) % t for x, y in zip(mu, mv)]
    assert [int(x) for x in o.decode(np.array(add, np.uint64))] == [(int(x) + int(y)) % t for x, y in zip(u, v)]
    prod = ring_mul(mu, mv, N, t)
    assert [int(x) for x in o.decode(np.array(prod, np.uint64))] == [int(x) * int(y) % t for x, y in zip(u, v)]
    # each slot value is A(theta^e) for every root e of the slot (constant on the orbit)
    A = mu[:: o.s]
    for j, e0 in enumerate(o.slot_exp):
        for e in orbit(int(e0)):
            z, acc = G.pow(th, e), (0, 0)
            for c in reversed(A):
                acc = G.mul(acc, z)
                acc = ((acc[0] + c) % t, acc[1])
            assert acc == (int(u[j]), 0)


@pytest.mark.parametrize("p,r,logN", [(17, 2, 5), (257, 2, 6), (13, 2, 6)])
def test_galois_elements_permute_slots_3n(p, r, logN):
    o = ctx(logN=logN, p=p, r=r, L=2, alpha=1)
    N, t, Mp = o.N, o.t, o.Mp
    slot_of = {}
    for j, e0 in enumerate(o.slot_exp):
        for i in range(Mp):
            slot_of[int(e0) * pow(p, i, Mp) % Mp] = j
    u = (np.arange(o.slots, dtype=np.uint64) + 3) % t
    m = [int(x) for x in o.encode(u)]
    for g in [5, 7, 3 * N - 1] + o.rotate_sum_elements():
        got = o.decode(np.array(substitute(m, g, N, t), np.uint64))
        # sigma_g(A(X^s)) = A(X^(s g)): slot of e now holds the value at g e
        assert [int(x) for x in got] == [int(u[slot_of[g * int(e) % Mp]]) for e in o.slot_exp]


@pytest.mark.parametrize("p,logN", [(17, 5), (257, 6), (13, 6), (5, 7), (257, 9)])
def test_rotate_sum_elements_cover_the_slot_group(p, logN):
    o = ctx(logN=logN, p=p, r=2, L=2, alpha=1)
    m = 3 * o.N
    H = {pow(p, i, m) for i in range(m)}  # the decomposition group <p> in (Z/3N)^*
    classes = {}
    for e in units(m):
        classes.setdefault(min(e * h % m for h in H), []).append(e)
    assert len(classes) == o.slots
    # x <- x + sigma_g(x) over the list sums sigma over all subset products
    prods = [1]
    for g in o.rotate_sum_elements():
        assert math.gcd(g, m) == 1
        prods = prods + [x * g % m for x in prods]
    reps = {min(x * h % m for h in H) for x in prods}
    assert len(prods) == o.slots and len(reps) == o.slots


# ---------------------------------------------------------------- BGV on the ring
@pytest.mark.parametrize("logN,p,r,L,bits", [(6, 17, 2, 18, 36), (5, 257, 2, 30, 55)])
def test_query_and_rotate_sum_3n(logN, p, r, L, bits):
    o = ctx(logN=logN, p=p, r=r, L=L, alpha=2, bits=bits)
    o.keygen(o.rotate_sum_elements())
    t = o.t
    rng = np.random.default_rng(logN + p)
    a, b, c1, c2 = (rng.integers(0, t, o.slots) for _ in range(4))
    enc = lambda v, n: o.encrypt(o.encode(v), n)
    ca, cb = enc(a, 1), enc(b, 2)
    assert (o.decrypt_slots(o.mul(ca, cb)) == (a.astype(object) * b) % t).all()
    assert (o.decrypt_slots(o.rotate_sum(ca)) == int(a.astype(object).sum() % t)).all()
    res = o.query([enc(a, 10)], [enc(b, 20)], [enc(c1, 30)], [enc(c2, 40)])
    assert (o.decrypt_slots(res) == plain.query([a], [b], [c1], [c2], t)).all()
    assert o.noise_budget(res) > 5


@pytest.mark.parametrize("p,r,L", [(7, 3, 30), (11, 4, 44), (67, 2, 30), (131, 3, 60)])
def test_lt_and_raise_p3mod4_3n(p, r, L):
    """The paper's (p, r) pairs with p = 3 mod 4 (Section 5, LT table) on m = 3N:
    Algorithm 4 then raising, decrypted against the plaintext definition."""
    o = ctx(logN=6, p=p, r=r, L=L, alpha=3, bits=58 if p == 131 else 55)
    o.keygen([])
    t = o.t
    rng = np.random.default_rng(p)
    A, B = rng.integers(0, t, o.slots), rng.integers(0, t, o.slots)
    lt = o.raise_modulus(o.compare_lt(o.encrypt(o.encode(A), 1), o.encrypt(o.encode(B), 2)))
    assert (o.decrypt_slots(lt) == np.array([plain.lt(x, y, t) for x, y in zip(A, B)])).all()
