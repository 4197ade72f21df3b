"""Pins for the CPU reference on the cyclotomic ring m = 5N/2 (Phi_m(X) =
Phi_10(X^(N/4)) = X^N - X^(3N/4) + X^(N/2) - X^(N/4) + 1, N = 2^k; Section 2.1
with a general m, the slot count l = n / Ord(m, p) of Section 5.1). Each check
is against something other than the reference itself: direct evaluation at
the roots, schoolbook products reduced by X^N = X^(3N/4) - X^(N/2) + X^(N/4) - 1,
a(X^g) reduced term by term, sympy's orders and primitive roots, Galois-ring
arithmetic written out here, brute-force group covers and plaintext semantics.
"""
import math

import numpy as np
import pytest
import sympy

import oracle as O
from oracle import plain

E5 = (1, 3, 7, 9)


def ctx(logN=5, p=17, r=2, L=3, alpha=2, bits=36, h=None, seed=11):
    N = 1 << logN
    return O.Oracle(logN=logN, L=L, alpha=alpha, bits=bits, p=p, r=r, h=h or min(8, N // 2), seed=seed, m_odd=5)


def bitrev(x, n):
    return int(format(x, "0%db" % n)[::-1], 2) if n else 0


def reduce_phi(c, N, mod):
    """c (any length) reduced modulo Phi_(5N/2), from the top degree down."""
    c = list(c) + [0] * max(0, N - len(c))
    for e in range(len(c) - 1, N - 1, -1):
        v, c[e] = c[e], 0
        c[e - N // 4] += v
        c[e - N // 2] -= v
        c[e - 3 * N // 4] += v
        c[e - N] -= v
    return [x % mod for x in c[:N]]


def ring_mul(a, b, N, mod):
    out = [0] * (2 * N - 1)
    for i, x in enumerate(a):
        if x:
            for j, y in enumerate(b):
                out[i + j] += x * y
    return reduce_phi(out, N, mod)


def substitute(a, g, N, mod):
    out = [0] * (g * (N - 1) + 1)
    for i, x in enumerate(a):
        out[g * i] += x
    return reduce_phi(out, N, mod)


def units(m):
    return [e for e in range(1, m) if math.gcd(e, m) == 1]


def test_cyclotomic_polynomial_is_phi_m():
    for logN in (3, 4, 6):
        N = 1 << logN
        x = sympy.symbols("x")
        phi = sympy.Poly(sympy.cyclotomic_poly(5 * N // 2, x), x).all_coeffs()[::-1]
        assert reduce_phi([0] * N + [1], N, 10 ** 9) == [(-c) % 10 ** 9 for c in phi[:N]]


def test_primes_are_the_largest_admissible_for_5n2():
    o = ctx(logN=5, L=5, alpha=2)
    q = [int(x) for x in o.primes()]
    M = 5 * o.N // 2 * o.t
    k = ((1 << 36) - 2) // M
    expect = []
    while len(expect) < len(q):
        c = k * M + 1
        if sympy.isprime(c):
            expect.append(c)
        k -= 1
    assert q == expect


@pytest.mark.parametrize("logN", [3, 4, 6])
def test_root_is_the_smallest_primitive_m_th_root(logN):
    o = ctx(logN=logN, L=2, alpha=1)
    m = 5 * o.N // 2
    for q, w in zip(o.primes(), o.psi()):
        q, w = int(q), int(w)
        c = pow(sympy.primitive_root(q), (q - 1) // m, q)
        assert min(pow(c, j, q) for j in units(m)) == w
        assert sympy.n_order(w, q) == m


@pytest.mark.parametrize("logN", [3, 5, 6])
def test_ntt_5n2_is_evaluation_at_the_roots(logN):
    o = ctx(logN=logN, L=2, alpha=1)
    N, n, m = o.N, o.N // 4, 5 * o.N // 2
    exps = [E5[i // n] + 10 * bitrev(i % n, logN - 2) for i in range(N)]
    assert sorted(exps) == units(m)
    rng = np.random.default_rng(logN)
    for pi, (q, w) in enumerate(zip(o.primes(), o.psi())):
        q, w = int(q), int(w)
        a = [int(x) for x in rng.integers(0, q, N, dtype=np.uint64)]
        A = o.ntt_fwd(pi, np.array(a, dtype=np.uint64))
        for i, e in enumerate(exps):
            z = pow(w, e, q)
            assert sum(c * pow(z, k, q) for k, c in enumerate(reduce_phi([0] * N + [1], N, q))) % q == pow(z, N, q)
            assert int(A[i]) == sum(c * pow(z, k, q) for k, c in enumerate(a)) % q
        assert [int(x) for x in o.ntt_inv(pi, A)] == a


def test_ntt_5n2_convolution_theorem():
    o = ctx(logN=5, L=2, alpha=1)
    rng = np.random.default_rng(3)
    q, N = int(o.primes()[0]), o.N
    a = [int(x) for x in rng.integers(0, q, N, dtype=np.uint64)]
    b = [int(x) for x in rng.integers(0, q, N, dtype=np.uint64)]
    A, B = o.ntt_fwd(0, np.array(a, np.uint64)), o.ntt_fwd(0, np.array(b, np.uint64))
    prod = np.array([(int(x) * int(y)) % q for x, y in zip(A, B)], dtype=np.uint64)
    assert [int(x) for x in o.ntt_inv(0, prod)] == ring_mul(a, b, N, q)


def test_automorphism_5n2_definition():
    o = ctx(logN=4, L=2, alpha=1)
    q, N, m = int(o.primes()[0]), o.N, 5 * o.N // 2
    rng = np.random.default_rng(5)
    a = [int(x) for x in rng.integers(0, q, N, dtype=np.uint64)]
    for g in [3, 7, 11, 13, m - 1]:
        got = [int(x) for x in o.automorph_coeff(0, g, np.array(a, np.uint64))]
        assert got == substitute(a, g, N, q)


class GR4:
    """GR(t, 2)[v] / (v^2 - w) over Z_t[u] / (u^2 - c), written out for the pins."""

    def __init__(self, c, w, t):
        self.c, self.w, self.t = c, w, t

    def m2(self, x, y):
        c, t = self.c, self.t
        return ((x[0] * y[0] + c * x[1] * y[1]) % t, (x[0] * y[1] + x[1] * y[0]) % t)

    def mul(self, x, y):
        a, b, cc, d = x[:2], x[2:], y[:2], y[2:]
        ac, bd, ad, bc = self.m2(a, cc), self.m2(b, d), self.m2(a, d), self.m2(b, cc)
        bdw = self.m2(bd, self.w)
        t = self.t
        return ((ac[0] + bdw[0]) % t, (ac[1] + bdw[1]) % t, (ad[0] + bc[0]) % t, (ad[1] + bc[1]) % t)

    def pow(self, x, e):
        r = (1, 0, 0, 0)
        while e:
            if e & 1:
                r = self.mul(r, x)
            x = self.mul(x, x)
            e >>= 1
        return r


SLOT_CASES = [(17, 2, 5), (257, 2, 6), (13, 2, 6), (11, 2, 6), (41, 3, 7), (7, 2, 5), (257, 3, 7)]


@pytest.mark.parametrize("p,r,logN", SLOT_CASES)
def test_slot_algebra_5n2(p, r, logN):
    o = ctx(logN=logN, p=p, r=r, L=2, alpha=1, bits=55 if p == 257 else 36)
    N, t, m = o.N, o.t, 5 * o.N // 2
    assert o.m == m and o.slots == N // sympy.n_order(p, m) and o.slots * o.d == N
    b = sympy.multiplicity(2, p ** 4 - 1)
    assert o.Mp == 5 * 2 ** min(b, logN - 1) and o.s * o.Mp == m and o.nprime * o.s == N
    assert sympy.legendre_symbol(o.gr_c, p) == -1
    G = GR4(o.gr_c, o.gr_w, t)
    G1 = GR4(o.gr_c, o.gr_w, p)
    assert G1.pow((o.gr_w[0], o.gr_w[1], 0, 0), (p * p - 1) // 2) != (1, 0, 0, 0)  # w is not a square in F_{p^2}
    th = o.theta
    assert G.pow(th, o.Mp) == (1, 0, 0, 0)
    assert G.pow(th, o.Mp // 2) != (1, 0, 0, 0) and G.pow(th, o.Mp // 5) != (1, 0, 0, 0)
    orbit = lambda e: {e * pow(p, i, o.Mp) % o.Mp for i in range(o.Mp)}
    cover = [orbit(int(e)) for e in o.slot_exp]
    assert sum(len(c) for c in cover) == len(units(o.Mp)) and set().union(*cover) == set(units(o.Mp))
    rng = np.random.default_rng(p + r + logN)
    u = rng.integers(0, t, o.slots, dtype=np.uint64)
    v = rng.integers(0, t, o.slots, dtype=np.uint64)
    mu, mv = [int(x) for x in o.encode(u)], [int(x) for x in o.encode(v)]
    assert all(x == 0 for i, x in enumerate(mu) if i % o.s)
    assert (o.decode(np.array(mu, np.uint64)) == u).all()
    prod = ring_mul(mu, mv, N, t)
    assert [int(x) for x in o.decode(np.array(prod, np.uint64))] == [int(x) * int(y) % t for x, y in zip(u, v)]
    A = mu[:: o.s]
    for j, e0 in enumerate(o.slot_exp[:4]):
        for e in orbit(int(e0)):
            z, acc = G.pow(th, e), (0, 0, 0, 0)
            for c in reversed(A):
                acc = G.mul(acc, z)
                acc = ((acc[0] + c) % t,) + acc[1:]
            assert acc == (int(u[j]), 0, 0, 0)


@pytest.mark.parametrize("p,logN", [(17, 5), (257, 6), (13, 6), (41, 7)])
def test_galois_elements_permute_slots_and_cover_5n2(p, logN):
    o = ctx(logN=logN, p=p, r=2, L=2, alpha=1)
    N, t, Mp, m = o.N, o.t, o.Mp, 5 * o.N // 2
    slot_of = {}
    for j, e0 in enumerate(o.slot_exp):
        for i in range(Mp):
            slot_of[int(e0) * pow(p, i, Mp) % Mp] = j
    u = (np.arange(o.slots, dtype=np.uint64) + 3) % t
    mm = [int(x) for x in o.encode(u)]
    for g in [3, 7, m - 1] + o.rotate_sum_elements():
        got = o.decode(np.array(substitute(mm, g, N, t), np.uint64))
        assert [int(x) for x in got] == [int(u[slot_of[g * int(e) % Mp]]) for e in o.slot_exp]
    H = {pow(p, i, m) for i in range(m)}
    prods = [1]
    for g in o.rotate_sum_elements():
        prods = prods + [x * g % m for x in prods]
    assert len(prods) == o.slots and len({min(x * h % m for h in H) for x in prods}) == o.slots


@pytest.mark.parametrize("logN,p,r,L,bits", [(6, 17, 2, 18, 36), (5, 257, 2, 30, 55)])
def test_query_and_rotate_sum_5n2(logN, p, r, L, bits):
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
