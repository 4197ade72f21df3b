"""Plaintext definitions of the query results (test infrastructure only).

LT over Z_{p^r} follows Algorithm 4: the comparison is on the centred
difference, [centred(c1 - c2 mod p^r) < 0] (balanced digits, Lemma 3).
"""
import numpy as np


def centred(x, m):
    x %= m
    return x - m if x > m // 2 else x


def lt(c1, c2, t):
    return 1 if centred(int(c1) - int(c2), t) < 0 else 0


def query(A, B, C1, C2, t):
    """sum over rows of a*b*[C1 < C2] mod t (Section 1, Fig. 1 shape)."""
    A, B, C1 = (np.asarray(x) for x in (A, B, C1))
    C2b = np.broadcast_to(np.asarray(C2), C1.shape)
    total = 0
    for a, b, c1, c2 in zip(A.ravel(), B.ravel(), C1.ravel(), C2b.ravel()):
        total += int(a) * int(b) * lt(c1, c2, t)
    return total % t


def balanced_digits(v, p, r):
    out = []
    for _ in range(r):
        z = v % p
        z = z - p if z > p // 2 else z
        out.append(z)
        v = (v - z) // p
    return out
