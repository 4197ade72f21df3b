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


def predicate(pred, x, y, t):
    """Section 4.3 predicates on the centred difference d = centred(x - y mod t):
    lt d < 0, le d <= 0, gt d > 0, ge d >= 0, eq d = 0, neq d != 0."""
    d = centred(int(x) - int(y), t)
    return int({"lt": d < 0, "le": d <= 0, "gt": d > 0, "ge": d >= 0, "eq": d == 0, "neq": d != 0}[pred])


def query_where(A, B, conds, t):
    """sum over rows of a*b*prod_k [X_k pred_k Y_k] mod t (conjunctive WHERE)."""
    A, B = np.asarray(A), np.asarray(B)
    total = 0
    for idx in np.ndindex(A.shape):
        keep = 1
        for pred, X, Y in conds:
            Yb = np.broadcast_to(np.asarray(Y), A.shape)
            keep *= predicate(pred, np.asarray(X)[idx], Yb[idx], t)
        total += int(A[idx]) * int(B[idx]) * keep
    return total % t


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
