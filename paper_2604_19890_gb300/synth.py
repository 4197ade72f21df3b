"""Seeded synthetic inputs (plaintext slot values only).

This module holds none of the method's arithmetic: it draws the column values
of the synthetic encrypted tables from numpy's PCG64 with a fixed seed, so
that the library and the CPU reference receive identical plaintexts. The
encryption randomness itself comes from the Philox streams inside each side.
"""
import numpy as np


def table(seed, n_ct, slots, t, columns=("a", "b", "c1", "c2"), half_range=False):
    """Uniform column values in [0, t) (or [0, (t+1)/2) for the half-range
    variant), shaped [n_ct][slots] per column."""
    rng = np.random.default_rng(seed)
    hi = (t + 1) // 2 if half_range else t
    return {c: rng.integers(0, hi, size=(n_ct, slots), dtype=np.int64).astype(np.uint64) for c in columns}


def threshold(seed, slots, t, value=None):
    """A threshold replicated in every slot (drawn uniformly unless given)."""
    rng = np.random.default_rng(seed + 7919)
    v = int(rng.integers(0, t)) if value is None else int(value)
    return np.full((1, slots), v, dtype=np.uint64)

