"""Full-size parity cases: parameter sets, seeded inputs and the operations whose
ciphertext words are compared between the CUDA path and the CPU reference.

Pure data plus the seeded input recipe (no method arithmetic, no import of the
reference or of the library). `make_fullsize_digests.py` runs these cases on
the CPU reference and stores a SHA-256 digest of every result's words;
`tests/test_gpu_fullsize.py` runs them on the GPU and compares digests.

Digest of a ciphertext: SHA-256 of its words as little-endian uint64 in the
order [component][limb][coefficient] (evaluation form), limbs 0..level-1.
"""
import hashlib

import numpy as np

from paper_2604_19890_gb300 import synth

# The named parameter sets (N = 2^13 / 17^2, N = 2^15 / 257^2, N = 2^16 /
# 257^3 on X^N + 1 and on m = 3N), chain lengths as the query needs them,
# seed 0x5EED0000 + id.
PRESETS = {
    0: dict(logN=13, L=18, alpha=2, bits=36, p=17, r=2, h=120, seed=0x5EED0000),
    1: dict(logN=15, L=30, alpha=2, bits=55, p=257, r=2, h=120, seed=0x5EED0001),
    2: dict(logN=16, L=41, alpha=3, bits=55, p=257, r=3, h=120, seed=0x5EED0002),
    # the same on the cyclotomic ring m = 3N (X^N - X^(N/2) + 1): 256 slots
    3: dict(logN=16, L=41, alpha=3, bits=55, p=257, r=3, h=120, seed=0x5EED0003, m_odd=3),
    # and on m = 5N/2 (X^N - X^(3N/4) + X^(N/2) - X^(N/4) + 1): 512 slots
    4: dict(logN=16, L=41, alpha=3, bits=55, p=257, r=3, h=120, seed=0x5EED0004, m_odd=5),
}

# Nonces of the encrypted inputs: column k uses nonce base + row index.
NONCE = {"a": 1000, "b": 2000, "c1": 3000, "c2": 4000}

CASES = {
    # Single operations at the largest parameter set (level 41, three special
    # primes): every key-switching mode the query uses at full size.
    "ops_n65536_257cubed": dict(kind="ops", params=PRESETS[2], value_seed=0x5EED2002),
    # SUM(a*a) WHERE c < 150 (threshold encrypted, replicated), 2 ciphertexts per column.
    "query_n8192_17sq": dict(kind="query", params=PRESETS[0], value_seed=0x5EED3000, n_ct=2,
                             threshold=150, square=True),
    # SUM(a*b) WHERE c < t, t uniform and encrypted, 1 ciphertext per column.
    "query_n32768_257sq": dict(kind="query", params=PRESETS[1], value_seed=0x5EED3001, n_ct=1,
                               threshold="random", square=False),
    # SUM(a*b) WHERE c1 < c2 (column against column), 1 ciphertext per column.
    "query_n65536_257cubed": dict(kind="query", params=PRESETS[2], value_seed=0x5EED3002, n_ct=1,
                                  threshold=None, square=False),
    # the same query on m = 3N, 256 slots
    "query_n65536_257cubed_m3n": dict(kind="query", params=PRESETS[3], value_seed=0x5EED3003, n_ct=1,
                                      threshold=None, square=False),
    # on m = 5N/2, 512 slots
    "query_n65536_257cubed_m5n2": dict(kind="query", params=PRESETS[4], value_seed=0x5EED3004, n_ct=1,
                                       threshold=None, square=False),
}

# Results of the "ops" case, in the order they are computed:
#   enc_a, enc_b         fresh encryptions (nonces 1 and 2)
#   tensor               a (x) b, three components
#   relin                relinearisation of the tensor (hybrid key switch, ModDown by P)
#   mul                  the evaluator's multiplication: tensor, relinearise and drop one prime
#   modswitch_1/3        a with its last 1 / 3 primes dropped
#   rotate_5, rotate_m1  a under X -> X^5 and X -> X^(2N-1), key-switched back
#   rotate_sum           total over all slots of `mul`
#   digit_0..r-1         Algorithm 3 on a
OPS_RESULTS = ["enc_a", "enc_b", "tensor", "relin", "mul", "modswitch_1", "modswitch_3", "rotate_5",
               "rotate_m1", "rotate_sum", "digit_0", "digit_1", "digit_2"]


def ops_inputs(case, slots, t):
    v = synth.table(case["value_seed"], 1, slots, t, columns=("a", "b"))
    return v["a"][0], v["b"][0]


def query_inputs(case, slots, t):
    """Column values {a, b, c1, c2} ([n_ct][slots]); c2 has one row for a threshold."""
    n = case["n_ct"]
    cols = synth.table(case["value_seed"], n, slots, t)
    thr = case["threshold"]
    if thr is not None:
        cols["c2"] = synth.threshold(case["value_seed"], slots, t, None if thr == "random" else thr)
    if case["square"]:
        cols["b"] = cols["a"]
    return cols


def digest(words):
    """SHA-256 of uint64 words [ncomp][level][N], little-endian."""
    w = np.ascontiguousarray(words, dtype="<u8")
    return hashlib.sha256(w.tobytes()).hexdigest()
