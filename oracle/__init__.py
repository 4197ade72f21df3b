"""ctypes wrapper around the plain CPU reference (liboracle.so).

TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the benchmark's
CPU-baseline leg. The product package never imports this module.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


# Section 4.3 predicates, in the order the C interfaces number them.
PREDICATES = ["lt", "le", "gt", "ge", "eq", "neq"]


def _pred(p):
    return PREDICATES.index(p) if isinstance(p, str) else int(p)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        vp, i32, u32, u64, i64, dbl = C.c_void_p, C.c_int, C.c_uint32, C.c_uint64, C.c_int64, C.c_double
        P = C.POINTER
        sig = {
            "orc_last_error": (C.c_char_p, []),
            "orc_ctx_new": (vp, [i32, i32, i32, i32, i32, i32, i32, i32, u64, i32]),
            "orc_ctx_ring": (i32, [vp, P(i32), P(u64), P(i32)]),
            "orc_ctx_free": (None, [vp]),
            "orc_ctx_info": (i32, [vp, P(i32), P(i32), P(u64), P(u64), P(i32)]),
            "orc_primes": (i32, [vp, P(u64)]),
            "orc_psi": (i32, [vp, P(u64)]),
            "orc_ntt_fwd": (i32, [vp, i32, P(u64)]),
            "orc_ntt_inv": (i32, [vp, i32, P(u64)]),
            "orc_automorph_coeff": (i32, [vp, i32, i32, P(u64)]),
            "orc_keygen": (i32, [vp, P(i32), i32]),
            "orc_secret": (i32, [vp, P(i64)]),
            "orc_secret_keygen": (i32, [vp]),
            "orc_ksk_export": (i32, [vp, i32, P(u64), P(u64)]),
            "orc_rotate_sum_elements": (i32, [vp, P(i32)]),
            "orc_encode": (i32, [vp, i32, P(u64), P(u64)]),
            "orc_decode": (i32, [vp, i32, P(u64), P(u64)]),
            "orc_g_table": (i32, [i32, i32, P(i64)]),
            "orc_flt_table": (i32, [i32, P(i64)]),
            "orc_g_table_reduced": (i32, [i32, i32, P(i64)]),
            "orc_set_reduced_g": (i32, [vp, i32]),
            "orc_encrypt": (vp, [vp, P(u64), u32, i32]),
            "orc_ct_info": (i32, [vp, P(i32), P(i32), P(i32)]),
            "orc_ct_export": (i32, [vp, P(u64)]),
            "orc_ct_import": (vp, [vp, P(u64), i32, i32, i32]),
            "orc_ct_free": (None, [vp]),
            "orc_decrypt": (i32, [vp, vp, P(u64)]),
            "orc_noise_budget": (dbl, [vp, vp]),
            "orc_add": (vp, [vp, vp, vp]),
            "orc_sub": (vp, [vp, vp, vp]),
            "orc_mul_scalar": (vp, [vp, vp, i64]),
            "orc_add_scalar": (vp, [vp, vp, i64]),
            "orc_tensor": (vp, [vp, vp, vp]),
            "orc_relin": (vp, [vp, vp]),
            "orc_modswitch": (vp, [vp, vp, i32]),
            "orc_rotate": (vp, [vp, vp, i32]),
            "orc_divide_by_p": (vp, [vp, vp]),
            "orc_mul": (vp, [vp, vp, vp]),
            "orc_relin_drop": (vp, [vp, vp]),
            "orc_set_t_exp": (vp, [vp, vp, i32]),
            "orc_eval_g": (vp, [vp, vp, i32]),
            "orc_reduce": (i32, [vp, vp, P(vp)]),
            "orc_compare_lt": (vp, [vp, vp, vp]),
            "orc_compare": (vp, [vp, i32, vp, vp]),
            "orc_query_where": (vp, [vp, P(vp), P(vp), i32, i32, P(i32), P(vp), P(vp), P(i32)]),
            "orc_raise": (vp, [vp, vp]),
            "orc_rotate_sum": (vp, [vp, vp]),
            "orc_query": (vp, [vp, P(vp), P(vp), P(vp), P(vp), i32, i32]),
            "orc_trace": (i32, [vp, i32]),
            "orc_ntt_count": (C.c_ulonglong, [i32]),
            "orc_set_threads": (i32, [i32]),
            "orc_trace_get": (i32, [vp, C.c_char_p, i32]),
            "orc_meter": (i32, [vp, i32]),
            "orc_meter_get": (i32, [vp, C.c_char_p, i32]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class OracleError(RuntimeError):
    pass


def _err():
    return OracleError(lib().orc_last_error().decode())


def _ptr(a, ty=C.c_uint64):
    return a.ctypes.data_as(C.POINTER(ty))


def _chk(rc):
    if rc != 0:
        raise _err()


def set_threads(n=0):
    """Worker threads of the reference's parallel limb loops (0: one per
    hardware thread; results do not depend on it). Returns the count in use."""
    return int(lib().orc_set_threads(int(n)))


def threads():
    return int(lib().orc_set_threads(-1))


def ntt_count(reset=False):
    """Limb transforms (forward + inverse) the reference has run in this process."""
    return int(lib().orc_ntt_count(1 if reset else 0))


def g_table(p, e):
    D = (e - 1) * (p - 1) + 1
    out = np.zeros(D + 1, dtype=np.int64)
    _chk(lib().orc_g_table(p, e, _ptr(out, C.c_int64)))
    return out


def g_table_reduced(p, e):
    """An equivalent G_{p,e} with the least sum of |centred coefficients| (e = 2, 3)."""
    D = (e - 1) * (p - 1) + 1
    out = np.zeros(D + 1, dtype=np.int64)
    _chk(lib().orc_g_table_reduced(p, e, _ptr(out, C.c_int64)))
    return out


def flt_table(p):
    out = np.zeros(p, dtype=np.int64)
    _chk(lib().orc_flt_table(p, _ptr(out, C.c_int64)))
    return out


class Ct:
    """Owning handle to one oracle ciphertext."""

    def __init__(self, ctx, h):
        if not h:
            raise _err()
        self.ctx = ctx
        self.h = h

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_ct_free(self.h)
            self.h = None

    def info(self):
        n, l, t = C.c_int(), C.c_int(), C.c_int()
        _chk(lib().orc_ct_info(self.h, C.byref(n), C.byref(l), C.byref(t)))
        return n.value, l.value, t.value

    @property
    def ncomp(self):
        return self.info()[0]

    @property
    def level(self):
        return self.info()[1]

    @property
    def t_exp(self):
        return self.info()[2]

    def words(self):
        """Ciphertext words as uint64[ncomp][level][N] (evaluation form)."""
        n, l, _ = self.info()
        out = np.zeros((n, l, self.ctx.N), dtype=np.uint64)
        _chk(lib().orc_ct_export(self.h, _ptr(out)))
        return out


class Oracle:
    """One parameter set of the CPU reference BGV."""

    def __init__(self, logN, L, alpha, bits, p, r, h=120, nmax=0, seed=1, m_odd=1):
        self.logN, self.N, self.L, self.alpha, self.bits = logN, 1 << logN, L, alpha, bits
        self.p, self.r, self.h_weight, self.seed = p, r, h, seed
        self.m_odd = m_odd or 1
        self.h = lib().orc_ctx_new(logN, L, alpha, bits, p, r, h, nmax, seed, self.m_odd)
        if not self.h:
            raise _err()
        s, d, t, w = C.c_int(), C.c_int(), C.c_uint64(), C.c_uint64()
        _chk(lib().orc_ctx_info(self.h, C.byref(s), C.byref(d), C.byref(t), C.byref(w), None))
        self.slots, self.d, self.t, self.omega = s.value, d.value, t.value, w.value
        se = np.zeros(self.slots, dtype=np.int32)
        _chk(lib().orc_ctx_info(self.h, C.byref(s), C.byref(d), C.byref(t), C.byref(w), _ptr(se, C.c_int)))
        self.slot_exp = se
        ri, th, gens = np.zeros(6, dtype=np.int32), np.zeros(6, dtype=np.uint64), np.zeros(64, dtype=np.int32)
        _chk(lib().orc_ctx_ring(self.h, _ptr(ri, C.c_int), _ptr(th), _ptr(gens, C.c_int)))
        # cyclotomic index m (2N or 3N); for m = 3N the slot algebra of Phi_M'(X^s) over GR(p^r, 2)
        self.m, self.Mp, self.s, self.nprime, self.gr_c = (int(x) for x in ri[:5])
        # m = 3N: theta = (t0, t1) in GR(p^r, 2); m = 5N/2: theta = (t0, t1, t2, t3) in GR(p^r, 4), gr_w = w
        self.theta = tuple(int(x) for x in th[:4]) if self.m_odd == 5 else (int(th[0]), int(th[1]))
        self.gr_w = (int(th[4]), int(th[5]))
        self.gens = [(int(gens[2 * i]), int(gens[2 * i + 1])) for i in range(int(ri[5]))]

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_ctx_free(self.h)
            self.h = None

    # -- tables
    def primes(self):
        out = np.zeros(self.L + self.alpha, dtype=np.uint64)
        _chk(lib().orc_primes(self.h, _ptr(out)))
        return out

    def psi(self):
        out = np.zeros(self.L + self.alpha, dtype=np.uint64)
        _chk(lib().orc_psi(self.h, _ptr(out)))
        return out

    def ntt_fwd(self, pi, a):
        x = np.ascontiguousarray(a, dtype=np.uint64).copy()
        _chk(lib().orc_ntt_fwd(self.h, pi, _ptr(x)))
        return x

    def ntt_inv(self, pi, a):
        x = np.ascontiguousarray(a, dtype=np.uint64).copy()
        _chk(lib().orc_ntt_inv(self.h, pi, _ptr(x)))
        return x

    def automorph_coeff(self, pi, g, a):
        x = np.ascontiguousarray(a, dtype=np.uint64).copy()
        _chk(lib().orc_automorph_coeff(self.h, pi, g, _ptr(x)))
        return x

    # -- keys
    def keygen(self, galois=None):
        if galois is None:
            galois = self.rotate_sum_elements()
        g = np.ascontiguousarray(galois, dtype=np.int32)
        _chk(lib().orc_keygen(self.h, _ptr(g, C.c_int), len(g)))

    def secret_keygen(self):
        """Secret key only (no key-switching keys): enough to encrypt and decrypt."""
        _chk(lib().orc_secret_keygen(self.h))

    def secret(self):
        out = np.zeros(self.N, dtype=np.int64)
        _chk(lib().orc_secret(self.h, _ptr(out, C.c_int64)))
        return out

    def ksk(self, g=0):
        dnum = (self.L + self.alpha - 1) // self.alpha
        b = np.zeros((dnum, self.L + self.alpha, self.N), dtype=np.uint64)
        a = np.zeros_like(b)
        _chk(lib().orc_ksk_export(self.h, g, _ptr(b), _ptr(a)))
        return b, a

    def rotate_sum_elements(self):
        out = np.zeros(64, dtype=np.int32)
        n = lib().orc_rotate_sum_elements(self.h, _ptr(out, C.c_int))
        if n < 0:
            raise _err()
        return [int(x) for x in out[:n]]

    # -- slots
    def encode(self, slots, t_exp=None):
        t_exp = self.r if t_exp is None else t_exp
        v = np.ascontiguousarray(slots, dtype=np.uint64)
        out = np.zeros(self.N, dtype=np.uint64)
        _chk(lib().orc_encode(self.h, t_exp, _ptr(v), _ptr(out)))
        return out

    def decode(self, coeffs, t_exp=None):
        t_exp = self.r if t_exp is None else t_exp
        m = np.ascontiguousarray(coeffs, dtype=np.uint64)
        out = np.zeros(self.slots, dtype=np.uint64)
        _chk(lib().orc_decode(self.h, t_exp, _ptr(m), _ptr(out)))
        return out

    # -- ciphertexts
    def encrypt(self, coeffs, nonce, t_exp=None):
        t_exp = self.r if t_exp is None else t_exp
        m = np.ascontiguousarray(coeffs, dtype=np.uint64)
        return Ct(self, lib().orc_encrypt(self.h, _ptr(m), nonce, t_exp))

    def encrypt_slots(self, slots, nonce):
        return self.encrypt(self.encode(slots), nonce)

    def ct_from_words(self, words, t_exp):
        w = np.ascontiguousarray(words, dtype=np.uint64)
        n, l, _ = w.shape
        return Ct(self, lib().orc_ct_import(self.h, _ptr(w), n, l, t_exp))

    def decrypt(self, ct):
        out = np.zeros(self.N, dtype=np.uint64)
        _chk(lib().orc_decrypt(self.h, ct.h, _ptr(out)))
        return out

    def decrypt_slots(self, ct):
        return self.decode(self.decrypt(ct), ct.t_exp)

    def set_reduced_g(self, on=True):
        """Evaluate G_{p,e} with the lattice-reduced coefficients (Section 4.2)."""
        _chk(lib().orc_set_reduced_g(self.h, 1 if on else 0))

    def noise_budget(self, ct):
        return lib().orc_noise_budget(self.h, ct.h)

    def add(self, a, b):
        return Ct(self, lib().orc_add(self.h, a.h, b.h))

    def sub(self, a, b):
        return Ct(self, lib().orc_sub(self.h, a.h, b.h))

    def mul_scalar(self, a, c):
        return Ct(self, lib().orc_mul_scalar(self.h, a.h, int(c)))

    def add_scalar(self, a, c):
        return Ct(self, lib().orc_add_scalar(self.h, a.h, int(c)))

    def tensor(self, a, b):
        return Ct(self, lib().orc_tensor(self.h, a.h, b.h))

    def relin(self, a):
        return Ct(self, lib().orc_relin(self.h, a.h))

    def modswitch(self, a, drop=1):
        return Ct(self, lib().orc_modswitch(self.h, a.h, drop))

    def rotate(self, a, g):
        return Ct(self, lib().orc_rotate(self.h, a.h, g))

    def divide_by_p(self, a):
        return Ct(self, lib().orc_divide_by_p(self.h, a.h))

    def mul(self, a, b):
        return Ct(self, lib().orc_mul(self.h, a.h, b.h))

    def relin_drop(self, a):
        return Ct(self, lib().orc_relin_drop(self.h, a.h))

    def with_t_exp(self, a, t_exp):
        return Ct(self, lib().orc_set_t_exp(self.h, a.h, t_exp))

    # -- space switching
    def eval_g(self, x, e):
        return Ct(self, lib().orc_eval_g(self.h, x.h, e))

    def reduce(self, a):
        out = (C.c_void_p * self.r)()
        _chk(lib().orc_reduce(self.h, a.h, out))
        return [Ct(self, out[i]) for i in range(self.r)]

    def compare_lt(self, a, b):
        return Ct(self, lib().orc_compare_lt(self.h, a.h, b.h))

    def compare(self, pred, a, b):
        """Section 4.3 predicate (PREDICATES name or index) of a against b, at t = p."""
        return Ct(self, lib().orc_compare(self.h, _pred(pred), a.h, b.h))

    def query_where(self, A, B, conds):
        """SUM(A*B) over rows where every (pred, X, Y) condition holds; Y may hold one ciphertext."""
        n, k = len(A), len(conds)
        arr = lambda xs: (C.c_void_p * len(xs))(*[x.h for x in xs])
        preds = (C.c_int32 * k)(*[_pred(c[0]) for c in conds])
        X = (C.c_void_p * (k * n))(*[x.h for c in conds for x in c[1]])
        Y = (C.c_void_p * (k * n))()
        for j, c in enumerate(conds):
            for i, y in enumerate(c[2]):
                Y[j * n + i] = y.h
        ny = (C.c_int32 * k)(*[len(c[2]) for c in conds])
        return Ct(self, lib().orc_query_where(self.h, arr(A), arr(B), n, k, preds, X, Y, ny))

    def raise_modulus(self, a):
        return Ct(self, lib().orc_raise(self.h, a.h))

    def rotate_sum(self, a):
        return Ct(self, lib().orc_rotate_sum(self.h, a.h))

    def query(self, A, B, C1, C2):
        n, n2 = len(A), len(C2)
        arr = lambda xs: (C.c_void_p * len(xs))(*[x.h for x in xs])
        return Ct(self, lib().orc_query(self.h, arr(A), arr(B), arr(C1), arr(C2), n, n2))

    def trace(self, on=True):
        lib().orc_trace(self.h, 1 if on else 0)

    def meter(self, on=True):
        """Records the noise budget of every stage result of the space-switching
        procedures (Algorithms 3 and 4, raising, the query) while on."""
        lib().orc_meter(self.h, 1 if on else 0)

    def meter_readings(self):
        """[(stage label, level, budget in bits)] recorded since meter(True)."""
        n = lib().orc_meter_get(self.h, None, 0)
        buf = C.create_string_buffer(n + 1)
        lib().orc_meter_get(self.h, buf, n + 1)
        out = []
        for line in buf.value.decode().splitlines():
            lab, lvl, bits = line.split()
            out.append((lab, int(lvl[1:]), float(bits)))
        return out

    def trace_text(self):
        n = lib().orc_trace_get(self.h, None, 0)
        buf = C.create_string_buffer(n + 1)
        lib().orc_trace_get(self.h, buf, n + 1)
        return buf.value.decode()
