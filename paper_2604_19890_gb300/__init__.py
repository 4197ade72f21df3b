"""Python binding of libss.so, the GB300 space-switching BGV library.

Argument marshalling only: every step runs in the library's CUDA kernels.
Device memory and streams come from PyTorch. There is no CPU fallback: the
binding raises if the compiled library is missing or no GPU is present.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libss.so")
HEADER = os.path.join(HERE, "..", "include", "ss.h")

SS_OK, SS_ERR_PARAM, SS_ERR_LEVEL, SS_ERR_NOISE, SS_ERR_TMOD = 0, 1, 2, 3, 4
SS_ERR_SHAPE, SS_ERR_OOM, SS_ERR_TIMEOUT, SS_ERR_CUDA = 5, 6, 7, 8
STATUS = {0: "SS_OK", 1: "SS_ERR_PARAM", 2: "SS_ERR_LEVEL", 3: "SS_ERR_NOISE", 4: "SS_ERR_TMOD",
          5: "SS_ERR_SHAPE", 6: "SS_ERR_OOM", 7: "SS_ERR_TIMEOUT", 8: "SS_ERR_CUDA"}


class SSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS.get(code, code), msg))
        self.code = code


class ss_params(C.Structure):
    _fields_ = [("logN", C.c_int32), ("L", C.c_int32), ("alpha", C.c_int32), ("bits", C.c_int32),
                ("p", C.c_int32), ("r", C.c_int32), ("h", C.c_int32), ("nmax", C.c_int32),
                ("seed", C.c_uint64), ("m_odd", C.c_int32), ("reserved", C.c_int32)]


class ss_ct(C.Structure):
    _fields_ = [("data", C.c_void_p), ("count", C.c_int32), ("ncomp", C.c_int32), ("level", C.c_int32),
                ("t_exp", C.c_int32), ("capacity", C.c_int32), ("reserved", C.c_int32)]


class ss_cond(C.Structure):
    _fields_ = [("pred", C.c_int32), ("pad", C.c_int32), ("x", C.POINTER(ss_ct)), ("y", C.POINTER(ss_ct))]


class ss_batch_item(C.Structure):
    _fields_ = [("ctx", C.c_int32), ("reduce", C.c_int32), ("a", ss_ct), ("b", ss_ct),
                ("prod", C.POINTER(ss_ct)), ("digits", C.POINTER(ss_ct))]


_lib = None

_SIGS = {
    "ss_last_error": (C.c_char_p, []),
    "ss_params_preset": (C.c_int, [C.c_int, C.POINTER(ss_params)]),
    "ss_context_create": (C.c_int, [C.POINTER(ss_params), C.POINTER(C.c_void_p)]),
    "ss_context_destroy": (None, [C.c_void_p]),
    "ss_context_info": (C.c_int, [C.c_void_p] + [C.POINTER(C.c_int32)] * 5 + [C.POINTER(C.c_uint64)]),
    "ss_keygen": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_int32]),
    "ss_rotate_sum_elements": (C.c_int32, [C.c_void_p, C.POINTER(C.c_int32), C.c_int32]),
    "ss_encode": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]),
    "ss_decode": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]),
    "ss_encrypt": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_uint32, C.c_int32, C.POINTER(ss_ct),
                             C.c_void_p]),
    "ss_decrypt": (C.c_int, [C.c_void_p, C.POINTER(ss_ct), C.c_void_p, C.c_void_p]),
    "ss_add": (C.c_int, [C.c_void_p, C.POINTER(ss_ct), C.POINTER(ss_ct), C.POINTER(ss_ct), C.c_void_p]),
    "ss_sub": (C.c_int, [C.c_void_p, C.POINTER(ss_ct), C.POINTER(ss_ct), C.POINTER(ss_ct), C.c_void_p]),
    "ss_mul_scalar": (C.c_int, [C.c_void_p, C.POINTER(ss_ct), C.c_int64, C.POINTER(ss_ct), C.c_void_p]),
    "ss_add_scalar": (C.c_int, [C.c_void_p, C.POINTER(ss_ct), C.c_int64, C.POINTER(ss_ct), C.c_void_p]),
    "ss_mul": (C.c_int, [C.c_void_p, C.POINTER(ss_ct), C.POINTER(ss_ct), C.POINTER(ss_ct), C.c_void_p]),
    "ss_relin": (C.c_int, [C.c_void_p, C.POINTER(ss_ct), C.POINTER(ss_ct), C.c_void_p]),
    "ss_linear_combinations": (C.c_int, [C.c_void_p, C.POINTER(ss_ct), C.c_int32, C.POINTER(C.c_int64), C.c_int32,
                                         C.POINTER(ss_ct), C.c_void_p]),
    "ss_query_bytes": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(C.c_uint64)]),
    "ss_set_g_table": (C.c_int, [C.c_void_p, C.c_int32]),
    "ss_mul_relin": (C.c_int, [C.c_void_p, C.POINTER(ss_ct), C.POINTER(ss_ct), C.POINTER(ss_ct), C.c_void_p]),
    "ss_relin_noalloc": (C.c_int, [C.c_void_p, C.POINTER(ss_ct), C.POINTER(ss_ct), C.c_void_p]),
    "ss_modswitch": (C.c_int, [C.c_void_p, C.POINTER(ss_ct), C.c_int32, C.POINTER(ss_ct), C.c_void_p]),
    "ss_rotate": (C.c_int, [C.c_void_p, C.POINTER(ss_ct), C.c_int32, C.POINTER(ss_ct), C.c_void_p]),
    "ss_rotate_sum": (C.c_int, [C.c_void_p, C.POINTER(ss_ct), C.POINTER(ss_ct), C.c_void_p]),
    "ss_linear_combination": (C.c_int, [C.c_void_p, C.POINTER(ss_ct), C.POINTER(C.c_int64), C.c_int32, C.c_int64,
                                        C.POINTER(ss_ct), C.c_void_p]),
    "ss_divide_by_p": (C.c_int, [C.c_void_p, C.POINTER(ss_ct), C.POINTER(ss_ct), C.c_void_p]),
    "ss_eval_g": (C.c_int, [C.c_void_p, C.POINTER(ss_ct), C.c_int32, C.POINTER(ss_ct), C.c_void_p]),
    "ss_reduce_to_digits": (C.c_int, [C.c_void_p, C.POINTER(ss_ct), C.POINTER(ss_ct), C.c_void_p]),
    "ss_compare_lt": (C.c_int, [C.c_void_p, C.POINTER(ss_ct), C.POINTER(ss_ct), C.POINTER(ss_ct), C.c_void_p]),
    "ss_raise_modulus": (C.c_int, [C.c_void_p, C.POINTER(ss_ct), C.POINTER(ss_ct), C.c_void_p]),
    "ss_query_sum_where_lt": (C.c_int, [C.c_void_p] + [C.POINTER(ss_ct)] * 5 + [C.c_void_p]),
    "ss_query_sum_where_lt_host": (C.c_int, [C.c_void_p] + [C.c_void_p] * 4 + [C.c_int32] * 3 +
                                   [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.c_void_p]),
    "ss_query_depth": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32)]),
    "ss_set_batch": (C.c_int, [C.c_void_p, C.c_int32]),
    "ss_ntt_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p]),
    "ss_ntt_inverse": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p]),
    "ss_trace": (C.c_int, [C.c_void_p, C.c_int32]),
    "ss_trace_get": (C.c_int32, [C.c_void_p, C.c_char_p, C.c_int32]),
    "ss_launch_count": (C.c_uint64, [C.c_void_p]),
    "ss_compare": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(ss_ct), C.POINTER(ss_ct), C.POINTER(ss_ct),
                             C.c_void_p]),
    "ss_query_sum_where": (C.c_int, [C.c_void_p, C.POINTER(ss_ct), C.POINTER(ss_ct), C.POINTER(ss_cond), C.c_int32,
                                     C.POINTER(ss_ct), C.c_void_p]),
    "ss_stage_stats": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_uint64), C.POINTER(C.c_double)]),
    "ss_alu_probe": (C.c_int, [C.c_int32, C.c_int32, C.POINTER(C.c_double)]),
    "ss_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(ss_batch_item), C.c_int32,
                                  C.POINTER(C.c_void_p)]),
    "ss_batch_config": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32]),
    "ss_batch_get_config": (C.c_int, [C.c_void_p] + [C.POINTER(C.c_int32)] * 5),
    "ss_batch_tune": (C.c_int, [C.c_void_p, C.c_void_p] + [C.POINTER(C.c_int32)] * 3),
    "ss_batch_capture": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ss_batch_run": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ss_batch_destroy": (None, [C.c_void_p]),
    "ss_server_create": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_uint64, C.POINTER(C.c_void_p)]),
    "ss_server_submit": (C.c_int, [C.c_void_p] + [C.POINTER(ss_ct)] * 5 + [C.POINTER(C.c_uint64)]),
    "ss_server_create_multi": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.c_int32, C.c_int32, C.c_uint64,
                                         C.POINTER(C.c_void_p)]),
    "ss_server_submit_to": (C.c_int, [C.c_void_p, C.c_int32] + [C.POINTER(ss_ct)] * 5 + [C.POINTER(C.c_uint64)]),
    "ss_server_wait": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "ss_server_stats": (C.c_int, [C.c_void_p] + [C.POINTER(C.c_uint64)] * 3),
    "ss_server_destroy": (None, [C.c_void_p]),
    "ss_kernel_timing": (C.c_int, [C.c_void_p, C.c_int32]),
    "ss_ntt_products": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "ss_kernel_stats": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_uint64), C.POINTER(C.c_double),
                                  C.POINTER(C.c_double)]),
}

KERNEL_CLASSES = ["ntt", "base_conversion", "keyswitch_inner_product", "tensor", "sub_scale", "automorphism",
                  "elementwise", "sampling"]
# Section 4.3 predicates in ss_predicate order
PREDICATES = ["lt", "le", "gt", "ge", "eq", "neq"]

QUERY_STAGES = ["reduction", "comparison", "aggregation", "modulus_raising", "masked_product", "sum"]


def alu_probe(kind, iters=4096):
    """Integer-pipe ceiling on the current device: kind 0 = 32-bit IMAD/s,
    kind 1 = 64-bit Shoup forward butterflies/s (registers only)."""
    out = C.c_double()
    _chk(lib().ss_alu_probe(int(kind), int(iters), C.byref(out)))
    return out.value


def declared_symbols():
    """Every function name include/ss.h declares."""
    import re
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ss_[a-z0-9_]+)\s*\(", txt)))


def lib():
    """Loads libss.so; raises if it has not been built (no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libss.so is not built; run __graft_entry__.build() (nvcc, sm_103a)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _chk(rc):
    if rc != SS_OK:
        raise SSError(rc, lib().ss_last_error().decode())


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the space-switching library needs a CUDA GPU")
    return torch


def _stream(torch, stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def preset(i):
    p = ss_params()
    _chk(lib().ss_params_preset(i, C.byref(p)))
    return p


class CtBatch:
    """A batch of ciphertexts in a torch int64 tensor [count][ncomp][capacity][N]."""

    def __init__(self, buf, count, ncomp, level, t_exp):
        self.buf, self.count, self.ncomp, self.level, self.t_exp = buf, count, ncomp, level, t_exp

    @property
    def capacity(self):
        return self.buf.shape[2]

    def desc(self):
        return ss_ct(self.buf.data_ptr(), self.count, self.ncomp, self.level, self.t_exp, self.capacity, 0)

    def update(self, d):
        self.ncomp, self.level, self.t_exp = d.ncomp, d.level, d.t_exp
        return self

    def words(self):
        """uint64 numpy array [count][ncomp][level][N] (evaluation form)."""
        x = self.buf[:, : self.ncomp, : self.level].contiguous().cpu().numpy()
        return x.view(np.uint64)

    def slice(self, b0, n):
        return CtBatch(self.buf[b0:b0 + n], n, self.ncomp, self.level, self.t_exp)


class Batch:
    """Batched form (ss_batch_*): pairs (ctx_index, a, b, reduce) of single
    ciphertexts over several contexts; outputs are allocated here."""

    def __init__(self, ctxs, pairs):
        self.ctxs = ctxs
        self.torch = ctxs[0].torch
        items = (ss_batch_item * len(pairs))()
        self._keep = []
        self.outputs = []
        for i, (ci, a, b, red) in enumerate(pairs):
            g = ctxs[ci]
            prod = g.empty(1, level=a.level - 1)
            pd = prod.desc()
            digs = [g.empty(1, level=a.level - 1) for _ in range(g.r)] if red else []
            dd = (ss_ct * max(1, len(digs)))(*[d.desc() for d in digs]) if red else None
            items[i] = ss_batch_item(ci, 1 if red else 0, a.desc(), b.desc(), C.pointer(pd),
                                     C.cast(dd, C.POINTER(ss_ct)) if red else None)
            self._keep.append((pd, dd, a, b))
            self.outputs.append((prod, pd, digs, dd))
        arr = (C.c_void_p * len(ctxs))(*[g.h.value for g in ctxs])
        h = C.c_void_p()
        _chk(lib().ss_batch_create(arr, len(ctxs), items, len(pairs), C.byref(h)))
        self.h = h
        self._items = items

    def results(self):
        """[(product CtBatch, [digit CtBatch...] or [])] with metadata from the last run."""
        out = []
        for prod, pd, digs, dd in self.outputs:
            prod.update(pd)
            ds = [d.update(dd[k]) for k, d in enumerate(digs)] if digs else []
            out.append((prod, ds))
        return out

    def config(self, chunk, nstreams, tile_log=11):
        _chk(lib().ss_batch_config(self.h, chunk, nstreams, tile_log))

    def get_config(self):
        v = [C.c_int32() for _ in range(5)]
        _chk(lib().ss_batch_get_config(self.h, *[C.byref(x) for x in v]))
        return dict(zip(["chunk", "nstreams", "tile_log", "groups", "skipped"], [x.value for x in v]))

    def tune(self, stream):
        v = [C.c_int32() for _ in range(3)]
        _chk(lib().ss_batch_tune(self.h, C.c_void_p(stream.cuda_stream), *[C.byref(x) for x in v]))
        return [x.value for x in v]

    def capture(self, stream):
        _chk(lib().ss_batch_capture(self.h, C.c_void_p(stream.cuda_stream)))

    def run(self, stream):
        _chk(lib().ss_batch_run(self.h, C.c_void_p(stream.cuda_stream)))

    def close(self):
        if getattr(self, "h", None):
            lib().ss_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Request loop with continuous batching (ss_server_*) over one context or
    a list of contexts (one HBM budget; queries merge only within a context)."""

    def __init__(self, ctx, workers=2, max_merge=8, hbm_budget=0):
        self.ctxs = list(ctx) if isinstance(ctx, (list, tuple)) else [ctx]
        self.ctx = self.ctxs[0]
        h = C.c_void_p()
        arr = (C.c_void_p * len(self.ctxs))(*[g.h.value for g in self.ctxs])
        _chk(lib().ss_server_create_multi(arr, len(self.ctxs), workers, max_merge, hbm_budget, C.byref(h)))
        self.h = h
        self._live = {}

    def submit(self, A, B, C1, C2, ctx_index=0):
        """Queues a query on context ctx_index; returns a ticket. Keeps the
        descriptors alive until wait()."""
        out = self.ctxs[ctx_index].empty(1, level=A.level)
        descs = [x.desc() for x in (A, B, C1, C2)] + [out.desc()]
        t = C.c_uint64()
        _chk(lib().ss_server_submit_to(self.h, ctx_index, *[C.byref(d) for d in descs], C.byref(t)))
        self._live[t.value] = (descs, out, (A, B, C1, C2))
        return t.value

    def wait(self, ticket, timeout_ms=-1):
        """Returns (result CtBatch, queued_ms, run_ms)."""
        q, r = C.c_double(), C.c_double()
        rc = lib().ss_server_wait(self.h, ticket, timeout_ms, C.byref(q), C.byref(r))
        if rc == SS_ERR_TIMEOUT:
            raise SSError(rc, lib().ss_last_error().decode())
        descs, out, _ = self._live.pop(ticket)
        _chk(rc)
        return out.update(descs[4]), q.value, r.value

    def stats(self):
        c, b, p = C.c_uint64(), C.c_uint64(), C.c_uint64()
        _chk(lib().ss_server_stats(self.h, C.byref(c), C.byref(b), C.byref(p)))
        return {"completed": c.value, "batches": b.value, "peak_inflight_bytes": p.value}

    def close(self):
        if getattr(self, "h", None):
            lib().ss_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    def __init__(self, params=None, preset_id=None, **kw):
        self.torch = _torch()
        if params is None:
            params = preset(preset_id) if preset_id is not None else ss_params()
            for k, v in kw.items():
                setattr(params, k, v)
        self.params = params
        h = C.c_void_p()
        _chk(lib().ss_context_create(C.byref(params), C.byref(h)))
        self.h = h
        n, L, a, s, d = (C.c_int32() for _ in range(5))
        _chk(lib().ss_context_info(h, C.byref(n), C.byref(L), C.byref(a), C.byref(s), C.byref(d), None))
        self.N, self.L, self.alpha, self.slots, self.d = n.value, L.value, a.value, s.value, d.value
        pr = (C.c_uint64 * (self.L + self.alpha))()
        _chk(lib().ss_context_info(h, None, None, None, None, None, pr))
        self.primes = np.array(list(pr), dtype=np.uint64)
        self.p, self.r = params.p, params.r
        self.t = self.p ** self.r
        # cyclotomic index: m = 2N (X^N + 1), 3N (X^N - X^(N/2) + 1) or 5N/2 (Phi_10(X^(N/4)))
        self.m_odd = params.m_odd if params.m_odd in (3, 5) else 1
        self.m = {1: 2 * self.N, 3: 3 * self.N, 5: 5 * self.N // 2}[self.m_odd]

    def close(self):
        if getattr(self, "h", None):
            lib().ss_context_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- keys, slots
    def rotate_sum_elements(self):
        out = (C.c_int32 * 64)()
        n = lib().ss_rotate_sum_elements(self.h, out, 64)
        return [int(out[i]) for i in range(n)]

    def keygen(self, galois=None):
        g = self.rotate_sum_elements() if galois is None else list(galois)
        arr = (C.c_int32 * max(1, len(g)))(*g)
        _chk(lib().ss_keygen(self.h, arr, len(g)))

    def encode(self, slots, t_exp=None):
        t_exp = self.r if t_exp is None else t_exp
        v = np.ascontiguousarray(slots, dtype=np.uint64)
        out = np.zeros(self.N, dtype=np.uint64)
        _chk(lib().ss_encode(self.h, t_exp, v.ctypes.data_as(C.POINTER(C.c_uint64)),
                             out.ctypes.data_as(C.POINTER(C.c_uint64))))
        return out

    def decode(self, coeffs, t_exp=None):
        t_exp = self.r if t_exp is None else t_exp
        m = np.ascontiguousarray(coeffs, dtype=np.uint64)
        out = np.zeros(self.slots, dtype=np.uint64)
        _chk(lib().ss_decode(self.h, t_exp, m.ctypes.data_as(C.POINTER(C.c_uint64)),
                             out.ctypes.data_as(C.POINTER(C.c_uint64))))
        return out

    # ---------------------------------------------------------------- memory
    def empty(self, count, level=None, ncomp=2, t_exp=None, capacity=None):
        level = self.L if level is None else level
        cap = level if capacity is None else capacity
        buf = self.torch.empty((count, ncomp, cap, self.N), dtype=self.torch.int64, device="cuda")
        return CtBatch(buf, count, ncomp, level, self.r if t_exp is None else t_exp)

    def from_words(self, words, t_exp):
        w = np.ascontiguousarray(words, dtype=np.uint64)
        if w.ndim == 3:
            w = w[None]
        buf = self.torch.from_numpy(w.view(np.int64).copy()).cuda()
        return CtBatch(buf, w.shape[0], w.shape[1], w.shape[2], t_exp)

    # ---------------------------------------------------------------- Enc / Dec
    def encrypt(self, coeffs, nonce0, t_exp=None, stream=None):
        t_exp = self.r if t_exp is None else t_exp
        torch = self.torch
        m = np.ascontiguousarray(coeffs, dtype=np.uint64)
        if m.ndim == 1:
            m = m[None]
        dm = torch.from_numpy(m.view(np.int64)).cuda()
        out = self.empty(m.shape[0], t_exp=t_exp)
        d = out.desc()
        _chk(lib().ss_encrypt(self.h, C.c_void_p(dm.data_ptr()), m.shape[0], nonce0, t_exp, C.byref(d),
                              _stream(torch, stream)))
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        return out.update(d)

    def encrypt_slots(self, slots, nonce0):
        s = np.atleast_2d(np.asarray(slots, dtype=np.uint64))
        return self.encrypt(np.stack([self.encode(x) for x in s]), nonce0)

    def decrypt(self, ct, stream=None):
        torch = self.torch
        out = torch.empty((ct.count, self.N), dtype=torch.int64, device="cuda")
        d = ct.desc()
        _chk(lib().ss_decrypt(self.h, C.byref(d), C.c_void_p(out.data_ptr()), _stream(torch, stream)))
        return out.cpu().numpy().view(np.uint64)

    def decrypt_slots(self, ct):
        m = self.decrypt(ct)
        return np.stack([self.decode(x, ct.t_exp) for x in m])

    # ---------------------------------------------------------------- operations
    def _out(self, a, level=None, ncomp=None):
        return self.empty(a.count, level=a.level if level is None else level,
                          ncomp=a.ncomp if ncomp is None else ncomp, t_exp=a.t_exp)

    def _call2(self, fn, a, b, out, stream=None):
        da, db, do = a.desc(), b.desc(), out.desc()
        _chk(fn(self.h, C.byref(da), C.byref(db), C.byref(do), _stream(self.torch, stream)))
        return out.update(do)

    def add(self, a, b):
        return self._call2(lib().ss_add, a, b, self._out(a))

    def sub(self, a, b):
        return self._call2(lib().ss_sub, a, b, self._out(a))

    def mul(self, a, b):
        return self._call2(lib().ss_mul, a, b, self._out(a, ncomp=3))

    def mul_relin(self, a, b):
        """Multiplication as the evaluator runs it: tensor, relinearise, drop one prime."""
        lvl = min(a.level, b.level) - 1
        return self._call2(lib().ss_mul_relin, a, b, self.empty(a.count, level=lvl, t_exp=a.t_exp))

    def compare_lt(self, a, b):
        return self._call2(lib().ss_compare_lt, a, b, self._out(a, ncomp=2))

    def _call1(self, fn, a, out, *extra):
        da, do = a.desc(), out.desc()
        if extra:
            _chk(fn(self.h, C.byref(da), *extra, C.byref(do), _stream(self.torch)))
        else:
            _chk(fn(self.h, C.byref(da), C.byref(do), _stream(self.torch)))
        return out.update(do)

    def mul_scalar(self, a, c):
        return self._call1(lib().ss_mul_scalar, a, self._out(a), C.c_int64(int(c)))

    def add_scalar(self, a, c):
        return self._call1(lib().ss_add_scalar, a, self._out(a), C.c_int64(int(c)))

    def relin(self, a):
        return self._call1(lib().ss_relin, a, self._out(a, ncomp=2))

    def relin_noalloc(self, a):
        """ss_relin without any device allocation (scratch in a static device array)."""
        return self._call1(lib().ss_relin_noalloc, a, self._out(a, ncomp=2))

    def modswitch(self, a, drop=1):
        return self._call1(lib().ss_modswitch, a, self._out(a, level=a.level - drop), C.c_int32(drop))

    def rotate(self, a, g):
        return self._call1(lib().ss_rotate, a, self._out(a), C.c_int32(g))

    def rotate_sum(self, a):
        return self._call1(lib().ss_rotate_sum, a, self._out(a))

    def linear_combination(self, terms, coeffs, cst=0):
        arr = (ss_ct * len(terms))(*[x.desc() for x in terms])
        cf = (C.c_int64 * len(terms))(*[int(c) for c in coeffs])
        out = self._out(terms[0])
        do = out.desc()
        _chk(lib().ss_linear_combination(self.h, arr, cf, len(terms), int(cst), C.byref(do), _stream(self.torch)))
        return out.update(do)

    def linear_combinations(self, terms, coeff_rows):
        """[sum_i row[i] * terms[i] for row in coeff_rows] in one pass (ss_linear_combinations)."""
        arr = (ss_ct * len(terms))(*[x.desc() for x in terms])
        flat = [int(c) for row in coeff_rows for c in row]
        cf = (C.c_int64 * len(flat))(*flat)
        outs = [self._out(terms[0], ncomp=2) for _ in coeff_rows]
        od = (ss_ct * len(outs))(*[o.desc() for o in outs])
        _chk(lib().ss_linear_combinations(self.h, arr, len(terms), cf, len(outs), od, _stream(self.torch)))
        return [o.update(od[k]) for k, o in enumerate(outs)]

    def divide_by_p(self, a):
        return self._call1(lib().ss_divide_by_p, a, self._out(a))

    def eval_g(self, x, e):
        return self._call1(lib().ss_eval_g, x, self._out(x), C.c_int32(e))

    def compare(self, pred, a, b):
        """Section 4.3 predicate ('lt', 'le', 'gt', 'ge', 'eq', 'neq' or its index) of a against b, at t = p."""
        pi = PREDICATES.index(pred) if isinstance(pred, str) else int(pred)
        out = self._out(a if a.count >= b.count else b, ncomp=2)
        da, db, do = a.desc(), b.desc(), out.desc()
        _chk(lib().ss_compare(self.h, pi, C.byref(da), C.byref(db), C.byref(do), _stream(self.torch)))
        return out.update(do)

    def query_where(self, A, B, conds, stream=None):
        """SUM(A*B) over the rows where every (pred, X, Y) condition holds (Y may have count 1)."""
        out = self.empty(1, level=A.level)
        descs = [(x.desc(), y.desc()) for _, x, y in conds]
        arr = (ss_cond * len(conds))()
        for k, (pred, _, _) in enumerate(conds):
            arr[k].pred = PREDICATES.index(pred) if isinstance(pred, str) else int(pred)
            arr[k].x = C.pointer(descs[k][0])
            arr[k].y = C.pointer(descs[k][1])
        da, db, do = A.desc(), B.desc(), out.desc()
        _chk(lib().ss_query_sum_where(self.h, C.byref(da), C.byref(db), arr, len(conds), C.byref(do),
                                      _stream(self.torch, stream)))
        return out.update(do)

    def raise_modulus(self, a):
        return self._call1(lib().ss_raise_modulus, a, self._out(a))

    def reduce(self, a):
        outs = [self._out(a) for _ in range(self.r)]
        arr = (ss_ct * self.r)(*[o.desc() for o in outs])
        da = a.desc()
        _chk(lib().ss_reduce_to_digits(self.h, C.byref(da), arr, _stream(self.torch)))
        return [o.update(arr[i]) for i, o in enumerate(outs)]

    def query(self, A, B, C1, C2, stream=None):
        out = self.empty(1, level=A.level)
        ds = [x.desc() for x in (A, B, C1, C2, out)]
        _chk(lib().ss_query_sum_where_lt(self.h, *[C.byref(d) for d in ds], _stream(self.torch, stream)))
        return out.update(ds[4])

    def query_host(self, A, B, C1, C2, level, stream=None):
        """Query on host arrays uint64[count][2][level][N]; returns (words, level, t_exp)."""
        out = np.zeros(2 * level * self.N, dtype=np.uint64)  # filled as uint64[2][out_level][N]
        ol, ot = C.c_int32(), C.c_int32()
        arrs = [np.ascontiguousarray(x, dtype=np.uint64) for x in (A, B, C1, C2)]
        _chk(lib().ss_query_sum_where_lt_host(self.h, *[C.c_void_p(x.ctypes.data) for x in arrs],
                                              arrs[0].shape[0], arrs[3].shape[0], level,
                                              C.c_void_p(out.ctypes.data), C.byref(ol), C.byref(ot),
                                              _stream(self.torch, stream)))
        return out[: 2 * ol.value * self.N].reshape(2, ol.value, self.N), ol.value, ot.value

    def query_depth(self, level=None):
        out = C.c_int32()
        _chk(lib().ss_query_depth(self.h, self.L if level is None else level, C.byref(out)))
        return out.value

    def query_bytes(self, n_ct, level=None):
        """Peak device bytes of a query over n_ct ciphertexts per column (admission estimate)."""
        out = C.c_uint64()
        _chk(lib().ss_query_bytes(self.h, int(n_ct), self.L if level is None else int(level), C.byref(out)))
        return out.value

    def set_g_table(self, mode):
        """0: canonical G_{p,e} coefficients; 1: the lattice-reduced representative."""
        _chk(lib().ss_set_g_table(self.h, int(mode)))

    def set_batch(self, b):
        _chk(lib().ss_set_batch(self.h, b))

    def ntt_forward(self, data, first_prime=0, nprimes=None, stream=None):
        npoly = data.numel() // self.N
        nprimes = npoly if nprimes is None else nprimes
        _chk(lib().ss_ntt_forward(self.h, C.c_void_p(data.data_ptr()), npoly, first_prime, nprimes,
                                  _stream(self.torch, stream)))

    def ntt_inverse(self, data, first_prime=0, nprimes=None, stream=None):
        npoly = data.numel() // self.N
        nprimes = npoly if nprimes is None else nprimes
        _chk(lib().ss_ntt_inverse(self.h, C.c_void_p(data.data_ptr()), npoly, first_prime, nprimes,
                                  _stream(self.torch, stream)))

    def trace(self, on=True):
        _chk(lib().ss_trace(self.h, 1 if on else 0))

    def trace_text(self):
        n = lib().ss_trace_get(self.h, None, 0)
        b = C.create_string_buffer(n + 1)
        lib().ss_trace_get(self.h, b, n + 1)
        return b.value.decode()

    def launches(self):
        return int(lib().ss_launch_count(self.h))

    def kernel_timing(self, on=True):
        _chk(lib().ss_kernel_timing(self.h, 1 if on else 0))

    def kernel_stats(self):
        """{class: (launches, total ms, algorithmic bytes)} since timing was switched on."""
        out = {}
        for i, name in enumerate(KERNEL_CLASSES):
            n, ms, b = C.c_uint64(), C.c_double(), C.c_double()
            _chk(lib().ss_kernel_stats(self.h, i, C.byref(n), C.byref(ms), C.byref(b)))
            out[name] = (n.value, ms.value, b.value)
        return out

    def ntt_products(self):
        """Shoup products the timed transforms performed since timing was switched on."""
        v = C.c_double()
        _chk(lib().ss_ntt_products(self.h, C.byref(v)))
        return v.value

    def stage_stats(self):
        """{stage: (runs, total ms)} of the query since timing was switched on."""
        out = {}
        for i, name in enumerate(QUERY_STAGES):
            n, ms = C.c_uint64(), C.c_double()
            _chk(lib().ss_stage_stats(self.h, i, C.byref(n), C.byref(ms)))
            out[name] = (n.value, ms.value)
        return out
