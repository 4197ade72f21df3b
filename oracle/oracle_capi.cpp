// C entry points of the plain CPU reference, for the Python test harness.
// TEST INFRASTRUCTURE ONLY (see oracle.hpp). Errors return NULL / -1 and the
// message is available from orc_last_error().
#include <cstring>
#include <string>

#include "oracle.hpp"

using namespace orc;

namespace {
thread_local std::string g_err;
struct Handle {
  Context C;
  Trace tr;
};
template <class F>
int guard(F f) {
  try { f(); return 0; } catch (const std::exception& e) { g_err = e.what(); return -1; }
}
template <class F>
void* guard_ptr(F f) {
  try { return f(); } catch (const std::exception& e) { g_err = e.what(); return nullptr; }
}
Context& ctx(void* h) { return static_cast<Handle*>(h)->C; }
Trace* trace(void* h) { return &static_cast<Handle*>(h)->tr; }
const Ct& ct(void* c) { return *static_cast<Ct*>(c); }
void* box(Ct&& c) { return new Ct(std::move(c)); }
}  // namespace

extern "C" {

const char* orc_last_error() { return g_err.c_str(); }

void* orc_ctx_new(int logN, int L, int alpha, int bits, int p, int r, int h, int nmax, uint64_t seed, int m_odd) {
  return guard_ptr([&]() -> void* {
    Params P;
    P.logN = logN; P.N = 1 << logN; P.L = L; P.alpha = alpha; P.bits = bits;
    P.p = p; P.r = r; P.h = h; P.nmax = nmax; P.seed = seed; P.m_odd = m_odd;
    Handle* H = new Handle();
    H->C = make_context(P);
    return H;
  });
}

void orc_ctx_free(void* h) { delete static_cast<Handle*>(h); }

int orc_ctx_info(void* h, int* slots, int* d, uint64_t* t, uint64_t* omega, int* slot_exp) {
  return guard([&] {
    Context& C = ctx(h);
    *slots = C.slots; *d = C.d; *t = C.t; *omega = C.omega;
    if (slot_exp) for (int j = 0; j < C.slots; ++j) slot_exp[j] = C.slot_exp[j];
  });
}

// m = 3N slot algebra: out[0..5] = m, M', s, n', c, number of generators;
// theta = (theta[0], theta[1]); gens[2i], gens[2i+1] = generator i and its order.
// m = 5N/2: theta[0..3] = theta4, theta[4..5] = w.
int orc_ctx_ring(void* h, int* out, uint64_t* theta, int* gens) {
  return guard([&] {
    Context& C = ctx(h);
    out[0] = C.m; out[1] = C.Mp; out[2] = C.s; out[3] = C.nprime; out[4] = (int)C.gr_c;
    out[5] = (int)C.gens.size();
    if (C.P.m_odd == 5) {
      for (int i = 0; i < 4; ++i) theta[i] = C.theta4[i];
      theta[4] = C.gr_w[0]; theta[5] = C.gr_w[1];
    } else {
      theta[0] = C.theta[0]; theta[1] = C.theta[1];
    }
    if (gens)
      for (size_t i = 0; i < C.gens.size(); ++i) { gens[2 * i] = C.gens[i].first; gens[2 * i + 1] = C.gens[i].second; }
  });
}

int orc_primes(void* h, uint64_t* out) {
  return guard([&] { for (size_t i = 0; i < ctx(h).primes.size(); ++i) out[i] = ctx(h).primes[i]; });
}

int orc_psi(void* h, uint64_t* out) {
  return guard([&] { for (size_t i = 0; i < ctx(h).psi.size(); ++i) out[i] = ctx(h).psi[i]; });
}

int orc_ntt_fwd(void* h, int pi, uint64_t* a) {
  return guard([&] {
    Poly x(a, a + ctx(h).P.N);
    ntt_fwd(ctx(h), pi, x);
    std::memcpy(a, x.data(), x.size() * 8);
  });
}

int orc_ntt_inv(void* h, int pi, uint64_t* a) {
  return guard([&] {
    Poly x(a, a + ctx(h).P.N);
    ntt_inv(ctx(h), pi, x);
    std::memcpy(a, x.data(), x.size() * 8);
  });
}

int orc_automorph_coeff(void* h, int pi, int g, uint64_t* a) {
  return guard([&] {
    Poly x(a, a + ctx(h).P.N);
    x = automorph_coeff(ctx(h), x, g, ctx(h).primes[pi]);
    std::memcpy(a, x.data(), x.size() * 8);
  });
}

int orc_keygen(void* h, const int* galois, int ng) {
  return guard([&] { keygen(ctx(h), std::vector<int>(galois, galois + ng)); });
}

int orc_secret_keygen(void* h) { return guard([&] { secret_keygen(ctx(h)); }); }

int orc_secret(void* h, int64_t* out) {
  return guard([&] { for (int n = 0; n < ctx(h).P.N; ++n) out[n] = ctx(h).sk[n]; });
}

// Key-switching key words: [digit][limb (L+alpha)][N] for b then a.
int orc_ksk_export(void* h, int g, uint64_t* b_out, uint64_t* a_out) {
  return guard([&] {
    Context& C = ctx(h);
    const KSKey& K = (g == 0) ? C.rlk : C.gk.at(g);
    size_t o = 0;
    for (size_t j = 0; j < K.b.size(); ++j)
      for (size_t i = 0; i < K.b[j].size(); ++i) {
        std::memcpy(b_out + o, K.b[j][i].data(), C.P.N * 8);
        std::memcpy(a_out + o, K.a[j][i].data(), C.P.N * 8);
        o += C.P.N;
      }
  });
}

int orc_rotate_sum_elements(void* h, int* out) {
  int n = -1;
  guard([&] {
    auto g = rotate_sum_elements(ctx(h));
    for (size_t i = 0; i < g.size(); ++i) out[i] = g[i];
    n = (int)g.size();
  });
  return n;
}

int orc_encode(void* h, int t_exp, const uint64_t* slots, uint64_t* coeffs) {
  return guard([&] {
    Context& C = ctx(h);
    auto m = encode(C, t_exp, std::vector<u64>(slots, slots + C.slots));
    std::memcpy(coeffs, m.data(), m.size() * 8);
  });
}

int orc_decode(void* h, int t_exp, const uint64_t* coeffs, uint64_t* slots) {
  return guard([&] {
    Context& C = ctx(h);
    auto v = decode(C, t_exp, std::vector<u64>(coeffs, coeffs + C.P.N));
    std::memcpy(slots, v.data(), v.size() * 8);
  });
}

int orc_g_table(int p, int e, int64_t* out) {
  return guard([&] {
    auto g = g_table(p, e);
    for (size_t i = 0; i < g.size(); ++i) out[i] = g[i];
  });
}

int orc_g_table_reduced(int p, int e, int64_t* out) {
  return guard([&] {
    auto g = g_table_reduced(p, e);
    for (size_t i = 0; i < g.size(); ++i) out[i] = g[i];
  });
}

int orc_set_reduced_g(void* h, int on) {
  return guard([&] { ctx(h).reduced_g = on != 0; });
}

int orc_flt_table(int p, int64_t* out) {
  return guard([&] {
    auto f = flt_table(p);
    for (size_t i = 0; i < f.size(); ++i) out[i] = f[i];
  });
}

// ------------------------------------------------------------- ciphertexts
void* orc_encrypt(void* h, const uint64_t* m, uint32_t nonce, int t_exp) {
  return guard_ptr([&] {
    Context& C = ctx(h);
    return box(encrypt(C, std::vector<u64>(m, m + C.P.N), nonce, t_exp));
  });
}

int orc_ct_info(void* c, int* ncomp, int* level, int* t_exp) {
  return guard([&] { *ncomp = ct(c).ncomp; *level = ct(c).level; *t_exp = ct(c).t_exp; });
}

int orc_ct_export(void* c, uint64_t* out) {
  return guard([&] {
    const Ct& x = ct(c);
    size_t o = 0;
    for (int k = 0; k < x.ncomp; ++k)
      for (int i = 0; i < x.level; ++i) {
        std::memcpy(out + o, x.c[k][i].data(), x.c[k][i].size() * 8);
        o += x.c[k][i].size();
      }
  });
}

void* orc_ct_import(void* h, const uint64_t* data, int ncomp, int level, int t_exp) {
  return guard_ptr([&] {
    Context& C = ctx(h);
    Ct x;
    x.ncomp = ncomp; x.level = level; x.t_exp = t_exp;
    x.c.assign(ncomp, std::vector<Poly>(level, Poly(C.P.N)));
    size_t o = 0;
    for (int k = 0; k < ncomp; ++k)
      for (int i = 0; i < level; ++i) {
        std::memcpy(x.c[k][i].data(), data + o, C.P.N * 8);
        o += C.P.N;
      }
    return box(std::move(x));
  });
}

void orc_ct_free(void* c) { delete static_cast<Ct*>(c); }

int orc_decrypt(void* h, void* c, uint64_t* m) {
  return guard([&] {
    auto v = decrypt(ctx(h), ct(c));
    std::memcpy(m, v.data(), v.size() * 8);
  });
}

double orc_noise_budget(void* h, void* c) {
  double b = -1e300;
  guard([&] { b = noise_budget(ctx(h), ct(c)); });
  return b;
}

void* orc_add(void* h, void* a, void* b) { return guard_ptr([&] { return box(add(ctx(h), ct(a), ct(b))); }); }
void* orc_sub(void* h, void* a, void* b) { return guard_ptr([&] { return box(sub(ctx(h), ct(a), ct(b))); }); }
void* orc_mul_scalar(void* h, void* a, int64_t c) {
  return guard_ptr([&] { return box(mul_scalar(ctx(h), ct(a), c)); });
}
void* orc_add_scalar(void* h, void* a, int64_t c) {
  return guard_ptr([&] { return box(add_scalar(ctx(h), ct(a), c)); });
}
void* orc_tensor(void* h, void* a, void* b) { return guard_ptr([&] { return box(tensor(ctx(h), ct(a), ct(b))); }); }
void* orc_relin(void* h, void* a) { return guard_ptr([&] { return box(relin(ctx(h), ct(a))); }); }
void* orc_modswitch(void* h, void* a, int drop) {
  return guard_ptr([&] { return box(modswitch(ctx(h), ct(a), drop)); });
}
void* orc_rotate(void* h, void* a, int g) { return guard_ptr([&] { return box(rotate(ctx(h), ct(a), g)); }); }
void* orc_divide_by_p(void* h, void* a) { return guard_ptr([&] { return box(divide_by_p(ctx(h), ct(a))); }); }
void* orc_relin_drop(void* h, void* a) { return guard_ptr([&] { return box(relin_drop(ctx(h), ct(a))); }); }
void* orc_mul(void* h, void* a, void* b) { return guard_ptr([&] { return box(mul(ctx(h), ct(a), ct(b))); }); }
void* orc_set_t_exp(void* h, void* a, int t_exp) {
  return guard_ptr([&] { Ct x = ct(a); x.t_exp = t_exp; (void)h; return box(std::move(x)); });
}

// ------------------------------------------------------- space switching
void* orc_eval_g(void* h, void* x, int e) {
  return guard_ptr([&] { return box(eval_g(ctx(h), ct(x), e, trace(h))); });
}

int orc_reduce(void* h, void* a, void** out) {
  return guard([&] {
    auto d = reduce_to_digits(ctx(h), ct(a), trace(h));
    for (size_t i = 0; i < d.size(); ++i) out[i] = box(std::move(d[i]));
  });
}

void* orc_compare_lt(void* h, void* a, void* b) {
  return guard_ptr([&] { return box(compare_lt(ctx(h), ct(a), ct(b), trace(h))); });
}

void* orc_compare(void* h, int pred, void* a, void* b) {
  return guard_ptr([&] { return box(compare(ctx(h), pred, ct(a), ct(b), trace(h))); });
}

// conds: n_cond (pred, X[n], Y[ny]) triples flattened: preds[k], X[k*n + i], Y[k*n + i] (ny[k] = 1 or n)
void* orc_query_where(void* h, void** A, void** B, int n, int n_cond, const int* preds, void** X, void** Y,
                      const int* ny) {
  return guard_ptr([&] {
    std::vector<Ct> a, b;
    for (int i = 0; i < n; ++i) { a.push_back(ct(A[i])); b.push_back(ct(B[i])); }
    std::vector<Cond> conds;
    for (int k = 0; k < n_cond; ++k) {
      Cond c;
      c.pred = preds[k];
      for (int i = 0; i < n; ++i) c.X.push_back(ct(X[(size_t)k * n + i]));
      for (int i = 0; i < ny[k]; ++i) c.Y.push_back(ct(Y[(size_t)k * n + i]));
      conds.push_back(std::move(c));
    }
    return box(query_sum_where(ctx(h), a, b, conds, trace(h)));
  });
}

void* orc_raise(void* h, void* a) { return guard_ptr([&] { return box(raise_modulus(ctx(h), ct(a), trace(h))); }); }

void* orc_rotate_sum(void* h, void* a) { return guard_ptr([&] { return box(rotate_sum(ctx(h), ct(a), trace(h))); }); }

void* orc_query(void* h, void** A, void** B, void** C1, void** C2, int n, int n2) {
  return guard_ptr([&] {
    std::vector<Ct> a, b, c1, c2;
    for (int i = 0; i < n; ++i) { a.push_back(ct(A[i])); b.push_back(ct(B[i])); c1.push_back(ct(C1[i])); }
    for (int i = 0; i < n2; ++i) c2.push_back(ct(C2[i]));
    return box(query_sum_where_lt(ctx(h), a, b, c1, c2, trace(h)));
  });
}

// Worker threads of the reference's parallel loops (0: one per hardware
// thread); returns the count in use.
int orc_set_threads(int n) {
  if (n >= 0) set_threads(n);
  return threads();
}

unsigned long long orc_ntt_count(int reset) {
  unsigned long long v = g_ntt_count;
  if (reset) g_ntt_count = 0;
  return v;
}

int orc_trace(void* h, int on) {
  Trace* t = trace(h);
  t->on = on != 0;
  t->ops.clear();
  return 0;
}

int orc_meter(void* h, int on) {
  Trace* t = trace(h);
  t->meter = on != 0;
  t->noise.clear();
  return 0;
}

// Copies the noise-meter lines (one per stage) into buf; returns the full length.
int orc_meter_get(void* h, char* buf, int len) {
  std::string s;
  for (auto& o : trace(h)->noise) { s += o; s += '\n'; }
  if (buf && len > 0) {
    int n = (int)std::min<size_t>(s.size(), (size_t)len - 1);
    std::memcpy(buf, s.data(), n);
    buf[n] = 0;
  }
  return (int)s.size();
}

// Copies the trace (one op per line) into buf; returns the full length.
int orc_trace_get(void* h, char* buf, int len) {
  std::string s;
  for (auto& o : trace(h)->ops) { s += o; s += '\n'; }
  if (buf && len > 0) {
    int n = (int)std::min<size_t>(s.size(), (size_t)len - 1);
    std::memcpy(buf, s.data(), n);
    buf[n] = 0;
  }
  return (int)s.size();
}

}  // extern "C"
