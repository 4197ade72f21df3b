// BGV operations on device-resident ciphertext batches: secret-key encryption
// (Algorithm 1), decryption (Algorithm 2), key generation, hybrid key switching
// (ModUp -> inner product -> ModDown), relinearisation, modulus switching and
// automorphisms. Each step is a kernel launch on the caller's stream; scratch
// comes from the stream-ordered pool.
#include <algorithm>
#include <cstring>

#include "philox.h"
#include "ss_internal.h"

namespace ss {

// ------------------------------------------------------------------ memory
void* pool_alloc(size_t bytes, cudaStream_t s) {
  void* p = nullptr;
  if (bytes == 0) return nullptr;
  cudaError_t e = cudaMallocAsync(&p, bytes, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error(SS_ERR_OOM, std::string("device pool allocation failed: ") + cudaGetErrorString(e));
  }
  return p;
}

void pool_free(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

Buf::~Buf() {
  if (owned && data) pool_free(data, stream);
}

BufP alloc_buf(Context& C, int count, int ncomp, int level, int t_exp, cudaStream_t s) {
  auto b = std::make_shared<Buf>();
  b->count = count;
  b->ncomp = ncomp;
  b->level = level;
  b->t_exp = t_exp;
  b->cap = level;
  b->stream = s;
  b->bytes = (size_t)count * ncomp * level * C.N * sizeof(u64);
  if (!is_dry(C)) {
    b->data = static_cast<u64*>(pool_alloc(b->bytes, s));
    b->owned = true;
  }
  return b;
}

BufP view_buf(const ss_ct& c) {
  auto b = std::make_shared<Buf>();
  b->data = c.data;
  b->count = c.count;
  b->ncomp = c.ncomp;
  b->level = c.level;
  b->t_exp = c.t_exp;
  b->cap = c.capacity;
  b->owned = false;
  return b;
}

BufP slice_buf(const BufP& a, int b0, int count, int N) {
  auto b = std::make_shared<Buf>(*a);
  b->owned = false;
  b->parent = a;
  b->count = count;
  if (a->data) b->data = a->data + (size_t)b0 * a->ncomp * a->cap * N;
  return b;
}

// ------------------------------------------------------------------ key switching
// On X^N + 1 a base conversion whose output is transformed forward next (the
// ModUp digits, the ModDown and modulus-switch corrections) multiplies the
// upper half of every output limb by the forward transform's node-1 twiddle
// psi^(N/2), so the transform's first stage needs no product (one Shoup
// product per word pair of the first stage saved; the words are unchanged).
// Other rings split node 1; below N = 1024 a base-conversion block would
// straddle the two halves.
static bool bconv_folds_w1(const Context& C) { return C.m_odd == 1 && C.N >= 1024; }
// Likewise an inverse transform whose output only feeds a base conversion (the
// ModUp digit source, the ModDown and modulus-switch dropped limbs) leaves its
// last stage's N^-1 and N^-1 psi^(-N/2) to the base conversion's per-source
// constants (PolySet::post_scale): that stage runs without products. Two-phase
// transforms only (N > 4096).
static bool bconv_folds_inverse(const Context& C) { return bconv_folds_w1(C) && C.N > 4096; }
static PolySet scaled_later(PolySet s, bool post) {
  s.post_scale = post;
  return s;
}

// out.comp0 = addend.comp0 + KS(in.comp)[0]; out.comp1 = (addend ? addend.comp1 : 0) + KS[1]
// addend_comp1 selects whether the addend's component 1 is added too.
static void keyswitch_impl(Context& C, const Buf& in, int comp, const KeyDev& K, const Buf* addend, bool add_c1,
                           Buf& out, cudaStream_t st) {
  const int N = C.N, l = in.level, B = in.count, a = C.alpha;
  const int dn = (l + a - 1) / a, nx = l + a;
  const long in_os = (long)in.ncomp * in.cap * N;
  const u64* d = in.data + (size_t)comp * in.cap * N;
  // 1. coefficient form of the digit source (read in place, written to dc)
  u64* dc = static_cast<u64*>(pool_alloc((size_t)B * l * N * 8, st));
  const bool post = bconv_folds_inverse(C);
  ntt_inverse_from(C, scaled_later(PolySet{dc, (long)l * N, B, l, 0, l}, post), d, in_os, st);
  // 2. ModUp of every digit to the other data primes and the special primes
  //    (X^N + 1: the base conversion also applies the transform's first twiddle)
  const long ext_os = (long)dn * nx * N;
  u64* ext = static_cast<u64*>(pool_alloc((size_t)B * ext_os * 8, st));
  const bool pre = bconv_folds_w1(C);
  for (int j = 0; j < dn; ++j) {
    int lo = j * a, hi = std::min(lo + a, l);
    size_t off = C.off_modup.at({j, hi});
    const u64* c1 = C.d_tables + off;
    const u64* c2 = c1 + 2 * (hi - lo);
    k_bconv(C, dc + (size_t)lo * N, (long)l * N, hi - lo, lo, c1, c2, ext + (size_t)j * nx * N, ext_os, nx, l, lo,
            hi, nullptr, B, st, -1, pre, post);
  }
  PolySet ps{ext, (long)nx * N, B * dn, nx, 0, l};
  ps.skip_w = a;
  ps.skip_mod = dn;
  ps.skip_level = l;
  ps.pre_w1 = pre;
  ntt_forward(C, ps, st);
  pool_free(dc, st);
  // 3. inner product with the key on the special primes (both components)
  const long sp_os = 2L * a * N;
  u64* acc = static_cast<u64*>(pool_alloc((size_t)B * sp_os * 8, st));
  k_ks_ip(C, d, in_os, ext, ext_os, K, l, acc, sp_os, B, st, l, a);
  // 4. ModDown: delta = t * conv_P->Q(t^-1 acc mod P) on the data primes
  ntt_inverse(C, scaled_later(PolySet{acc, (long)a * N, 2 * B, a, C.L, 0}, post), st);
  u64* delta = static_cast<u64*>(pool_alloc((size_t)2 * B * l * N * 8, st));
  const u64* c1 = C.d_tables + C.off_md_c1[in.t_exp];
  const u64* c2 = C.d_tables + C.off_md_c2;
  const u64* tpost = C.d_tmod + (size_t)in.t_exp * C.ntot * 2;
  k_bconv(C, acc, (long)a * N, a, C.L, c1, c2, delta, (long)l * N, l, l, 0, 0, tpost, 2 * B, st, -1, pre, post);
  PolySet pd{delta, (long)l * N, 2 * B, l, 0, l};
  pd.pre_w1 = pre;
  ntt_forward(C, pd, st);
  pool_free(acc, st);
  // 5. inner product on the data primes fused with out = (acc - delta) P^-1 (+ addend)
  const u64* pinv = C.d_tables + C.off_md_pinv;
  k_ks_ip_fused(C, d, in_os, ext, ext_os, K, l, l, false, addend, add_c1, delta, l, nullptr, pinv, out, B, st);
  pool_free(ext, st);
  pool_free(delta, st);
}

void op_keyswitch(Context& C, const Buf& in, int comp, const KeyDev& K, const Buf* addend, Buf& out,
                  cudaStream_t st) {
  keyswitch_impl(C, in, comp, K, addend, true, out, st);
}

void op_relin(Context& C, const Buf& a, Buf& out, cudaStream_t st) {
  if (a.ncomp != 3) throw Error(SS_ERR_SHAPE, "relinearisation needs a 3-component ciphertext");
  if (!C.have_keys) throw Error(SS_ERR_PARAM, "no keys");
  out.ncomp = 2;
  out.level = a.level;
  out.t_exp = a.t_exp;
  keyswitch_impl(C, a, 2, C.rlk, &a, true, out, st);
}

// Relinearise and drop the last prime in one ModDown: after the key-switch
// inner product acc (over Q_l and P), the extended ciphertext is P*d_c + acc_c;
// with D = {q_{l-1}} and the special primes (contiguous in acc: limbs l-1 ..
// l+alpha-1), out_c = ((P d_c + acc_c) - t conv([t^{-1}(P d_c + acc_c)]_D)) /
// (q_{l-1} P) on the first l-1 primes.
void op_relin_drop(Context& C, const Buf& in, Buf& out, cudaStream_t st) {
  if (in.ncomp != 3) throw Error(SS_ERR_SHAPE, "relinearisation needs a 3-component ciphertext");
  if (!C.have_keys) throw Error(SS_ERR_PARAM, "no keys");
  const int N = C.N, l = in.level, B = in.count, a = C.alpha;
  if (l < 2) throw Error(SS_ERR_LEVEL, "no prime left to drop");
  const int dn = (l + a - 1) / a, nx = l + a, nl = l - 1;
  out.ncomp = 2;
  out.level = nl;
  out.t_exp = in.t_exp;
  const long in_os = (long)in.ncomp * in.cap * N;
  const u64* d = in.data + (size_t)2 * in.cap * N;
  // 1-3: ModUp and inner product, as in keyswitch_impl
  u64* dc = static_cast<u64*>(pool_alloc((size_t)B * l * N * 8, st));
  const bool post = bconv_folds_inverse(C);
  ntt_inverse_from(C, scaled_later(PolySet{dc, (long)l * N, B, l, 0, l}, post), d, in_os, st);
  const long ext_os = (long)dn * nx * N;
  u64* ext = static_cast<u64*>(pool_alloc((size_t)B * ext_os * 8, st));
  const bool pre = bconv_folds_w1(C);
  for (int j = 0; j < dn; ++j) {
    int lo = j * a, hi = std::min(lo + a, l);
    const u64* c1 = C.d_tables + C.off_modup.at({j, hi});
    const u64* c2 = c1 + 2 * (hi - lo);
    k_bconv(C, dc + (size_t)lo * N, (long)l * N, hi - lo, lo, c1, c2, ext + (size_t)j * nx * N, ext_os, nx, l, lo,
            hi, nullptr, B, st, -1, pre, post);
  }
  PolySet ps{ext, (long)nx * N, B * dn, nx, 0, l};
  ps.skip_w = a;
  ps.skip_mod = dn;
  ps.skip_level = l;
  ps.pre_w1 = pre;
  ntt_forward(C, ps, st);
  pool_free(dc, st);
  // 3. inner product on q_{l-1} and the special primes (the limbs the ModDown drops)
  const int ns = a + 1;
  const long sp_os = 2L * ns * N;
  u64* acc = static_cast<u64*>(pool_alloc((size_t)B * sp_os * 8, st));
  k_ks_ip(C, d, in_os, ext, ext_os, C.rlk, l, acc, sp_os, B, st, l - 1, ns);
  // 4. ModDown by q_{l-1} P: delta = t conv([t^-1 (P d + acc)]_D) on the first l-1 primes
  const u64* pmod = C.d_tables + C.off_pmod;
  k_fixup_last(C, acc, sp_os, ns, 0, in, l, pmod, B, st);
  ntt_inverse(C, scaled_later(PolySet{acc, (long)ns * N, 2 * B, ns, l - 1, 1}, post), st);
  u64* delta = static_cast<u64*>(pool_alloc((size_t)2 * B * nl * N * 8, st));
  const u64* c2 = C.d_tables + C.off_rd[l];
  const u64* inv = c2 + (size_t)(a + 1) * C.ntot;
  const u64* c1 = C.d_tables + C.off_rd_c1.at({l, in.t_exp});
  const u64* tpost = C.d_tmod + (size_t)in.t_exp * C.ntot * 2;
  k_bconv(C, acc, (long)ns * N, ns, l - 1, c1, c2, delta, (long)nl * N, nl, nl, 0, 0, tpost, 2 * B, st, 1, pre, post);
  PolySet pd{delta, (long)nl * N, 2 * B, nl, 0, nl};
  pd.pre_w1 = pre;
  ntt_forward(C, pd, st);
  pool_free(acc, st);
  // 5. inner product on the kept primes fused with the combine
  //    out_c = ((P d_c + acc_c) - delta_c) (q_{l-1} P)^-1
  k_ks_ip_fused(C, d, in_os, ext, ext_os, C.rlk, l, nl, true, &in, true, delta, nl, pmod, inv, out, B, st);
  pool_free(ext, st);
  pool_free(delta, st);
}

void op_modswitch(Context& C, const Buf& a, int k, Buf& out, cudaStream_t st) {
  const int N = C.N, l = a.level, nl = l - k, B = a.count, nc = a.ncomp;
  if (k <= 0) throw Error(SS_ERR_PARAM, "modswitch drop must be positive");
  if (nl < 1) throw Error(SS_ERR_LEVEL, "modswitch below one prime");
  out.ncomp = nc;
  out.level = nl;
  out.t_exp = a.t_exp;
  u64* x = static_cast<u64*>(pool_alloc((size_t)B * nc * k * N * 8, st));
  SS_CUDA(cudaMemcpy2DAsync(x, (size_t)k * N * 8, a.data + (size_t)nl * N, (size_t)a.cap * N * 8, (size_t)k * N * 8,
                            (size_t)B * nc, cudaMemcpyDeviceToDevice, st));
  const bool pre = bconv_folds_w1(C), post = bconv_folds_inverse(C);
  ntt_inverse(C, scaled_later(PolySet{x, (long)k * N, B * nc, k, nl, k}, post), st);
  u64* delta = static_cast<u64*>(pool_alloc((size_t)B * nc * nl * N * 8, st));
  size_t off = C.off_ms.at({l, k});
  const u64* c2 = C.d_tables + off;
  const u64* qinv = c2 + (size_t)k * C.ntot;
  const u64* c1 = C.d_tables + C.off_ms_c1.at(std::make_tuple(l, k, a.t_exp));
  const u64* tpost = C.d_tmod + (size_t)a.t_exp * C.ntot * 2;
  k_bconv(C, x, (long)k * N, k, nl, c1, c2, delta, (long)nl * N, nl, nl, 0, 0, tpost, B * nc, st, -1, pre, post);
  PolySet pd{delta, (long)nl * N, B * nc, nl, 0, nl};
  pd.pre_w1 = pre;
  ntt_forward(C, pd, st);
  k_sub_scale(C, a.data, (long)a.cap * N, delta, (long)nl * N, qinv, nullptr, 0, out.data, (long)out.cap * N, nl,
              B * nc, st);
  pool_free(x, st);
  pool_free(delta, st);
}

void op_rotate(Context& C, const Buf& a, int g, Buf& out, cudaStream_t st) {
  if (a.ncomp != 2) throw Error(SS_ERR_SHAPE, "rotation needs a 2-component ciphertext");
  auto it = C.gk.find(g);
  if (it == C.gk.end()) throw Error(SS_ERR_PARAM, "no Galois key for this element");
  BufP s = alloc_buf(C, a.count, 2, a.level, a.t_exp, st);
  k_automorph(C, a, g, *s, st);
  out.ncomp = 2;
  out.level = a.level;
  out.t_exp = a.t_exp;
  keyswitch_impl(C, *s, 1, it->second, s.get(), false, out, st);
}

// ------------------------------------------------------------------ encryption
void op_encrypt(Context& C, const u64* m, int B, u32 nonce0, int t_exp, Buf& out, cudaStream_t st) {
  if (!C.have_keys) throw Error(SS_ERR_PARAM, "no keys");
  if (t_exp < 1 || t_exp > C.r) throw Error(SS_ERR_TMOD, "bad t_exp");
  const int N = C.N, L = C.L;
  if (out.cap < L) throw Error(SS_ERR_SHAPE, "output capacity below L");
  out.ncomp = 2;
  out.level = L;
  out.t_exp = t_exp;
  const long os = 2L * out.cap * N;
  u64* c0 = out.data;
  u64* c1 = out.data + (size_t)out.cap * N;
  k_uniform(C, c1, os, B, L, 0, L, nonce0, TAG_ENC_A, st);
  i64* e = static_cast<i64*>(pool_alloc((size_t)B * N * 8, st));
  k_cbd(C, e, B, nonce0, TAG_ENC_E, st);
  k_lift_small(C, e, m, C.tpow[t_exp], c0, os, B, L, 0, L, st);
  ntt_forward(C, PolySet{c0, os, B, L, 0, L}, st);
  k_mul_sub(C, c0, os, c1, os, C.d_sk, c0, os, B, L, 0, L, 0, st);
  pool_free(e, st);
}

void op_decrypt(Context& C, const Buf& a, u64* d_out, cudaStream_t st) {
  if (!C.have_keys) throw Error(SS_ERR_PARAM, "no keys");
  const int N = C.N, l = a.level, B = a.count;
  u64* v = static_cast<u64*>(pool_alloc((size_t)B * l * N * 8, st));
  k_dec_dot(C, a, v, st);
  ntt_inverse(C, PolySet{v, (long)l * N, B, l, 0, l}, st);
  SS_CUDA(cudaMemsetAsync(d_out, 0, (size_t)B * N * 8, st));
  k_crt(C, v, B, l, a.t_exp, d_out, st);
  pool_free(v, st);
}

// ------------------------------------------------------------------ keys
static std::vector<i64> sample_secret(const Context& C) {
  const int N = C.N;
  std::vector<int> idx(N);
  for (int i = 0; i < N; ++i) idx[i] = i;
  std::vector<i64> s(N, 0);
  u32 k0 = (u32)(C.prm.seed & 0xffffffffu), k1 = (u32)(C.prm.seed >> 32);
  for (int i = 0; i < C.prm.h; ++i) {
    Philox4 r = philox((u32)i, 0u, 0u, TAG_SK, k0, k1);
    u64 w = ((u64)r.x[1] << 32) | r.x[0];
    int j = i + (int)(w % (u64)(N - i));
    std::swap(idx[i], idx[j]);
    s[idx[i]] = (r.x[2] & 1u) ? -1 : 1;
  }
  return s;
}

static void make_ksk(Context& C, const u64* sprime, u32 key_id, KeyDev& K, cudaStream_t st) {
  const int N = C.N, T = C.ntot, dn = C.dnum;
  size_t words = (size_t)dn * T * N;
  SS_CUDA(cudaMalloc(&K.a, words * 8));
  SS_CUDA(cudaMalloc(&K.b, words * 8));
  i64* e = static_cast<i64*>(pool_alloc((size_t)N * 8, st));
  for (int j = 0; j < dn; ++j) {
    u32 id = key_id * 256u + (u32)j;
    u64* a = K.a + (size_t)j * T * N;
    u64* b = K.b + (size_t)j * T * N;
    k_uniform(C, a, 0, 1, T, 0, T, id, TAG_KSK_A, st);
    k_cbd(C, e, 1, id, TAG_KSK_E, st);
    k_lift_small(C, e, nullptr, C.t, b, 0, 1, T, 0, T, st);
    ntt_forward(C, PolySet{b, 0, 1, T, 0, T}, st);
    k_mul_sub(C, b, 0, a, 0, C.d_sk, b, 0, 1, T, 0, T, 0, st);
    k_ksk_gadget(C, K.b, sprime, j, st);
  }
  k_to_montgomery(C, K.a, dn * T, st);
  k_to_montgomery(C, K.b, dn * T, st);
  pool_free(e, st);
}

void op_keygen(Context& C, const std::vector<int>& galois) {
  cudaStream_t st = nullptr;
  const int N = C.N, T = C.ntot;
  for (int g : galois)
    if (g <= 0 || g >= C.m || g % 2 == 0 || (C.m_odd > 1 && g % C.m_odd == 0))
      throw Error(SS_ERR_PARAM, "Galois element must be a unit in (0, m)");
  C.sk = sample_secret(C);
  // s in evaluation form on every prime
  std::vector<u64> sc((size_t)T * N);
  for (int i = 0; i < T; ++i)
    for (int n = 0; n < N; ++n) sc[(size_t)i * N + n] = nt::lift(C.sk[n], C.primes[i]);
  cudaFree(C.d_sk);
  cudaFree(C.d_sk2);
  SS_CUDA(cudaMalloc(&C.d_sk, sc.size() * 8));
  SS_CUDA(cudaMalloc(&C.d_sk2, sc.size() * 8));
  SS_CUDA(cudaMemcpy(C.d_sk, sc.data(), sc.size() * 8, cudaMemcpyHostToDevice));
  ntt_forward(C, PolySet{C.d_sk, 0, 1, T, 0, T}, st);
  k_square(C, C.d_sk, C.d_sk2, T, st);
  cudaFree(C.rlk.a);
  cudaFree(C.rlk.b);
  for (auto& kv : C.gk) { cudaFree(kv.second.a); cudaFree(kv.second.b); }
  C.gk.clear();
  make_ksk(C, C.d_sk2, 0, C.rlk, st);
  Buf sview;
  sview.data = C.d_sk;
  sview.count = 1;
  sview.ncomp = 1;
  sview.level = T;
  sview.cap = T;
  for (int g : galois) {
    if (C.gk.count(g)) continue;
    u64* sg = static_cast<u64*>(pool_alloc((size_t)T * N * 8, st));
    Buf o = sview;
    o.data = sg;
    k_automorph(C, sview, g, o, st);
    make_ksk(C, sg, (u32)g, C.gk[g], st);
    pool_free(sg, st);
  }
  SS_CUDA(cudaStreamSynchronize(st));
  C.have_keys = true;
}

}  // namespace ss

namespace ss {

// ------------------------------------------------------------------ kernel timing
static cudaEvent_t kt_event(Context& C) {
  if (!C.kt.pool.empty()) {
    cudaEvent_t e = C.kt.pool.back();
    C.kt.pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  SS_CUDA(cudaEventCreate(&e));
  return e;
}

int kt_begin(Context& C, cudaStream_t st) {
  if (!C.kt.on || ntt_merger()) return -1;  // no per-launch timing in the batched form's lanes
  KTimer::Rec r;
  r.a = kt_event(C);
  r.b = kt_event(C);
  r.cls = 0;
  r.bytes = 0;
  SS_CUDA(cudaEventRecord(r.a, st));
  C.kt.recs.push_back(r);
  return (int)C.kt.recs.size() - 1;
}

void kt_end(Context& C, int rec, int cls, double bytes, cudaStream_t st) {
  if (rec < 0) return;
  KTimer::Rec& r = C.kt.recs[rec];
  r.cls = cls;
  r.bytes = bytes;
  SS_CUDA(cudaEventRecord(r.b, st));
  if (C.kt.recs.size() > 4096) kt_collect(C);
}

int stage_begin(Context& C, int stage, cudaStream_t st) {
  if (!C.kt.on || is_dry(C)) return -1;
  KTimer::SRec r;
  r.a = kt_event(C);
  r.b = kt_event(C);
  r.stage = stage;
  r.closed = false;
  SS_CUDA(cudaEventRecord(r.a, st));
  C.kt.srecs.push_back(r);
  return (int)C.kt.srecs.size() - 1;
}

void stage_end(Context& C, int rec, cudaStream_t st) noexcept {
  if (rec < 0 || rec >= (int)C.kt.srecs.size()) return;
  if (cudaEventRecord(C.kt.srecs[rec].b, st) == cudaSuccess) C.kt.srecs[rec].closed = true;
}

// Stage records are folded in only when none is still open (a stage scope
// keeps its index until it closes).
static void stage_collect(Context& C) {
  for (auto& r : C.kt.srecs)
    if (!r.closed) return;
  for (auto& r : C.kt.srecs) {
    SS_CUDA(cudaEventSynchronize(r.b));
    float ms = 0;
    SS_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
    C.kt.st_count[r.stage] += 1;
    C.kt.st_ms[r.stage] += ms;
    C.kt.pool.push_back(r.a);
    C.kt.pool.push_back(r.b);
  }
  C.kt.srecs.clear();
}

void kt_collect(Context& C) {
  stage_collect(C);
  if (C.kt.recs.empty()) return;
  SS_CUDA(cudaEventSynchronize(C.kt.recs.back().b));
  for (auto& r : C.kt.recs) {
    float ms = 0;
    SS_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
    C.kt.launches[r.cls] += 1;
    C.kt.ms[r.cls] += ms;
    C.kt.bytes[r.cls] += r.bytes;
    C.kt.pool.push_back(r.a);
    C.kt.pool.push_back(r.b);
  }
  C.kt.recs.clear();
}

}  // namespace ss
