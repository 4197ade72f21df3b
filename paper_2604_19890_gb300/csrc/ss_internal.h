// Internal declarations of the GB300 space-switching library.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/ss.h"

namespace ss {

typedef uint64_t u64;
typedef int64_t i64;
typedef uint32_t u32;

struct Error : std::runtime_error {
  ss_status code;
  Error(ss_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define SS_CUDA(x)                                                                          \
  do {                                                                                      \
    cudaError_t e_ = (x);                                                                   \
    if (e_ != cudaSuccess)                                                                  \
      throw ::ss::Error(e_ == cudaErrorMemoryAllocation ? SS_ERR_OOM : SS_ERR_CUDA,         \
                        std::string(#x) + ": " + cudaGetErrorString(e_));                   \
  } while (0)

// ------------------------------------------------------------ host number theory
namespace nt {
u64 mul(u64 a, u64 b, u64 m);
u64 pow(u64 a, u64 e, u64 m);
u64 inv(u64 a, u64 m);
u64 lift(i64 c, u64 m);
bool prime(u64 n);
u64 shoup(u64 w, u64 q);  // floor(w * 2^64 / q)
int brv(int x, int logn);
std::vector<u64> chain(int bits, u64 step, int count);
u64 root2n(u64 q, int N);
std::vector<i64> g_coeffs(int p, int e);  // centred mod p^e, odd, degree (e-1)(p-1)+1
std::vector<i64> g_coeffs_reduced(int p, int e);  // equivalent, least sum of |coefficients| (e = 2, 3)
std::vector<i64> flt_coeffs(int p);       // centred mod p
}  // namespace nt

// Modulus descriptor shared with device code (layout matches Modulus in modarith.cuh)
struct ModDesc {
  u64 q, mu;
  int kbits, pad;
  u64 qinv;  // -q^-1 mod 2^64
};

// A batch of ciphertexts with one shape; either a view of caller memory or a
// pool allocation released on the owning stream.
struct Buf {
  u64* data = nullptr;
  int count = 0, ncomp = 0, level = 0, t_exp = 0, cap = 0;
  size_t bytes = 0;
  cudaStream_t stream = nullptr;
  bool owned = false;
  std::shared_ptr<Buf> parent;  // keeps the allocation of a slice alive
  ~Buf();
  u64* limb(int b, int c, int i, int N) const { return data + ((size_t)(b * ncomp + c) * cap + i) * N; }
};
typedef std::shared_ptr<Buf> BufP;

// Key-switching key, stored in Montgomery form (every word times 2^64 mod its
// prime) for the inner product's Montgomery reduction.
struct KeyDev {
  u64* b = nullptr;  // [dnum][L+alpha][N]
  u64* a = nullptr;
};

// Kernel classes for the optional per-launch timing (CUDA events on the
// launching stream) and their algorithmic byte counts.
enum KClass { KC_NTT = 0, KC_BCONV, KC_KSIP, KC_TENSOR, KC_SUBSCALE, KC_AUTOMORPH, KC_ELEM, KC_SAMPLE, KC_N };

// Stages of the query for the per-stage breakdown (Section 5's runtime
// breakdown of LT: reduction, comparison, aggregation, modulus raising; plus
// the masked product and the SUM).
enum Stage { ST_REDUCE = 0, ST_COMPARE, ST_AGGREGATE, ST_RAISE, ST_PRODUCT, ST_SUM, ST_N };

struct KTimer {
  bool on = false;
  struct Rec {
    cudaEvent_t a, b;
    int cls;
    double bytes;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  unsigned long long launches[KC_N] = {};
  double ms[KC_N] = {}, bytes[KC_N] = {};
  double ntt_products = 0;  // Shoup products of the timed transforms (ss_ntt_products)
  struct SRec {
    cudaEvent_t a, b;
    int stage;
    bool closed;
  };
  std::vector<SRec> srecs;
  unsigned long long st_count[ST_N] = {};
  double st_ms[ST_N] = {};
};

#ifndef SS_NTT_TILE_LOG
#define SS_NTT_TILE_LOG 11
#endif

struct Context {
  ss_params prm;
  int N = 0, logN = 0, L = 0, alpha = 0, ntot = 0, dnum = 0;
  int p = 0, r = 0;
  u64 t = 0;  // p^r
  std::vector<u64> tpow;  // p^e, e = 0..r
  std::vector<u64> primes, psi;  // psi: primitive m-th root of unity per prime
  int m_odd = 1, m = 0;           // odd part of the cyclotomic index; m = 2N (m_odd 1), 3N (3) or 5N/2 (5)
  int slots = 0, d = 0;
  u64 omega = 0;
  std::vector<int> slot_exp;
  // decryption reconstructs, and decoding reads, the coefficients k * dec_stride, k < dec_count
  int dec_stride = 0, dec_count = 0;
  // m = 3N slot algebra: Phi_3N(X) = Phi_M'(X^s), roots theta^e in GR(p^r, 2) = Z_{p^r}[u]/(u^2 - gr_c)
  int Mp = 0, s_stride = 0, nprime = 0;
  u64 gr_c = 0, theta[2] = {0, 0};
  // m = 5N/2: Phi_m(X) = Phi_M'(X^s), M' = 5*2^b', roots theta4 in GR(p^r, 4) = GR(p^r, 2)[v]/(v^2 - gr_w)
  u64 gr_w[2] = {0, 0}, theta4[4] = {0, 0, 0, 0};
  std::vector<std::pair<int, int>> gens;  // slot-group generators mod M' with their orders

  // device tables
  ModDesc* d_mod = nullptr;           // [ntot]
  u64* d_tw = nullptr;                // per prime 4N words: (psi_brv, shoup) pairs, then (psiinv_brv, shoup) pairs
  u64* d_r64 = nullptr;               // [ntot][4] 2^64 mod q; X^N + 1: 2^64 psi^(N/2) (forward node 1),
                                      //   2^64 N^-1, 2^64 N^-1 psi^(-N/2) (the inverse's last stage)
  u64* d_ninv = nullptr;              // [ntot][4] N^{-1}, shoup, N^{-1} psi^{-N/2} (m = 3N: 2 N^{-1}), shoup
  u64* d_split = nullptr;             // m = 5N/2: [ntot][12][2] four-way split constants (forward 5, inverse 7)
  u64* d_pinv = nullptr;              // [ntot][2] p^{-1}, shoup
  u64* d_tmod = nullptr;              // [r+1][ntot][2]: p^e mod q, shoup
  u64* d_tables = nullptr;            // base-conversion constants (offsets below)
  size_t tables_words = 0;
  // ModUp: key (j, e) -> offset of c1[k], c1s[k], c2[k][ntot]
  std::map<std::pair<int, int>, size_t> off_modup;
  // ModDown: t_exp -> offset of c1[alpha], c1s[alpha]; c2 [alpha][ntot]; Pinv[ntot][2]
  std::vector<size_t> off_md_c1;
  size_t off_md_c2 = 0, off_md_pinv = 0;
  // relinearise-and-drop: level -> offset of c2[alpha+1][ntot], inv[ntot][2]; (level, t_exp) -> c1;
  // P mod q per data prime [ntot][2]
  std::vector<size_t> off_rd;
  std::map<std::pair<int, int>, size_t> off_rd_c1;
  size_t off_pmod = 0;
  // modswitch: (level, k) -> offset of c2[k][ntot], Qinv[ntot][2]; (level,k,t_exp) -> c1
  std::map<std::pair<int, int>, size_t> off_ms;
  std::map<std::tuple<int, int, int>, size_t> off_ms_c1;
  // decryption CRT: inv of prefix products, per-level half-Q digits, prefix mod t
  u64* d_crt = nullptr;
  std::vector<size_t> off_crt_half;  // per level
  size_t off_crt_pinv = 0, off_crt_qmodt = 0;

  // keys
  bool have_keys = false;
  std::vector<i64> sk;
  u64* d_sk = nullptr;  // NTT(s) per prime [ntot][N]
  u64* d_sk2 = nullptr; // NTT(s^2) per prime [ntot][N]
  KeyDev rlk;
  std::map<int, KeyDev> gk;

  // evaluator
  int batch = 8;
  bool reduced_g = false;  // evaluate G_{p,e} with the lattice-reduced coefficients
  int ntt_tile_log = SS_NTT_TILE_LOG;  // words per CTA tile of the two-phase transform: 2^11 or 2^12
  bool trace_on = false;
  std::vector<std::string> trace;
  std::atomic<unsigned long long> launches{0};  // shared by server worker threads
  KTimer kt;

  ~Context();
};

// ------------------------------------------------------------------ memory
BufP alloc_buf(Context& C, int count, int ncomp, int level, int t_exp, cudaStream_t s);
BufP view_buf(const ss_ct& c);
BufP slice_buf(const BufP& a, int b0, int count, int N);
void* pool_alloc(size_t bytes, cudaStream_t s);
void pool_free(void* p, cudaStream_t s);

// ------------------------------------------------------------------ launchers
// Polys (o, i) at base + o*outer_stride + i*N, i < nl; global prime of limb i:
// i < nq ? q0 + i : L + (i - nq). Limbs inside [skip_lo, skip_hi) of digit
// (o % skip_mod) * skip_w .. are skipped when skip_w > 0 (ModUp outputs).
// pre_w1 (forward, ring X^N + 1): the upper half of every polynomial already
// carries the node-1 twiddle psi^(N/2) (the base conversion that wrote it
// applied it), so the first stage adds and subtracts without its product.
// post_scale (inverse, ring X^N + 1, N > 4096): the last stage adds and
// subtracts without its products and leaves N^-1 (lower half) and
// N^-1 psi^(-N/2) (upper half) to the consumer, a base conversion that folds
// them into its per-source constants; the words are then unreduced (< 4q).
struct PolySet {
  u64* base;
  long outer_stride;
  int n_outer, nl, q0, nq;
  int skip_w = 0, skip_mod = 1, skip_level = 0;
  bool pre_w1 = false;
  bool post_scale = false;
};
void ntt_forward(Context& C, const PolySet& s, cudaStream_t st);
void ntt_inverse(Context& C, const PolySet& s, cudaStream_t st);
// Inverse transform of the polynomials at src (same shape as s, outer stride
// src_os) written to s: the first phase reads src, so src is left unchanged.
void ntt_inverse_from(Context& C, const PolySet& s, const u64* src, long src_os, cudaStream_t st);
// Transforms of several contexts (ring dimensions N >= 8192) merged: each
// phase of all of them runs as one persistent launch over their tiles.
struct NttReq {
  Context* C;
  PolySet s;
  const u64* src;  // out-of-place source of an inverse transform, or null
  long src_os;
};
void ntt_multi(const std::vector<NttReq>& reqs, bool fwd, int tile_log, cudaStream_t st);
// Collects the transforms that several cooperating host threads issue (the
// batched form's lanes) and launches them merged. While a thread's hook is
// set, its transforms of rings N >= 8192 go to submit(), which returns once
// the merged launch that includes them is enqueued (ordered after st and
// before st's later work).
struct NttMerger {
  virtual void submit(const NttReq& r, bool fwd, cudaStream_t st) = 0;
  virtual ~NttMerger() {}
};
NttMerger*& ntt_merger();  // this thread's hook (null: launch directly)
// One key-switch inner-product launch, recorded for merging (its argument
// block is private to the kernels' file).
struct KsReq {
  Context* C;
  int nlimbs;
  alignas(16) unsigned char job[256];
};
// Inner products of several lanes (any contexts, levels, epilogues) as
// persistent launches over all their blocks.
void ks_multi(const std::vector<KsReq>& reqs, cudaStream_t st);
struct KsMerger {
  virtual void submit_ks(const KsReq& r, cudaStream_t st) = 0;
  virtual ~KsMerger() {}
};
KsMerger*& ks_merger();  // this thread's hook (null: launch directly)

void k_binary(Context& C, int op, const Buf& a, const Buf& b, Buf& out, cudaStream_t st);  // 0 add, 1 sub
void k_scalar(Context& C, int op, const Buf& a, i64 c, Buf& out, cudaStream_t st);       // 0 mul, 1 add(c0), 2 mul p^-1
void k_copy_limbs(Context& C, const Buf& a, Buf& out, int level, cudaStream_t st);
void k_tensor(Context& C, const Buf& a, const Buf& b, Buf& out, cudaStream_t st);
// sources s < nsq are data primes sp0 + s, the rest special primes L + (s - nsq) (nsq < 0: all sp0 + s)
void k_bconv(Context& C, const u64* src, long src_os, int ns, int sp0, const u64* c1, const u64* c2, u64* dst,
             long dst_os, int nd, int nq, int skip_lo, int skip_hi, const u64* post, int n_outer, cudaStream_t st,
             int nsq = -1, bool pre_w1 = false, bool post_scale = false);
// acc_c[acc_limb] += P * d_c[l-1] (acc: nx limbs per component)
void k_fixup_last(Context& C, u64* acc, long acc_os, int nx, int acc_limb, const Buf& d, int l, const u64* pmod,
                  int B, cudaStream_t st);
void k_sub_scale(Context& C, const u64* a, long a_os, const u64* dl, long d_os, const u64* scale, const u64* add,
                 long add_os, u64* out, long out_os, int nl, int n_outer, cudaStream_t st);
void k_to_montgomery(Context& C, u64* data, int npoly, cudaStream_t st);
// key-switch inner product for the limbs [m0, m0 + nlimbs) of the extended
// basis (nlimbs < 0: to the end); acc holds nlimbs limbs per component
void k_ks_ip(Context& C, const u64* d, long d_os, const u64* ext, long ext_os, const KeyDev& K, int level,
             u64* acc, long acc_os, int n_outer, cudaStream_t st, int m0 = 0, int nlimbs = -1);
// inner product over the data limbs [0, nlimbs) with the ModDown epilogue
// (drop: relinearise-and-drop combine; else subtract, scale by P^-1, add x)
void k_ks_ip_fused(Context& C, const u64* d, long d_os, const u64* ext, long ext_os, const KeyDev& K, int level,
                   int nlimbs, bool drop, const Buf* x, bool add_c1, const u64* delta, int nl, const u64* pm,
                   const u64* scale, Buf& out, int n_outer, cudaStream_t st);
void k_automorph(Context& C, const Buf& a, int g, Buf& out, cudaStream_t st);
void k_uniform(Context& C, u64* out, long out_os, int n_outer, int nl, int q0, int nq, u32 id0, u32 tag,
               cudaStream_t st);
void k_cbd(Context& C, i64* out, int n_outer, u32 id0, u32 tag, cudaStream_t st);
void k_lift_small(Context& C, const i64* e, const u64* m, u64 tmul, u64* out, long out_os, int n_outer, int nl,
                  int q0, int nq, cudaStream_t st);
void k_mul_sub(Context& C, const u64* x, long x_os, const u64* a, long a_os, const u64* s, u64* out, long out_os,
               int n_outer, int nl, int q0, int nq, int s_stride_primes, cudaStream_t st);
void k_dec_dot(Context& C, const Buf& a, u64* out, cudaStream_t st);
void k_crt(Context& C, const u64* v, int count, int level, int t_exp, u64* out, cudaStream_t st);
void k_ksk_gadget(Context& C, u64* b, const u64* sprime, int j, cudaStream_t st);
void k_square(Context& C, const u64* a, u64* out, int nprimes, cudaStream_t st);
void k_batch_sum(Context& C, const Buf& a, Buf& out, cudaStream_t st);
// outs[j] = sum_i cs[j][i] ys[i]; every input read once (all of one shape and level)
void k_lincomb_multi(Context& C, const std::vector<const Buf*>& ys, const std::vector<std::vector<i64>>& cs,
                     const std::vector<Buf*>& outs, cudaStream_t st);
void k_lincomb(Context& C, const std::vector<const Buf*>& ys, const std::vector<i64>& cs, i64 cst, Buf& out,
               cudaStream_t st);

// ------------------------------------------------------------------ operations
void op_encrypt(Context& C, const u64* d_coeffs, int count, u32 nonce0, int t_exp, Buf& out, cudaStream_t st);
void op_decrypt(Context& C, const Buf& a, u64* d_out, cudaStream_t st);
void op_keygen(Context& C, const std::vector<int>& galois);
void op_keyswitch(Context& C, const Buf& in, int comp, const KeyDev& K, const Buf* addend, Buf& out,
                  cudaStream_t st);  // out = addend + KS(in.comp)
void op_relin(Context& C, const Buf& a, Buf& out, cudaStream_t st);
// relinearise a 3-component batch and drop its last prime in one ModDown by q_{l-1} P
void op_relin_drop(Context& C, const Buf& a, Buf& out, cudaStream_t st);
void op_modswitch(Context& C, const Buf& a, int drop, Buf& out, cudaStream_t st);
void op_rotate(Context& C, const Buf& a, int g, Buf& out, cudaStream_t st);
// relinearisation with its scratch in a static device array (allocates nothing)
void op_relin_noalloc(Context& C, const Buf& a, Buf& out, cudaStream_t st);
size_t relin_noalloc_words(const Context& C, int level, int count);
size_t relin_noalloc_capacity();

// evaluator (batched, one plan for every ciphertext of a batch)
BufP ev_modswitch_to(Context& C, const BufP& a, int level, cudaStream_t st);
BufP ev_mul(Context& C, const BufP& a, const BufP& b, cudaStream_t st);
BufP ev_add(Context& C, const BufP& a, const BufP& b, cudaStream_t st);
BufP ev_sub(Context& C, const BufP& a, const BufP& b, cudaStream_t st);
BufP ev_scalar(Context& C, int op, const BufP& a, i64 c, cudaStream_t st);
BufP ev_lincomb(Context& C, const std::vector<std::pair<BufP, i64>>& terms, i64 cst, cudaStream_t st);
BufP ev_eval_g(Context& C, const BufP& x, int e, cudaStream_t st);
std::vector<BufP> ev_reduce(Context& C, const BufP& a, cudaStream_t st);
BufP ev_compare_lt(Context& C, const BufP& a, const BufP& b, cudaStream_t st);
BufP ev_raise(Context& C, const BufP& a, cudaStream_t st);
BufP ev_rotate_sum(Context& C, const BufP& a, cudaStream_t st);
BufP ev_query(Context& C, const BufP& A, const BufP& B, const BufP& C1, const BufP& C2, cudaStream_t st);
BufP ev_compare_eq(Context& C, const BufP& a, const BufP& b, cudaStream_t st);
BufP ev_compare(Context& C, int pred, const BufP& a, const BufP& b, cudaStream_t st);
struct QCond {
  int pred;
  BufP X, Y;  // X[i] pred Y[i]; Y may hold one ciphertext
};
// ab_ready (optional): event after which A and B hold their data; the first
// product waits for it, so their upload can overlap the comparisons.
BufP ev_query_where(Context& C, const BufP& A, const BufP& B, const std::vector<QCond>& conds, cudaStream_t st,
                    cudaEvent_t ab_ready = nullptr);
struct QueryCols {
  BufP A, B, C1, C2;
};
std::vector<BufP> ev_query_multi(Context& C, const std::vector<QueryCols>& qs, cudaStream_t st);
size_t query_bytes_estimate(const Context& C, int n_ct, int level);
// batches of one shape joined along the batch axis (a part of count 1 is repeated)
BufP ev_concat(Context& C, const std::vector<std::pair<BufP, int>>& parts, cudaStream_t st);
int plan_query_depth(Context& C, int level);
std::vector<int> rotate_sum_elements(const Context& C);

// host-side setup
void build_context(Context& C, const ss_params& prm);
std::vector<u64> encode(const Context& C, int t_exp, const u64* slots);
std::vector<u64> decode(const Context& C, int t_exp, const u64* coeffs);

int kt_begin(Context& C, cudaStream_t st);
void kt_end(Context& C, int rec, int cls, double bytes, cudaStream_t st);
void kt_collect(Context& C);
double alu_probe(int kind, int iters);
int stage_begin(Context& C, int stage, cudaStream_t st);
void stage_end(Context& C, int rec, cudaStream_t st) noexcept;
// Times the enclosing scope as one query stage when kernel timing is on.
struct StageScope {
  Context& C;
  int rec;
  cudaStream_t st;
  StageScope(Context& c, int stage, cudaStream_t s) : C(c), rec(stage_begin(c, stage, s)), st(s) {}
  ~StageScope() { stage_end(C, rec, st); }
};

// Plan-only evaluation. While a PlanScope for a context is open on the calling
// thread, the evaluator tracks shapes, levels and plaintext moduli of that
// context's operations but allocates, launches and traces nothing. The state is
// per thread, so planning never affects other threads (server workers) using
// the same context.
bool is_dry(const Context& C);
struct PlanScope {
  const Context* prev;
  explicit PlanScope(const Context& C);
  ~PlanScope();
};
// Runs f as a plan first (an error such as SS_ERR_NOISE is thrown before any
// work is enqueued), then for real.
template <class F>
auto plan_then_run(Context& C, F&& f) -> decltype(f()) {
  {
    PlanScope ps(C);
    f();
  }
  return f();
}

inline void note(Context& C, const std::string& s) {
  if (C.trace_on && !is_dry(C)) C.trace.push_back(s);
}

}  // namespace ss
