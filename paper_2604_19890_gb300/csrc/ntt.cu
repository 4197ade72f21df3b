// NTT / inverse NTT over RNS limbs (Section 2.1 ring arithmetic), for the
// cyclotomic rings X^N + 1 (m = 2N) and X^N - X^(N/2) + 1 (m = 3N).
//
// Forward: merged-twist Cooley-Tukey with twiddles psi^bitrev(m+i); natural
// coefficients in, evaluation form out with word j = a(psi^(2 bitrev(j)+1)).
// Inverse: Gentleman-Sande with psi^-bitrev(m+i), then times N^-1.
// m = 3N: the same trees with node 1 replaced by the split into
// X^(N/2) - rho and X^(N/2) - rho^5 (R3 kernels) and the subtree twiddles of
// those two factors; word h N/2 + j = a(omega^(e_h + 6 bitrev(j))).
//
// A length-N transform is split N = N1 * N2. Its first log2(N1) stages act on
// the N2 columns (stride N2) independently, the remaining log2(N2) stages on
// the N1 contiguous chunks of N2 words. Each phase is one kernel: a CTA
// stages a tile of CPB columns (or chunks) in shared memory (32 KiB), runs
// its stages there with Harvey lazy butterflies (residues in [0, 4q) forward,
// [0, 2q) inverse) and writes the tile back. N <= 4096 runs in one phase.
#include "modarith.cuh"
#include "ss_internal.h"

namespace ss {

namespace {

constexpr int TILE = 4096;  // words per CTA tile (32 KiB of shared memory)

// resident CTAs per SM the radix-16 phases are compiled for (forward, inverse)
#ifndef SS_NTT_PREFETCH
#define SS_NTT_PREFETCH 1  // inverse chunk phase: first-stage twiddles loaded before the staging
#endif
#ifndef SS_NTT_MINB_F
#define SS_NTT_MINB_F 3
#endif
#ifndef SS_NTT_MINB_I
#define SS_NTT_MINB_I 3
#endif
#ifndef SS_NTT_MINB_R5
#define SS_NTT_MINB_R5 3  // m = 5N/2 column phases (the factored split fits the same 80 registers)
#endif

struct NttArgs {
  u64* base;
  long outer_stride;
  int n_outer, nl, q0, nq, L, N;
  int skip_w, skip_mod, skip_level;
  const Modulus* mods;
  const u64* tw;     // per prime 4N words: (w, w') pairs forward, then inverse
  const u64* ninv;   // per prime (N^-1, shoup, N^-1 psi^(-N/2), shoup)
  const u64* split;  // m = 5N/2: per prime 12 (value, shoup) pairs of the four-way split (split4_fwd/inv)
  const u64* src;    // out-of-place first phase: polynomial (o, i) is read at src + o src_os + i N
  long src_os;
  int pre_w1;        // forward, X^N + 1: upper halves already carry psi^(N/2) (PolySet::pre_w1)
  int post_scale;    // inverse, X^N + 1: last stage without its products (PolySet::post_scale)
};

// Blocks walk the polynomials limb-major (all outer copies of limb 0, then of
// limb 1, ...) so consecutive blocks share a prime and its twiddles stay in L2.
__device__ __forceinline__ bool poly_of(const NttArgs& A, int poly, u64*& ptr, int& pidx) {
  int i = poly / A.n_outer, o = poly % A.n_outer;
  if (A.skip_w > 0) {
    int j = o % A.skip_mod;
    int lo = j * A.skip_w, hi = min(lo + A.skip_w, A.skip_level);
    if (i >= lo && i < hi && i < A.nq) return false;
  }
  ptr = A.base + (long)o * A.outer_stride + (long)i * A.N;
  pidx = i < A.nq ? A.q0 + i : A.L + (i - A.nq);
  return true;
}

// Shared-memory word for linear tile index `lin`: one pad word per 8, which
// spreads the strided round accesses over all banks.
__device__ __forceinline__ int swz(int lin) { return lin + (lin >> 3); }

#ifndef SS_NTT_XSWZ
#define SS_NTT_XSWZ 1  // chunk phases of the radix-16 kernels: XOR swizzle instead of the padded one
#endif
// Chunk tiles of the radix-16 kernels: within every aligned group of 16 words
// the low four index bits are XORed with the next four. A half-warp then hits
// 16 distinct bank pairs both when it touches 16 consecutive words (rounds of
// spacing >= 16, the linear staging loops: the XOR is one permutation of the
// group) and when it touches one word of each of 16 consecutive groups
// (rounds of spacing 1: thread B holds words 16B .. 16B+15), where the padded
// swizzle left two threads on each bank pair. It needs no padding.
template <bool COLS>
__device__ __forceinline__ int swz16(int lin) {
  if (COLS || !SS_NTT_XSWZ) return swz(lin);
  return lin ^ ((lin >> 4) & 15);
}

// v < 64q  ->  v mod q. The quotient estimate k = floor(t * mq / 2^24) from
// t = floor(v / 2^(kb-8)) and mq = floor(2^(kb+16) / q) satisfies
// v/q - 2 < k <= v/q, so v - k q lies in [0, 2q) and one subtraction ends it.
__device__ __forceinline__ u64 reduce_lazy(u64 v, u64 q, int kb, uint32_t mq) {
  const uint32_t t = (uint32_t)(v >> (kb - 8));
  const uint32_t k = (t * mq) >> 24;
  const u64 r = v - (u64)k * q;
  return r >= q ? r - q : r;
}

// m = 5N/2: the four-way split of Phi_10(X^(N/4)) on four words a_j (the
// quarters' words at one position), factored through the quadratics
// y^2 - c y + 1 = (y - xi^e)(y - xi^-e), c = xi^e + xi^-e, e = 1 and 3. Both
// c are roots of c^2 = c + 1 (c_1 + c_3 = 1, c_1 c_3 = -1), so a mod the
// quadratic is (a0 - a2 - c a3) + (a1 + c (a2 + a3)) y and the two
// quadratics share the products c_1 a3 and c_1 (a2 + a3); each remainder is
// then evaluated at its two roots. Forward: 6 Shoup products per 4 words,
// inputs below 4q give outputs below 16q, in the order xi^1, xi^3, xi^7, xi^9.
// Inverse (inputs below 2q): the remainders from the root values, then
// a3 = (r0 - s0) / (1 - 2 c_1), a2 + a3 = (s1 - r1) / (1 - 2 c_1),
// a1 = r1 - c_1 (a2 + a3), a0 = r0 + a2 + c_1 a3, scaled by 4/N: 10 products,
// canonical. Constants per prime (value, Shoup pairs): forward c_1, xi, xi^3,
// xi^7, xi^9; inverse (xi - xi^9)^-1, xi, (xi^3 - xi^7)^-1, xi^3,
// (1 - 2 c_1)^-1 4/N, 4/N, c_1.
constexpr int kSplitWords = 24;
__device__ __forceinline__ void split4_fwd(u64& a0, u64& a1, u64& a2, u64& a3, const ulonglong2* __restrict__ c,
                                           u64 q) {
  const ulonglong2 c1 = __ldg(c);
  const u64 t3 = shoup_lazy(a3, c1.x, c1.y, q);
  const u64 t23 = shoup_lazy(a2 + a3, c1.x, c1.y, q);
  const u64 r0 = a0 + 6 * q - a2 - t3;
  const u64 r1 = a1 + t23;
  const u64 s0 = a0 + t3 + 8 * q - a2 - a3;
  const u64 s1 = a1 + a2 + a3 + 2 * q - t23;
  const ulonglong2 x1 = __ldg(c + 1), x3 = __ldg(c + 2), x7 = __ldg(c + 3), x9 = __ldg(c + 4);
  a0 = r0 + shoup_lazy(r1, x1.x, x1.y, q);
  a3 = r0 + shoup_lazy(r1, x9.x, x9.y, q);
  a1 = s0 + shoup_lazy(s1, x3.x, x3.y, q);
  a2 = s0 + shoup_lazy(s1, x7.x, x7.y, q);
}
__device__ __forceinline__ void split4_inv(u64& b0, u64& b1, u64& b2, u64& b3, const ulonglong2* __restrict__ c,
                                           u64 q) {
  const ulonglong2 k1 = __ldg(c + 5), x1 = __ldg(c + 6), k3 = __ldg(c + 7), x3 = __ldg(c + 8);
  const u64 r1 = shoup(b0 - b3 + 2 * q, k1.x, k1.y, q);
  const u64 r0 = b0 + q - shoup(r1, x1.x, x1.y, q);
  const u64 s1 = shoup(b1 - b2 + 2 * q, k3.x, k3.y, q);
  const u64 s0 = b1 + q - shoup(s1, x3.x, x3.y, q);
  const ulonglong2 d = __ldg(c + 9), sg = __ldg(c + 10), c1 = __ldg(c + 11);
  const u64 a3 = shoup(r0 - s0 + 3 * q, d.x, d.y, q);
  const u64 S = shoup(s1 - r1 + q, d.x, d.y, q);
  const u64 a2 = S >= a3 ? S - a3 : S + q - a3;
  const u64 u1 = shoup(r1, sg.x, sg.y, q), v1 = shoup(S, c1.x, c1.y, q);
  const u64 a1 = u1 >= v1 ? u1 - v1 : u1 + q - v1;
  u64 a0 = shoup(r0, sg.x, sg.y, q) + a2 + shoup(a3, c1.x, c1.y, q);
  if (a0 >= 2 * q) a0 -= 2 * q;
  if (a0 >= q) a0 -= q;
  b0 = a0;
  b1 = a1;
  b2 = a2;
  b3 = a3;
}

// One round of up to three radix-2 stages held in registers. The thread owns
// the eight words r_k = rbase + k*u (rbase = B*8u + o, o < u); the round's
// stages have half-distances t = u*2^j for j in [JLO, JHI] and pair the
// registers (k, k + 2^j). Butterflies of one 2t-block share one twiddle,
// index (mg << sg) + r/(2t), sg = logS - 1 - log2(t).
// R3 (m = 3N): node 1 (twiddle index 1) is the split of X^N - X^(N/2) + 1 into
// X^(N/2) - rho and X^(N/2) - rho^5 (rho^5 = 1 - rho): forward (U, V) ->
// (U + rho V, U + V - rho V); inverse t = (U - V)(2 rho - 1)^-1 ->
// (U + V - t, 2t), both scaled by N^-1 with the rest afterwards.
template <bool FWD, int JLO, int JHI, int RING>
__device__ __forceinline__ void ntt_round(u64 (&x)[8], int rbase, int logu, int logS, int mg,
                                          const ulonglong2* __restrict__ tw, u64 q, bool pre1) {
  const u64 q2 = 2 * q;
#pragma unroll
  for (int jj = JLO; jj <= JHI; ++jj) {
    const int j = FWD ? JHI + JLO - jj : jj;
    const int d = 1 << j;
    const int logt = logu + j;
    const int sg = logS - 1 - logt;
#pragma unroll
    for (int blk = 0; blk < 4 / d; ++blk) {
      const int k0 = blk * 2 * d;
      const int widx = (mg << sg) + ((rbase + (k0 << logu)) >> (logt + 1));
      const ulonglong2 wv = __ldg(tw + widx);
      const u64 w = wv.x, wp = wv.y;
#pragma unroll
      for (int p = 0; p < d; ++p) {
        const int k = k0 + p;
        u64 U = x[k], V = x[k + d];
        if (RING == 3 && widx == 1) {
          if (FWD) {  // residues stay below 4q
            if (U >= q2) U -= q2;
            if (V >= q2) V -= q2;
            const u64 t = shoup_lazy(V, w, wp, q);
            u64 z = V + q2 - t;
            if (z >= q2) z -= q2;
            x[k] = U + t;
            x[k + d] = U + z;
          } else {
            const u64 t = shoup_lazy(U - V + q2, w, wp, q);
            x[k] = U + V + q2 - t;
            x[k + d] = t + t;
          }
        } else if (FWD) {
          if (U >= q2) U -= q2;
          if (!(pre1 && widx == 1)) V = shoup_lazy(V, w, wp, q);  // pre1: node 1's product already applied
          x[k] = U + V;
          x[k + d] = U - V + q2;
        } else {
          u64 s = U + V;
          if (s >= q2) s -= q2;
          x[k] = s;
          x[k + d] = shoup_lazy(U - V + q2, w, wp, q);
        }
      }
    }
  }
}

template <bool FWD, int RING>
__device__ __forceinline__ void ntt_round_dispatch(int jlo, int jhi, u64 (&x)[8], int rbase, int logu, int logS, int mg,
                                                   const ulonglong2* tw, u64 q, bool pre1) {
  switch (jlo * 3 + jhi) {
    case 0: ntt_round<FWD, 0, 0, RING>(x, rbase, logu, logS, mg, tw, q, pre1); break;
    case 1: ntt_round<FWD, 0, 1, RING>(x, rbase, logu, logS, mg, tw, q, pre1); break;
    case 2: ntt_round<FWD, 0, 2, RING>(x, rbase, logu, logS, mg, tw, q, pre1); break;
    case 4: ntt_round<FWD, 1, 1, RING>(x, rbase, logu, logS, mg, tw, q, pre1); break;
    case 5: ntt_round<FWD, 1, 2, RING>(x, rbase, logu, logS, mg, tw, q, pre1); break;
    default: ntt_round<FWD, 2, 2, RING>(x, rbase, logu, logS, mg, tw, q, pre1); break;
  }
}

// One phase: the tile is CPB sub-transforms of S = 2^logS words (columns of
// stride N/S when COLS, else contiguous chunks), staged in shared memory.
// blockDim = CPB*S/8. Residues stay lazy ([0,4q) forward, [0,2q) inverse)
// except in the LAST phase, which writes canonical values (times N^-1 for
// the inverse).
template <bool FWD, bool COLS, bool LAST, int RING = 1>
__global__ void __launch_bounds__(512) k_ntt(NttArgs A, int logS, int logCPB, int m0) {
  extern __shared__ u64 sm[];
  u64* ptr;
  int pidx;
  if (!poly_of(A, blockIdx.y, ptr, pidx)) return;
  const u64 q = A.mods[pidx].q;
  const ulonglong2* tw = reinterpret_cast<const ulonglong2*>(A.tw + (size_t)pidx * 4 * A.N + (FWD ? 0 : 2 * A.N));
  const int S = 1 << logS, CPB = 1 << logCPB, W = S << logCPB;
  const int tid = threadIdx.x, T = blockDim.x;
  const int tile = blockIdx.x;
  const long colbase = (long)tile * CPB;
  const int stride = A.N >> logS;
  // global -> shared, coalesced: consecutive lin are consecutive addresses
  for (int lin = tid; lin < W; lin += T) {
    long g = COLS ? (long)(lin >> logCPB) * stride + colbase + (lin & (CPB - 1)) : (long)tile * W + lin;
    sm[swz(lin)] = ptr[g];
  }
  __syncthreads();
  // m = 5N/2 (one phase over CPB = 4 chunks, the four factors): the split
  // first, residues brought below 2q for the rounds
  const ulonglong2* spl = RING == 5 ? reinterpret_cast<const ulonglong2*>(A.split + (size_t)pidx * kSplitWords) : nullptr;
  if (RING == 5 && FWD) {
    const int n4 = W >> 2;
    for (int i = tid; i < n4; i += T) {
      u64 a0 = sm[swz(i)], a1 = sm[swz(i + n4)], a2 = sm[swz(i + 2 * n4)], a3 = sm[swz(i + 3 * n4)];
      split4_fwd(a0, a1, a2, a3, spl, q);
      u64* o4[4] = {&a0, &a1, &a2, &a3};
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        u64 v = *o4[h];  // below 16q
        if (v >= 8 * q) v -= 8 * q;
        if (v >= 4 * q) v -= 4 * q;
        if (v >= 2 * q) v -= 2 * q;
        sm[swz(i + h * n4)] = v;
      }
    }
    __syncthreads();
  }
  const int rounds = (logS + 2) / 3;
  for (int rho = 0; rho < rounds; ++rho) {
    // log2 of the smallest (a) and largest (b) half-distance of this round
    const int ns = min(3, logS - 3 * rho);
    const int b = FWD ? logS - 1 - 3 * rho : 3 * rho + ns - 1;
    const int a = b - ns + 1;
    const int logu = max(0, b - 2);
    int c, o, B;
    if (COLS) {
      c = tid & (CPB - 1);
      int rest = tid >> logCPB;
      o = rest & ((1 << logu) - 1);
      B = rest >> logu;
    } else {
      o = tid & ((1 << logu) - 1);
      int rest = tid >> logu;
      int logB = logS - 3 - logu;
      B = rest & ((1 << logB) - 1);
      c = rest >> logB;
    }
    const int rbase = (B << (logu + 3)) + o;
    const int mg = m0 + (COLS ? 0 : tile * CPB + c);
    u64 x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      int r = rbase + (k << logu);
      x[k] = sm[swz(COLS ? (r << logCPB) + c : (c << logS) + r)];
    }
    ntt_round_dispatch<FWD, RING>(a - logu, b - logu, x, rbase, logu, logS, mg, tw, q, RING == 1 && A.pre_w1);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      int r = rbase + (k << logu);
      sm[swz(COLS ? (r << logCPB) + c : (c << logS) + r)] = x[k];
    }
    __syncthreads();
  }
  if (RING == 5 && !FWD) {  // the split last, with the 4/N scaling: canonical
    const int n4 = W >> 2;
    for (int i = tid; i < n4; i += T) {
      u64 b0 = sm[swz(i)], b1 = sm[swz(i + n4)], b2 = sm[swz(i + 2 * n4)], b3 = sm[swz(i + 3 * n4)];
      split4_inv(b0, b1, b2, b3, spl, q);
      sm[swz(i)] = b0;
      sm[swz(i + n4)] = b1;
      sm[swz(i + 2 * n4)] = b2;
      sm[swz(i + 3 * n4)] = b3;
    }
    __syncthreads();
  }
  u64 ni = 0, nip = 0;
  if (LAST && !FWD) { ni = A.ninv[4 * pidx]; nip = A.ninv[4 * pidx + 1]; }
  for (int lin = tid; lin < W; lin += T) {
    u64 v = sm[swz(lin)];
    if (LAST) {
      if (FWD) {
        if (v >= 2 * q) v -= 2 * q;
        if (v >= q) v -= q;
      } else if (RING != 5) {
        v = shoup(v, ni, nip, q);
      }
    }
    long g = COLS ? (long)(lin >> logCPB) * stride + colbase + (lin & (CPB - 1)) : (long)tile * W + lin;
    ptr[g] = v;
  }
}

// ---------------------------------------------------------------- radix-16 phases
// Same scheme with sixteen words per thread (four stages per register round,
// two rounds per 256-point phase) for the two-phase transforms (N >= 8192).
// Round 0 reads global memory straight into registers and the last round
// writes straight back whenever that access is coalesced (always for column
// tiles; for chunk tiles when the round's spacing u >= 16), otherwise the
// tile passes through shared memory once more.
// blockDim = CPB*S/16, S = 2^LOGS with 5 <= LOGS <= 8. Every round's stage
// range is a compile-time constant, so the sixteen words stay in registers.
// The forward butterfly here never reduces its upper input: each stage adds
// less than 2q to the bound, so inputs below 4q leave a log2 N <= 16 stage
// transform below 36q (40q with the m = 3N split, 44q with m = 5N/2's) < 64q < 2^64 (primes below
// 2^58), and the last phase brings every word back to [0, q) once (reduce_lazy).
// One CTA tile (`tile` of polynomial `poly`) of one phase; the body of the
// per-transform kernel k_ntt16 and of the persistent kernel k_ntt16_multi.
// R3 (m = 3N, column phases only): the first forward stage and the last
// inverse stage are node 1, the split of X^N - X^(N/2) + 1 (see ntt_round).
// Forward it adds up to 6q to the bound, so the transform stays below 40q.
// Inverse it is fused with N^-1: with c = (2 rho - 1)^-1 N^-1 (inverse
// twiddle word 0), high = (U - V) 2c, low = (U + V) N^-1 - (U - V) c.
template <bool FWD, bool COLS, bool LAST, int LOGS, bool SRC, int RING = 1>
__device__ __forceinline__ void ntt16_tile(const NttArgs& A, int logCPB, int m0, int tile, int poly) {
  extern __shared__ u64 sm[];
  u64* ptr;
  int pidx;
  if (!poly_of(A, poly, ptr, pidx)) return;
  const u64 q = A.mods[pidx].q;
  const ulonglong2* tw = reinterpret_cast<const ulonglong2*>(A.tw + (size_t)pidx * 4 * A.N + (FWD ? 0 : 2 * A.N));
  constexpr int S = 1 << LOGS;
  const int CPB = 1 << logCPB, W = S << logCPB;
  const int tid = threadIdx.x, T = blockDim.x;
  const int stride = A.N >> LOGS;
  u64* gbase = COLS ? ptr + (long)tile * CPB : ptr + (long)tile * W;
  const u64* gsrc = gbase;
  if (SRC) {  // same polynomial, read from the out-of-place source
    const int i = poly / A.n_outer, o = poly % A.n_outer;
    const u64* rb = A.src + (long)o * A.src_os + (long)i * A.N;
    gsrc = COLS ? rb + (long)tile * CPB : rb + (long)tile * W;
  }
  constexpr int NR = (LOGS + 3) / 4;
  constexpr int B0 = FWD ? LOGS - 1 : (LOGS < 4 ? LOGS : 4) - 1;
  constexpr int NSL = LOGS - 4 * (NR - 1);
  constexpr int BL = FWD ? LOGS - 1 - 4 * (NR - 1) : 4 * (NR - 1) + NSL - 1;
  constexpr bool DIN = COLS || (B0 - 3 >= 4);
  constexpr bool DOUT = COLS || (BL - 3 >= 4);
  // Inverse chunk phase (staged through shared memory): the first stage's
  // eight twiddles of this thread are consecutive; load them before the
  // staging so their latency overlaps it.
  constexpr bool PRE = SS_NTT_PREFETCH && !FWD && !DIN && !COLS;
  ulonglong2 pre[PRE ? 8 : 1];
  if (PRE) {
    const int logB = LOGS - 4;
    const int B = tid & ((1 << logB) - 1), c = tid >> logB;
    const int mg = m0 + tile * CPB + c;
    const ulonglong2* tp = tw + (mg << (LOGS - 1)) + (B << 3);
#pragma unroll
    for (int i = 0; i < (PRE ? 8 : 1); ++i) pre[i] = __ldg(tp + i);
  }
  if (!DIN) {
    for (int lin = tid; lin < W; lin += T) sm[swz16<COLS>(lin)] = gsrc[lin];
    __syncthreads();
  }
  u64 ni = 0, nip = 0;
  u64 wni = 0, wnip = 0;
  u64 cni = 0, cnip = 0;
  if (LAST && !FWD) {
    ni = A.ninv[4 * pidx];
    nip = A.ninv[4 * pidx + 1];
    wni = A.ninv[4 * pidx + 2];
    wnip = A.ninv[4 * pidx + 3];
    if (RING == 3) {
      const ulonglong2 c0 = __ldg(tw);
      cni = c0.x;
      cnip = c0.y;
    }
  }
  const int kb = A.mods[pidx].kbits;
  const uint32_t mq = (uint32_t)(A.mods[pidx].mu >> 47);
#pragma unroll
  for (int rho = 0; rho < NR; ++rho) {
    const int ns = (LOGS - 4 * rho) < 4 ? (LOGS - 4 * rho) : 4;
    const int b = FWD ? LOGS - 1 - 4 * rho : 4 * rho + ns - 1;
    const int a = b - ns + 1;
    const int logu = b - 3 > 0 ? b - 3 : 0;
    int c, o, B;
    if (COLS) {
      c = tid & (CPB - 1);
      int rest = tid >> logCPB;
      o = rest & ((1 << logu) - 1);
      B = rest >> logu;
    } else {
      o = tid & ((1 << logu) - 1);
      int rest = tid >> logu;
      const int logB = LOGS - 4 - logu;
      B = rest & ((1 << logB) - 1);
      c = rest >> logB;
    }
    const int rbase = (B << (logu + 4)) + o;
    const int mg = m0 + (COLS ? 0 : tile * CPB + c);
    u64 x[16];
    if (rho == 0 && DIN) {
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        int r = rbase + (k << logu);
        x[k] = COLS ? gsrc[(long)r * stride + c] : gsrc[(c << LOGS) + r];
      }
    } else {
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        int r = rbase + (k << logu);
        x[k] = sm[swz16<COLS>(COLS ? (r << logCPB) + c : (c << LOGS) + r)];
      }
    }
    // stages j in [a - logu, b - logu]: d = 2^j registers apart
    const u64 q2 = 2 * q;
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int jlo = a - logu, jhi = b - logu;
      const int j = FWD ? jhi - jj : jlo + jj;
      if (jj < ns) {
        const int d = 1 << j;
        const int logt = logu + j;
        const int sg = LOGS - 1 - logt;
        // the inverse transform's last stage (one twiddle, psi^(-N/2)) also
        // applies N^-1: sums times N^-1, differences times N^-1 psi^(-N/2)
        const bool fold = LAST && !FWD && rho == NR - 1 && jj == ns - 1;
        const bool split = RING == 3 && COLS && FWD && rho == 0 && jj == 0;
        // node 1 of X^N + 1 (the column phase's first forward stage) on inputs
        // whose upper half already carries its twiddle: no product
        const bool pre1 = RING == 1 && COLS && FWD && rho == 0 && jj == 0 && A.pre_w1;
        // m = 5N/2: the first two forward stages and the last two inverse
        // stages of the column phase are the four-way split on the registers
        // k, k+4, k+8, k+12 (the quarters), k < 4
        if (RING == 5 && COLS && FWD && rho == 0 && jj < 2) {
          if (jj == 0) {
            const ulonglong2* spl = reinterpret_cast<const ulonglong2*>(A.split + (size_t)pidx * kSplitWords);
#pragma unroll
            for (int k = 0; k < 4; ++k) split4_fwd(x[k], x[k + 4], x[k + 8], x[k + 12], spl, q);
          }
          continue;
        }
        if (RING == 5 && COLS && LAST && !FWD && rho == NR - 1 && jj >= ns - 2) {
          if (jj == ns - 1) {
            const ulonglong2* spl = reinterpret_cast<const ulonglong2*>(A.split + (size_t)pidx * kSplitWords);
#pragma unroll
            for (int k = 0; k < 4; ++k) split4_inv(x[k], x[k + 4], x[k + 8], x[k + 12], spl, q);
          }
          continue;
        }
#pragma unroll
        for (int blk = 0; blk < 8; ++blk) {
          if (blk < 8 / d) {
            const int k0 = blk * 2 * d;
            u64 w = wni, wp = wnip;
            if (PRE && rho == 0 && jj == 0) {
              w = pre[PRE ? blk : 0].x;
              wp = pre[PRE ? blk : 0].y;
            } else if (!fold && !pre1) {
              const int widx = (mg << sg) + ((rbase + (k0 << logu)) >> (logt + 1));
              const ulonglong2 wv = __ldg(tw + widx);
              w = wv.x;
              wp = wv.y;
            }
#pragma unroll
            for (int p = 0; p < 8; ++p) {
              if (p < d) {
                const int k = k0 + p;
                u64 U = x[k], V = x[k + d];
                if (fold && RING == 3) {
                  const u64 dv = U - V + q2;
                  const u64 lo = shoup(U + V, ni, nip, q), cr = shoup(dv, cni, cnip, q);
                  x[k] = lo >= cr ? lo - cr : lo + q - cr;
                  x[k + d] = shoup(dv, w, wp, q);
                } else if (fold && A.post_scale) {  // N^-1 and N^-1 psi^(-N/2) left to the consumer
                  x[k] = U + V;
                  x[k + d] = U - V + q2;
                } else if (fold) {
                  x[k] = shoup(U + V, ni, nip, q);
                  x[k + d] = shoup(U - V + q2, w, wp, q);
                } else if (split) {
                  const u64 t = shoup_lazy(V, w, wp, q);
                  x[k] = U + t;
                  x[k + d] = U + V + q2 - t;
                } else if (pre1) {  // U, V < q
                  x[k] = U + V;
                  x[k + d] = U - V + q2;
                } else if (FWD) {
                  V = shoup_lazy(V, w, wp, q);
                  x[k] = U + V;
                  x[k + d] = U - V + q2;
                } else {
                  u64 s2 = U + V;
                  if (s2 >= q2) s2 -= q2;
                  x[k] = s2;
                  x[k + d] = shoup_lazy(U - V + q2, w, wp, q);
                }
              }
            }
          }
        }
      }
    }
    if (rho == NR - 1 && DOUT) {
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        int r = rbase + (k << logu);
        u64 v = x[k];
        if (LAST && FWD) v = reduce_lazy(v, q, kb, mq);  // the inverse's last stage already reduced and scaled
        if (COLS) gbase[(long)r * stride + c] = v;
        else gbase[(c << LOGS) + r] = v;
      }
    } else {
      if (rho > 0 || !DIN) __syncthreads();  // every read of the previous layout is done
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        int r = rbase + (k << logu);
        sm[swz16<COLS>(COLS ? (r << logCPB) + c : (c << LOGS) + r)] = x[k];
      }
      __syncthreads();
    }
  }
  if (!DOUT) {
    for (int lin = tid; lin < W; lin += T) {
      u64 v = sm[swz16<COLS>(lin)];
      if (LAST && FWD) v = reduce_lazy(v, q, kb, mq);
      gbase[lin] = v;
    }
  }
}

template <bool FWD, bool COLS, bool LAST, int LOGS, bool SRC = false, int RING = 1>
__global__ void __launch_bounds__(256, RING == 5 ? SS_NTT_MINB_R5 : (FWD ? SS_NTT_MINB_F : SS_NTT_MINB_I))
    k_ntt16(NttArgs A, int logCPB, int m0) {
  ntt16_tile<FWD, COLS, LAST, LOGS, SRC, RING>(A, logCPB, m0, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------- persistent multi-transform phase
// One phase of up to kMaxNttJobs transforms of any ring dimensions N >= 8192
// (each job: one polynomial set of one context, with its own moduli and
// twiddles) in one launch: the tiles of all jobs form one work list, job j
// owning tiles [start_j, start_j + polys_j * tiles_j); every CTA of a grid
// sized to the resident CTAs of the device walks the list with stride
// gridDim.x. All jobs share the tile size (blockDim = tile / 16), so tiles
// of different N run side by side; the sub-transform length of a job's phase
// (2^logS, 5 <= logS <= 8) selects the instantiation per tile.
constexpr int kMaxNttJobs = 24;
struct NttJob {
  NttArgs A;
  int logS, logCPB, m0, tiles, start;
  int ring;  // the context's m_odd: 3 (m = 3N) or 5 (m = 5N/2) give the column phase its split; 1 none
};
struct NttMulti {
  int njobs, total;
  NttJob j[kMaxNttJobs];
};

// a separate function per instantiation, so each keeps its own register allocation
template <bool FWD, bool COLS, bool LAST, int LOGS, bool SRC, int RING = 1>
__device__ __noinline__ void ntt16_tile_fn(const NttArgs& A, int logCPB, int m0, int tile, int poly) {
  ntt16_tile<FWD, COLS, LAST, LOGS, SRC, RING>(A, logCPB, m0, tile, poly);
}

template <bool FWD, bool COLS, bool LAST, bool SRC>
__global__ void __launch_bounds__(256, FWD ? SS_NTT_MINB_F : SS_NTT_MINB_I)
    k_ntt16_multi(const __grid_constant__ NttMulti M) {
  for (int t = blockIdx.x; t < M.total; t += gridDim.x) {
    int j = 0;
    while (j + 1 < M.njobs && t >= M.j[j + 1].start) ++j;
    const NttJob& J = M.j[j];
    const int local = t - J.start;
    const int poly = local / J.tiles, tile = local - poly * J.tiles;
    if constexpr (COLS) {
      if (J.ring == 3 || J.ring == 5) {
        if (J.ring == 3) {
          switch (J.logS) {
            case 5: ntt16_tile_fn<FWD, COLS, LAST, 5, SRC, 3>(J.A, J.logCPB, J.m0, tile, poly); break;
            case 6: ntt16_tile_fn<FWD, COLS, LAST, 6, SRC, 3>(J.A, J.logCPB, J.m0, tile, poly); break;
            case 7: ntt16_tile_fn<FWD, COLS, LAST, 7, SRC, 3>(J.A, J.logCPB, J.m0, tile, poly); break;
            default: ntt16_tile_fn<FWD, COLS, LAST, 8, SRC, 3>(J.A, J.logCPB, J.m0, tile, poly); break;
          }
        } else {
          switch (J.logS) {
            case 6: ntt16_tile_fn<FWD, COLS, LAST, 6, SRC, 5>(J.A, J.logCPB, J.m0, tile, poly); break;
            case 7: ntt16_tile_fn<FWD, COLS, LAST, 7, SRC, 5>(J.A, J.logCPB, J.m0, tile, poly); break;
            default: ntt16_tile_fn<FWD, COLS, LAST, 8, SRC, 5>(J.A, J.logCPB, J.m0, tile, poly); break;
          }
        }
        __syncthreads();
        continue;
      }
    }
    switch (J.logS) {
      case 5: ntt16_tile_fn<FWD, COLS, LAST, 5, SRC>(J.A, J.logCPB, J.m0, tile, poly); break;
      case 6: ntt16_tile_fn<FWD, COLS, LAST, 6, SRC>(J.A, J.logCPB, J.m0, tile, poly); break;
      case 7: ntt16_tile_fn<FWD, COLS, LAST, 7, SRC>(J.A, J.logCPB, J.m0, tile, poly); break;
      default: ntt16_tile_fn<FWD, COLS, LAST, 8, SRC>(J.A, J.logCPB, J.m0, tile, poly); break;
    }
    __syncthreads();  // the next tile reuses the shared memory
  }
}

template <bool FWD, bool COLS, bool LAST, bool SRC = false, int RING = 1>
void launch16(int logS, dim3 g, int thr, size_t smem, cudaStream_t st, const NttArgs& A, int logc, int m0) {
  switch (logS) {
    case 5: k_ntt16<FWD, COLS, LAST, 5, SRC, RING><<<g, thr, smem, st>>>(A, logc, m0); break;
    case 6: k_ntt16<FWD, COLS, LAST, 6, SRC, RING><<<g, thr, smem, st>>>(A, logc, m0); break;
    case 7: k_ntt16<FWD, COLS, LAST, 7, SRC, RING><<<g, thr, smem, st>>>(A, logc, m0); break;
    default: k_ntt16<FWD, COLS, LAST, 8, SRC, RING><<<g, thr, smem, st>>>(A, logc, m0); break;
  }
}

NttArgs make_args(Context& C, const PolySet& s) {
  NttArgs A;
  A.base = s.base;
  A.outer_stride = s.outer_stride;
  A.n_outer = s.n_outer;
  A.nl = s.nl;
  A.q0 = s.q0;
  A.nq = s.nq;
  A.L = C.L;
  A.N = C.N;
  A.skip_w = s.skip_w;
  A.skip_mod = s.skip_mod;
  A.skip_level = s.skip_level;
  A.mods = reinterpret_cast<const Modulus*>(C.d_mod);
  A.tw = C.d_tw;
  A.ninv = C.d_ninv;
  A.split = C.d_split;
  A.src = nullptr;
  A.src_os = 0;
  if (s.pre_w1 && C.m_odd != 1) throw Error(SS_ERR_PARAM, "node-1 twiddle folding is for the ring X^N + 1");
  if (s.post_scale && (C.m_odd != 1 || C.N <= TILE))
    throw Error(SS_ERR_PARAM, "deferred inverse scaling is for two-phase transforms on the ring X^N + 1");
  A.pre_w1 = s.pre_w1 ? 1 : 0;
  A.post_scale = s.post_scale ? 1 : 0;
  return A;
}

double active_polys(const PolySet& s);

// Shoup products of one transform of the set: N/2 per stage and polynomial,
// less node 1's when folded (pre_w1), plus the inverse's N^-1: on the sums of
// the last stage (two-phase transforms, N/2) or on every word (single-phase,
// N), none when the last stage is deferred (post_scale: no products there)
double ntt_products(const Context& C, const PolySet& s, bool fwd) {
  const double half = C.N / 2.0;
  const int inv_extra = s.post_scale ? -1 : (C.N <= TILE ? 2 : 1);
  return active_polys(s) * half * (C.logN + (fwd ? (s.pre_w1 ? -1 : 0) : inv_extra));
}

// polynomials a transform actually touches (ModUp outputs skip the digit's own limbs)
double active_polys(const PolySet& s) {
  double n = (double)s.n_outer * s.nl;
  if (s.skip_w > 0)
    for (int o = 0; o < s.n_outer; ++o) {
      int lo = (o % s.skip_mod) * s.skip_w, hi = std::min(lo + s.skip_w, s.skip_level);
      if (hi > lo) n -= hi - lo;
    }
  return n;
}

}  // namespace

NttMerger*& ntt_merger() {
  static thread_local NttMerger* m = nullptr;
  return m;
}

// log2 of the chunk length N2 of the two-phase split: 256, except that the
// m = 5N/2 ring needs at least 64 column words (its inverse split takes the
// column phase's last two stages in one register round)
static int chunk_log(const Context& C) { return C.m_odd == 5 && C.logN - 8 < 6 ? C.logN - 6 : 8; }

// src: optional out-of-place source read by the first phase (inverse only)
static void launch(Context& C, const PolySet& s, bool fwd, cudaStream_t st, const u64* src = nullptr,
                   long src_os = 0) {
  int npoly = s.n_outer * s.nl;
  if (npoly == 0) return;
  if (ntt_merger() && C.N > TILE && !is_dry(C)) {
    ntt_merger()->submit(NttReq{&C, s, src, src_os}, fwd, st);
    return;
  }
  if (npoly > 65535) throw Error(SS_ERR_SHAPE, "too many polynomials in one transform");
  NttArgs A = make_args(C, s);
  const int N = C.N, logN = C.logN;
  auto smem = [](int words) { return (size_t)(words + words / 8) * 8; };
  if (N <= TILE) {
    if (src)  // one in-place phase: copy first
      SS_CUDA(cudaMemcpy2DAsync(s.base, (size_t)s.outer_stride * 8, src, (size_t)src_os * 8, (size_t)s.nl * N * 8,
                                s.n_outer, cudaMemcpyDeviceToDevice, st));
    int kr = kt_begin(C, st);
    dim3 g(1, npoly);
    int thr = N / 8;
    if (C.m_odd == 5) {  // the split, then the four factors as chunks of N/4 (nodes 4..7 and below)
      if (fwd) k_ntt<true, false, true, 5><<<g, thr, smem(N), st>>>(A, logN - 2, 2, 4);
      else k_ntt<false, false, true, 5><<<g, thr, smem(N), st>>>(A, logN - 2, 2, 4);
    } else if (C.m_odd == 3) {
      if (fwd) k_ntt<true, false, true, 3><<<g, thr, smem(N), st>>>(A, logN, 0, 1);
      else k_ntt<false, false, true, 3><<<g, thr, smem(N), st>>>(A, logN, 0, 1);
    } else {
      if (fwd) k_ntt<true, false, true><<<g, thr, smem(N), st>>>(A, logN, 0, 1);
      else k_ntt<false, false, true><<<g, thr, smem(N), st>>>(A, logN, 0, 1);
    }
    ++C.launches;
    if (kr >= 0) C.kt.ntt_products += ntt_products(C, s, fwd);
    kt_end(C, kr, KC_NTT, 16.0 * N * active_polys(s), st);
  } else {
    int kr = kt_begin(C, st);
    const int log2n = chunk_log(C), log1 = logN - log2n;  // N = N1 * N2, N2 = 2^log2n
    const int tl = C.ntt_tile_log == 11 ? 11 : 12, tile = 1 << tl;
    const int logc1 = tl - log1, logc2 = tl - log2n;
    dim3 g1(1 << (log2n - logc1), npoly), g2(1 << (log1 - logc2), npoly);
    const int thr = tile / 16;
    if (fwd) {
      if (C.m_odd == 3) launch16<true, true, false, false, 3>(log1, g1, thr, smem(tile), st, A, logc1, 1);
      else if (C.m_odd == 5) launch16<true, true, false, false, 5>(log1, g1, thr, smem(tile), st, A, logc1, 1);
      else launch16<true, true, false>(log1, g1, thr, smem(tile), st, A, logc1, 1);
      launch16<true, false, true>(log2n, g2, thr, smem(tile), st, A, logc2, 1 << log1);
    } else {
      if (src) {
        NttArgs A1 = A;
        A1.src = src;
        A1.src_os = src_os;
        launch16<false, false, false, true>(log2n, g2, thr, smem(tile), st, A1, logc2, 1 << log1);
      } else {
        launch16<false, false, false>(log2n, g2, thr, smem(tile), st, A, logc2, 1 << log1);
      }
      if (C.m_odd == 3) launch16<false, true, true, false, 3>(log1, g1, thr, smem(tile), st, A, logc1, 1);
      else if (C.m_odd == 5) launch16<false, true, true, false, 5>(log1, g1, thr, smem(tile), st, A, logc1, 1);
      else launch16<false, true, true>(log1, g1, thr, smem(tile), st, A, logc1, 1);
    }
    C.launches += 2;
    if (kr >= 0) C.kt.ntt_products += ntt_products(C, s, fwd);
    kt_end(C, kr, KC_NTT, 16.0 * N * active_polys(s), st);
  }
  SS_CUDA(cudaGetLastError());
}

static int resident_ctas() {
  static std::atomic<int> n{0};
  int v = n.load();
  if (!v) {
    int dev = 0, sms = 0;
    SS_CUDA(cudaGetDevice(&dev));
    SS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    v = sms * SS_NTT_MINB_F;
    n.store(v);
  }
  return v;
}

template <bool FWD, bool COLS, bool LAST, bool SRC>
static void launch_multi(const NttMulti& M, int thr, size_t smem, cudaStream_t st) {
  if (M.total == 0) return;
  const int grid = std::min(M.total, resident_ctas());
  k_ntt16_multi<FWD, COLS, LAST, SRC><<<grid, thr, smem, st>>>(M);
  SS_CUDA(cudaGetLastError());
}

void ntt_multi(const std::vector<NttReq>& reqs, bool fwd, int tile_log, cudaStream_t st) {
  const int tl = tile_log == 11 ? 11 : 12, tile = 1 << tl, thr = tile / 16;
  const size_t smem = (size_t)(tile + tile / 8) * 8;
  for (size_t b0 = 0; b0 < reqs.size(); b0 += kMaxNttJobs) {
    const size_t b1 = std::min(reqs.size(), b0 + kMaxNttJobs);
    // phase 1 (columns forward, chunks inverse) and phase 2 of every job
    NttMulti P1, P2;
    P1.njobs = P2.njobs = 0;
    P1.total = P2.total = 0;
    double bytes = 0, prods = 0;
    for (size_t r = b0; r < b1; ++r) {
      const NttReq& q = reqs[r];
      Context& C = *q.C;
      if (C.N < 8192) throw Error(SS_ERR_PARAM, "merged transforms need N >= 8192");
      const int npoly = q.s.n_outer * q.s.nl;
      if (npoly == 0) continue;
      NttArgs A = make_args(C, q.s);
      const int l2 = chunk_log(C), log1 = C.logN - l2, logc1 = tl - log1, logc2 = tl - l2;
      NttJob cols{A, log1, logc1, 1, 1 << (l2 - logc1), 0, C.m_odd};
      NttJob chunks{A, l2, logc2, 1 << log1, 1 << (log1 - logc2), 0, 1};
      if (!fwd) {  // the chunk phase reads the source (the polynomials themselves when in place)
        chunks.A.src = q.src ? q.src : q.s.base;
        chunks.A.src_os = q.src ? q.src_os : q.s.outer_stride;
      }
      NttJob& j1 = P1.j[P1.njobs++];
      NttJob& j2 = P2.j[P2.njobs++];
      j1 = fwd ? cols : chunks;
      j2 = fwd ? chunks : cols;
      j1.start = P1.total;
      j2.start = P2.total;
      P1.total += npoly * j1.tiles;
      P2.total += npoly * j2.tiles;
      bytes += 16.0 * C.N * active_polys(q.s);
      prods += ntt_products(C, q.s, fwd);
    }
    if (P1.njobs == 0) continue;
    Context& C0 = *reqs[b0].C;
    int kr = kt_begin(C0, st);
    if (fwd) {
      launch_multi<true, true, false, false>(P1, thr, smem, st);
      launch_multi<true, false, true, false>(P2, thr, smem, st);
    } else {
      launch_multi<false, false, false, true>(P1, thr, smem, st);
      launch_multi<false, true, true, false>(P2, thr, smem, st);
    }
    C0.launches += 2;
    if (kr >= 0) C0.kt.ntt_products += prods;
    kt_end(C0, kr, KC_NTT, bytes, st);
  }
}

void ntt_forward(Context& C, const PolySet& s, cudaStream_t st) { launch(C, s, true, st); }

void ntt_inverse(Context& C, const PolySet& s, cudaStream_t st) { launch(C, s, false, st); }

void ntt_inverse_from(Context& C, const PolySet& s, const u64* src, long src_os, cudaStream_t st) {
  launch(C, s, false, st, src, src_os);
}

}  // namespace ss
