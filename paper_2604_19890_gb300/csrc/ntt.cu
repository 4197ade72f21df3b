// Negacyclic NTT / inverse NTT over RNS limbs (Section 2.1 ring arithmetic).
//
// Forward: merged-twist Cooley-Tukey with twiddles psi^bitrev(m+i); natural
// coefficients in, evaluation form out with word j = a(psi^(2 bitrev(j)+1)).
// Inverse: Gentleman-Sande with psi^-bitrev(m+i), then times N^-1.
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
constexpr int THREADS = 256;

struct NttArgs {
  u64* base;
  long outer_stride;
  int nl, q0, nq, L, N;
  int skip_w, skip_mod, skip_level;
  const Modulus* mods;
  const u64* tw;     // per prime 4N words
  const u64* ninv;   // per prime (N^-1, shoup)
};

__device__ __forceinline__ bool poly_of(const NttArgs& A, int poly, u64*& ptr, int& pidx) {
  int o = poly / A.nl, i = poly % A.nl;
  if (A.skip_w > 0) {
    int j = o % A.skip_mod;
    int lo = j * A.skip_w, hi = min(lo + A.skip_w, A.skip_level);
    if (i >= lo && i < hi && i < A.nq) return false;
  }
  ptr = A.base + (long)o * A.outer_stride + (long)i * A.N;
  pidx = i < A.nq ? A.q0 + i : A.L + (i - A.nq);
  return true;
}

// COLS: the tile is CPB columns (stride N/S between rows); else CPB chunks of S.
// Forward stages sigma = 0..s-1 with global twiddle index (m0 + g0) 2^sigma + group.
template <bool COLS, bool LAST>
__global__ void __launch_bounds__(THREADS) k_ntt_fwd(NttArgs A, int S, int logS, int CPB, int m0) {
  extern __shared__ u64 sm[];
  // map polys so that consecutive blocks share a prime (twiddles stay in L2)
  int poly = blockIdx.y;
  u64* ptr;
  int pidx;
  if (!poly_of(A, poly, ptr, pidx)) return;
  const Modulus md = A.mods[pidx];
  const u64 q = md.q, q2 = 2 * q;
  const u64* tw = A.tw + (size_t)pidx * 4 * A.N;
  const u64* tws = tw + A.N;
  const int tile = blockIdx.x;
  const int words = CPB * S;
  const int stride = A.N / S;  // column stride (COLS)
  // load
  for (int e = threadIdx.x; e < words; e += blockDim.x) {
    if (COLS) {
      int c = e % CPB, r = e / CPB;
      sm[e] = ptr[(long)r * stride + tile * CPB + c];
    } else {
      sm[e] = ptr[(long)tile * words + e];
    }
  }
  __syncthreads();
  const int half = words / 2;
  for (int sg = 0; sg < logS; ++sg) {
    int t = S >> (sg + 1);
    for (int b = threadIdx.x; b < half; b += blockDim.x) {
      int c, bb;
      if (COLS) { c = b % CPB; bb = b / CPB; }
      else { c = b / (S / 2); bb = b % (S / 2); }
      int grp = bb / t, pos = bb % t;
      int r = grp * 2 * t + pos;
      int g0 = COLS ? 0 : tile * CPB + c;
      int widx = ((m0 + g0) << sg) + grp;
      u64 w = __ldg(tw + widx), wp = __ldg(tws + widx);
      int i0, i1;
      if (COLS) { i0 = r * CPB + c; i1 = (r + t) * CPB + c; }
      else { i0 = c * S + r; i1 = i0 + t; }
      u64 U = sm[i0], V = sm[i1];
      if (U >= q2) U -= q2;
      V = shoup_lazy(V, w, wp, q);
      sm[i0] = U + V;
      sm[i1] = U - V + q2;
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < words; e += blockDim.x) {
    u64 x = sm[e];
    if (LAST) {
      if (x >= q2) x -= q2;
      if (x >= q) x -= q;
    }
    if (COLS) {
      int c = e % CPB, r = e / CPB;
      ptr[(long)r * stride + tile * CPB + c] = x;
    } else {
      ptr[(long)tile * words + e] = x;
    }
  }
}

template <bool COLS, bool LAST>
__global__ void __launch_bounds__(THREADS) k_ntt_inv(NttArgs A, int S, int logS, int CPB, int m0) {
  extern __shared__ u64 sm[];
  int poly = blockIdx.y;
  u64* ptr;
  int pidx;
  if (!poly_of(A, poly, ptr, pidx)) return;
  const Modulus md = A.mods[pidx];
  const u64 q = md.q, q2 = 2 * q;
  const u64* tw = A.tw + (size_t)pidx * 4 * A.N + 2 * A.N;
  const u64* tws = tw + A.N;
  const int tile = blockIdx.x;
  const int words = CPB * S;
  const int stride = A.N / S;
  for (int e = threadIdx.x; e < words; e += blockDim.x) {
    if (COLS) {
      int c = e % CPB, r = e / CPB;
      sm[e] = ptr[(long)r * stride + tile * CPB + c];
    } else {
      sm[e] = ptr[(long)tile * words + e];
    }
  }
  __syncthreads();
  const int half = words / 2;
  for (int sg = logS - 1; sg >= 0; --sg) {
    int t = S >> (sg + 1);
    for (int b = threadIdx.x; b < half; b += blockDim.x) {
      int c, bb;
      if (COLS) { c = b % CPB; bb = b / CPB; }
      else { c = b / (S / 2); bb = b % (S / 2); }
      int grp = bb / t, pos = bb % t;
      int r = grp * 2 * t + pos;
      int g0 = COLS ? 0 : tile * CPB + c;
      int widx = ((m0 + g0) << sg) + grp;
      u64 w = __ldg(tw + widx), wp = __ldg(tws + widx);
      int i0, i1;
      if (COLS) { i0 = r * CPB + c; i1 = (r + t) * CPB + c; }
      else { i0 = c * S + r; i1 = i0 + t; }
      u64 U = sm[i0], V = sm[i1];
      u64 s = U + V;
      if (s >= q2) s -= q2;
      sm[i0] = s;
      sm[i1] = shoup_lazy(U - V + q2, w, wp, q);
    }
    __syncthreads();
  }
  u64 ni = 0, nip = 0;
  if (LAST) { ni = A.ninv[2 * pidx]; nip = A.ninv[2 * pidx + 1]; }
  for (int e = threadIdx.x; e < words; e += blockDim.x) {
    u64 x = sm[e];
    if (LAST) x = shoup(x, ni, nip, q);
    if (COLS) {
      int c = e % CPB, r = e / CPB;
      ptr[(long)r * stride + tile * CPB + c] = x;
    } else {
      ptr[(long)tile * words + e] = x;
    }
  }
}

NttArgs make_args(Context& C, const PolySet& s) {
  NttArgs A;
  A.base = s.base;
  A.outer_stride = s.outer_stride;
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
  return A;
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

int ilog2(int x) {
  int l = 0;
  while ((1 << l) < x) ++l;
  return l;
}

}  // namespace

void ntt_forward(Context& C, const PolySet& s, cudaStream_t st) {
  int npoly = s.n_outer * s.nl;
  if (npoly == 0) return;
  if (npoly > 65535) throw Error(SS_ERR_SHAPE, "too many polynomials in one transform");
  NttArgs A = make_args(C, s);
  int N = C.N, logN = C.logN;
  size_t smem = TILE * 8;
  int kr = kt_begin(C, st);
  if (N <= TILE) {
    int thr = std::min(THREADS, N / 2);
    k_ntt_fwd<false, true><<<dim3(1, npoly), thr, N * 8, st>>>(A, N, logN, 1, 1);
    ++C.launches;
  } else {
    int N2 = 256, N1 = N / N2;
    int log1 = ilog2(N1);
    int cpb1 = TILE / N1, cpb2 = TILE / N2;
    k_ntt_fwd<true, false><<<dim3(N2 / cpb1, npoly), THREADS, smem, st>>>(A, N1, log1, cpb1, 1);
    k_ntt_fwd<false, true><<<dim3(N1 / cpb2, npoly), THREADS, smem, st>>>(A, N2, 8, cpb2, N1);
    C.launches += 2;
  }
  kt_end(C, kr, KC_NTT, 16.0 * N * active_polys(s), st);
  SS_CUDA(cudaGetLastError());
}

void ntt_inverse(Context& C, const PolySet& s, cudaStream_t st) {
  int npoly = s.n_outer * s.nl;
  if (npoly == 0) return;
  if (npoly > 65535) throw Error(SS_ERR_SHAPE, "too many polynomials in one transform");
  NttArgs A = make_args(C, s);
  int N = C.N, logN = C.logN;
  size_t smem = TILE * 8;
  int kr = kt_begin(C, st);
  if (N <= TILE) {
    int thr = std::min(THREADS, N / 2);
    k_ntt_inv<false, true><<<dim3(1, npoly), thr, N * 8, st>>>(A, N, logN, 1, 1);
    ++C.launches;
  } else {
    int N2 = 256, N1 = N / N2;
    int log1 = ilog2(N1);
    int cpb1 = TILE / N1, cpb2 = TILE / N2;
    k_ntt_inv<false, false><<<dim3(N1 / cpb2, npoly), THREADS, smem, st>>>(A, N2, 8, cpb2, N1);
    k_ntt_inv<true, true><<<dim3(N2 / cpb1, npoly), THREADS, smem, st>>>(A, N1, log1, cpb1, 1);
    C.launches += 2;
  }
  kt_end(C, kr, KC_NTT, 16.0 * N * active_polys(s), st);
  SS_CUDA(cudaGetLastError());
}

}  // namespace ss
