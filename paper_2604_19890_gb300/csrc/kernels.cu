// Streaming kernels of the BGV hot path: elementwise RNS arithmetic, the
// tensor product, fast base conversion (ModUp / ModDown / modulus switching),
// the key-switching inner product, automorphisms in evaluation form, Philox
// sampling and the CRT step of decryption.
//
// All of them are bound by HBM traffic on limb-major [.. ][limb][N] arrays:
// threads walk the coefficient index n, so every warp touches 32 consecutive
// 8-byte words of one limb (256 B, fully coalesced).
#include <cstdio>
#include <cstring>
#include <atomic>

#include "modarith.cuh"
#include "philox.h"
#include "ss_internal.h"

namespace ss {

#define LAUNCHED() do { ++C.launches; SS_CUDA(cudaGetLastError()); } while (0)
// launch bracketed by timing events (when kernel timing is on) with its algorithmic bytes
#define TIMED(cls, bytes, ...)                      \
  do {                                              \
    int kr_ = kt_begin(C, st);                      \
    __VA_ARGS__;                                    \
    kt_end(C, kr_, (cls), (double)(bytes), st);     \
  } while (0)

namespace {

constexpr int TPB = 256;

#ifndef SS_KSIP_OB
#define SS_KSIP_OB 2  // ciphertexts per thread in the key-switch inner product
#endif
#ifndef SS_BCONV_V
#define SS_BCONV_V 2  // coefficients per thread in base conversion (1 to 4 sources)
#endif
#ifndef SS_KSIP_V
#define SS_KSIP_V 2  // coefficients per thread in the key-switch inner product
#endif
#ifndef SS_KSIP_UNROLL
#define SS_KSIP_UNROLL 0  // digits per iteration of the inner product's loop (0: the compiler's choice)
#endif
#ifndef SS_KSIP_MINB
#define SS_KSIP_MINB 4  // resident CTAs per SM the inner product is compiled for (64 registers)
#endif
#ifndef SS_KSIP_STAGES
#define SS_KSIP_STAGES 3  // digits in flight per thread of the inner product (cp.async ring; 0: direct loads)
#endif
#ifndef SS_KSIP_ASYNC_MINB
#define SS_KSIP_ASYNC_MINB 4  // resident CTAs per SM of the cp.async inner product (48 KiB ring each, 64 registers)
#endif
constexpr int kKsipUnroll = SS_KSIP_UNROLL > 0 ? SS_KSIP_UNROLL : 1;

static_assert(sizeof(Modulus) == sizeof(ModDesc), "device modulus descriptors share one layout");
__device__ __forceinline__ const Modulus& MOD(const ModDesc* m, int i) {
  return reinterpret_cast<const Modulus*>(m)[i];
}

// Two consecutive words per thread through 16-byte loads and stores (every
// limb starts on a 16-byte boundary: N is even and bases are 256-byte aligned).
__device__ __forceinline__ ulonglong2 ld2(const u64* p) { return *reinterpret_cast<const ulonglong2*>(p); }
__device__ __forceinline__ void st2(u64* p, u64 x, u64 y) { *reinterpret_cast<ulonglong2*>(p) = make_ulonglong2(x, y); }
// V consecutive words (V = 1, 2 or 4; 16-byte accesses for V > 1)
template <int V>
__device__ __forceinline__ void ldv(const u64* p, u64 (&v)[V]) {
  if (V == 1) {
    v[0] = *p;
  } else {
#pragma unroll
    for (int i = 0; i < V; i += 2) {
      const ulonglong2 t = ld2(p + i);
      v[i] = t.x;
      v[i + 1 < V ? i + 1 : i] = t.y;
    }
  }
}
template <int V>
__device__ __forceinline__ void stv(u64* p, const u64 (&v)[V]) {
  if (V == 1) {
    *p = v[0];
  } else {
#pragma unroll
    for (int i = 0; i < V; i += 2) st2(p + i, v[i], v[i + 1 < V ? i + 1 : i]);
  }
}

// (h 2^32 + l) mod q for 64-bit partial sums h, l (the value is below 2^96)
__device__ __forceinline__ u64 reduce_split(u64 h, u64 l, const Modulus& md) {
  const u64 lo = (h << 32) + l;
  const u64 hi = (h >> 32) + (lo < l ? 1 : 0);
  return barrett_reduce128(hi, lo, md);
}

// y * c (|c| < 2^32) added into a 128-bit sum as two 32-bit products
__device__ __forceinline__ void add_small(Acc128& a, u64 y, uint32_t m) {
  const u64 p0 = (u64)(uint32_t)y * m, p1 = (u64)(uint32_t)(y >> 32) * m;
  a.add(p0);
  a.add(p1 << 32);
  a.hi += p1 >> 32;
}

dim3 grid_for(int N, int polys) {
  int bx = (N + TPB - 1) / TPB;
  return dim3(bx, polys);
}

// ---------------------------------------------------------------- add / sub
__global__ void k_binary_impl(int op, const u64* a, const u64* b, u64* out, int N, int ncomp, int level, int acap,
                              int bcap, int ocap, int bcast, const ModDesc* mods) {
  int poly = blockIdx.y;  // (bt, c, i)
  int i = poly % level, c = (poly / level) % ncomp, bt = poly / (level * ncomp);
  int n = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (n >= N) return;
  u64 q = MOD(mods, i).q;
  int bb = bcast ? 0 : bt;
  const ulonglong2 x = ld2(a + ((size_t)(bt * ncomp + c) * acap + i) * N + n);
  const ulonglong2 y = ld2(b + ((size_t)(bb * ncomp + c) * bcap + i) * N + n);
  u64* o = out + ((size_t)(bt * ncomp + c) * ocap + i) * N + n;
  if (op == 0) st2(o, add_mod(x.x, y.x, q), add_mod(x.y, y.y, q));
  else st2(o, sub_mod(x.x, y.x, q), sub_mod(x.y, y.y, q));
}

// ---------------------------------------------------------------- scalars
__global__ void k_scalar_impl(int op, const u64* a, i64 c, u64* out, int N, int ncomp, int level, int acap,
                              int ocap, const ModDesc* mods, const u64* pinv) {
  __shared__ u64 sw[2];
  int poly = blockIdx.y;
  int i = poly % level, comp = (poly / level) % ncomp, bt = poly / (level * ncomp);
  const Modulus& md = MOD(mods, i);
  u64 q = md.q;
  if (threadIdx.x == 0) {
    u64 w;
    if (op == 2) {
      sw[0] = pinv[2 * i];
      sw[1] = pinv[2 * i + 1];
    } else {
      if (c >= 0) w = (u64)c % q;
      else { u64 k = (u64)(-(c + 1)) % q; w = q - 1 - k; }
      sw[0] = w;
      sw[1] = (u64)(((u128)w << 64) / q);
    }
  }
  __syncthreads();
  int n = 2 * (blockIdx.x * blockDim.x + threadIdx.x);  // two consecutive words per thread
  if (n >= N) return;
  const ulonglong2 x = ld2(a + ((size_t)(bt * ncomp + comp) * acap + i) * N + n);
  u64 y0, y1;
  if (op == 1) {
    y0 = comp == 0 ? add_mod(x.x, sw[0], q) : x.x;
    y1 = comp == 0 ? add_mod(x.y, sw[0], q) : x.y;
  } else {
    y0 = shoup(x.x, sw[0], sw[1], q);
    y1 = shoup(x.y, sw[0], sw[1], q);
  }
  st2(out + ((size_t)(bt * ncomp + comp) * ocap + i) * N + n, y0, y1);
}

__global__ void k_copy_impl(const u64* a, u64* out, int N, int ncomp, int level, int acap, int ocap) {
  int poly = blockIdx.y;
  int i = poly % level, comp = (poly / level) % ncomp, bt = poly / (level * ncomp);
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  out[((size_t)(bt * ncomp + comp) * ocap + i) * N + n] = a[((size_t)(bt * ncomp + comp) * acap + i) * N + n];
}

// ---------------------------------------------------------------- tensor
__global__ void k_tensor_impl(const u64* a, const u64* b, u64* out, int N, int level, int acap, int bcap, int ocap,
                              const ModDesc* mods) {
  int poly = blockIdx.y;  // (bt, i)
  int i = poly % level, bt = poly / level;
  int n = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (n >= N) return;
  const Modulus& md = MOD(mods, i);
  size_t la = (size_t)acap * N, lb = (size_t)bcap * N, lo = (size_t)ocap * N;
  const u64* A = a + (size_t)bt * 2 * la + (size_t)i * N + n;
  const u64* B = b + (size_t)bt * 2 * lb + (size_t)i * N + n;
  u64* O = out + (size_t)bt * 3 * lo + (size_t)i * N + n;
  const ulonglong2 a0 = ld2(A), a1 = ld2(A + la), b0 = ld2(B), b1 = ld2(B + lb);
  st2(O, mul_mod(a0.x, b0.x, md), mul_mod(a0.y, b0.y, md));
  Acc128 x, y;
  x.zero();
  y.zero();
  x.mac_wide(a0.x, b1.x);
  x.mac_wide(a1.x, b0.x);
  y.mac_wide(a0.y, b1.y);
  y.mac_wide(a1.y, b0.y);
  st2(O + lo, barrett_reduce128(x.hi, x.lo, md), barrett_reduce128(y.hi, y.lo, md));
  st2(O + 2 * lo, mul_mod(a1.x, b1.x, md), mul_mod(a1.y, b1.y, md));
}

// ---------------------------------------------------------------- base conversion
// dst limb m (global prime g(m) = m < nq ? m : L + m - nq), m outside
// [skip_lo, skip_hi):  sum_s [src_s * c1_s]_{q_s} * c2[s][g(m)]  (mod q_g), then
// times post[g] when post != null. Source s lives on prime sp0 + s (s < nsq)
// or L + s - nsq. Per block, each target's modulus, its Montgomery inverse and
// the constants c2[s][g] * post[g] * 2^64 mod q_g are staged once in shared
// memory (row m: q, -q^-1 mod 2^64, c2'[0..ns)); every output is then a
// 128-bit sum of ns products and one Montgomery reduction, which removes the
// 2^64 and leaves the post factor applied. The sum stays below ns q_s q_g <
// q_g 2^64 (primes below 2^58, ns <= 64), as the reduction needs.
// V = 2: two consecutive coefficients per thread (16-byte accesses, the
// staged constants read once for both).
// tw != null (ModUp on the ring X^N + 1): outputs of the upper half
// (coefficients n >= N/2) also carry the forward transform's node-1 twiddle
// w_1 = psi^(N/2) of their prime, so the transform skips its first stage's
// product (PolySet::pre_w1). A block's V*blockDim coefficients lie in one
// half (the host checks that they divide N/2), so a block of the upper half
// stages c2'[s] w_1 2^64 instead (the factor 2^64 w_1 mod q comes from the
// per-prime table r64 beside 2^64 mod q; no product per output).
// dscale (sources from an inverse transform with PolySet::post_scale): the
// source words still lack N^-1 (lower half) or N^-1 psi^(-N/2) (upper half),
// and may be up to 4q; the first step then uses c1_s times that factor in
// Montgomery form (staged per block after the targets' rows) and a Montgomery
// reduction in place of the Shoup product, which accepts any 64-bit word.
template <int NS, int V>
__global__ void __launch_bounds__(256) k_bconv_impl(const u64* __restrict__ src, long src_os, int ns, int sp0, int nsq,
                                                    const u64* __restrict__ c1, const u64* __restrict__ c2, int T,
                                                    u64* __restrict__ dst, long dst_os, int nd, int nq, int L,
                                                    int skip_lo, int skip_hi, const u64* __restrict__ post, int N,
                                                    const ModDesc* mods, const u64* __restrict__ r64, int pre,
                                                    int dscale) {
  extern __shared__ u64 sh[];
  const int ns_ = NS > 0 ? NS : ns;
  const int W = 2 + ns_;
  const int half = 2 * V * blockIdx.x * blockDim.x >= N ? 1 : 0;  // block-uniform
  const int upper = pre ? half : 0;
  if (dscale)
    for (int s = threadIdx.x; s < ns_; s += blockDim.x) {
      const int gs = s < nsq ? sp0 + s : L + (s - nsq);
      sh[nd * W + s] = mul_mod(__ldg(c1 + 2 * s), __ldg(r64 + 4 * gs + 2 + half), MOD(mods, gs));
    }
  for (int m = threadIdx.x; m < nd; m += blockDim.x) {
    const int g = m < nq ? m : L + (m - nq);
    const Modulus& md = MOD(mods, g);
    u64* e = sh + m * W;
    e[0] = md.q;
    e[1] = md.qinv;
    const u64 R = __ldg(r64 + 4 * g + upper);  // 2^64 (times w_1) mod q
    for (int s = 0; s < ns_; ++s) {
      u64 v = c2[(long)s * T + g];
      if (post) v = shoup(v, post[2 * g], post[2 * g + 1], md.q);
      e[2 + s] = mul_mod(v, R, md);
    }
  }
  __syncthreads();
  const int o = blockIdx.y;
  const int n = V * (blockIdx.x * blockDim.x + threadIdx.x);
  if (n >= N) return;
  constexpr int MAXS = NS > 0 ? NS : 64;
  u64 y[V][MAXS];
#pragma unroll
  for (int s = 0; s < MAXS; ++s) {
    if (s < ns_) {
      const int gs = s < nsq ? sp0 + s : L + (s - nsq);
      const Modulus& ms = MOD(mods, gs);
      u64 v[V];
      ldv<V>(src + o * src_os + (long)s * N + n, v);
      if (dscale) {
        const u64 cm = sh[nd * W + s];
#pragma unroll
        for (int i = 0; i < V; ++i) y[i][s] = redc128(mulhi64(v[i], cm), v[i] * cm, ms.q, ms.qinv);
      } else {
#pragma unroll
        for (int i = 0; i < V; ++i) y[i][s] = shoup(v[i], c1[2 * s], c1[2 * s + 1], ms.q);
      }
    }
  }
  u64* out = dst + o * dst_os + n;
  for (int part = 0; part < 2; ++part) {
    const int m0 = part == 0 ? 0 : skip_hi, m1 = part == 0 ? min(skip_lo, nd) : nd;
    for (int m = m0; m < m1; ++m) {
      const u64* e = sh + m * W;
      Acc128 acc[V];
#pragma unroll
      for (int v = 0; v < V; ++v) acc[v].zero();
#pragma unroll
      for (int s = 0; s < MAXS; ++s) {
        if (s < ns_) {
          const u64 cs = e[2 + s];
#pragma unroll
          for (int v = 0; v < V; ++v) acc[v].mac_wide(y[v][s], cs);
        }
      }
      const u64 qm = e[0], qi = e[1];
      u64 r[V];
#pragma unroll
      for (int i = 0; i < V; ++i) r[i] = redc128(acc[i].hi, acc[i].lo, qm, qi);
      stv<V>(out + (long)m * N, r);
    }
  }
}

// Base conversion from more than four sources (a modulus switch that drops
// many primes at once): the same staged constants and arithmetic as
// k_bconv_impl, but the sources stream through registers once per chunk of TC
// targets, so a thread holds TC x V 128-bit sums instead of every source word.
// The sums are exact, so the outputs are the same words in any order. pre: the
// node-1 twiddle folded into the upper half, dscale: the inverse's deferred last
// stage folded into the source constants, as in k_bconv_impl.
template <int TC, int V>
__global__ void __launch_bounds__(256) k_bconv_many_impl(const u64* __restrict__ src, long src_os, int ns, int sp0,
                                                         int nsq, const u64* __restrict__ c1,
                                                         const u64* __restrict__ c2, int T, u64* __restrict__ dst,
                                                         long dst_os, int nd, int nq, int L, int skip_lo, int skip_hi,
                                                         const u64* __restrict__ post, int N, const ModDesc* mods,
                                                         const u64* __restrict__ r64, int pre, int dscale) {
  extern __shared__ u64 sh[];
  const int W = 2 + ns;
  const int half = 2 * V * blockIdx.x * blockDim.x >= N ? 1 : 0;  // block-uniform
  const int upper = pre ? half : 0;
  if (dscale)
    for (int s = threadIdx.x; s < ns; s += blockDim.x) {
      const int gs = s < nsq ? sp0 + s : L + (s - nsq);
      sh[nd * W + s] = mul_mod(__ldg(c1 + 2 * s), __ldg(r64 + 4 * gs + 2 + half), MOD(mods, gs));
    }
  for (int m = threadIdx.x; m < nd; m += blockDim.x) {
    const int g = m < nq ? m : L + (m - nq);
    const Modulus& md = MOD(mods, g);
    u64* e = sh + m * W;
    e[0] = md.q;
    e[1] = md.qinv;
    const u64 R = __ldg(r64 + 4 * g + upper);  // 2^64 (times w_1) mod q
    for (int s = 0; s < ns; ++s) {
      u64 v = c2[(long)s * T + g];
      if (post) v = shoup(v, post[2 * g], post[2 * g + 1], md.q);
      e[2 + s] = mul_mod(v, R, md);
    }
  }
  __syncthreads();
  const int o = blockIdx.y;
  const int n = V * (blockIdx.x * blockDim.x + threadIdx.x);
  if (n >= N) return;
  const int lo_end = min(skip_lo, nd);
  const int nt = lo_end + (nd - skip_hi);  // targets [0, skip_lo) and [skip_hi, nd)
  const u64* sp = src + o * src_os + n;
  u64* out = dst + o * dst_os + n;
  for (int t0 = 0; t0 < nt; t0 += TC) {
    int tm[TC];
#pragma unroll
    for (int c = 0; c < TC; ++c) {
      const int t = min(t0 + c, nt - 1);
      tm[c] = t < lo_end ? t : skip_hi + (t - lo_end);
    }
    Acc128 acc[TC][V];
#pragma unroll
    for (int c = 0; c < TC; ++c)
#pragma unroll
      for (int i = 0; i < V; ++i) acc[c][i].zero();
    for (int s = 0; s < ns; ++s) {
      const int gs = s < nsq ? sp0 + s : L + (s - nsq);
      const Modulus& ms = MOD(mods, gs);
      u64 v[V];
      ldv<V>(sp + (long)s * N, v);
      if (dscale) {
        const u64 cm = sh[nd * W + s];
#pragma unroll
        for (int i = 0; i < V; ++i) v[i] = redc128(mulhi64(v[i], cm), v[i] * cm, ms.q, ms.qinv);
      } else {
        const u64 w = __ldg(c1 + 2 * s), wp = __ldg(c1 + 2 * s + 1);
#pragma unroll
        for (int i = 0; i < V; ++i) v[i] = shoup(v[i], w, wp, ms.q);
      }
#pragma unroll
      for (int c = 0; c < TC; ++c) {
        const u64 cs = sh[tm[c] * W + 2 + s];
#pragma unroll
        for (int i = 0; i < V; ++i) acc[c][i].mac_wide(v[i], cs);
      }
    }
#pragma unroll
    for (int c = 0; c < TC; ++c) {
      if (t0 + c < nt) {
        const u64* e = sh + tm[c] * W;
        u64 r[V];
#pragma unroll
        for (int i = 0; i < V; ++i) r[i] = redc128(acc[c][i].hi, acc[c][i].lo, e[0], e[1]);
        stv<V>(out + (long)tm[c] * N, r);
      }
    }
  }
}

// out[m] = (a[m] - d[m]) * scale[m] (+ add[m]); limb m is data prime m.
__global__ void k_sub_scale_impl(const u64* a, long a_os, const u64* dl, long d_os, const u64* scale, const u64* add,
                                 long add_os, u64* out, long out_os, int nl, int N, const ModDesc* mods) {
  int poly = blockIdx.y;
  int m = poly % nl, o = poly / nl;
  int n = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (n >= N) return;
  const u64 q = MOD(mods, m).q;
  const u64 w = __ldg(scale + 2 * m), wp = __ldg(scale + 2 * m + 1);
  const ulonglong2 av = ld2(a + (long)o * a_os + (long)m * N + n), dv = ld2(dl + (long)o * d_os + (long)m * N + n);
  u64 x0 = shoup(sub_mod(av.x, dv.x, q), w, wp, q), x1 = shoup(sub_mod(av.y, dv.y, q), w, wp, q);
  if (add) {
    const ulonglong2 ad = ld2(add + (long)o * add_os + (long)m * N + n);
    x0 = add_mod(x0, ad.x, q);
    x1 = add_mod(x1, ad.y, q);
  }
  st2(out + (long)o * out_os + (long)m * N + n, x0, x1);
}

// ---------------------------------------------------------------- key-switch inner product
// s_c = sum_j ext_j[m] * key_j[c][g(m)] over the digits j, with ext_j[m] = d[m]
// on the digit's own primes: 128-bit lazy sums for a group of OB ciphertexts
// and V consecutive coefficients of limb m (each key word is loaded once for
// the group).
template <int OB, int V>
__device__ __forceinline__ void ks_sums(const u64* __restrict__ d, long d_os, const u64* __restrict__ ext,
                                        long ext_os, const u64* __restrict__ kb, const u64* __restrict__ ka, int m,
                                        int g, int n, int nb, int level, int alpha, int T, int N, Acc128 (&s0)[OB][V],
                                        Acc128 (&s1)[OB][V]) {
  const int dn = (level + alpha - 1) / alpha;
  const int nlx = level + alpha;
  const int jown = m < level ? m / alpha : -1;
  const u64* kbp = kb + (size_t)g * N + n;
  const u64* kap = ka + (size_t)g * N + n;
  const size_t kstride = (size_t)T * N;
  const u64* ep = ext + (long)m * N + n;
  const u64* dp = d + (long)m * N + n;
  const long jstride = (long)nlx * N;
#pragma unroll
  for (int b = 0; b < OB; ++b)
#pragma unroll
    for (int v = 0; v < V; ++v) {
      s0[b][v].zero();
      s1[b][v].zero();
    }
#if SS_KSIP_UNROLL > 0
#pragma unroll kKsipUnroll
#endif
  for (int j = 0; j < dn; ++j) {
    u64 wb[V], wa[V];
    ldv<V>(kbp + j * kstride, wb);
    ldv<V>(kap + j * kstride, wa);
    u64 x[OB][V];
#pragma unroll
    for (int b = 0; b < OB; ++b)
      if (b < nb) ldv<V>(j == jown ? dp + b * d_os : ep + b * ext_os + j * jstride, x[b]);
#pragma unroll
    for (int b = 0; b < OB; ++b) {
      if (b < nb) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
          s0[b][v].mac_wide(x[b][v], wb[v]);
          s1[b][v].mac_wide(x[b][v], wa[v]);
        }
      }
    }
  }
}

// The same sums with the loads of each digit issued SS_KSIP_STAGES - 1 digits
// ahead as asynchronous global-to-shared copies (cp.async, 16 bytes: this
// thread's two coefficients of one row), so that several digits' key and
// extended words are in flight per thread without holding registers. Every
// thread reads back only the words it copied itself, so no block barrier is
// needed. Ring layout: [slot][row][thread] of 16 bytes, row 0 the key's b
// part, 1 its a part, 2 + b the extended (or own-digit) words of ciphertext b;
// consecutive threads read consecutive 16 bytes (no bank conflicts).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(K) : "memory");
}

template <int OB, int S>
__device__ __forceinline__ void ks_sums_async(const u64* __restrict__ d, long d_os, const u64* __restrict__ ext,
                                              long ext_os, const u64* __restrict__ kb, const u64* __restrict__ ka,
                                              int m, int g, int n, int nb, int level, int alpha, int T, int N,
                                              ulonglong2* ring, Acc128 (&s0)[OB][2], Acc128 (&s1)[OB][2]) {
  constexpr int R = 2 + OB;
  const int dn = (level + alpha - 1) / alpha;
  const int nlx = level + alpha;
  const int jown = m < level ? m / alpha : -1;
  const u64* kbp = kb + (size_t)g * N + n;
  const u64* kap = ka + (size_t)g * N + n;
  const size_t kstride = (size_t)T * N;
  const u64* ep = ext + (long)m * N + n;
  const u64* dp = d + (long)m * N + n;
  const long jstride = (long)nlx * N;
  const int nt = blockDim.x;
  ulonglong2* mine = ring + threadIdx.x;
#pragma unroll
  for (int b = 0; b < OB; ++b)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      s0[b][v].zero();
      s1[b][v].zero();
    }
  auto issue = [&](int j) {
    if (j < dn) {
      ulonglong2* slot = mine + (j % S) * R * nt;
      cp_async16(slot, kbp + j * kstride);
      cp_async16(slot + nt, kap + j * kstride);
#pragma unroll
      for (int b = 0; b < OB; ++b)
        if (b < nb) cp_async16(slot + (2 + b) * nt, j == jown ? dp + b * d_os : ep + b * ext_os + j * jstride);
    }
    cp_async_commit();  // an empty group past the last digit keeps the count uniform
  };
#pragma unroll
  for (int j = 0; j < S - 1; ++j) issue(j);
  for (int j = 0; j < dn; ++j) {
    issue(j + S - 1);
    cp_async_wait<S - 1>();  // the group of digit j has landed
    const ulonglong2* slot = mine + (j % S) * R * nt;
    const ulonglong2 wb = slot[0], wa = slot[nt];
#pragma unroll
    for (int b = 0; b < OB; ++b) {
      if (b < nb) {
        const ulonglong2 x = slot[(2 + b) * nt];
        s0[b][0].mac_wide(x.x, wb.x);
        s0[b][1].mac_wide(x.y, wb.y);
        s1[b][0].mac_wide(x.x, wa.x);
        s1[b][1].mac_wide(x.y, wa.y);
      }
    }
  }
}

// Arguments of one key-switch inner-product launch (see ks_block).
struct KsJob {
  int type;  // 0: reduced sums to acc; 1: fused ModDown by P; 2: fused relinearise-and-drop
  const u64* d;
  long d_os;
  const u64* ext;
  long ext_os;
  const u64 *kb, *ka;
  int level, alpha, L, T;
  u64* acc;  // type 0
  long acc_os;
  int m0, acc_nl;
  const u64* x;  // types 1, 2
  long x_os;
  int x_cap, add_c1;
  const u64* delta;
  int nl;
  const u64 *pm, *scale;
  u64* out;
  long out_os;
  int out_cap;
  int n_outer, N;
  const ModDesc* mods;
  int gx, start;  // blocks along x; first work item (persistent launches)
};

// One block (bx, by) of a key-switch inner product: one thread per (group of
// OB ciphertexts, limb, V coefficients); the ciphertext group runs fastest over
// bx, so the blocks that read one stretch of the key run back to back and all
// but the first find it in L2. The sums are reduced once (Montgomery: the keys
// are stored times 2^64 mod q and a sum is below dn q^2 < q 2^64).
//  TYPE 0: acc[comp][m - m0] = sum_j ext_j[m] * key_j[comp][g(m)] for the limbs
//          m = m0 + by of the extended basis (data primes, then special
//          primes); acc holds acc_nl limbs per component.
//  TYPE 1, 2: the data limb m = by with the ModDown epilogue fused, so these
//          limbs of the sum never reach memory. With acc_c[m] the reduced sum
//          and delta_c[m] the converted correction ([ciphertext][2][nl][N],
//          computed beforehand from the dropped limbs), scale (s, s') Shoup
//          pairs per limb:
//    TYPE 2 (relinearise and drop q_{l-1}):
//          out_c[m] = ((P x_c[m] + acc_c[m]) - delta_c[m]) * (q_{l-1} P)^{-1},
//          x_c the input's components 0 and 1, P mod q_m in pm;
//    TYPE 1 (ModDown by P):
//          out_c[m] = (acc_c[m] - delta_c[m]) * P^{-1} (+ x_c[m] when x is
//          given; component 1 only when add_c1).
template <int OB, int TYPE, int STAGES = 0>
__device__ __forceinline__ void ks_block(const KsJob& J, int bx, int by) {
  constexpr int V = STAGES > 0 ? 2 : SS_KSIP_V;  // consecutive coefficients per thread (1, 2 or 4)
  const int N = J.N;
  const int ngroups = (J.n_outer + OB - 1) / OB;
  const int o0 = (bx % ngroups) * OB;
  const int n = V * ((bx / ngroups) * blockDim.x + threadIdx.x);
  const int m = TYPE == 0 ? J.m0 + by : by;  // local limb over level + alpha
  if (n >= N) return;
  const int nb = min(OB, J.n_outer - o0);
  const int g = m < J.level ? m : J.L + (m - J.level);
  const Modulus md = MOD(J.mods, g);
  Acc128 s0[OB][V], s1[OB][V];
  if constexpr (STAGES > 0) {
    extern __shared__ ulonglong2 ks_ring[];
    ks_sums_async<OB, STAGES>(J.d + o0 * J.d_os, J.d_os, J.ext + o0 * J.ext_os, J.ext_os, J.kb, J.ka, m, g, n, nb,
                              J.level, J.alpha, J.T, N, ks_ring, s0, s1);
  } else {
    ks_sums<OB, V>(J.d + o0 * J.d_os, J.d_os, J.ext + o0 * J.ext_os, J.ext_os, J.kb, J.ka, m, g, n, nb, J.level,
                   J.alpha, J.T, N, s0, s1);
  }
  if (TYPE == 0) {
    u64* out = J.acc + o0 * J.acc_os + (long)(m - J.m0) * N + n;
#pragma unroll
    for (int b = 0; b < OB; ++b) {
      if (b < nb) {
        u64 r0[V], r1[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
          r0[v] = redc128(s0[b][v].hi, s0[b][v].lo, md.q, md.qinv);
          r1[v] = redc128(s1[b][v].hi, s1[b][v].lo, md.q, md.qinv);
        }
        stv<V>(out + b * J.acc_os, r0);
        stv<V>(out + b * J.acc_os + (long)J.acc_nl * N, r1);
      }
    }
    return;
  }
  const u64 q = md.q;
  const u64 sc = __ldg(J.scale + 2 * m), scp = __ldg(J.scale + 2 * m + 1);
  u64 pw = 0, pwp = 0;
  if (TYPE == 2) {
    pw = __ldg(J.pm + 2 * m);
    pwp = __ldg(J.pm + 2 * m + 1);
  }
#pragma unroll
  for (int b = 0; b < OB; ++b) {
    if (b < nb) {
      const int o = o0 + b;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        u64 dl[V], r[V];
        ldv<V>(J.delta + ((long)(o * 2 + c) * J.nl + m) * N + n, dl);
        u64 xv[V];
        const bool has_x = J.x != nullptr && (TYPE == 2 || c == 0 || J.add_c1);
        if (has_x) ldv<V>(J.x + (long)o * J.x_os + ((long)c * J.x_cap + m) * N + n, xv);
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const u64 a = redc128(c ? s1[b][v].hi : s0[b][v].hi, c ? s1[b][v].lo : s0[b][v].lo, q, md.qinv);
          if (TYPE == 2) {
            r[v] = shoup(sub_mod(add_mod(shoup(xv[v], pw, pwp, q), a, q), dl[v], q), sc, scp, q);
          } else {
            r[v] = shoup(sub_mod(a, dl[v], q), sc, scp, q);
            if (has_x) r[v] = add_mod(r[v], xv[v], q);
          }
        }
        stv<V>(J.out + (long)o * J.out_os + ((long)c * J.out_cap + m) * N + n, r);
      }
    }
  }
}

template <int OB, int TYPE>
__global__ void __launch_bounds__(256, SS_KSIP_MINB) k_ks_ip_impl(const __grid_constant__ KsJob J) {
  ks_block<OB, TYPE>(J, blockIdx.x, blockIdx.y);
}

// dynamic shared memory: SS_KSIP_STAGES slots x (2 + OB) rows x 256 threads x 16 bytes
template <int OB, int TYPE>
__global__ void __launch_bounds__(256, SS_KSIP_ASYNC_MINB) k_ks_ip_async(const __grid_constant__ KsJob J) {
  ks_block<OB, TYPE, SS_KSIP_STAGES>(J, blockIdx.x, blockIdx.y);
}

// Several inner-product launches (any contexts, levels and types) as one
// persistent launch: the blocks of all jobs form one work list that every
// CTA walks with stride gridDim.x.
constexpr int kMaxKsJobs = 16;
struct KsMulti {
  int njobs, total;
  KsJob j[kMaxKsJobs];
};

template <int OB>
__global__ void __launch_bounds__(256, SS_KSIP_MINB) k_ks_ip_multi(const __grid_constant__ KsMulti M) {
  for (int t = blockIdx.x; t < M.total; t += gridDim.x) {
    int j = 0;
    while (j + 1 < M.njobs && t >= M.j[j + 1].start) ++j;
    const KsJob& J = M.j[j];
    const int local = t - J.start;
    const int by = local / J.gx, bx = local - by * J.gx;
    switch (J.type) {
      case 0: ks_block<OB, 0>(J, bx, by); break;
      case 1: ks_block<OB, 1>(J, bx, by); break;
      default: ks_block<OB, 2>(J, bx, by); break;
    }
  }
}

// ---------------------------------------------------------------- automorphism
// evaluation form, m = 2N: word j holds a(psi^(2 brv(j)+1)); sigma_g(a) at that
// point is a(psi^(g (2 brv(j)+1))), i.e. the word at brv((g (2 brv(j)+1) mod 2N - 1)/2).
// m = 3N: word h N/2 + j holds a(psi^E), E = e_h + 6 brv(j) (e_0 = 1, e_1 = 5,
// brv over log2(N/2) bits); sigma_g(a) there is the word of exponent g E mod 3N,
// whose residue mod 6 (1 or 5) gives its half and (gE - e)/6 its index.
// m = 5N/2: word h N/4 + j holds a(psi^E), E = e_h + 10 brv(j), e = (1, 3, 7, 9),
// brv over log2(N/4) bits; the residue of g E mod 10 gives the source quarter.
template <int RING>
__global__ void k_automorph_impl(const u64* a, u64* out, int g, int N, int logN, int nrows, int acap, int ocap,
                                 int level) {
  int poly = blockIdx.y;  // (bt*ncomp + c, i)
  int i = poly % level, row = poly / level;
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  unsigned src;
  if (RING == 5) {
    const int lq = logN - 2, n4 = N >> 2;
    const unsigned h = (unsigned)j >> lq, r = (unsigned)j & (unsigned)(n4 - 1);
    const unsigned E = (2u * h + 1u + (h >= 2u ? 2u : 0u)) + 10u * (__brev(r) >> (32 - lq));  // e_h = 1, 3, 7, 9
    const unsigned k = (unsigned)(((unsigned long long)g * E) % (5ull * (unsigned)N / 2ull));
    const unsigned km = k % 10u;  // 1, 3, 7 or 9
    const unsigned hs = km < 5u ? km / 2u : (km - 3u) / 2u;
    src = hs * (unsigned)n4 + (__brev((k - km) / 10u) >> (32 - lq));
  } else if (RING == 3) {
    const int lh = logN - 1, n2 = N >> 1;
    const unsigned h = (unsigned)j >> lh, r = (unsigned)j & (unsigned)(n2 - 1);
    const unsigned E = (h ? 5u : 1u) + 6u * (__brev(r) >> (32 - lh));
    const unsigned k = (unsigned)(((unsigned long long)g * E) % (3ull * (unsigned)N));
    const unsigned hs = (k % 6u == 1u) ? 0u : 1u;
    const unsigned rs = (k - (hs ? 5u : 1u)) / 6u;
    src = hs * (unsigned)n2 + (__brev(rs) >> (32 - lh));
  } else {
    unsigned rj = __brev((unsigned)j) >> (32 - logN);
    unsigned k = (unsigned)(((unsigned long long)g * (2 * rj + 1)) % (2u * (unsigned)N));
    src = __brev((k - 1) / 2) >> (32 - logN);
  }
  out[((size_t)row * ocap + i) * N + j] = a[((size_t)row * acap + i) * N + src];
}

// ---------------------------------------------------------------- sampling
__global__ void k_uniform_impl(u64* out, long out_os, int nl, int q0, int nq, int L, u32 id0, u32 tag, u32 k0,
                               u32 k1, int N, const ModDesc* mods) {
  int poly = blockIdx.y;
  int i = poly % nl, o = poly / nl;
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  int g = i < nq ? q0 + i : L + (i - nq);
  const Modulus& md = MOD(mods, g);
  Philox4 r = philox((u32)n, (u32)g, id0 + (u32)o, tag, k0, k1);
  u64 lo = ((u64)r.x[1] << 32) | r.x[0];
  u64 hi = ((u64)r.x[3] << 32) | r.x[2];
  // (hi 2^64 + lo) mod q = (hi mod q)(2^64 mod q) + lo mod q
  u64 R = barrett_reduce128(1, 0, md);
  u64 h = barrett_reduce128(0, hi, md);
  u64 v = add_mod(mul_mod(h, R, md), barrett_reduce128(0, lo, md), md.q);
  out[(long)o * out_os + (long)i * N + n] = v;
}

__global__ void k_cbd_impl(i64* out, u32 id0, u32 tag, u32 k0, u32 k1, int N) {
  int o = blockIdx.y;
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  Philox4 r = philox((u32)n, 0u, id0 + (u32)o, tag, k0, k1);
  out[(long)o * N + n] = (i64)__popc(r.x[0] & 0x1FFFFFu) - (i64)__popc(r.x[1] & 0x1FFFFFu);
}

// out[o][i] = (m[o] + tmul * e[o]) mod q_g  (coefficient form)
__global__ void k_lift_small_impl(const i64* e, const u64* m, u64 tmul, u64* out, long out_os, int nl, int q0,
                                  int nq, int L, int N, const ModDesc* mods) {
  int poly = blockIdx.y;
  int i = poly % nl, o = poly / nl;
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  int g = i < nq ? q0 + i : L + (i - nq);
  const Modulus& md = MOD(mods, g);
  u64 q = md.q;
  i64 ev = e ? e[(long)o * N + n] : 0;
  u64 el = ev >= 0 ? (u64)ev : q - (u64)(-ev);
  u64 v = mul_mod(el, tmul, md);  // tmul, m < p^r < q (checked at context creation)
  if (m) v = add_mod(v, m[(long)o * N + n], q);
  out[(long)o * out_os + (long)i * N + n] = v;
}

// out = x - a * s  (evaluation form); s indexed by global prime
__global__ void k_mul_sub_impl(const u64* x, long x_os, const u64* a, long a_os, const u64* s, u64* out, long out_os,
                               int nl, int q0, int nq, int L, int N, const ModDesc* mods) {
  int poly = blockIdx.y;
  int i = poly % nl, o = poly / nl;
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  int g = i < nq ? q0 + i : L + (i - nq);
  const Modulus& md = MOD(mods, g);
  u64 p = mul_mod(a[(long)o * a_os + (long)i * N + n], s[(long)g * N + n], md);
  out[(long)o * out_os + (long)i * N + n] = sub_mod(x[(long)o * x_os + (long)i * N + n], p, md.q);
}

// every word of limb (poly mod T) times 2^64 mod its prime
__global__ void k_to_mont_impl(u64* a, int T, int N, const ModDesc* mods) {
  const int poly = blockIdx.y;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const Modulus& md = MOD(mods, poly % T);
  const u64 R = barrett_reduce128(1, 0, md);
  u64* w = a + (size_t)poly * N + n;
  *w = mul_mod(*w, R, md);
}

struct GadgetArgs {
  u64 pmod[16];
};

// b_j[i] += (P mod q_i) * s'[i] for the data primes i of digit j
__global__ void k_gadget_impl(u64* b, const u64* sp, int j, int alpha, int L, int T, int N, GadgetArgs G,
                              const ModDesc* mods) {
  int k = blockIdx.y;
  int i = j * alpha + k;
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N || i >= L) return;
  const Modulus& md = MOD(mods, i);
  size_t o = ((size_t)j * T + i) * N + n;
  b[o] = add_mod(b[o], mul_mod(G.pmod[k], sp[(size_t)i * N + n], md), md.q);
}

// v = c0 + c1 s (+ c2 s^2)
__global__ void k_dec_dot_impl(const u64* a, int ncomp, int level, int cap, const u64* s, const u64* s2, u64* v,
                               int N, const ModDesc* mods) {
  int poly = blockIdx.y;  // (bt, i)
  int i = poly % level, bt = poly / level;
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const Modulus& md = MOD(mods, i);
  size_t lc = (size_t)cap * N;
  const u64* A = a + (size_t)bt * ncomp * lc + (size_t)i * N + n;
  Acc128 acc;
  acc.zero();
  acc.add(A[0]);
  acc.mac(A[lc], s[(size_t)i * N + n]);
  if (ncomp == 3) acc.mac(A[2 * lc], s2[(size_t)i * N + n]);
  v[((size_t)bt * level + i) * N + n] = barrett_reduce128(acc.hi, acc.lo, md);
}

// Garner mixed-radix CRT of one coefficient, centred against (Q-1)/2, mod p^e.
__global__ void k_crt_impl(const u64* v, int level, int N, int stride, int count, const u64* pinv, const u64* half,
                           const u64* qmodt, u64 te, u64* out, const ModDesc* mods) {
  int bt = blockIdx.y;
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  int n = k * stride;
  u64 dig[200];
  for (int i = 0; i < level; ++i) {
    const Modulus& md = MOD(mods, i);
    u64 q = md.q;
    u64 x = v[((size_t)bt * level + i) * N + n];
    u64 acc = 0;
    for (int j = i - 1; j >= 0; --j) {
      u64 qj = MOD(mods, j).q;
      u64 qjm = qj >= q ? qj - q : qj;
      acc = add_mod(mul_mod(acc, qjm, md), dig[j], q);
    }
    dig[i] = i == 0 ? x : mul_mod(sub_mod(x, acc, q), pinv[i], md);
  }
  int neg = 0;
  for (int i = level - 1; i >= 0; --i) {
    if (dig[i] != half[i]) { neg = dig[i] > half[i]; break; }
  }
  u64 m = 0;
  for (int i = 0; i < level; ++i) m = (m + (u64)(((u128)(dig[i] % te) * qmodt[i]) % te)) % te;
  if (neg) m = (m + te - qmodt[level]) % te;
  out[(size_t)bt * N + n] = m;
}

// out = sum_t c_t * y_t (+ cst on component 0), one 128-bit lazy sum per word.
// Scalars are centred integers with |c| < q, so the lift is one add.
struct LinArgs {
  const u64* ptr[16];
  int cap[16];
  i64 c[16];
};

// out = sum_t c_t y_t (+ cst on component 0), one word per thread. All term
// words are loaded before any arithmetic so the loads overlap.
__global__ void __launch_bounds__(256) k_lincomb_impl(LinArgs A, int nterms, i64 cst, int small, int tiny, u64* out,
                                                      int ocap, int N, int ncomp, int level, const ModDesc* mods) {
  const int poly = blockIdx.y;  // (bt, comp, i)
  const int i = poly % level, comp = (poly / level) % ncomp, bt = poly / (level * ncomp);
  const int n = 2 * (blockIdx.x * blockDim.x + threadIdx.x);  // two consecutive words per thread
  if (n >= N) return;
  const Modulus& md = MOD(mods, i);
  const u64 q = md.q;
  const size_t row = (size_t)(bt * ncomp + comp);
  ulonglong2 y[16];
#pragma unroll
  for (int t = 0; t < 16; ++t)
    if (t < nterms) y[t] = ld2(A.ptr[t] + (row * A.cap[t] + i) * N + n);
  u64 r0, r1;
  if (tiny) {
    // |c| < 2^27 (constant included), at most 16 terms, words below 2^58: the
    // 32-bit halves of every word times |c| sum in 64 bits without overflow;
    // terms arrive sorted: the first `small` - 1 have c >= 0, the rest c < 0
    const int npos = small - 1;
    u64 pl0 = 0, ph0 = 0, nl0 = 0, nh0 = 0, pl1 = 0, ph1 = 0, nl1 = 0, nh1 = 0;
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      if (t < nterms) {
        const i64 c = A.c[t];
        const uint32_t m = (uint32_t)(t < npos ? c : -c);
        if (t < npos) {
          pl0 += (u64)(uint32_t)y[t].x * m;
          ph0 += (u64)(uint32_t)(y[t].x >> 32) * m;
          pl1 += (u64)(uint32_t)y[t].y * m;
          ph1 += (u64)(uint32_t)(y[t].y >> 32) * m;
        } else {
          nl0 += (u64)(uint32_t)y[t].x * m;
          nh0 += (u64)(uint32_t)(y[t].x >> 32) * m;
          nl1 += (u64)(uint32_t)y[t].y * m;
          nh1 += (u64)(uint32_t)(y[t].y >> 32) * m;
        }
      }
    }
    if (comp == 0 && cst > 0) {
      pl0 += (u64)cst;
      pl1 += (u64)cst;
    }
    if (comp == 0 && cst < 0) {
      nl0 += (u64)(-cst);
      nl1 += (u64)(-cst);
    }
    r0 = sub_mod(reduce_split(ph0, pl0, md), reduce_split(nh0, nl0, md), q);
    r1 = sub_mod(reduce_split(ph1, pl1, md), reduce_split(nh1, nl1, md), q);
  } else if (small) {
    // |c| < 2^32: y * |c| is two 32x32 products; positive and negative terms
    // are summed apart (each sum < 2^92) and reduced once each.
    // terms arrive sorted: the first `small` - 1 have c >= 0, the rest c < 0
    Acc128 p0, n0, p1, n1;
    p0.zero();
    n0.zero();
    p1.zero();
    n1.zero();
    const int npos = small - 1;
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      if (t < nterms) {
        const i64 c = A.c[t];
        const uint32_t m = (uint32_t)(t < npos ? c : -c);
        if (t < npos) {
          add_small(p0, y[t].x, m);
          add_small(p1, y[t].y, m);
        } else {
          add_small(n0, y[t].x, m);
          add_small(n1, y[t].y, m);
        }
      }
    }
    if (comp == 0 && cst > 0) {
      p0.add((u64)cst);
      p1.add((u64)cst);
    }
    if (comp == 0 && cst < 0) {
      n0.add((u64)(-cst));
      n1.add((u64)(-cst));
    }
    r0 = sub_mod(barrett_reduce128(p0.hi, p0.lo, md), barrett_reduce128(n0.hi, n0.lo, md), q);
    r1 = sub_mod(barrett_reduce128(p1.hi, p1.lo, md), barrett_reduce128(n1.hi, n1.lo, md), q);
  } else {
    // |c| < q (checked on the host): c mod q is c or q - |c|
    Acc128 s0, s1;
    s0.zero();
    s1.zero();
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      if (t < nterms) {
        const i64 c = A.c[t];
        const u64 w = c >= 0 ? (u64)c : q - (u64)(-c);
        s0.mac_wide(y[t].x, w);
        s1.mac_wide(y[t].y, w);
      }
    }
    if (comp == 0 && cst != 0) {
      const u64 w = cst >= 0 ? (u64)cst : q - (u64)(-cst);
      s0.add(w);
      s1.add(w);
    }
    r0 = barrett_reduce128(s0.hi, s0.lo, md);
    r1 = barrett_reduce128(s1.hi, s1.lo, md);
  }
  st2(out + (row * ocap + i) * N + n, r0, r1);
}

// Several linear combinations of the same inputs in one pass:
// out_j = sum_i c[j][i] y_i for j < nout, every y_i read once. Scalars are
// below 2^32 in magnitude (two 32-bit products per term, positive and
// negative sums apart) or, with `small` = 0, below the smallest prime.
struct LinMultiArgs {
  const u64* ptr[16];
  int cap[16];
  u64* out[16];
  int ocap[16];
  i64 c[16][16];
};

// Two consecutive words per thread.
__global__ void __launch_bounds__(256) k_lincomb_multi_impl(LinMultiArgs A, int nin, int nout, int small, int tiny,
                                                            int N, int ncomp, int level, const ModDesc* mods) {
  const int poly = blockIdx.y;  // (bt, comp, i)
  const int i = poly % level, comp = (poly / level) % ncomp, bt = poly / (level * ncomp);
  const int n = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (n >= N) return;
  const Modulus& md = MOD(mods, i);
  const u64 q = md.q;
  const size_t row = (size_t)(bt * ncomp + comp);
  ulonglong2 y[16];
#pragma unroll
  for (int t = 0; t < 16; ++t)
    if (t < nin) y[t] = ld2(A.ptr[t] + (row * A.cap[t] + i) * N + n);
  for (int j = 0; j < nout; ++j) {
    u64 r0, r1;
    if (tiny) {
      // |c| < 2^27, at most 16 terms, words below 2^58: the low and high 32-bit
      // halves of every word times |c| sum without overflow in 64 bits
      u64 pl0 = 0, ph0 = 0, nl0 = 0, nh0 = 0, pl1 = 0, ph1 = 0, nl1 = 0, nh1 = 0;
#pragma unroll
      for (int t = 0; t < 16; ++t) {
        if (t < nin) {
          const i64 c = A.c[j][t];
          if (c > 0) {
            const uint32_t m = (uint32_t)c;
            pl0 += (u64)(uint32_t)y[t].x * m;
            ph0 += (u64)(uint32_t)(y[t].x >> 32) * m;
            pl1 += (u64)(uint32_t)y[t].y * m;
            ph1 += (u64)(uint32_t)(y[t].y >> 32) * m;
          } else if (c < 0) {
            const uint32_t m = (uint32_t)(-c);
            nl0 += (u64)(uint32_t)y[t].x * m;
            nh0 += (u64)(uint32_t)(y[t].x >> 32) * m;
            nl1 += (u64)(uint32_t)y[t].y * m;
            nh1 += (u64)(uint32_t)(y[t].y >> 32) * m;
          }
        }
      }
      r0 = sub_mod(reduce_split(ph0, pl0, md), reduce_split(nh0, nl0, md), q);
      r1 = sub_mod(reduce_split(ph1, pl1, md), reduce_split(nh1, nl1, md), q);
    } else if (small) {
      Acc128 p0, n0, p1, n1;
      p0.zero();
      n0.zero();
      p1.zero();
      n1.zero();
#pragma unroll
      for (int t = 0; t < 16; ++t) {
        if (t < nin) {
          const i64 c = A.c[j][t];
          if (c > 0) {
            add_small(p0, y[t].x, (uint32_t)c);
            add_small(p1, y[t].y, (uint32_t)c);
          } else if (c < 0) {
            add_small(n0, y[t].x, (uint32_t)(-c));
            add_small(n1, y[t].y, (uint32_t)(-c));
          }
        }
      }
      r0 = sub_mod(barrett_reduce128(p0.hi, p0.lo, md), barrett_reduce128(n0.hi, n0.lo, md), q);
      r1 = sub_mod(barrett_reduce128(p1.hi, p1.lo, md), barrett_reduce128(n1.hi, n1.lo, md), q);
    } else {
      Acc128 s0, s1;
      s0.zero();
      s1.zero();
#pragma unroll
      for (int t = 0; t < 16; ++t) {
        if (t < nin) {
          const i64 c = A.c[j][t];
          if (c != 0) {
            const u64 w = c > 0 ? (u64)c : q - (u64)(-c);
            s0.mac_wide(y[t].x, w);
            s1.mac_wide(y[t].y, w);
          }
        }
      }
      r0 = barrett_reduce128(s0.hi, s0.lo, md);
      r1 = barrett_reduce128(s1.hi, s1.lo, md);
    }
    st2(A.out[j] + (row * A.ocap[j] + i) * N + n, r0, r1);
  }
}

// acc_c[l-1] += P * d_c[l-1] (mod q_{l-1}) for c = 0, 1: the last data limb of
// the extended ciphertext P*d + acc before it joins the dropped primes. That
// limb is limb acc_limb of acc's nx limbs per component.
__global__ void k_fixup_last_impl(u64* acc, long acc_os, int nx, int acc_limb, const u64* d, long d_os, int dcap,
                                  int l, const u64* pmod, int N, const ModDesc* mods) {
  int o = blockIdx.y;  // (bt, c)
  int bt = o >> 1, c = o & 1;
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int i = l - 1;
  u64 q = MOD(mods, i).q;
  u64* a = acc + (long)bt * acc_os + ((long)c * nx + acc_limb) * N + n;
  u64 x = d[(long)bt * d_os + ((long)c * dcap + i) * N + n];
  *a = add_mod(*a, shoup(x, pmod[2 * i], pmod[2 * i + 1], q), q);
}

// out[g] = a[g]^2 for every prime g (evaluation form)
__global__ void k_square_impl(const u64* a, u64* out, int N, const ModDesc* mods) {
  int g = blockIdx.y;
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  u64 x = a[(size_t)g * N + n];
  out[(size_t)g * N + n] = mul_mod(x, x, MOD(mods, g));
}

// out[c][i] = sum_b a[b][c][i]
__global__ void k_batch_sum_impl(const u64* a, u64* out, int count, int ncomp, int level, int acap, int ocap, int N,
                                 const ModDesc* mods) {
  int poly = blockIdx.y;  // (c, i)
  int i = poly % level, c = poly / level;
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  u64 q = MOD(mods, i).q;
  u64 s = 0;
  for (int b = 0; b < count; ++b) s = add_mod(s, a[((size_t)(b * ncomp + c) * acap + i) * N + n], q);
  out[((size_t)c * ocap + i) * N + n] = s;
}

}  // namespace

// ======================================================================= launchers
void k_fixup_last(Context& C, u64* acc, long acc_os, int nx, int acc_limb, const Buf& d, int l, const u64* pmod,
                  int B, cudaStream_t st) {
  TIMED(KC_ELEM, 3.0 * 2 * B * C.N * 8.0,
        k_fixup_last_impl<<<grid_for(C.N, 2 * B), TPB, 0, st>>>(acc, acc_os, nx, acc_limb, d.data,
                                                                 (long)d.ncomp * d.cap * C.N, d.cap, l, pmod, C.N,
                                                                 C.d_mod));
  LAUNCHED();
}

void k_square(Context& C, const u64* a, u64* out, int nprimes, cudaStream_t st) {
  k_square_impl<<<grid_for(C.N, nprimes), TPB, 0, st>>>(a, out, C.N, C.d_mod);
  ++C.launches;
  SS_CUDA(cudaGetLastError());
}

void k_lincomb(Context& C, const std::vector<const Buf*>& ys, const std::vector<i64>& cs, i64 cst, Buf& out,
               cudaStream_t st) {
  int nt = (int)ys.size();
  if (nt < 1 || nt > 16) throw Error(SS_ERR_PARAM, "linear combination of 1..16 terms");
  LinArgs A;
  bool small = cst > -(1LL << 32) && cst < (1LL << 32);
  for (int t = 0; t < nt; ++t) small = small && cs[t] > -(1LL << 32) && cs[t] < (1LL << 32);
  bool tiny = small && cst > -(1LL << 27) && cst < (1LL << 27);
  for (int t = 0; t < nt; ++t) tiny = tiny && cs[t] > -(1LL << 27) && cs[t] < (1LL << 27);
  if (!small) {  // the general path lifts c as c or q - |c|: every |c| must lie below every prime
    const u64 qmin = 1ULL << (C.prm.bits - 1);
    for (int t = 0; t <= nt; ++t) {
      const i64 c = t < nt ? cs[t] : cst;
      if (c == INT64_MIN || (u64)(c < 0 ? -c : c) >= qmin)
        throw Error(SS_ERR_PARAM, "linear-combination scalar too large for the primes");
    }
  }
  int npos = 0, k2 = 0;
  if (small) {  // non-negative scalars first (the sum does not depend on the order)
    for (int t = 0; t < nt; ++t)
      if (cs[t] >= 0) { A.ptr[k2] = ys[t]->data; A.cap[k2] = ys[t]->cap; A.c[k2] = cs[t]; ++k2; ++npos; }
    for (int t = 0; t < nt; ++t)
      if (cs[t] < 0) { A.ptr[k2] = ys[t]->data; A.cap[k2] = ys[t]->cap; A.c[k2] = cs[t]; ++k2; }
  } else {
    for (int t = 0; t < nt; ++t) { A.ptr[t] = ys[t]->data; A.cap[t] = ys[t]->cap; A.c[t] = cs[t]; }
  }
  int polys = out.count * out.ncomp * out.level;
  TIMED(KC_ELEM, (nt + 1.0) * polys * C.N * 8.0,
        k_lincomb_impl<<<grid_for(C.N / 2, polys), TPB, 0, st>>>(A, nt, cst, small ? npos + 1 : 0, tiny ? 1 : 0, out.data,
                                                                  out.cap, C.N,
                                                              out.ncomp, out.level, C.d_mod));
  LAUNCHED();
}

void k_lincomb_multi(Context& C, const std::vector<const Buf*>& ys, const std::vector<std::vector<i64>>& cs,
                     const std::vector<Buf*>& outs, cudaStream_t st) {
  const int nin = (int)ys.size(), nout = (int)outs.size();
  if (nin < 1 || nin > 16 || nout < 1 || nout > 16 || (int)cs.size() != nout)
    throw Error(SS_ERR_PARAM, "multi-output linear combination of 1..16 inputs and outputs");
  LinMultiArgs A;
  bool small = true, tiny = C.prm.bits <= 58;
  const u64 qmin = 1ULL << (C.prm.bits - 1);
  for (int j = 0; j < nout; ++j) {
    if ((int)cs[j].size() != nin) throw Error(SS_ERR_PARAM, "coefficient row length");
    A.out[j] = outs[j]->data;
    A.ocap[j] = outs[j]->cap;
    for (int t = 0; t < nin; ++t) {
      const i64 c = cs[j][t];
      if (c == INT64_MIN || (u64)(c < 0 ? -c : c) >= qmin)
        throw Error(SS_ERR_PARAM, "linear-combination scalar too large for the primes");
      small = small && c > -(1LL << 32) && c < (1LL << 32);
      tiny = tiny && c > -(1LL << 27) && c < (1LL << 27);
      A.c[j][t] = c;
    }
  }
  for (int t = 0; t < nin; ++t) {
    A.ptr[t] = ys[t]->data;
    A.cap[t] = ys[t]->cap;
  }
  const Buf& o0 = *outs[0];
  const int polys = o0.count * o0.ncomp * o0.level;
  TIMED(KC_ELEM, (double)(nin + nout) * polys * C.N * 8.0,
        k_lincomb_multi_impl<<<grid_for(C.N / 2, polys), TPB, 0, st>>>(A, nin, nout, small ? 1 : 0, tiny ? 1 : 0, C.N,
                                                                        o0.ncomp,
                                                                    o0.level, C.d_mod));
  LAUNCHED();
}

void k_batch_sum(Context& C, const Buf& a, Buf& out, cudaStream_t st) {
  k_batch_sum_impl<<<grid_for(C.N, a.ncomp * a.level), TPB, 0, st>>>(a.data, out.data, a.count, a.ncomp, a.level,
                                                                      a.cap, out.cap, C.N, C.d_mod);
  ++C.launches;
  SS_CUDA(cudaGetLastError());
}



void k_binary(Context& C, int op, const Buf& a, const Buf& b, Buf& out, cudaStream_t st) {
  int polys = a.count * a.ncomp * a.level;
  TIMED(KC_ELEM, 3.0 * polys * (double)C.N * 8.0,
  k_binary_impl<<<grid_for(C.N / 2, polys), TPB, 0, st>>>(op, a.data, b.data, out.data, C.N, a.ncomp, a.level, a.cap,
                                                       b.cap, out.cap, b.count == 1 && a.count > 1, C.d_mod));
  LAUNCHED();
}

void k_scalar(Context& C, int op, const Buf& a, i64 c, Buf& out, cudaStream_t st) {
  int polys = a.count * a.ncomp * a.level;
  TIMED(KC_ELEM, 2.0 * polys * (double)C.N * 8.0,
  k_scalar_impl<<<grid_for(C.N / 2, polys), TPB, 0, st>>>(op, a.data, c, out.data, C.N, a.ncomp, a.level, a.cap,
                                                       out.cap, C.d_mod, C.d_pinv));
  LAUNCHED();
}

void k_copy_limbs(Context& C, const Buf& a, Buf& out, int level, cudaStream_t st) {
  int polys = a.count * a.ncomp * level;
  TIMED(KC_ELEM, 2.0 * polys * (double)C.N * 8.0,
  k_copy_impl<<<grid_for(C.N, polys), TPB, 0, st>>>(a.data, out.data, C.N, a.ncomp, level, a.cap, out.cap));
  LAUNCHED();
}

void k_tensor(Context& C, const Buf& a, const Buf& b, Buf& out, cudaStream_t st) {
  int polys = a.count * a.level;
  TIMED(KC_TENSOR, 7.0 * polys * (double)C.N * 8.0,
  k_tensor_impl<<<grid_for(C.N / 2, polys), TPB, 0, st>>>(a.data, b.data, out.data, C.N, a.level, a.cap, b.cap, out.cap,
                                                       C.d_mod));
  LAUNCHED();
}

void k_bconv(Context& C, const u64* src, long src_os, int ns, int sp0, const u64* c1, const u64* c2, u64* dst,
             long dst_os, int nd, int nq, int skip_lo, int skip_hi, const u64* post, int n_outer, cudaStream_t st,
             int nsq, bool pre_w1, bool post_scale) {
  if (nsq < 0) nsq = ns;  // every source is the data or special prime sp0 + s
  dim3 g = grid_for(C.N, n_outer);
  if (ns < 1 || ns > 64) throw Error(SS_ERR_PARAM, "base conversion from 1..64 primes");
  static_assert(SS_BCONV_V == 2, "both base-conversion kernels cover 2 * 256 coefficients per block");
  if ((pre_w1 || post_scale) && (C.m_odd != 1 || (C.N / 2) % (SS_BCONV_V * TPB) != 0))
    throw Error(SS_ERR_PARAM, "twiddle folding needs the ring X^N + 1 and N >= 1024");
  if (skip_hi <= skip_lo) skip_lo = skip_hi = nd;
  const int pre = pre_w1 ? 1 : 0, dscale = post_scale ? 1 : 0;
  size_t smem = (size_t)(nd * (2 + ns) + dscale * ns) * 8;
  if (smem > 48 * 1024) throw Error(SS_ERR_PARAM, "base conversion tables exceed 48 KiB of shared memory");
  int kr_ = kt_begin(C, st);
#define SS_BCONV(NSV, VV)                                                                                        \
  k_bconv_impl<NSV, VV><<<dim3((g.x + VV - 1) / VV, g.y), TPB, smem, st>>>(                                       \
      src, src_os, ns, sp0, nsq, c1, c2, C.ntot, dst, dst_os, nd, nq, C.L, skip_lo, skip_hi, post, C.N, C.d_mod,     \
      C.d_r64, pre, dscale)
  switch (ns) {
    case 1: SS_BCONV(1, SS_BCONV_V); break;
    case 2: SS_BCONV(2, SS_BCONV_V); break;
    case 3: SS_BCONV(3, SS_BCONV_V); break;
    case 4: SS_BCONV(4, SS_BCONV_V); break;
    default:
      k_bconv_many_impl<4, 2><<<dim3((g.x + 1) / 2, g.y), TPB, smem, st>>>(
          src, src_os, ns, sp0, nsq, c1, c2, C.ntot, dst, dst_os, nd, nq, C.L, skip_lo, skip_hi, post, C.N, C.d_mod,
          C.d_r64, pre, dscale);
      break;
  }
#undef SS_BCONV
  kt_end(C, kr_, KC_BCONV, (double)(ns + nd - (skip_hi - skip_lo)) * n_outer * C.N * 8.0, st);
  LAUNCHED();
}

void k_sub_scale(Context& C, const u64* a, long a_os, const u64* dl, long d_os, const u64* scale, const u64* add,
                 long add_os, u64* out, long out_os, int nl, int n_outer, cudaStream_t st) {
  TIMED(KC_SUBSCALE, (add ? 4.0 : 3.0) * nl * n_outer * (double)C.N * 8.0,
  k_sub_scale_impl<<<grid_for(C.N / 2, nl * n_outer), TPB, 0, st>>>(a, a_os, dl, d_os, scale, add, add_os, out, out_os,
                                                                 nl, C.N, C.d_mod));
  LAUNCHED();
}

void k_to_montgomery(Context& C, u64* data, int npoly, cudaStream_t st) {
  k_to_mont_impl<<<grid_for(C.N, npoly), TPB, 0, st>>>(data, C.ntot, C.N, C.d_mod);
  LAUNCHED();
}

static KsJob ks_job(Context& C, int type, const u64* d, long d_os, const u64* ext, long ext_os, const KeyDev& K,
                    int level, int n_outer, int nlimbs) {
  KsJob J{};
  J.type = type;
  J.d = d;
  J.d_os = d_os;
  J.ext = ext;
  J.ext_os = ext_os;
  J.kb = K.b;
  J.ka = K.a;
  J.level = level;
  J.alpha = C.alpha;
  J.L = C.L;
  J.T = C.ntot;
  J.n_outer = n_outer;
  J.N = C.N;
  J.mods = C.d_mod;
  const int nx_blocks = (C.N / SS_KSIP_V + TPB - 1) / TPB;
  J.gx = ((n_outer + SS_KSIP_OB - 1) / SS_KSIP_OB) * nx_blocks;
  (void)nlimbs;
  return J;
}

static_assert(sizeof(KsJob) <= sizeof(KsReq::job), "inner-product job fits the merge request");

static void ks_launch(Context& C, const KsJob& J, int nlimbs, double bytes, cudaStream_t st) {
  if (ks_merger()) {
    KsReq r;
    r.C = &C;
    r.nlimbs = nlimbs;
    std::memcpy(r.job, &J, sizeof(J));
    ks_merger()->submit_ks(r, st);
    return;
  }
  constexpr int OB = SS_KSIP_OB;
  const dim3 grid((unsigned)J.gx, (unsigned)nlimbs);
#if SS_KSIP_STAGES > 0
  static_assert(SS_KSIP_V == 2, "the cp.async inner product copies two coefficients per thread");
  constexpr size_t ring = (size_t)SS_KSIP_STAGES * (2 + OB) * TPB * 16;
  if (ring > 48 * 1024) {  // beyond the default limit: opt in once per device (the attribute is per device)
    static std::atomic<unsigned long long> done{0};
    int dev = 0;
    SS_CUDA(cudaGetDevice(&dev));
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(done.load() & bit)) {
      SS_CUDA(cudaFuncSetAttribute(k_ks_ip_async<OB, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ring));
      SS_CUDA(cudaFuncSetAttribute(k_ks_ip_async<OB, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ring));
      SS_CUDA(cudaFuncSetAttribute(k_ks_ip_async<OB, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ring));
      done.fetch_or(bit);
    }
  }
  switch (J.type) {
    case 0: TIMED(KC_KSIP, bytes, (k_ks_ip_async<OB, 0><<<grid, TPB, ring, st>>>(J))); break;
    case 1: TIMED(KC_KSIP, bytes, (k_ks_ip_async<OB, 1><<<grid, TPB, ring, st>>>(J))); break;
    default: TIMED(KC_KSIP, bytes, (k_ks_ip_async<OB, 2><<<grid, TPB, ring, st>>>(J))); break;
  }
#else
  switch (J.type) {
    case 0: TIMED(KC_KSIP, bytes, (k_ks_ip_impl<OB, 0><<<grid, TPB, 0, st>>>(J))); break;
    case 1: TIMED(KC_KSIP, bytes, (k_ks_ip_impl<OB, 1><<<grid, TPB, 0, st>>>(J))); break;
    default: TIMED(KC_KSIP, bytes, (k_ks_ip_impl<OB, 2><<<grid, TPB, 0, st>>>(J))); break;
  }
#endif
  LAUNCHED();
}

void k_ks_ip(Context& C, const u64* d, long d_os, const u64* ext, long ext_os, const KeyDev& K, int level, u64* acc,
             long acc_os, int n_outer, cudaStream_t st, int m0, int nlimbs) {
  const int dn = (level + C.alpha - 1) / C.alpha;
  if (nlimbs < 0) nlimbs = level + C.alpha - m0;
  KsJob J = ks_job(C, 0, d, d_os, ext, ext_os, K, level, n_outer, nlimbs);
  J.acc = acc;
  J.acc_os = acc_os;
  J.m0 = m0;
  J.acc_nl = nlimbs;
  // each key limb is read once per launch; ext limbs and the sums once per ciphertext
  ks_launch(C, J, nlimbs, ((double)dn * nlimbs * (n_outer + 2.0) + 2.0 * nlimbs * n_outer) * (double)C.N * 8.0, st);
}

void k_ks_ip_fused(Context& C, const u64* d, long d_os, const u64* ext, long ext_os, const KeyDev& K, int level,
                   int nlimbs, bool drop, const Buf* x, bool add_c1, const u64* delta, int nl, const u64* pm,
                   const u64* scale, Buf& out, int n_outer, cudaStream_t st) {
  const int dn = (level + C.alpha - 1) / C.alpha;
  KsJob J = ks_job(C, drop ? 2 : 1, d, d_os, ext, ext_os, K, level, n_outer, nlimbs);
  J.x = x ? x->data : nullptr;
  J.x_os = x ? (long)x->ncomp * x->cap * C.N : 0;
  J.x_cap = x ? x->cap : 0;
  J.add_c1 = add_c1 ? 1 : 0;
  J.delta = delta;
  J.nl = nl;
  J.pm = pm;
  J.scale = scale;
  J.out = out.data;
  J.out_os = (long)out.ncomp * out.cap * C.N;
  J.out_cap = out.cap;
  const int nx = x ? (drop || add_c1 ? 2 : 1) : 0;
  ks_launch(C, J, nlimbs,
            ((double)dn * nlimbs * (n_outer + 2.0) + (4.0 + nx) * nlimbs * n_outer) * (double)C.N * 8.0, st);
}

KsMerger*& ks_merger() {
  static thread_local KsMerger* m = nullptr;
  return m;
}

// Jobs of several lanes as persistent launches of at most kMaxKsJobs jobs each.
void ks_multi(const std::vector<KsReq>& reqs, cudaStream_t st) {
  static std::atomic<int> resident_{0};
  int resident = resident_.load();
  if (!resident) {
    int dev = 0, sms = 0, per = 0;
    SS_CUDA(cudaGetDevice(&dev));
    SS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_ks_ip_multi<SS_KSIP_OB>, TPB, 0));
    resident = sms * std::max(1, per);
    resident_.store(resident);
  }
  for (size_t b0 = 0; b0 < reqs.size(); b0 += kMaxKsJobs) {
    const size_t b1 = std::min(reqs.size(), b0 + kMaxKsJobs);
    KsMulti M;
    M.njobs = 0;
    M.total = 0;
    for (size_t r = b0; r < b1; ++r) {
      KsJob J;
      std::memcpy(&J, reqs[r].job, sizeof(J));
      J.start = M.total;
      M.total += J.gx * reqs[r].nlimbs;
      M.j[M.njobs++] = J;
    }
    if (M.total == 0) continue;
    k_ks_ip_multi<SS_KSIP_OB><<<std::min(M.total, resident), TPB, 0, st>>>(M);
    SS_CUDA(cudaGetLastError());
    ++reqs[b0].C->launches;
  }
}

void k_automorph(Context& C, const Buf& a, int g, Buf& out, cudaStream_t st) {
  int rows = a.count * a.ncomp;
  TIMED(KC_AUTOMORPH, 2.0 * rows * a.level * (double)C.N * 8.0,
  if (C.m_odd == 5) k_automorph_impl<5><<<grid_for(C.N, rows * a.level), TPB, 0, st>>>(
      a.data, out.data, g, C.N, C.logN, rows, a.cap, out.cap, a.level);
  else if (C.m_odd == 3) k_automorph_impl<3><<<grid_for(C.N, rows * a.level), TPB, 0, st>>>(
      a.data, out.data, g, C.N, C.logN, rows, a.cap, out.cap, a.level);
  else k_automorph_impl<1><<<grid_for(C.N, rows * a.level), TPB, 0, st>>>(
      a.data, out.data, g, C.N, C.logN, rows, a.cap, out.cap, a.level));
  LAUNCHED();
}

static void seed_words(const Context& C, u32& k0, u32& k1) {
  k0 = (u32)(C.prm.seed & 0xffffffffu);
  k1 = (u32)(C.prm.seed >> 32);
}

void k_uniform(Context& C, u64* out, long out_os, int n_outer, int nl, int q0, int nq, u32 id0, u32 tag,
               cudaStream_t st) {
  u32 k0, k1;
  seed_words(C, k0, k1);
  k_uniform_impl<<<grid_for(C.N, n_outer * nl), TPB, 0, st>>>(out, out_os, nl, q0, nq, C.L, id0, tag, k0, k1, C.N,
                                                               C.d_mod);
  LAUNCHED();
}

void k_cbd(Context& C, i64* out, int n_outer, u32 id0, u32 tag, cudaStream_t st) {
  u32 k0, k1;
  seed_words(C, k0, k1);
  k_cbd_impl<<<grid_for(C.N, n_outer), TPB, 0, st>>>(out, id0, tag, k0, k1, C.N);
  LAUNCHED();
}

void k_lift_small(Context& C, const i64* e, const u64* m, u64 tmul, u64* out, long out_os, int n_outer, int nl,
                  int q0, int nq, cudaStream_t st) {
  k_lift_small_impl<<<grid_for(C.N, n_outer * nl), TPB, 0, st>>>(e, m, tmul, out, out_os, nl, q0, nq, C.L, C.N,
                                                                  C.d_mod);
  LAUNCHED();
}

void k_mul_sub(Context& C, const u64* x, long x_os, const u64* a, long a_os, const u64* s, u64* out, long out_os,
               int n_outer, int nl, int q0, int nq, int, cudaStream_t st) {
  k_mul_sub_impl<<<grid_for(C.N, n_outer * nl), TPB, 0, st>>>(x, x_os, a, a_os, s, out, out_os, nl, q0, nq, C.L, C.N,
                                                               C.d_mod);
  LAUNCHED();
}

void k_ksk_gadget(Context& C, u64* b, const u64* sprime, int j, cudaStream_t st) {
  GadgetArgs G;
  int lo = j * C.alpha, hi = std::min(lo + C.alpha, C.L);
  if (hi - lo > 16) throw Error(SS_ERR_PARAM, "alpha > 16");
  for (int i = lo; i < hi; ++i) {
    u64 q = C.primes[i], P = 1;
    for (int k = C.L; k < C.ntot; ++k) P = nt::mul(P, C.primes[k] % q, q);
    G.pmod[i - lo] = P;
  }
  if (hi <= lo) return;
  k_gadget_impl<<<grid_for(C.N, hi - lo), TPB, 0, st>>>(b, sprime, j, C.alpha, C.L, C.ntot, C.N, G, C.d_mod);
  LAUNCHED();
}

void k_dec_dot(Context& C, const Buf& a, u64* v, cudaStream_t st) {
  k_dec_dot_impl<<<grid_for(C.N, a.count * a.level), TPB, 0, st>>>(a.data, a.ncomp, a.level, a.cap, C.d_sk, C.d_sk2,
                                                                     v, C.N, C.d_mod);
  LAUNCHED();
}

void k_crt(Context& C, const u64* v, int count, int level, int t_exp, u64* out, cudaStream_t st) {
  if (level > 200) throw Error(SS_ERR_PARAM, "level too large for CRT");
  const u64* pinv = C.d_crt + C.off_crt_pinv;
  const u64* half = C.d_crt + C.off_crt_half[level];
  const u64* qmodt = C.d_crt + C.off_crt_qmodt + (size_t)t_exp * (C.L + 1);
  dim3 g((C.dec_count + 127) / 128, count);
  k_crt_impl<<<g, 128, 0, st>>>(v, level, C.N, C.dec_stride, C.dec_count, pinv, half, qmodt, C.tpow[t_exp], out,
                                C.d_mod);
  LAUNCHED();
}

}  // namespace ss
