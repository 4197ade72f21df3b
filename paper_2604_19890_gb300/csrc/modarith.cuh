// Device modular arithmetic for RNS limbs held in 64-bit words.
//
// Primes q satisfy 2^(k-1) < q < 2^k with k <= 62, so 4q fits a word and the
// transforms can keep lazy residues in [0, 4q) (Harvey's butterfly). The GPU
// has no 64x64 multiplier: every product below compiles to 32-bit
// IMAD.WIDE/IMAD.HI sequences, so the code keeps the number of wide products
// minimal:
//   * Shoup product with a precomputed companion w' = floor(w 2^64 / q):
//     one high product, two low products, one conditional subtract.
//   * Barrett reduction of a value x < 2^(63+k) (a product or a lazy sum of
//     products) with mu = floor(2^(63+k) / q):
//       qhat = hi64((x >> (k-1)) * mu),  r = x - qhat q in [0, 3q).
#pragma once
#include <cstdint>

typedef uint64_t u64;
typedef unsigned __int128 u128;

struct Modulus {
  u64 q;
  u64 mu;     // floor(2^(63+k) / q)
  int kbits;  // bit length of q
  int pad;
  u64 qinv;   // -q^-1 mod 2^64 (Montgomery reduction)
};

__device__ __forceinline__ u64 mulhi64(u64 a, u64 b) { return __umul64hi(a, b); }

// x = (hi, lo) < 2^(63+k)  ->  x mod q in [0, q)
__device__ __forceinline__ u64 barrett_reduce128(u64 hi, u64 lo, const Modulus& m) {
  int s = m.kbits - 1;
  u64 xs = (lo >> s) | (hi << (64 - s));  // s in [1, 61]
  u64 qh = mulhi64(xs, m.mu);
  u64 r = lo - qh * m.q;
  if (r >= m.q) r -= m.q;
  if (r >= m.q) r -= m.q;
  return r;
}

__device__ __forceinline__ u64 mul_mod(u64 a, u64 b, const Modulus& m) {
  return barrett_reduce128(mulhi64(a, b), a * b, m);
}

// Montgomery reduction: x = (hi, lo) < q 2^64 -> x 2^-64 mod q in [0, q).
// With m = lo * qinv mod 2^64, x + m q is divisible by 2^64; the low words
// cancel with a carry exactly when lo != 0, and (x + m q) / 2^64 < 2q.
__device__ __forceinline__ u64 redc128(u64 hi, u64 lo, u64 q, u64 qinv) {
  const u64 m = lo * qinv;
  const u64 t = hi + mulhi64(m, q) + (lo != 0 ? 1 : 0);
  return t >= q ? t - q : t;
}

// 128-bit accumulator of products; reduce once at the end.
struct Acc128 {
  u64 lo, hi;
  __device__ __forceinline__ void zero() { lo = 0; hi = 0; }
  __device__ __forceinline__ void mac(u64 a, u64 b) {
    u64 l = a * b, h = mulhi64(a, b);
    lo += l;
    hi += h + (lo < l ? 1 : 0);
  }
  // the same product-accumulate through the compiler's 128-bit arithmetic
  __device__ __forceinline__ void mac_wide(u64 a, u64 b) {
    const u128 s = (((u128)hi << 64) | lo) + (u128)a * b;
    lo = (u64)s;
    hi = (u64)(s >> 64);
  }
  __device__ __forceinline__ void add(u64 a) {
    lo += a;
    hi += (lo < a ? 1 : 0);
  }
};

__device__ __forceinline__ u64 add_mod(u64 a, u64 b, u64 q) {
  u64 s = a + b;
  return s >= q ? s - q : s;
}

__device__ __forceinline__ u64 sub_mod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }

// a * w mod q, result in [0, 2q); any a < 2^64, w < q.
__device__ __forceinline__ u64 shoup_lazy(u64 a, u64 w, u64 wp, u64 q) {
  u64 qh = mulhi64(a, wp);
  return a * w - qh * q;
}

__device__ __forceinline__ u64 shoup(u64 a, u64 w, u64 wp, u64 q) {
  u64 r = shoup_lazy(a, w, wp, q);
  return r >= q ? r - q : r;
}
