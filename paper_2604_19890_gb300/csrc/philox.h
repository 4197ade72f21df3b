// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11),
// usable from host and device code of this library.
//
// Sampling streams (key = the 64-bit context seed split into two words;
// counter = {index, limb, id, tag}):
//   tag 1: secret-key selection, counter {i, 0, 0, 1}
//   tag 2/3: encryption randomness (uniform c1 / error), id = nonce
//   tag 4/5: key-switching keys (uniform a_j / error e_j), id = key*256 + digit
// Uniform residues take all 128 output bits modulo q; errors are centred
// binomial with eta = 21 (popcount of 21 bits minus popcount of 21 bits).
#pragma once
#include <cstdint>

#ifdef __CUDACC__
#define SS_HD __host__ __device__ __forceinline__
#else
#define SS_HD inline
#endif

namespace ss {

enum : uint32_t { TAG_SK = 1, TAG_ENC_A = 2, TAG_ENC_E = 3, TAG_KSK_A = 4, TAG_KSK_E = 5 };

SS_HD void mulhilo32(uint32_t a, uint32_t b, uint32_t& hi, uint32_t& lo) {
  uint64_t p = (uint64_t)a * (uint64_t)b;
  hi = (uint32_t)(p >> 32);
  lo = (uint32_t)p;
}

struct Philox4 {
  uint32_t x[4];
};

SS_HD Philox4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1) {
  for (int round = 0; round < 10; ++round) {
    uint32_t h0, l0, h1, l1;
    mulhilo32(0xD2511F53u, c0, h0, l0);
    mulhilo32(0xCD9E8D57u, c2, h1, l1);
    uint32_t y0 = h1 ^ c1 ^ k0, y2 = h0 ^ c3 ^ k1;
    c0 = y0;
    c1 = l1;
    c2 = y2;
    c3 = l0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  Philox4 r;
  r.x[0] = c0; r.x[1] = c1; r.x[2] = c2; r.x[3] = c3;
  return r;
}

SS_HD int popc21(uint32_t v) {
  v &= 0x1FFFFFu;
  int c = 0;
  while (v) { v &= v - 1; ++c; }
  return c;
}

}  // namespace ss
