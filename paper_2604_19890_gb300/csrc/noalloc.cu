// Relinearisation that allocates nothing.
//
// Some callers cannot allocate device memory while they run: a host
// framework that owns every byte of device memory through its own allocator,
// or a service that must not risk an allocation stalling or failing in the
// middle of a request. For them, this variant of ss_relin takes its scratch
// from one file-scope device array that exists from the moment the library's
// module is loaded until the process exits (on every GPU that loads it).
//
// Limits and rules:
//  * the array holds kScratchWords 64-bit words (64 MiB); a call needs
//    count * (l + dnum*(l+alpha) + 2*(l+alpha) + 2*l) * N words at level l
//    with dnum = ceil(l/alpha), and larger calls are rejected;
//  * every call shares the array and leaves its last contents in place;
//    each word a call reads has been written earlier in the same call, so
//    nothing needs clearing, but calls that overlap on the GPU (two streams,
//    or two host threads) race on the array;
//  * the first call on a device looks up the array's device address with that
//    device current; make that first call before any stream capture.
#include <algorithm>
#include <mutex>
#include <string>

#include "ss_internal.h"

namespace ss {

namespace {

constexpr size_t kScratchWords = size_t(8) << 20;  // 64 MiB
static __device__ __align__(256) u64 g_relin_scratch[kScratchWords];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
u64* g_scratch_ptr[kMaxDevices] = {};

u64* scratch_for_current_device() {
  int dev = 0;
  SS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) throw Error(SS_ERR_PARAM, "device ordinal out of range for the static scratch");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    u64* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void**)&p, g_relin_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      throw Error(SS_ERR_CUDA, std::string("cudaGetSymbolAddress of the relinearisation scratch failed: ") +
                                   cudaGetErrorString(e));
    }
    g_scratch_ptr[dev] = p;
  }
  return g_scratch_ptr[dev];
}

}  // namespace

size_t relin_noalloc_words(const Context& C, int level, int count) {
  const int a = C.alpha, dn = (level + a - 1) / a, nx = level + a;
  return (size_t)count * ((size_t)level + (size_t)dn * nx + 2 * (size_t)nx + 2 * (size_t)level) * C.N;
}

size_t relin_noalloc_capacity() { return kScratchWords; }

// out = (c0, c1) + KS(c2) with the relinearisation key, every intermediate in
// the static array: ModUp, inner product with the key, ModDown.
void op_relin_noalloc(Context& C, const Buf& in, Buf& out, cudaStream_t st) {
  if (in.ncomp != 3) throw Error(SS_ERR_SHAPE, "relinearisation needs a 3-component ciphertext");
  if (!C.have_keys) throw Error(SS_ERR_PARAM, "no keys");
  const int N = C.N, l = in.level, B = in.count, a = C.alpha;
  const int dn = (l + a - 1) / a, nx = l + a;
  const size_t need = relin_noalloc_words(C, l, B);
  if (need > kScratchWords)
    throw Error(SS_ERR_PARAM, "ss_relin_noalloc needs " + std::to_string(need * 8) + " bytes of scratch; the static "
                              "array holds " + std::to_string(kScratchWords * 8) + " bytes (use ss_relin)");
  u64* base = scratch_for_current_device();
  u64* dc = base;
  u64* ext = dc + (size_t)B * l * N;
  u64* acc = ext + (size_t)B * dn * nx * N;
  u64* delta = acc + (size_t)B * 2 * nx * N;
  out.ncomp = 2;
  out.level = l;
  out.t_exp = in.t_exp;
  const long in_os = (long)in.ncomp * in.cap * N;
  const u64* d = in.data + (size_t)2 * in.cap * N;
  SS_CUDA(cudaMemcpy2DAsync(dc, (size_t)l * N * 8, d, (size_t)in_os * 8, (size_t)l * N * 8, B,
                            cudaMemcpyDeviceToDevice, st));
  ntt_inverse(C, PolySet{dc, (long)l * N, B, l, 0, l}, st);
  const long ext_os = (long)dn * nx * N;
  for (int j = 0; j < dn; ++j) {
    int lo = j * a, hi = std::min(lo + a, l);
    const u64* c1 = C.d_tables + C.off_modup.at({j, hi});
    const u64* c2 = c1 + 2 * (hi - lo);
    k_bconv(C, dc + (size_t)lo * N, (long)l * N, hi - lo, lo, c1, c2, ext + (size_t)j * nx * N, ext_os, nx, l, lo,
            hi, nullptr, B, st);
  }
  PolySet ps{ext, (long)nx * N, B * dn, nx, 0, l};
  ps.skip_w = a;
  ps.skip_mod = dn;
  ps.skip_level = l;
  ntt_forward(C, ps, st);
  const long acc_os = 2L * nx * N;
  k_ks_ip(C, d, in_os, ext, ext_os, C.rlk, l, acc, acc_os, B, st);
  ntt_inverse(C, PolySet{acc + (size_t)l * N, (long)nx * N, 2 * B, a, C.L, 0}, st);
  const u64* c1 = C.d_tables + C.off_md_c1[in.t_exp];
  const u64* c2 = C.d_tables + C.off_md_c2;
  const u64* post = C.d_tmod + (size_t)in.t_exp * C.ntot * 2;
  k_bconv(C, acc + (size_t)l * N, (long)nx * N, a, C.L, c1, c2, delta, (long)l * N, l, l, 0, 0, post, 2 * B, st);
  ntt_forward(C, PolySet{delta, (long)l * N, 2 * B, l, 0, l}, st);
  const u64* pinv = C.d_tables + C.off_md_pinv;
  for (int c = 0; c < 2; ++c)
    k_sub_scale(C, acc + (size_t)c * nx * N, acc_os, delta + (size_t)c * l * N, 2L * l * N, pinv,
                in.data + (size_t)c * in.cap * N, in_os, out.data + (size_t)c * out.cap * N,
                (long)out.ncomp * out.cap * N, l, B, st);
}

}  // namespace ss
