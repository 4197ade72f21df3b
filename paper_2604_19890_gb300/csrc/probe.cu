// Integer-pipe ceilings for the roofline of the ALU-bound kernels: register-only
// loops that issue the arithmetic of the transforms with no memory traffic.
//   kind 0: 32-bit multiply-adds (IMAD) per second;
//   kind 1: forward butterflies per second in Harvey's form: reduce the upper
//           input below 2q, one 64-bit Shoup product, lazy add and subtract;
//   kind 2: 32 x 32 -> 64-bit widening multiply-adds (IMAD.WIDE) per second,
//           the partial products a 64-bit modular product is built from.
// One full wave of CTAs (as many per SM as fit) runs the loop.
#include "modarith.cuh"
#include <algorithm>

#include "ss_internal.h"

namespace ss {
namespace {

__global__ void __launch_bounds__(256) k_probe_imad(uint32_t* out, int iters, uint32_t seed) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = tid * 2654435761u + k;
  const uint32_t b = seed | 1u, c = seed >> 3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = a[k] * b + c;
  }
  uint32_t x = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) x ^= a[k];
  out[tid] = x;
}

__global__ void __launch_bounds__(256) k_probe_wide(u64* out, int iters, uint32_t seed) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  u64 a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = (u64)tid * 2654435761u + k;
  const uint32_t b = seed | 1u;
  const u64 c = ((u64)seed << 29) | 7u;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = (u64)(uint32_t)a[k] * b + c;  // low 32 bits times b, 64-bit sum
  }
  u64 x = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) x ^= a[k];
  out[tid] = x;
}

__global__ void __launch_bounds__(256) k_probe_butterfly(u64* out, int iters, u64 q, u64 w, u64 wp) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  u64 x[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) x[k] = (tid * 16u + k) % q;
  const u64 q2 = 2 * q;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      u64 U = x[k];
      if (U >= q2) U -= q2;
      const u64 V = shoup_lazy(x[k + 8], w, wp, q);
      x[k] = U + V;
      x[k + 8] = U - V + q2;
    }
  }
  u64 s = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) s ^= x[k];
  out[tid] = s;
}

}  // namespace

// Runs one probe on the current device and returns its rate per second.
double alu_probe(int kind, int iters) {
  cudaDeviceProp prop;
  int dev = 0;
  SS_CUDA(cudaGetDevice(&dev));
  SS_CUDA(cudaGetDeviceProperties(&prop, dev));
  const int threads = 256;
  int per_sm = 0;
  if (kind == 0) SS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_imad, threads, 0));
  else if (kind == 1) SS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_butterfly, threads, 0));
  else SS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_wide, threads, 0));
  const int blocks = prop.multiProcessorCount * std::max(1, per_sm), n = blocks * threads;
  void* buf = nullptr;
  SS_CUDA(cudaMalloc(&buf, (size_t)n * 8));
  cudaStream_t st;
  SS_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  cudaEvent_t e0, e1;
  SS_CUDA(cudaEventCreate(&e0));
  SS_CUDA(cudaEventCreate(&e1));
  // a 55-bit prime and a twiddle with its Shoup companion, as in the transforms
  const u64 q = 36028797018652673ULL, w = 12345678901234567ULL % q;
  const u64 wp = (u64)(((unsigned __int128)w << 64) / q);
  float ms = 0;
  for (int rep = 0; rep < 2; ++rep) {  // the first pass warms up
    SS_CUDA(cudaEventRecord(e0, st));
    if (kind == 0) k_probe_imad<<<blocks, threads, 0, st>>>((uint32_t*)buf, iters, 0x9E3779B9u);
    else if (kind == 1) k_probe_butterfly<<<blocks, threads, 0, st>>>((u64*)buf, iters, q, w, wp);
    else k_probe_wide<<<blocks, threads, 0, st>>>((u64*)buf, iters, 0x9E3779B9u);
    SS_CUDA(cudaEventRecord(e1, st));
    SS_CUDA(cudaEventSynchronize(e1));
    SS_CUDA(cudaGetLastError());
    SS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  cudaFree(buf);
  const double ops = (double)n * iters * 8.0;  // 8 operations per thread and iteration
  return ops / (ms * 1e-3);
}

}  // namespace ss
