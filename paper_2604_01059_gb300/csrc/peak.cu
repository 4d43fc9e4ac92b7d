// Integer-issue microbenchmark of the GPU (no counterpart in the paper): the
// throughput of the instruction classes the sampling kernel is built from,
// used to state the ALU roofline of that kernel.  Each thread runs eight
// independent dependency chains so that issue, not latency, limits the rate.
#include <cuda_runtime.h>

#include <string>

#include "common.h"

namespace tsim {
namespace {

constexpr int kIters = 4096;

// op 0: 32-bit three-input logic (LOP3), op 1: 32-bit multiply-add (IMAD),
// op 2: 32x32 -> 64-bit multiply (IMAD.WIDE, as in Philox), op 3: popcount
template <int OP>
__global__ void k_peak(uint32_t seed, uint32_t* out) {
  uint32_t a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = seed * (threadIdx.x + 1) + i * 0x9E3779B9u;
  const uint32_t m = seed | 1u, n = seed ^ 0x5bd1e995u;
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (OP == 0) a[i] = (a[i] ^ m) ^ (a[(i + 1) & 7] & n);
      if (OP == 1) a[i] = a[i] * m + n;
      if (OP == 2) {
        const uint64_t p = (uint64_t)a[i] * m;
        a[i] = (uint32_t)(p >> 32) ^ (uint32_t)p;
      }
      if (OP == 3) a[i] = __popc(a[i] ^ m) + a[i];
    }
  }
  uint32_t r = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) r ^= a[i];
  if (r == 0x12345678u) out[0] = r;  // keeps the work alive
}

}  // namespace
}  // namespace tsim

extern "C" tsim_status tsim_measure_int_peak(int op, double* ops_per_s) {
  using namespace tsim;
  if (!ops_per_s || op < 0 || op > 3) return TSIM_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TSIM_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return TSIM_ERR_CUDA;
  uint32_t* out = nullptr;
  if (cudaMalloc(&out, 4) != cudaSuccess) return TSIM_ERR_OOM;
  const int threads = 256, blocks = sms * 8;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto run = [&](uint32_t seed) {
    switch (op) {
      case 0: k_peak<0><<<blocks, threads>>>(seed, out); break;
      case 1: k_peak<1><<<blocks, threads>>>(seed, out); break;
      case 2: k_peak<2><<<blocks, threads>>>(seed, out); break;
      default: k_peak<3><<<blocks, threads>>>(seed, out); break;
    }
  };
  run(3);  // warm-up
  cudaEventRecord(e0);
  for (int r = 0; r < 5; ++r) run(7 + r);
  cudaEventRecord(e1);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess || ms <= 0) return TSIM_ERR_CUDA;
  // instructions per inner step: LOP3 chain 2 ops, IMAD 1, IMAD.WIDE 1 (+1 xor), popc 1 (+2)
  const double per_step[4] = {2.0, 1.0, 1.0, 1.0};
  *ops_per_s = 5.0 * blocks * threads * (double)kIters * 8 * per_step[op] / (ms * 1e-3);
  return TSIM_OK;
}
