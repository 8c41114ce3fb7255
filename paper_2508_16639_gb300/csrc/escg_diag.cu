// escg_diag.cu -- diagnostics (include/escg_diag.h): integer-issue-rate
// probe used as the roofline denominator of the Monte Carlo kernels.
#include <cstdio>
#include <cuda_runtime.h>

#include "escg_diag.h"

namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;

// Each thread runs kChains independent chains; one iteration of a chain is
// one 32x32->64 multiply-add (both halves used) and one three-input XOR,
// i.e. the two instruction kinds of a Philox round.
__global__ void int_probe_kernel(uint32_t* out, unsigned long long* cycles, uint32_t seed) {
  uint32_t a[kChains], b[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    a[c] = seed + threadIdx.x * 7919u + c * 104729u + blockIdx.x;
    b[c] = a[c] ^ 0x9E3779B9u;
  }
  const long long t0 = clock64();
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      const uint64_t p = (uint64_t)a[c] * 0xD2511F53u + b[c];
      a[c] = (uint32_t)(p >> 32) ^ b[c] ^ (uint32_t)it;
      b[c] = (uint32_t)p;
    }
  }
  const long long t1 = clock64();
  uint32_t acc = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc ^= a[c] + b[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
  if (threadIdx.x == 0) atomicMax(cycles, (unsigned long long)(t1 - t0));
}

}  // namespace

extern "C" int escg_diag_int_throughput(double* ops_per_s, double* ops_per_sm_clk) {
  if (!ops_per_s) return ESCG_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ESCG_ECUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 256, per_sm = 8, grid = sms * per_sm;
  uint32_t* out = nullptr;
  unsigned long long* cyc = nullptr;
  if (cudaMalloc(&out, sizeof(uint32_t) * grid * threads) != cudaSuccess) return ESCG_ENOMEM;
  if (cudaMalloc(&cyc, sizeof(unsigned long long)) != cudaSuccess) {
    cudaFree(out);
    return ESCG_ENOMEM;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int_probe_kernel<<<grid, threads>>>(out, cyc, 1u);  // warm-up
  cudaMemset(cyc, 0, sizeof(unsigned long long));
  cudaEventRecord(e0);
  int_probe_kernel<<<grid, threads>>>(out, cyc, 2u);
  cudaEventRecord(e1);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  unsigned long long c = 0;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaMemcpy(&c, cyc, sizeof c, cudaMemcpyDeviceToHost);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  cudaFree(cyc);
  if (e != cudaSuccess || ms <= 0.f) return ESCG_ECUDA;
  // two integer instructions per chain iteration: one 32x32+32->64-bit
  // multiply-add and one three-input XOR
  const double ops = (double)grid * threads * kIters * kChains * 2.0;
  *ops_per_s = ops / (ms * 1e-3);
  if (ops_per_sm_clk) *ops_per_sm_clk = c ? ops / ((double)sms * (double)c) : 0.0;
  return ESCG_OK;
}
