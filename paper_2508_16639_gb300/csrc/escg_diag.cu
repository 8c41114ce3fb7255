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

// The instruction mix of one elementary step (24 integer instructions, the
// count the roofline divides by): a quarter of a Philox4x32-10 call (5 wide
// multiplies, 5 three-input XORs), the split of the word (1 shift), the cell
// and neighbour offsets (2 byte permutes, 2 shifts, 2 adds), the action
// select (2 compares, 1 select), the transition-table index (1 multiply-add,
// 1 add) and the unpacking of the new pair (1 and, 1 shift).  Written in PTX
// so that every instruction is kept; kChains independent chains per thread.
__device__ __forceinline__ void alg_step(uint32_t& a, uint32_t& b, uint32_t k, uint32_t tx) {
  uint64_t p0, p1;
  uint32_t l0, h0, l1, h1, t0, t1, t2, t3, t4, t5, sel, q;
#pragma unroll
  for (int r = 0; r < 2; ++r) {   // 2 x (2 wide multiplies + 2 XORs)
    asm("mul.wide.u32 %0, %1, %2;" : "=l"(p0) : "r"(a), "r"(0xD2511F53u));
    asm("mul.wide.u32 %0, %1, %2;" : "=l"(p1) : "r"(b), "r"(0xCD9E8D57u));
    asm("mov.b64 {%0, %1}, %2;" : "=r"(l0), "=r"(h0) : "l"(p0));
    asm("mov.b64 {%0, %1}, %2;" : "=r"(l1), "=r"(h1) : "l"(p1));
    asm("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(a) : "r"(h1), "r"(l0), "r"(k));
    asm("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(b) : "r"(h0), "r"(l1), "r"(k));
  }
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(p0) : "r"(a), "r"(0xD2511F53u));
  asm("mov.b64 {%0, %1}, %2;" : "=r"(l0), "=r"(h0) : "l"(p0));
  asm("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(a) : "r"(h0), "r"(b), "r"(l0));
  asm("shl.b32 %0, %1, 4;" : "=r"(t0) : "r"(a));                            // action draw
  asm("prmt.b32 %0, %1, 0, %2;" : "=r"(t1) : "r"(0x51500100u), "r"(a));     // cell offset
  asm("prmt.b32 %0, %1, 0, %2;" : "=r"(t2) : "r"(0x51A04F00u), "r"(b));     // neighbour offset
  asm("shr.b32 %0, %1, 28;" : "=r"(t3) : "r"(a));
  asm("shr.b32 %0, %1, 30;" : "=r"(t4) : "r"(b));
  asm("add.s32 %0, %1, %2;" : "=r"(t5) : "r"(t1), "r"(t3));
  asm("add.s32 %0, %1, %2;" : "=r"(t3) : "r"(t2), "r"(t4));
  asm("{ .reg .pred p0, p1; setp.lt.u32 p0, %1, %2; setp.lt.u32 p1, %1, %3; selp.b32 %0, %4, %5, p0; "
      "@p1 add.u32 %0, %0, 1; }"
      : "=r"(sel) : "r"(t0), "r"(tx), "r"(tx ^ 0x80000000u), "r"(t5), "r"(t3));   // 2 compares, select, add
  asm("mad.lo.u32 %0, %1, 6, %2;" : "=r"(q) : "r"(sel), "r"(t3));            // table index
  asm("and.b32 %0, %1, 0xFFFFFF0F;" : "=r"(b) : "r"(q));                     // unpack
  asm("shr.b32 %0, %1, 4;" : "=r"(a) : "r"(q));
}

__global__ void alg_probe_kernel(uint32_t* out, unsigned long long* cycles, uint32_t seed) {
  uint32_t a[kChains], b[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    a[c] = seed + threadIdx.x * 7919u + c * 104729u + blockIdx.x;
    b[c] = a[c] ^ 0x9E3779B9u;
  }
  const long long t0 = clock64();
  for (int it = 0; it < kIters / 4; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) alg_step(a[c], b[c], (uint32_t)it, 0x7F000000u);
  }
  const long long t1 = clock64();
  uint32_t acc = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc ^= a[c] + b[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
  if (threadIdx.x == 0) atomicMax(cycles, (unsigned long long)(t1 - t0));
}

// Copies of one L2-resident buffer into another, `passes` times in one
// launch (16-byte vectors, loads through L2 as the Monte Carlo kernels' tile
// loads; volatile PTX so that no pass is elided), grid-stride.
__global__ void l2_copy_kernel(const uint4* src, uint4* dst, size_t n, int passes) {
  for (int p = 0; p < passes; ++p)
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
      uint4 v;
      asm volatile("ld.global.cg.v4.u32 {%0, %1, %2, %3}, [%4];"
                   : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(src + i));
      asm volatile("st.global.v4.u32 [%0], {%1, %2, %3, %4};" ::"l"(dst + i), "r"(v.x), "r"(v.y), "r"(v.z),
                   "r"(v.w) : "memory");
    }
}

}  // namespace

extern "C" int escg_diag_alg_throughput(double* alg_per_s, double* alg_per_sm_clk) {
  if (!alg_per_s) return ESCG_EINVAL;
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
  alg_probe_kernel<<<grid, threads>>>(out, cyc, 1u);  // warm-up
  cudaMemset(cyc, 0, sizeof(unsigned long long));
  cudaEventRecord(e0);
  alg_probe_kernel<<<grid, threads>>>(out, cyc, 2u);
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
  const double steps = (double)grid * threads * (kIters / 4) * kChains;
  *alg_per_s = 24.0 * steps / (ms * 1e-3);
  if (alg_per_sm_clk) *alg_per_sm_clk = c ? 24.0 * steps / ((double)sms * (double)c) : 0.0;
  return ESCG_OK;
}

extern "C" int escg_diag_l2_copy(size_t bytes, int reps, double* gbs) {
  if (!gbs || bytes < 16 || reps < 1) return ESCG_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ESCG_ECUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t n = bytes / 16;
  uint4 *a = nullptr, *b = nullptr;
  if (cudaMalloc(&a, n * 16) != cudaSuccess) return ESCG_ENOMEM;
  if (cudaMalloc(&b, n * 16) != cudaSuccess) {
    cudaFree(a);
    return ESCG_ENOMEM;
  }
  cudaMemset(a, 1, n * 16);
  cudaMemset(b, 2, n * 16);
  const int threads = 256, grid = sms * 8;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  l2_copy_kernel<<<grid, threads>>>(a, b, n, 3);   // brings both buffers into L2
  cudaEventRecord(e0);
  l2_copy_kernel<<<grid, threads>>>(a, b, n, reps);
  cudaEventRecord(e1);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(a);
  cudaFree(b);
  if (e != cudaSuccess || ms <= 0.f) return ESCG_ECUDA;
  *gbs = 2.0 * (double)(n * 16) * reps / (ms * 1e-3) / 1e9;   // bytes read + written
  return ESCG_OK;
}

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
