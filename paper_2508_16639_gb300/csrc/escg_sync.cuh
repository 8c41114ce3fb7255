// escg_sync.cuh -- memory-ordering helpers shared by the persistent kernels
// (acquire / release flags, epoch-tagged 64-bit record words, named
// barriers) and the count-log writer.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "escg_internal.h"

namespace escg_impl {

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_volatile(const uint32_t* p) {
  return *reinterpret_cast<const volatile uint32_t*>(p);
}

__device__ __forceinline__ unsigned long long ld_word(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_word(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void bar_named(uint32_t id, uint32_t n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Writes the log entry of MCS m_end from counts c[0..S]; stasis check.
static __device__ void write_log_entry(RunState* st, LogBuffers lb, int S, uint32_t m_end, uint32_t log_every,
                                      const unsigned long long* c, int stop_at_extinction) {
  const uint32_t idx = m_end / log_every - st->log_num0;
  const uint32_t slot = idx % (uint32_t)kLogCap;
  int alive = 0;
  for (int v = 0; v < kMaxStates; ++v) {
    const unsigned long long x = (v <= S) ? c[v] : 0ull;
    lb.counts[(size_t)slot * kMaxStates + v] = x;
    if (v >= 1 && v <= S && x > 0) ++alive;
  }
  lb.mcs[slot] = m_end;
  atomicMax(&st->n_log, idx + 1u);
  if (stop_at_extinction && alive <= 1) {
    st->mcs = m_end;
    st->stopped = 1;
  }
}

}  // namespace escg_impl
