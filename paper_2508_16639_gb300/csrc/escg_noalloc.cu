// escg_noalloc.cu -- escg_run_noalloc: Monte Carlo steps on a caller-owned
// device lattice without any memory allocation by the library.
//
// Some callers cannot let a library allocate: code that owns a fixed device
// memory budget (an application with its own pool, an inference or HPC
// service that pre-reserves all GPU memory at start-up), and loops where a
// cudaMalloc/cudaFree would synchronise the device or is forbidden.  For them
// this entry point keeps all the scratch state the persistent kernel needs --
// run state, block epochs and the transition table -- in one
// file-scope device array of fixed size, which every GPU that loads the
// library holds until the process exits.
#include <cmath>
#include <cstring>
#include <mutex>

#include "escg.h"
#include "escg_internal.h"

namespace escg_impl {

// Scratch layout (bytes): RunState | block epochs | transition table.  The
// kernels find block spans and fine segments in closed form (AxisGeom in the
// kernel parameters), so no partition tables are kept.
constexpr int kNoallocMaxL = 4096;
constexpr size_t kNoallocScratchBytes = 64 * 1024;
constexpr size_t kNoallocStateBytes = (sizeof(RunState) + 255) / 256 * 256;
constexpr int kNoallocMaxP = 2 * ((kNoallocMaxL + 64) / 128);      // 64 coarse blocks per axis
constexpr size_t kNoallocDoneOff = kNoallocStateBytes;
constexpr size_t kNoallocDoneBytes = 4 * (size_t)kNoallocMaxP * kNoallocMaxP;
constexpr size_t kNoallocTransOff = (kNoallocDoneOff + kNoallocDoneBytes + 255) / 256 * 256;
constexpr size_t kNoallocTransBytes = 4 * (size_t)kTransWords;
static_assert(kNoallocTransOff >= kNoallocDoneOff + kNoallocDoneBytes, "epochs overlap the transition table");
static_assert(kNoallocTransOff + kNoallocTransBytes <= kNoallocScratchBytes, "scratch too small");

static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoallocScratchBytes];

// Set-up of one call, passed by value in the kernel parameters (2 KB): the
// transition table comes from the host builder that every other entry point
// uses (build_transitions), so there is one copy of the rule.
struct NoallocSetup {
  uint32_t mcs_begin;
  int32_t n_blocks;                // P * P
  uint32_t trans[kTransWords];
};

// One CTA: clears the run state, sets every block epoch to mcs_begin and
// copies the transition table into the scratch array.
__global__ void noalloc_setup_kernel(uint8_t* scratch, const __grid_constant__ NoallocSetup a) {
  RunState* st = reinterpret_cast<RunState*>(scratch);
  uint32_t* done = reinterpret_cast<uint32_t*>(scratch + kNoallocDoneOff);
  uint32_t* words = reinterpret_cast<uint32_t*>(scratch);
  uint32_t* tr = reinterpret_cast<uint32_t*>(scratch + kNoallocTransOff);
  for (int i = threadIdx.x; i < (int)(sizeof(RunState) / 4); i += blockDim.x) words[i] = 0;
  for (int i = threadIdx.x; i < a.n_blocks; i += blockDim.x) done[i] = a.mcs_begin;
  for (int i = threadIdx.x; i < kTransWords; i += blockDim.x) tr[i] = a.trans[i];
  __syncthreads();
  if (threadIdx.x == 0) st->mcs = a.mcs_begin;
}

__global__ void noalloc_counts_kernel(const uint8_t* scratch, int S, uint64_t* out) {
  const RunState* st = reinterpret_cast<const RunState*>(scratch);
  if ((int)threadIdx.x <= S) out[threadIdx.x] = st->cur[threadIdx.x];
}

}  // namespace escg_impl

using namespace escg_impl;

namespace {

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64] = {};

// Device address of the scratch array on the current device (looked up once
// per device: the array's name is only a host-side stand-in in host code).
int noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    set_last_error("escg_run_noalloc: no usable current CUDA device");
    return ESCG_ECUDA;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_last_error("escg_run_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return ESCG_ECUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return ESCG_OK;
}

}  // namespace

extern "C" int escg_run_noalloc(uint8_t* d_lattice, int32_t L, int32_t S, const uint8_t* digraph,
                                const escg_rates* rates, uint64_t seed, uint64_t mcs_begin, uint64_t n_mcs,
                                uint64_t* d_counts_out, void* cuda_stream) {
  if (!d_lattice || !digraph || !rates) {
    set_last_error("escg_run_noalloc: NULL lattice, digraph or rates");
    return ESCG_EINVAL;
  }
  if (reinterpret_cast<uintptr_t>(d_lattice) % 16 != 0) {
    set_last_error("escg_run_noalloc: d_lattice must be 16-byte aligned (rows are read as 16-byte vectors)");
    return ESCG_EINVAL;
  }
  if (reinterpret_cast<uintptr_t>(d_counts_out) % 8 != 0) {
    set_last_error("escg_run_noalloc: d_counts_out must be 8-byte aligned");
    return ESCG_EINVAL;
  }
  if (L < 8 || L > kNoallocMaxL) {
    set_last_error("escg_run_noalloc: L=%d outside [8, %d] (the fixed scratch array holds at most "
                   "that size)", L, kNoallocMaxL);
    return ESCG_EINVAL;
  }
  if (S < 2 || S > 15) {
    set_last_error("escg_run_noalloc: S=%d outside [2, 15]", S);
    return ESCG_EINVAL;
  }
  for (int i = 0; i < S * S; ++i)
    if (digraph[i] > 1 || (i / S == i % S && digraph[i])) {
      set_last_error("escg_run_noalloc: digraph must be 0/1 with a zero diagonal");
      return ESCG_EINVAL;
    }
  const double I = rates->interact, Pr = rates->reproduce, X = rates->exchange;
  const double R = (X + I) + Pr;
  if (!(I >= 0 && Pr >= 0 && X >= 0) || !(R > 0) || std::isinf(R)) {
    set_last_error("escg_run_noalloc: rates must be finite, >= 0 and not all zero");
    return ESCG_EINVAL;
  }
  // written so that no sum can wrap around 2^64
  if (mcs_begin >= 0x80000000ull || n_mcs >= 0x80000000ull - mcs_begin) {
    set_last_error("escg_run_noalloc: MCS numbers must stay below 2^31");
    return ESCG_EINVAL;
  }
  void* scratch_v = nullptr;
  int rc = noalloc_scratch(&scratch_v);
  if (rc != ESCG_OK) return rc;
  uint8_t* scratch = static_cast<uint8_t*>(scratch_v);
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  int dev = 0;
  cudaGetDevice(&dev);

  const int h = (L + 64) / 128, P = 2 * (h < 1 ? 1 : h);
  int GQ = 0;
  for (int k = 0; k < P; ++k) GQ += 2 * ((L / P + (k < L % P ? 1 : 0)) / 4);
  LatticeDesc d;
  std::memset(&d, 0, sizeof d);
  d.lat = d_lattice;
  d.L = L;
  d.pitch = escg_lattice_pitch(L);
  d.P = P;
  d.GQ = GQ;
  d.cs = d.fs = d.fc = nullptr;   // partition in closed form only (d.ax, d.ay)
  d.H = L;   // square
  d.Py = P;
  d.csy = d.fsy = d.fcy = nullptr;
  d.ax = make_axis_geom(L, P);
  d.ay = d.ax;
  d.bits = 8;
  d.trans = scratch + kNoallocTransOff;
  d.key0 = (uint32_t)seed;
  d.key1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    d.rk[2 * r] = d.key0 + (uint32_t)r * 0x9E3779B9u;
    d.rk[2 * r + 1] = d.key1 + (uint32_t)r * 0xBB67AE85u;
  }
  const uint64_t tx = (uint64_t)std::floor(std::ldexp(X / R, 32) + 0.5);
  const uint64_t txi = (uint64_t)std::floor(std::ldexp((X + I) / R, 32) + 0.5);
  d.tx = tx >> 32 ? 0xFFFFFFFFu : (uint32_t)tx;
  d.txi = txi >> 32 ? 0xFFFFFFFFu : (uint32_t)txi;
  d.S = S;
  d.nbh = 4;
  d.reflect = 0;
  d.uniform64 = (L % 64 == 0 && L / 64 == P && d.pitch % 16 == 0) ? 1 : 0;
  fill_perm24(d.perm24);

  NoallocSetup su;
  std::memset(&su, 0, sizeof su);
  su.mcs_begin = (uint32_t)mcs_begin;
  su.n_blocks = P * P;
  build_transitions(S, digraph, nullptr, tx, txi, su.trans);
  noalloc_setup_kernel<<<1, 256, 0, stream>>>(scratch, su);
  cudaError_t e = cudaGetLastError();
  RunState* st = reinterpret_cast<RunState*>(scratch);
  // Every byte of the caller's lattice must be a state 0..S (the transition
  // table is indexed by the pair); otherwise the run state stops, so that
  // the kernels below leave the lattice alone, and the call fails.
  if (e == cudaSuccess) e = launch_validate(d, &st->error, kErrBadValue, &st->stopped, stream);
  const int grid_max = persistent_grid(dev, d.uniform64 != 0);
  const uint64_t per_mcs = (uint64_t)P * P;
  const uint64_t max_chunk = ((1ull << 31) - (uint64_t)grid_max) / per_mcs;
  uint64_t m = mcs_begin;
  const uint64_t end = mcs_begin + n_mcs;
  while (e == cudaSuccess && m < end) {
    const uint64_t n = end - m < max_chunk ? end - m : max_chunk;
    PersistentArgs a;
    std::memset(&a, 0, sizeof a);
    a.d = d;
    a.st = st;
    a.done = reinterpret_cast<uint32_t*>(scratch + kNoallocDoneOff);
    a.lb = LogBuffers{nullptr, nullptr};   // no log points below 2^31 with this period
    a.m_begin = (uint32_t)m;
    a.n_mcs = (uint32_t)n;
    a.log_every = 0x80000000u;
    a.stop_at_extinction = 0;
    a.spin_limit = 2000000;
    a.stall_block = -1;
    const uint64_t items = n * per_mcs;
    const int grid = (int)(items < (uint64_t)grid_max ? items : (uint64_t)grid_max);
    e = launch_persistent(a, grid, stream);
    m += n;
  }
  if (e == cudaSuccess && d_counts_out) {
    e = launch_count(d, st, stream);
    if (e == cudaSuccess) {
      noalloc_counts_kernel<<<1, 32, 0, stream>>>(scratch, S, d_counts_out);
      e = cudaGetLastError();
    }
  }
  uint32_t err_word = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&err_word, &st->error, sizeof err_word, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) {
    set_last_error("escg_run_noalloc: %s", cudaGetErrorString(e));
    return ESCG_ECUDA;
  }
  if (err_word & kErrBadValue) {
    set_last_error("escg_run_noalloc: the lattice holds a value outside 0..S=%d; it was left unchanged", S);
    return ESCG_EINVAL;
  }
  if (err_word & kErrTimeout) {
    set_last_error("escg_run_noalloc: a bounded device-side wait timed out");
    return ESCG_ETIMEOUT;
  }
  return ESCG_OK;
}
