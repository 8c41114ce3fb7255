// escg_noalloc.cu -- escg_run_noalloc: Monte Carlo steps on a caller-owned
// device lattice without any memory allocation by the library.
//
// Some callers cannot let a library allocate: code that owns a fixed device
// memory budget (an application with its own pool, an inference or HPC
// service that pre-reserves all GPU memory at start-up), and loops where a
// cudaMalloc/cudaFree would synchronise the device or is forbidden.  For them
// this entry point keeps all the scratch state the persistent kernel needs --
// run state, block epochs, partition and transition tables -- in one
// file-scope device array of fixed size, which every GPU that loads the
// library holds until the process exits.
#include <cmath>
#include <cstring>
#include <mutex>

#include "escg.h"
#include "escg_internal.h"

namespace escg_impl {

// Scratch layout (bytes): RunState | epochs | partition tables | transitions.
constexpr int kNoallocMaxL = 4096;
constexpr size_t kNoallocScratchBytes = 64 * 1024;
constexpr size_t kNoallocStateBytes = (sizeof(RunState) + 255) / 256 * 256;
constexpr int kNoallocMaxP = 2 * ((kNoallocMaxL + 64) / 128);      // 64
constexpr int kNoallocMaxGQ = kNoallocMaxL / 2;                     // fine segments per axis
constexpr size_t kNoallocDoneOff = kNoallocStateBytes;
constexpr size_t kNoallocTabOff = kNoallocDoneOff + 4 * (size_t)kNoallocMaxP * kNoallocMaxP;
constexpr size_t kNoallocTransOff =
    kNoallocTabOff + 4 * (size_t)((kNoallocMaxP + 1) * 2 + kNoallocMaxGQ + 1 + 63) / 64 * 64;
static_assert(kNoallocTransOff + 4 * kTransWords <= kNoallocScratchBytes, "scratch too small");

static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoallocScratchBytes];

struct NoallocSetup {
  int32_t L, S;
  uint32_t mcs_begin;
  uint8_t digraph[kMaxStates * kMaxStates];
};

__device__ __forceinline__ void nsplit(int n, int parts, int32_t* start) {
  const int q = n / parts, r = n % parts;
  start[0] = 0;
  for (int k = 0; k < parts; ++k) start[k + 1] = start[k] + q + (k < r ? 1 : 0);
}

// One CTA: clears the run state, sets every block epoch to mcs_begin, and
// writes the schedule-v1 partition tables and the Alg. 3 transition table
// of this call into the scratch array.
__global__ void noalloc_setup_kernel(uint8_t* scratch, NoallocSetup a) {
  RunState* st = reinterpret_cast<RunState*>(scratch);
  const int L = a.L, h = (L + 64) / 128, P = 2 * (h < 1 ? 1 : h);
  uint32_t* done = reinterpret_cast<uint32_t*>(scratch + kNoallocDoneOff);
  uint32_t* words = reinterpret_cast<uint32_t*>(scratch);
  for (int i = threadIdx.x; i < (int)(sizeof(RunState) / 4); i += blockDim.x) words[i] = 0;
  for (int i = threadIdx.x; i < P * P; i += blockDim.x) done[i] = a.mcs_begin;
  if (threadIdx.x == 0) {
    st->mcs = a.mcs_begin;
    int32_t* cs = reinterpret_cast<int32_t*>(scratch + kNoallocTabOff);
    nsplit(L, P, cs);
    int GQ = 0;
    for (int k = 0; k < P; ++k) GQ += 2 * ((cs[k + 1] - cs[k]) / 4);
    int32_t* fs = cs + (P + 1);
    int32_t* fc = fs + (GQ + 1);
    int g = 0;
    for (int k = 0; k < P; ++k) {
      const int w = cs[k + 1] - cs[k], Q = 2 * (w / 4);
      fc[k] = g;
      const int q0 = w / Q, r0 = w % Q;
      int x = cs[k];
      for (int q = 0; q < Q; ++q) {
        fs[g + q] = x;
        x += q0 + (q < r0 ? 1 : 0);
      }
      g += Q;
    }
    fs[GQ] = L;
    fc[P] = GQ;
    const int S = a.S, s1 = S + 1;
    uint8_t* tr = scratch + kNoallocTransOff;
    // every edge certain: interaction thresholds 2^32 (stored as 0xFFFFFFFF)
    uint32_t* thr = reinterpret_cast<uint32_t*>(tr) + kTransPairs;
    for (int k = 0; k < s1 * s1; ++k) thr[k] = 0xFFFFFFFFu;
    for (int act = 0; act < 4; ++act)
      for (int x = 0; x < s1; ++x)
        for (int y = 0; y < s1; ++y) {
          const bool xy = x && y && a.digraph[(x - 1) * S + (y - 1)];
          const bool yx = x && y && a.digraph[(y - 1) * S + (x - 1)];
          int nx = x, ny = y;
          if (x != y) {
            if (act == 0) {
              nx = y;
              ny = x;
            } else if (act == 1) {
              if (xy)
                ny = 0;
              else if (yx)
                nx = 0;
            } else if (act == 2) {
              if (y == 0)
                ny = x;
              else if (x == 0)
                nx = y;
            }
          }
          tr[(x * s1 + y) * 4 + act] = (uint8_t)(nx | (ny << 4));
        }
  }
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
  if (mcs_begin + n_mcs >= 0x80000000ull) {
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
  d.cs = reinterpret_cast<const int32_t*>(scratch + kNoallocTabOff);
  d.fs = d.cs + (P + 1);
  d.fc = d.fs + (GQ + 1);
  d.H = L;   // square
  d.Py = P;
  d.csy = d.cs;
  d.fsy = d.fs;
  d.fcy = d.fc;
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
  d.uniform64 = (L % 64 == 0 && L / 64 == P && d.pitch % 16 == 0) ? 1 : 0;
  fill_perm24(d.perm24);

  NoallocSetup su;
  std::memset(&su, 0, sizeof su);
  su.L = L;
  su.S = S;
  su.mcs_begin = (uint32_t)mcs_begin;
  std::memcpy(su.digraph, digraph, (size_t)S * S);
  noalloc_setup_kernel<<<1, 256, 0, stream>>>(scratch, su);
  cudaError_t e = cudaGetLastError();
  RunState* st = reinterpret_cast<RunState*>(scratch);
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
  if (err_word & kErrTimeout) {
    set_last_error("escg_run_noalloc: a bounded device-side wait timed out");
    return ESCG_ETIMEOUT;
  }
  return ESCG_OK;
}
