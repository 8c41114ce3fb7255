// escg_internal.h -- declarations shared by the library's translation units
// (kernel launchers and the device-side run state).  Not part of the C ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "escg_types.h"

namespace escg_impl {

// Device-side run state of one lattice (lives in device memory).
struct RunState {
  uint32_t mcs;        // absolute MCS number the lattice has reached
  uint32_t stopped;    // stasis reached with stop_at_extinction
  uint32_t error;      // error bits (kErrTimeout, ...)
  uint32_t abort;      // set by a CTA that gave up; others leave quickly
  uint32_t n_log;      // number of count-log entries written so far
  uint32_t ticket;     // work-item dispenser of the persistent kernel
  uint32_t pad[2];
  unsigned long long cur[kMaxStates];  // counts being accumulated
};

constexpr uint32_t kErrTimeout = 1u;
constexpr int kLogCap = 4096;  // ring of logged count vectors per lattice

// Host-side launchers (all asynchronous on `stream`).
void upload_perm_table();  // once per process/device
cudaError_t launch_init(const LatticeDesc& d, uint64_t T_empty, cudaStream_t stream);
// Accumulates the lattice histogram into st->cur (which must be zero).
cudaError_t launch_count(const LatticeDesc& d, RunState* st, cudaStream_t stream);
// After a chunk ending at MCS m_end: st->mcs = m_end (unless stopped); if
// `log` appends st->cur to the ring (entry n_log, MCS m_end) and, with
// stop_at_extinction, sets st->stopped when <= 1 species is alive.
cudaError_t launch_finalize(const LatticeDesc& d, RunState* st, unsigned long long* log_counts,
                            uint32_t* log_mcs, uint32_t m_end, int log, int stop_at_extinction,
                            cudaStream_t stream);
// One coarse phase (slot 0..3 of MCS m): one CTA per active block.
cudaError_t launch_phase(const LatticeDesc& d, RunState* st, uint32_t m, int slot,
                         cudaStream_t stream);
// MCS [m_begin, m_begin + n_mcs) in one persistent dataflow launch.
// done: P*P epoch counters, zeroed by the caller together with st->ticket.
// stall_block >= 0 (test hook) never publishes that block's epoch.
cudaError_t launch_persistent(const LatticeDesc& d, RunState* st, uint32_t* done, uint32_t m_begin,
                              uint32_t n_mcs, int grid, uint32_t spin_limit, int stall_block,
                              cudaStream_t stream);
// Occupancy-derived grid size of the persistent kernel.
int persistent_grid(int device);
int persistent_block_threads();

}  // namespace escg_impl
