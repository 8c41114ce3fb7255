// escg_internal.h -- declarations shared by the library's translation units
// (kernel launchers and the device-side run state).  Not part of the C ABI.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "escg_types.h"

namespace escg_impl {

constexpr int kLogCap = 4096;   // ring of logged count vectors per lattice
constexpr int kPendRing = 64;   // log points a persistent launch may have open

// Device-side run state of one lattice (lives in device memory).
struct RunState {
  uint32_t mcs;        // absolute MCS number the lattice has reached
  uint32_t stopped;    // stasis reached with stop_at_extinction
  uint32_t error;      // error bits (kErrTimeout, ...)
  uint32_t abort;      // set by a CTA that gave up; others leave quickly
  uint32_t n_log;      // count-log entries written (entry i = log number log_num0 + i)
  uint32_t log_num0;   // log number (MCS / log_every) of entry 0
  uint32_t ticket;     // work-item dispenser of the persistent kernel
  uint32_t exited;     // CTAs of the current persistent launch that have left
  unsigned long long cur[kMaxStates];             // counts being accumulated
  unsigned long long acc[kPendRing][kMaxStates];  // open log points (fused counts)
  uint32_t pend[kPendRing];                       // blocks done per open log point
};

constexpr uint32_t kErrTimeout = 1u;
constexpr uint32_t kErrBadValue = 2u;   // a restored lattice held a value outside 0..S

struct LogBuffers {
  unsigned long long* counts;  // [kLogCap][kMaxStates]
  uint32_t* mcs;               // [kLogCap]
};

// Sets the thread-local message returned by escg_last_error().
void set_last_error(const char* fmt, ...);

// Fills out[kTransWords] with the transition table of LatticeDesc::trans for
// S species, dominance digraph D (S*S), optional edge probabilities prob
// (S*S, nullptr: every edge certain) and the 64-bit rate thresholds.
void build_transitions(int S, const uint8_t* D, const double* prob, uint64_t tx, uint64_t txi,
                       uint32_t* out);

// Host-side launchers (all asynchronous on `stream`).
cudaError_t launch_init(const LatticeDesc& d, uint64_t T_empty, cudaStream_t stream);
// Packed lattice (d.bits 4 or 2) from / to a byte image of byte_pitch-byte rows.
cudaError_t launch_pack(const LatticeDesc& d, const uint8_t* bytes, int byte_pitch, cudaStream_t stream);
cudaError_t launch_unpack(const LatticeDesc& d, uint8_t* bytes, int byte_pitch, cudaStream_t stream);
cudaError_t launch_fill_u32(uint32_t* p, int n, uint32_t value, cudaStream_t stream);
// Sets *bad |= flag if any lattice byte is outside 0..S, and then *stop = 1
// unless stop is null.
cudaError_t launch_validate(const LatticeDesc& d, uint32_t* bad, uint32_t flag, uint32_t* stop,
                            cudaStream_t stream);
// Zeroes *st and sets its MCS number and first log number.
cudaError_t launch_state_reset(RunState* st, uint32_t mcs, uint32_t log_num0, cudaStream_t stream);
// Accumulates the lattice histogram into st->cur (which must be zero).
cudaError_t launch_count(const LatticeDesc& d, RunState* st, cudaStream_t stream);
// After work ending at MCS m_end: st->mcs = m_end (unless stopped); if `log`
// appends st->cur as the entry of MCS m_end and, with stop_at_extinction,
// sets st->stopped when <= 1 species is alive.  check_total != 0: the counts
// must add up to it (every byte a state 0..S), else st->error |=
// kErrBadValue and st->stopped = 1 (a restored lattice checked by its count).
cudaError_t launch_finalize(const LatticeDesc& d, RunState* st, LogBuffers lb, uint32_t m_end,
                            uint32_t log_every, int log, int stop_at_extinction, cudaStream_t stream,
                            uint64_t check_total = 0);
// One coarse phase (slot 0..3 of MCS m): one CTA per active block.
cudaError_t launch_phase(const LatticeDesc& d, RunState* st, uint32_t m, int slot,
                         cudaStream_t stream);

struct PersistentArgs {
  LatticeDesc d;
  RunState* st;
  uint32_t* done;        // [P*P] absolute MCS count each block has completed
  LogBuffers lb;
  uint32_t m_begin, n_mcs;
  uint32_t log_every;
  int32_t stop_at_extinction;
  uint32_t spin_limit;
  int32_t stall_block;   // test hook: never publish this block's epoch (-1: off)
  unsigned long long* ob;  // boundary records of the mailbox kernel ([P*P][4][32]), else null
  int32_t fuse_counts;     // 1: counts of log points fused into the visits; 0: the host counts
  int32_t threads;         // flag kernel on uniform one-byte lattices: 128 (two quads per
                           // thread, up to 8 CTAs per SM) or 0 / 256 (one quad per thread)
  // div_rcp32 of the ticket decode's divisors (blocks per MCS, blocks per
  // coarse phase, half the blocks per row); filled in by launch_persistent
  uint32_t rcp_nb, rcp_per, rcp_half;
};
// MCS [m_begin, m_begin + n_mcs) in one persistent dataflow launch, counts
// of log points fused in.
cudaError_t launch_persistent(const PersistentArgs& a, int grid, cudaStream_t stream);
// Occupancy-derived grid size of the persistent kernel for a lattice.
int persistent_grid(int device, bool uniform);
// The same for the 128-thread build of the uniform flag kernel (up to 8 per SM).
int persistent_grid128(int device);

// Whole-lattice residency: one CTA runs MCS [m_begin, m_begin + n_mcs) with
// the lattice in shared memory (counts of log points written in-kernel).
bool resident_fits(const LatticeDesc& d, int device);
cudaError_t launch_resident(const PersistentArgs& a, cudaStream_t stream);

// Uniform geometry, boundary-mailbox variant (the default persistent path):
// a visit publishes its four boundary records (edge line + rim line per
// side, 4 lattice bytes and the epoch per 8-byte word) and only its interior
// to the lattice; neighbours read the records instead of waiting on epoch
// flags.  a.ob must hold kRecordWords words per block.
constexpr int kRecordWords = 128;
cudaError_t launch_persistent_ll(const PersistentArgs& a, int grid, cudaStream_t stream);
int persistent_ll_grid(int device);
// Block-owner variant (uniform geometry, one byte per site): CTA g owns
// coarse group g (2x2 blocks) for the whole launch with their tiles in
// shared memory and exchanges boundary records like the mailbox kernel (a.ob,
// kRecordWords per block); it leaves the lattice array complete.
// All (P/2)(Py/2) CTAs must be resident at once: persistent_own_config returns
// the grid size, the CTA size (128 or 256 threads), the shared-memory
// padding that spreads the grid over the SMs and the CTAs per SM that
// leaves, or 0 when the device cannot hold the whole grid.  min_per_sm > 0
// packs at least that many CTAs per SM (fewer SMs, the rest left to other
// streams' kernels).
int persistent_own_config(const LatticeDesc& d, int device, int* dyn_bytes, int* threads, int* ctas_per_sm,
                          int min_per_sm = 0);
cudaError_t launch_persistent_own(const PersistentArgs& a, int dyn_bytes, int threads, cudaStream_t stream);
// Block owners on any partition of the von Neumann rule (escg_owner.cu):
// periodic or reflecting, squares and rectangles, any bits per site; blocks
// of at most kMaxBlock sites with fine segments of 2 or 3 sites.  Records of
// kGRecordWords words per block (4 sides x 2 lines x 32 word slots); the
// grid of (P/2)(Py/2) CTAs must be resident at once.
constexpr int kGRecordWords = 256;
struct GownConfig {
  int dyn_bytes;     // dynamic shared memory: 4 tiles, the drawn words, padding
  int threads;       // 256 or 512 (one quad per thread)
  int ctas_per_sm;
  int tile_stride;   // bytes per tile in dynamic shared memory
  int prefetch;      // 512 threads, half of them drawing the next visit's words
};
struct GownArgs {
  PersistentArgs p;
  int32_t tile_stride;
};
// Grid size (0: this lattice or device cannot run the kernel) and launch
// configuration; min_per_sm as for persistent_own_config.
int persistent_gown_config(const LatticeDesc& d, int device, GownConfig* cfg, int min_per_sm = 0);
cudaError_t launch_persistent_gown(const PersistentArgs& a, const GownConfig& cfg, cudaStream_t stream);
// Completes the lattice array after a mailbox launch that ended at MCS
// m_end: every edge cell of a block that a neighbour's visit wrote last (in
// MCS m_end - 1) takes the value from that neighbour's record.  Does nothing
// unless the lattice reached m_end (st->mcs).
cudaError_t launch_ll_merge(const LatticeDesc& d, const unsigned long long* ob, const RunState* st,
                            uint32_t m_end, cudaStream_t stream);

// Uniform geometry (64x64 blocks): TMA-staged, warp-specialised variant.
// map: 2-D uint8 tensor map of the lattice (dims L x L, row stride pitch,
// box 112 x 66).
struct TmaArgs {   // aligned like CUtensorMap
  CUtensorMap map;
  PersistentArgs p;
};
cudaError_t launch_persistent_tma(const TmaArgs& a, int grid, cudaStream_t stream);

// 2-D uint8 tensor map of a lattice (dims L x L, row stride pitch, box
// box_w x box_h bytes; out-of-bounds elements read as zero).
bool encode_lattice_map(CUtensorMap* map, uint8_t* lattice, int L, int pitch, int box_w, int box_h);
int persistent_tma_grid(int device);

}  // namespace escg_impl
