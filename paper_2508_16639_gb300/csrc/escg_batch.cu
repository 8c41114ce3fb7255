// escg_batch.cu -- batched ensembles (include/escg.h, escg_batch_*): many
// independent replicas of uneven L in shared persistent launches.
//
// Device layout: one arena holds every replica's lattice, partition tables,
// transition table and block epochs; SlotDesc (static, per replica) and
// SlotState (dynamic) arrays describe them.  A run is a sequence of chunks of
// log_every MCS.  Each chunk is two kernels on the batch's stream:
//   batch_compact_kernel  advances every active replica's MCS by the last
//                         chunk, retires replicas that went extinct or spent
//                         their budget, admits new ones, and rebuilds the
//                         work table (one entry per block of a coarse phase
//                         of every active replica);
//   batch_kernel          persistent: CTAs take work items (chunk MCS index,
//                         coarse slot, table entry) from a ticket counter, wait
//                         for the block's 8 neighbours in its own replica
//                         (bounded spin), and visit the block exactly as the
//                         single-lattice kernels do; the counts of the chunk's
//                         final MCS (a log point) are fused in, and the last
//                         block of a replica decides its stasis.
// The chunk sequence needs no host round trip, so it is captured once in a
// CUDA graph and replayed.  A replica's trajectory depends only on its own
// parameters: items of different replicas never share data.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <unordered_map>
#include <vector>

#include "escg.h"
#include "escg_device.cuh"
#include "escg_internal.h"
#include "escg_resident.cuh"
#include "escg_rule8.cuh"
#include "escg_tma.cuh"

namespace escg_impl {

struct SlotDesc {
  LatticeDesc d;
  uint32_t* done;       // [P*P] absolute epochs
  uint32_t max_mcs;     // budget: absolute MCS number to stop at
  int32_t stop_at_extinction;
  int32_t nb4;          // blocks per coarse phase = P*P/4 in the chunk kernel's table (0: resident)
  int32_t rclass;       // 0: chunk kernel; 1..3: whole-lattice residency class
};

struct SlotState {
  uint32_t mcs;         // absolute MCS reached (advanced by the compaction)
  uint32_t stopped;     // stasis reached
  uint32_t pend;        // blocks done at the open log point
  uint32_t counts_mcs;  // MCS of `counts`
  unsigned long long acc[kMaxStates];
  unsigned long long counts[kMaxStates];   // counts at the last log point
};

struct BatchCtl {
  uint32_t n_active, tot4, chunk, ticket;
  uint32_t exited, error, abort, n_admit;
  uint32_t last_chunk;  // MCS the previous batch_kernel launch covered
  uint32_t res_ticket[3];  // dispensers of the resident kernels (classes 1..3)
  uint32_t pad[4];
};

struct BatchArgs {
  const SlotDesc* slots;
  SlotState* states;
  BatchCtl* ctl;
  const uint32_t* table;   // (slot << 16) | block-of-phase
  uint32_t log_every;
  uint32_t spin_limit;
};

__device__ __forceinline__ uint32_t b_ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void b_st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t b_ld_volatile(const uint32_t* p) {
  return *reinterpret_cast<const volatile uint32_t*>(p);
}

// Counts of the whole lattice of every slot (one CTA per slot), written as
// the slot's log entry of its current MCS; sets stopped when <= 1 species
// is alive and the slot stops at extinction.  Used once, at creation/admission.
__global__ void batch_count_kernel(const SlotDesc* slots, SlotState* states, const uint32_t* which, int n) {
  const int w = blockIdx.x;
  if (w >= n) return;
  const int s = which ? (int)which[w] : w;
  const LatticeDesc& d = slots[s].d;
  __shared__ uint32_t hist[kMaxStates];
  if (threadIdx.x < kMaxStates) hist[threadIdx.x] = 0;
  __syncthreads();
  count_vectors(d, threadIdx.x, blockDim.x, hist);
  __syncthreads();
  if (threadIdx.x == 0) {
    SlotState& st = states[s];
    int alive = 0;
    for (int v = 0; v < kMaxStates; ++v) {
      const unsigned long long c = (v <= d.S) ? hist[v] : 0ull;
      st.counts[v] = c;
      st.acc[v] = 0;
      if (v >= 1 && v <= d.S && c > 0) ++alive;
    }
    st.counts_mcs = st.mcs;
    st.pend = 0;
    if (slots[s].stop_at_extinction && alive <= 1) st.stopped = 1;
  }
}

// Single CTA.  Advances the active replicas by the last chunk, retires the
// finished ones, admits the slots listed in `admit`, and rebuilds the work
// table and the launch control block for the next chunk.
constexpr int kCompactThreads = 1024;
__global__ void __launch_bounds__(kCompactThreads) batch_compact_kernel(const SlotDesc* slots, SlotState* states,
                                                                        BatchCtl* ctl, uint32_t* active,
                                                                        uint32_t* active_tmp, uint32_t* table,
                                                                        const uint32_t* admit, uint32_t chunk) {
  __shared__ uint32_t s_scan[kCompactThreads];
  __shared__ uint32_t s_keep_total, s_n_old, s_n_admit, s_last;
  const int t = threadIdx.x;
  if (t == 0) {
    s_n_old = ctl->n_active;
    s_n_admit = ctl->n_admit;
    s_last = ctl->last_chunk;
  }
  __syncthreads();
  const uint32_t n_old = s_n_old, n_admit = s_n_admit, last = s_last;
  const uint32_t n_all = n_old + n_admit;
  // 1. advance and decide which slots stay (old active first, then admitted)
  const uint32_t per = (n_all + kCompactThreads - 1) / kCompactThreads;
  const uint32_t lo = t * per, hi = min(n_all, lo + per);
  uint32_t keep_count = 0;
  for (uint32_t a = lo; a < hi; ++a) {
    const uint32_t s = a < n_old ? active[a] : admit[a - n_old];
    SlotState& st = states[s];
    if (a < n_old && !st.stopped) {
      const uint32_t nm = st.mcs + last;
      st.mcs = nm < slots[s].max_mcs ? nm : slots[s].max_mcs;
    } else if (a < n_old && st.stopped) {
      st.mcs = st.counts_mcs;
    }
    if (!st.stopped && st.mcs < slots[s].max_mcs) ++keep_count;
  }
  s_scan[t] = keep_count;
  __syncthreads();
  for (int off = 1; off < kCompactThreads; off <<= 1) {   // inclusive scan
    const uint32_t v = t >= off ? s_scan[t - off] : 0u;
    __syncthreads();
    s_scan[t] += v;
    __syncthreads();
  }
  uint32_t pos = s_scan[t] - keep_count;
  if (t == kCompactThreads - 1) s_keep_total = s_scan[t];
  for (uint32_t a = lo; a < hi; ++a) {
    const uint32_t s = a < n_old ? active[a] : admit[a - n_old];
    const SlotState& st = states[s];
    if (!st.stopped && st.mcs < slots[s].max_mcs) active_tmp[pos++] = s;
  }
  __syncthreads();
  const uint32_t n_new = s_keep_total;
  // 2. work table: nb4 entries per kept slot, in active order
  const uint32_t per2 = (n_new + kCompactThreads - 1) / kCompactThreads;
  const uint32_t lo2 = t * per2, hi2 = min(n_new, lo2 + per2);
  uint32_t sum = 0;
  for (uint32_t a = lo2; a < hi2; ++a) sum += (uint32_t)slots[active_tmp[a]].nb4;
  __syncthreads();
  s_scan[t] = sum;
  __syncthreads();
  for (int off = 1; off < kCompactThreads; off <<= 1) {
    const uint32_t v = t >= off ? s_scan[t - off] : 0u;
    __syncthreads();
    s_scan[t] += v;
    __syncthreads();
  }
  uint32_t e = s_scan[t] - sum;
  for (uint32_t a = lo2; a < hi2; ++a) {
    const uint32_t s = active_tmp[a];
    active[a] = s;
    const uint32_t nb4 = (uint32_t)slots[s].nb4;
    for (uint32_t j = 0; j < nb4; ++j) table[e++] = (s << 16) | j;
  }
  __syncthreads();
  if (t == kCompactThreads - 1) {
    ctl->n_active = n_new;
    ctl->tot4 = s_scan[t];
    ctl->chunk = chunk;
    ctl->ticket = 0;
    ctl->exited = 0;
    ctl->n_admit = 0;
    ctl->res_ticket[0] = ctl->res_ticket[1] = ctl->res_ticket[2] = 0;
    ctl->last_chunk = 0;   // consumed; the next batch_kernel launch sets it
  }
}

// Persistent multi-replica chunk kernel.
template <int THREADS>
__global__ void __launch_bounds__(THREADS) batch_kernel(BatchArgs a) {
  __shared__ VisitSmem sm;
  __shared__ SlotDesc sd;
  __shared__ uint32_t s_quit, s_skip, s_abort, s_slot, s_m, s_ord;
  __shared__ int32_t s_k, s_bx, s_by, s_col;
  BatchCtl* ctl = a.ctl;
  const int tid = threadIdx.x;
  const uint32_t tot4 = ctl->tot4, chunk = ctl->chunk;
  const uint64_t total = (uint64_t)chunk * 4u * tot4;
  for (;;) {
    if (tid == 0) {
      const uint32_t t = atomicAdd(&ctl->ticket, 1u);
      uint32_t quit = ((uint64_t)t >= total) || b_ld_volatile(&ctl->abort);
      if (!quit) {
        const uint32_t i = t / (4u * tot4), rem = t - i * 4u * tot4;
        const uint32_t k = rem / tot4, e = a.table[rem - k * tot4];
        s_slot = e >> 16;
        s_k = (int32_t)k;
        s_m = i;   // chunk-relative for now
        s_by = (int32_t)(e & 0xFFFFu);   // block index within the phase
      }
      s_quit = quit;
      s_abort = 0;
    }
    if (tid < kMaxStates) sm.hist[tid] = 0;
    __syncthreads();
    if (s_quit) break;
    {  // the replica's descriptor
      const uint32_t* src = reinterpret_cast<const uint32_t*>(a.slots + s_slot);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&sd);
      for (int w = tid; w < (int)(sizeof(SlotDesc) / 4); w += THREADS) dst[w] = src[w];
    }
    __syncthreads();
    const LatticeDesc& d = sd.d;
    if (tid == 0) {
      const uint32_t m = a.states[s_slot].mcs + s_m;
      s_m = m;
      s_skip = m >= sd.max_mcs;
      if (!s_skip) {
        const uint32_t ord = colour_order(philox10_rk(make_uint4(0u, 0u, m, kTagOrder), d.rk).x, d.perm24);
        const int colour = order_at(ord, s_k), j = s_by, half = d.P >> 1;
        s_ord = ord;
        s_col = colour;
        s_bx = 2 * (j % half) + (colour & 1);
        s_by = 2 * (j / half) + (colour >> 1);
      }
    }
    load_trans(d, sm.trans);
    __syncthreads();
    if (s_skip) continue;   // beyond this replica's budget
    const uint32_t m = s_m, ord = s_ord;
    const int k = s_k, colour = s_col, bx = s_bx, by = s_by, P = d.P;
    if (tid < 9) {
      const int dx = tid % 3 - 1, dy = tid / 3 - 1;
      const int nx = (bx + dx + P) % P, ny = (by + dy + P) % P;
      const int ncol = colour ^ ((dx & 1) | ((dy & 1) << 1));
      const uint32_t need = (tid == 4) ? m : (slot_of(ord, ncol) < k ? m + 1u : m);
      const uint32_t* flag = sd.done + ny * P + nx;
      uint32_t spins = 0;
      while (b_ld_acquire(flag) < need) {
        if ((spins & 15u) == 15u && b_ld_volatile(&ctl->abort)) {
          s_abort = 1;
          break;
        }
        if (++spins > a.spin_limit) {
          atomicOr(&ctl->error, kErrTimeout);
          atomicExch(&ctl->abort, 1u);
          s_abort = 1;
          break;
        }
        __nanosleep(64);
      }
    }
    __syncthreads();
    if (s_abort) break;
    visit_generic(d, bx, by, m, sm);
    const bool log_point = ((m + 1u) % a.log_every) == 0u;
    if (log_point) {
      const int sV = slot_of(ord, colour ^ 2), sH = slot_of(ord, colour ^ 1), sD = slot_of(ord, colour ^ 3);
      count_visit_generic(d, bx, by, sm, k, sV, sH, sD);
    }
    __syncthreads();
    if (log_point) {
      SlotState* st = a.states + s_slot;
      if (tid <= d.S && sm.hist[tid]) atomicAdd(&st->acc[tid], (unsigned long long)sm.hist[tid]);
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        if (atomicAdd(&st->pend, 1u) == (uint32_t)(P * P) - 1u) {
          __threadfence();
          int alive = 0;
          for (int v = 0; v < kMaxStates; ++v) {
            const unsigned long long c = atomicExch(&st->acc[v], 0ull);
            st->counts[v] = c;
            if (v >= 1 && v <= d.S && c > 0) ++alive;
          }
          st->counts_mcs = m + 1u;
          st->pend = 0;
          if (sd.stop_at_extinction && alive <= 1) st->stopped = 1;
        }
      }
    }
    if (tid == 0) b_st_release(sd.done + by * P + bx, m + 1u);   // release orders the tile stores
  }
  // the last CTA to leave records how far this launch advanced the replicas
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(&ctl->exited, 1u) == gridDim.x - 1u) {
      ctl->exited = 0;
      ctl->last_chunk = chunk;
    }
  }
}

// ---------------------------------------------------------------------------
// Whole-lattice residency for replicas that fit one CTA's shared memory
// (escg_resident.cuh).  Classes by image size, so that small replicas share
// an SM: 1 up to kResBytes1 (128 threads), 2 up to kResBytes2 (256), 3 up to
// the device's per-CTA limit (1024).  CTAs take the active replicas of their
// class from a dispenser and run each one's chunk from its lattice in
// shared memory: no work table, no epochs, no waits; the chunk's final MCS
// (a log point) sets the replica's counts and stasis exactly as the chunk
// kernel's last block does.
constexpr int kResBytes1 = 16 * 1024, kResBytes2 = 56 * 1024;

// 64 registers a thread (8, 4 and 1 CTAs per SM for the three classes).
template <int THREADS, int CLASS>
__global__ void __launch_bounds__(THREADS, 65536 / (THREADS * 64)) batch_resident_kernel(BatchArgs a,
                                                                                          const uint32_t* active) {
  extern __shared__ __align__(16) uint8_t res_dyn[];
  __shared__ ResidentSmem rs;
  __shared__ SlotDesc sd;
  __shared__ uint32_t s_slot, s_quit;
  BatchCtl* ctl = a.ctl;
  const int tid = threadIdx.x;
  const uint32_t n_active = ctl->n_active, chunk = ctl->chunk;
  for (;;) {
    if (tid == 0) {
      uint32_t quit = 0, s = 0;
      for (;;) {
        const uint32_t t = atomicAdd(&ctl->res_ticket[CLASS - 1], 1u);
        if (t >= n_active || b_ld_volatile(&ctl->abort)) {
          quit = 1;
          break;
        }
        s = active[t];
        if (a.slots[s].rclass == CLASS) break;
      }
      s_slot = s;
      s_quit = quit;
    }
    __syncthreads();
    if (s_quit) break;
    {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(a.slots + s_slot);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&sd);
      for (int w = tid; w < (int)(sizeof(SlotDesc) / 4); w += THREADS) dst[w] = src[w];
    }
    __syncthreads();
    const LatticeDesc& d = sd.d;
    SlotState* st = a.states + s_slot;
    const uint32_t m0 = st->mcs;
    const uint32_t m_end = min(m0 + chunk, sd.max_mcs);
    if (m0 >= m_end) continue;   // uniform: every thread read the same words
    const int sp = resident_pitch(d.L);
    uint8_t* img = res_dyn;
    uint8_t* snap = res_dyn + (d.H + 2) * sp;
    load_trans(d, rs.trans);
    resident_load(d, img, sp);
    __syncthreads();
    resident_run(d, img, sp, snap, rs, m0, m_end, a.log_every, [&](uint32_t mm, const uint32_t* hist) {
      int alive = 0;
      for (int v = 0; v < kMaxStates; ++v) {
        const unsigned long long c = (v <= d.S) ? hist[v] : 0ull;
        st->counts[v] = c;
        if (v >= 1 && v <= d.S && c > 0) ++alive;
      }
      st->counts_mcs = mm;
      const bool stop = sd.stop_at_extinction && alive <= 1;
      if (stop) st->stopped = 1;
      return stop;
    });
    resident_store(d, img, sp);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Warp-specialised variant of the chunk kernel.  The last warp (producer)
// prepares the next work item in one of two buffers while the CONS consumer
// threads compute on the other: it takes tickets (skipping items beyond a
// replica's budget), copies the replica's descriptor, transition table and
// the block's fine partition into shared memory, waits for the block's 8
// neighbours, and stages block + rim with one TMA box load through the
// replica's tensor map (box 144 x 98 bytes from (floor16(x0-1), y0-1); the
// wrap-around rim cells of blocks on the lattice edge, which the box fills
// with zeros, are patched afterwards).
constexpr int kBSP = 144, kBRows = kMaxBlock + 2;
constexpr uint32_t kBBoxBytes = (uint32_t)(kBSP * kBRows);   // 14112
constexpr int kBTileStride = 14208;                          // 128-byte multiple
// Suspending waits of the warp-specialised chunk kernel: hint and bound
// (about 4 s at 2 GHz, the order of the flag waits' spin limit).
constexpr uint32_t kBMbarHintNs = 2000;
constexpr long long kBMbarMaxCycles = 8000000000ll;

struct BItem {
  uint32_t m, ord, forder, quit;
  int32_t slot, k, bx, by, colour, x0, y0, bw, bh, xoff, fx0, fy0, Qx, Qy;
  int16_t fsx[kMaxFine + 2], fsy[kMaxFine + 2];
};

struct BatchTmaSmem {
  alignas(128) uint8_t tile[2][kBTileStride];
  uint2 trans2[2][kTransPairs];   // the replica's transition table, one 8-byte entry per pair (rule8)
  SlotDesc sd[2];
  BItem item[2];
  alignas(8) uint64_t full[2], empty[2], tma[2];
  uint32_t hist[kMaxStates];
};

struct BatchTmaArgs {
  BatchArgs a;
  const CUtensorMap* maps;   // one per slot
};

__device__ __forceinline__ void btma_fail(BatchCtl* ctl) {
  atomicOr(&ctl->error, kErrTimeout);
  atomicExch(&ctl->abort, 1u);
}

__device__ void btma_producer(const BatchTmaArgs& ta, BatchTmaSmem& sm, uint64_t total, uint32_t tot4) {
  const BatchArgs& a = ta.a;
  BatchCtl* ctl = a.ctl;
  const int lane = threadIdx.x & 31;
  for (uint32_t n = 0;; ++n) {
    const int b = (int)(n & 1u);
    const uint32_t use = n >> 1;
    // next ticket whose MCS is within its replica's budget
    uint32_t quit = 0, slot = 0, j = 0, k = 0, m = 0;
    if (lane == 0) {
      for (;;) {
        const uint32_t t = atomicAdd(&ctl->ticket, 1u);
        if ((uint64_t)t >= total || b_ld_volatile(&ctl->abort)) {
          quit = 1;
          break;
        }
        const uint32_t i = t / (4u * tot4), rem = t - i * 4u * tot4;
        k = rem / tot4;
        const uint32_t e = a.table[rem - k * tot4];
        slot = e >> 16;
        j = e & 0xFFFFu;
        m = a.states[slot].mcs + i;
        if (m < a.slots[slot].max_mcs) break;
      }
      if (!mbar_wait_sleep(&sm.empty[b], (use & 1u) ^ 1u, kBMbarHintNs, kBMbarMaxCycles)) {
        btma_fail(ctl);
        quit = 1;
      }
    }
    quit = __shfl_sync(0xFFFFFFFFu, quit, 0);
    if (quit) {
      if (lane == 0) sm.item[b].quit = 1;
      __syncwarp();
      mbar_arrive(&sm.full[b]);
      return;
    }
    slot = __shfl_sync(0xFFFFFFFFu, slot, 0);
    j = __shfl_sync(0xFFFFFFFFu, j, 0);
    k = __shfl_sync(0xFFFFFFFFu, k, 0);
    m = __shfl_sync(0xFFFFFFFFu, m, 0);
    {  // replica descriptor into this buffer
      const uint32_t* src = reinterpret_cast<const uint32_t*>(a.slots + slot);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&sm.sd[b]);
      for (int w = lane; w < (int)(sizeof(SlotDesc) / 4); w += 32) dst[w] = src[w];
    }
    __syncwarp();
    const SlotDesc& sd = sm.sd[b];
    const LatticeDesc& d = sd.d;
    const int P = d.P, half = P >> 1;
    uint32_t ord = 0;
    if (lane == 0) ord = colour_order(philox10_rk(make_uint4(0u, 0u, m, kTagOrder), d.rk).x, d.perm24);
    ord = __shfl_sync(0xFFFFFFFFu, ord, 0);
    const int colour = order_at(ord, (int)k);
    const int bx = 2 * ((int)j % half) + (colour & 1), by = 2 * ((int)j / half) + (colour >> 1);
    uint32_t forder = 0;
    if (lane == 1)
      forder = colour_order(philox10_rk(make_uint4(0u, (uint32_t)(by * P + bx), m, kTagFineOrder), d.rk).x,
                            d.perm24);
    forder = __shfl_sync(0xFFFFFFFFu, forder, 1);
    // block span and fine segments from the closed-form partition (no
    // dependent table loads on the producer's path)
    const BlockSpan X = block_span(d.ax, bx), Y = block_span(d.ay, by);
    const int x0 = X.s0, bw = X.w, y0 = Y.s0, bh = Y.w;
    const int fx0 = X.f0, Qx = X.Q, fy0 = Y.f0, Qy = Y.Q;
    BItem& it = sm.item[b];
    for (int q = lane; q <= Qx; q += 32) it.fsx[q] = (int16_t)seg_start(X, q);
    for (int q = lane; q <= Qy; q += 32) it.fsy[q] = (int16_t)seg_start(Y, q);
    fill_trans8(sm.trans2[b], d.trans, d.S, lane, 32);
    // wait until the 8 neighbours (and the block itself) have completed
    // every visit that precedes this one in schedule order
    uint32_t fail = 0;
    if (lane < 9) {
      const int dx = lane % 3 - 1, dy = lane / 3 - 1;
      const int nx = (bx + dx + P) % P, ny = (by + dy + P) % P;
      const int ncol = colour ^ ((dx & 1) | ((dy & 1) << 1));
      const uint32_t need = (lane == 4) ? m : (slot_of(ord, ncol) < (int)k ? m + 1u : m);
      const uint32_t* flag = sd.done + ny * P + nx;
      uint32_t spins = 0;
      while (b_ld_acquire(flag) < need) {
        if ((spins & 15u) == 15u && b_ld_volatile(&ctl->abort)) {
          fail = 1;
          break;
        }
        if (++spins > a.spin_limit) {
          btma_fail(ctl);
          fail = 1;
          break;
        }
        __nanosleep(64);
      }
      fence_proxy_async_global();   // what was acquired is read by the TMA next
    }
    const int xal = (x0 - 1) & ~15;   // floor to a 16-byte boundary (x0 - 1 >= -1)
    uint32_t ok = __any_sync(0xFFFFFFFFu, fail != 0) ? 0u : 1u;
    // wrap-around rim cells of blocks on the lattice edge (the box fills them
    // with zeros): loaded now, beside the box, and placed once it has landed.
    // Blocks are at most 96 sites wide: 3 cells per lane and edge.
    const int L = d.L, pitch = d.pitch, xoff = x0 - xal;
    const uint8_t* lat = d.lat;
    uint8_t wrow[3] = {0, 0, 0}, wcol[3] = {0, 0, 0};
    const bool top = by == 0, left = bx == 0;   // P >= 2: otherwise bottom / right
    const bool wrap_row = by == 0 || by == P - 1, wrap_col = bx == 0 || bx == P - 1;
    if (ok) {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const int c = lane + 32 * i;
        if (wrap_row && c < bw) wrow[i] = __ldcg(lat + (top ? (size_t)(L - 1) * pitch : (size_t)0) + x0 + c);
        if (wrap_col && c < bh) wcol[i] = __ldcg(lat + (size_t)(y0 + c) * pitch + (left ? L - 1 : 0));
      }
    }
    if (ok && lane == 0) {
      fence_proxy_async_smem();   // the consumers' accesses of this tile precede the TMA's
      mbar_arrive_expect_tx(&sm.tma[b], kBBoxBytes);
      tma_load_2d(sm.tile[b], ta.maps + slot, xal, y0 - 1, &sm.tma[b]);
      if (!mbar_wait_sleep(&sm.tma[b], use & 1u, kBMbarHintNs, kBMbarMaxCycles)) {
        btma_fail(ctl);
        mbar_wait_sleep(&sm.tma[b], use & 1u, kBMbarHintNs, kBMbarMaxCycles);   // no copy left in flight
        ok = 0;
      }
    }
    ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
    if (!ok) {
      if (lane == 0) it.quit = 1;
      __syncwarp();
      mbar_arrive(&sm.full[b]);
      return;
    }
    uint8_t* tile = sm.tile[b];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int c = lane + 32 * i;
      if (wrap_row && c < bw) tile[(top ? 0 : (bh + 1) * kBSP) + xoff + c] = wrow[i];
      if (wrap_col && c < bh) tile[(c + 1) * kBSP + xoff + (left ? -1 : bw)] = wcol[i];
    }
    if (lane == 0) {
      it.m = m; it.ord = ord; it.forder = forder; it.quit = 0;
      it.slot = (int32_t)slot; it.k = (int32_t)k; it.bx = bx; it.by = by; it.colour = colour;
      it.x0 = x0; it.y0 = y0; it.bw = bw; it.bh = bh; it.xoff = xoff;
      it.fx0 = fx0; it.fy0 = fy0; it.Qx = Qx; it.Qy = Qy;
    }
    __syncwarp();
    mbar_arrive(&sm.full[b]);   // 32 arrivals complete the phase
  }
}

// Write-back of a TMA-staged tile (lattice column xal + t at tile column t,
// xal = x0 - xoff a multiple of 16) by the CONS consumer threads: two rows
// per warp and pass, 16 lanes per row, one aligned 8-byte group per lane --
// the interior rows and the rim rows that the box read from the lattice
// whole (sites beyond the rims and the corners included, which belong to the
// block's eight neighbours, idle during the visit, and go back as the box
// read them), the lattice's last group of a row byte by byte (no row
// padding written); a wrapped rim row (placed beside the box, the block's
// columns only) byte by byte over those columns, and the wrapped rim-column
// cells of the interior rows one byte each.
template <int CONS>
__device__ __forceinline__ void btma_store(const LatticeDesc& d, int x0, int y0, int bw, int bh, int bx, int by,
                                           const uint8_t* tile, int xoff) {
  const int L = d.L, P = d.P, lane = threadIdx.x & 31, l16 = lane & 15;
  const int g_lo = max(x0 - 1, 0) >> 3, g_hi = min(x0 + bw, L - 1) >> 3;
  const bool act = l16 <= g_hi - g_lo;
  const int gcol = (g_lo + l16) * 8, tcol = gcol - (x0 - xoff);
  const bool wrap_top = by == 0, wrap_bot = by == P - 1;
  const bool wl = x0 == 0 && l16 == 0, wr = x0 + bw == L && l16 == g_hi - g_lo;
  if (!act) return;
  for (int r = 2 * (int)(threadIdx.x >> 5) + (lane >> 4) - 1; r <= bh; r += 2 * (CONS / 32)) {
    const bool wrapped = (r < 0 && wrap_top) || (r >= bh && wrap_bot);
    const int gy = r < 0 ? (wrap_top ? L - 1 : y0 - 1) : (r >= bh ? (wrap_bot ? 0 : y0 + bh) : y0 + r);
    uint8_t* row = d.lat + (size_t)gy * d.pitch;
    const uint8_t* trow = tile + (r + 1) * kBSP;
    const uint2 v = *reinterpret_cast<const uint2*>(trow + tcol);
    if (!wrapped && gcol + 8 <= L) {
      *reinterpret_cast<uint2*>(row + gcol) = v;
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int c = gcol + e;
        if (c < L && (!wrapped || (c >= x0 && c < x0 + bw)))
          row[c] = (uint8_t)(((e < 4) ? v.x : v.y) >> (8 * (e & 3)));
      }
    }
    if (r >= 0 && r < bh) {
      if (wl) row[L - 1] = trow[xoff - 1];
      if (wr) row[0] = trow[xoff + bw];
    }
  }
}

template <int CONS>
__device__ void btma_consumer(const BatchTmaArgs& ta, BatchTmaSmem& sm) {
  const BatchArgs& a = ta.a;
  BatchCtl* ctl = a.ctl;
  const int tid = threadIdx.x;
  // More blocks per coarse phase than CTAs: the chunk is throughput-bound,
  // and the regular (all 2 x 2) quads go first through the short step.
  // Otherwise each replica's chain of visits is the bound, and row-major
  // order spreads a fine phase's largest sub-blocks over all warps.
  const bool reg_first = ctl->tot4 > gridDim.x;
  for (uint32_t n = 0;; ++n) {
    const int b = (int)(n & 1u);
    const uint32_t use = n >> 1;
    if (!mbar_wait_sleep(&sm.full[b], use & 1u, kBMbarHintNs, kBMbarMaxCycles)) {
      if (tid == 0) btma_fail(ctl);
      return;
    }
    const BItem& it = sm.item[b];
    if (it.quit) return;
    const SlotDesc& sd = sm.sd[b];
    const LatticeDesc& d = sd.d;
    uint8_t* tile = sm.tile[b];
    const uint2* t2 = sm.trans2[b];
    const uint32_t m = it.m, ord = it.ord, s1 = (uint32_t)d.S + 1u, tx = d.tx, txi = d.txi;
    const int xoff = it.xoff, bw = it.bw, bh = it.bh, nquads = (it.Qx >> 1) * (it.Qy >> 1);
    // regular (all 2 x 2) quads first, as in visit_generic
    BlockSpan X, Y;
    X.Q = it.Qx;
    X.fq = bw / it.Qx;
    X.fr = bw - X.fq * it.Qx;
    Y.Q = it.Qy;
    Y.fq = bh / it.Qy;
    Y.fr = bh - Y.fq * it.Qy;
    const QuadMap qm = quad_map(X, Y);
    if (tid < kMaxStates) sm.hist[tid] = 0;
    for (int fi = 0; fi < 4; ++fi) {
      const int fcol = order_at(it.forder, fi);
      const int cx = fcol & 1, cy = fcol >> 1;
      for (int q = tid; q < nquads; q += CONS) {
        int qx, qy;
        if (reg_first) {
          quad_at(qm, q, qx, qy);
        } else {
          qy = (int)(((uint32_t)q * qm.inv_hx) >> 16);
          qx = q - qy * qm.hx;
        }
        const int fx = 2 * qx + cx, fy = 2 * qy + cy;
        const int sx = it.fsx[fx], wx = it.fsx[fx + 1] - sx;
        const int sy = it.fsy[fy], wy = it.fsy[fy + 1] - sy;
        if (reg_first && q < qm.n_reg) {   // a 2 x 2 sub-block: one Philox call, four attempts
          const uint32_t g = (uint32_t)(it.fy0 + fy) * (uint32_t)d.GQ + (uint32_t)(it.fx0 + fx);
          const int base = (sy + 1) * kBSP + xoff + sx;
          const uint4 x = philox10_rk(make_uint4(0u, g, m, kTagStep), d.rk);
          attempt8_2x2(tile, t2, x.x, base, kBSP, tx, txi, s1);
          attempt8_2x2(tile, t2, x.y, base, kBSP, tx, txi, s1);
          attempt8_2x2(tile, t2, x.z, base, kBSP, tx, txi, s1);
          attempt8_2x2(tile, t2, x.w, base, kBSP, tx, txi, s1);
          continue;
        }
        const uint32_t nk = (uint32_t)(wx * wy), n4 = 4u * nk;
        const uint32_t g = (uint32_t)(it.fy0 + fy) * (uint32_t)d.GQ + (uint32_t)(it.fx0 + fx);
        // ceil(65536 / wx) for the fine widths 2, 3, 4
        const uint32_t inv_wx = wx == 2 ? 32768u : (wx == 3 ? 21846u : 16384u);
        const int base = (sy + 1) * kBSP + xoff + sx;
        for (uint32_t jj = 0; 4u * jj < nk; ++jj) {
          const uint4 x = philox10_rk(make_uint4(jj, g, m, kTagStep), d.rk);
          const uint32_t wv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (4u * jj + (uint32_t)e < nk) attempt8(tile, t2, wv[e], n4, base, wx, inv_wx, kBSP, tx, txi, s1);
        }
      }
      bar_sync_consumers(CONS);
    }
    const bool log_point = ((m + 1u) % a.log_every) == 0u;
    if (log_point) {
      const int k = it.k, colour = it.colour;
      const int sV = slot_of(ord, colour ^ 2), sH = slot_of(ord, colour ^ 1), sD = slot_of(ord, colour ^ 3);
      count_tile_generic(tile, kBSP, xoff, bw, bh, sm.hist, CONS / 32, k, sV, sH, sD);
    }
    // write back the block interior and rim strips
    btma_store<CONS>(d, it.x0, it.y0, bw, bh, it.bx, it.by, tile, xoff);
    bar_sync_consumers(CONS);
    const int P = d.P, slot = it.slot, bx = it.bx, by = it.by;
    if (log_point) {
      SlotState* st = a.states + slot;
      if (tid <= d.S && sm.hist[tid]) atomicAdd(&st->acc[tid], (unsigned long long)sm.hist[tid]);
      bar_sync_consumers(CONS);
      if (tid == 0) {
        __threadfence();
        if (atomicAdd(&st->pend, 1u) == (uint32_t)(P * P) - 1u) {
          __threadfence();
          int alive = 0;
          for (int v = 0; v < kMaxStates; ++v) {
            const unsigned long long c = atomicExch(&st->acc[v], 0ull);
            st->counts[v] = c;
            if (v >= 1 && v <= d.S && c > 0) ++alive;
          }
          st->counts_mcs = m + 1u;
          st->pend = 0;
          if (sd.stop_at_extinction && alive <= 1) st->stopped = 1;
        }
      }
    }
    if (tid == 0) {
      b_st_release(sd.done + by * P + bx, m + 1u);   // release orders the tile stores
      mbar_arrive(&sm.empty[b]);                     // the buffer may be refilled
    }
  }
}

template <int CONS>
__global__ void __launch_bounds__(CONS + 32) batch_tma_kernel(const __grid_constant__ BatchTmaArgs ta) {
  __shared__ BatchTmaSmem sm;
  BatchCtl* ctl = ta.a.ctl;
  const int tid = threadIdx.x;
  const uint32_t tot4 = ctl->tot4, chunk = ctl->chunk;
  const uint64_t total = (uint64_t)chunk * 4u * tot4;
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sm.full[b], 32);
      mbar_init(&sm.empty[b], 1);
      mbar_init(&sm.tma[b], 1);
    }
    fence_mbar_init();
  }
  __syncthreads();
  if (tid >= CONS)
    btma_producer(ta, sm, total, tot4);
  else
    btma_consumer<CONS>(ta, sm);
  __syncthreads();
  // the last CTA to leave records how far this launch advanced the replicas
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(&ctl->exited, 1u) == gridDim.x - 1u) {
      ctl->exited = 0;
      ctl->last_chunk = chunk;
    }
  }
}

}  // namespace escg_impl

using namespace escg_impl;

namespace {

struct BPartition {
  int P = 0, GQ = 0;
  std::vector<int32_t> cs, fs, fc;
};

void bsplit(int n, int parts, int32_t* start) {
  const int q = n / parts, r = n % parts;
  start[0] = 0;
  for (int k = 0; k < parts; ++k) start[k + 1] = start[k] + q + (k < r ? 1 : 0);
}

BPartition bpartition(int L) {
  BPartition p;
  const int h = (L + 64) / 128;
  p.P = 2 * (h < 1 ? 1 : h);
  p.cs.resize(p.P + 1);
  bsplit(L, p.P, p.cs.data());
  p.fc.resize(p.P + 1);
  for (int k = 0; k < p.P; ++k) {
    const int w = p.cs[k + 1] - p.cs[k], Q = 2 * (w / 4);
    std::vector<int32_t> loc(Q + 1);
    bsplit(w, Q, loc.data());
    p.fc[k] = (int)p.fs.size();
    for (int q = 0; q < Q; ++q) p.fs.push_back(p.cs[k] + loc[q]);
  }
  p.GQ = (int)p.fs.size();
  p.fc[p.P] = p.GQ;
  p.fs.push_back(L);
  return p;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// First-fit allocator of 256-byte-aligned regions of the device arena, with
// coalescing of freed neighbours.
class Arena {
 public:
  void init(size_t cap) {
    free_.clear();
    free_[0] = cap;
    cap_ = cap;
    used_ = 0;
  }
  bool alloc(size_t n, size_t* off) {
    n = align_up(n, 256);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < n) continue;
      *off = it->first;
      const size_t rem = it->second - n, start = it->first + n;
      free_.erase(it);
      if (rem) free_[start] = rem;
      used_ += n;
      return true;
    }
    return false;
  }
  void release(size_t off, size_t n) {
    n = align_up(n, 256);
    used_ -= n;
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }
  size_t capacity() const { return cap_; }

 private:
  std::map<size_t, size_t> free_;
  size_t cap_ = 0, used_ = 0;
};

// A replica's footprint in the arena: lattice | tables | transitions | epochs.
struct SlotPlan {
  BPartition part;
  size_t lat = 0, tab = 0, trans = 0, done = 0, bytes = 0;
  uint64_t TE = 0;
};

int plan_slot(const escg_replica_spec& sp, SlotPlan* pl, int idx) {
  if (sp.L < 8 || sp.L > 16384 || sp.S < 2 || sp.S > 15 || !sp.digraph) {
    set_last_error("replica %d: bad L=%d / S=%d / digraph", idx, sp.L, sp.S);
    return ESCG_EINVAL;
  }
  for (int a = 0; a < sp.S * sp.S; ++a)
    if (sp.digraph[a] > 1 || (a / sp.S == a % sp.S && sp.digraph[a])) {
      set_last_error("replica %d: digraph must be 0/1 with a zero diagonal", idx);
      return ESCG_EINVAL;
    }
  if (sp.dominance_prob)
    for (int a = 0; a < sp.S * sp.S; ++a)
      if (!(sp.dominance_prob[a] >= 0.0 && sp.dominance_prob[a] <= 1.0)) {
        set_last_error("replica %d: dominance_prob must be in [0,1]", idx);
        return ESCG_EINVAL;
      }
  const double I = sp.rates.interact, Pr = sp.rates.reproduce, X = sp.rates.exchange;
  if (!(I >= 0 && Pr >= 0 && X >= 0) || !((X + I) + Pr > 0) || std::isinf((X + I) + Pr) ||
      !(sp.p_empty >= 0.0 && sp.p_empty <= 1.0) || sp.max_mcs > 0xFFFFFFFFull) {
    set_last_error("replica %d: bad rates / p_empty / max_mcs", idx);
    return ESCG_EINVAL;
  }
  pl->part = bpartition(sp.L);
  for (int k = 0; k < pl->part.P; ++k)
    if (pl->part.cs[k + 1] - pl->part.cs[k] > kMaxBlock) {
      set_last_error("replica %d: partition exceeds block limits", idx);
      return ESCG_EINVAL;
    }
  const BPartition& p = pl->part;
  size_t off = 0;
  pl->lat = off;
  off = align_up(off + (size_t)sp.L * escg_lattice_pitch(sp.L), 256);
  pl->tab = off;
  off = align_up(off + 4 * (p.cs.size() + p.fs.size() + p.fc.size()), 256);
  pl->trans = off;
  off = align_up(off + sizeof(uint32_t) * kTransWords, 256);
  pl->done = off;
  off = align_up(off + 4 * (size_t)p.P * p.P, 256);
  pl->bytes = off;
  pl->TE = (uint64_t)std::floor(std::ldexp(sp.p_empty, 32) + 0.5);
  return ESCG_OK;
}

// Shared machinery of batches and servers: a pool of replica slots over one
// device arena, and the chunked persistent execution.
struct Engine {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  uint32_t log_every = 10;
  int threads = 0;          // CTA size in use (0: autotune on the first chunks)
  bool use_graph = true;
  int max_slots = 0;
  uint8_t* arena_mem = nullptr;
  Arena arena;
  SlotDesc* d_slots = nullptr;
  SlotState* d_states = nullptr;
  BatchCtl* d_ctl = nullptr;
  uint32_t* d_active = nullptr;
  uint32_t* d_active_tmp = nullptr;
  uint32_t* d_table = nullptr;
  uint32_t* d_admit = nullptr;
  CUtensorMap* d_maps = nullptr;  // one TMA tensor map per slot
  bool tma = true;                // warp-specialised TMA chunk kernel
  int grid_tma[3] = {0, 0, 0};
  uint32_t* h_pinned = nullptr;   // pinned host words (admit list staging, counters)
  size_t table_cap = 0;
  std::vector<SlotDesc> h_slots;
  std::vector<size_t> slot_off, slot_bytes;
  std::vector<uint32_t> pending_admit;
  int grid[3] = {0, 0, 0};
  bool resident = false;          // whole-lattice residency for replicas that fit
  int res_bytes3 = 0;             // dynamic shared memory of class 3
  int grid_res[4] = {0, 0, 0, 0};
  uint64_t launches = 0;
  cudaGraphExec_t graph = nullptr;
  uint32_t spin_limit = 2000000;
  static constexpr int kGraphChunks = 16;
};

int tsel(int threads) { return threads == 64 ? 0 : (threads == 128 ? 1 : 2); }

cudaError_t launch_batch_kernel(Engine* e, int threads) {
  BatchArgs a{e->d_slots, e->d_states, e->d_ctl, e->d_table, e->log_every, e->spin_limit};
  if (e->tma) {
    BatchTmaArgs ta{a, e->d_maps};
    const int g = e->grid_tma[tsel(threads)];
    if (threads == 64)
      batch_tma_kernel<64><<<g, 64 + 32, 0, e->stream>>>(ta);
    else if (threads == 128)
      batch_tma_kernel<128><<<g, 128 + 32, 0, e->stream>>>(ta);
    else
      batch_tma_kernel<256><<<g, 256 + 32, 0, e->stream>>>(ta);
    return cudaGetLastError();
  }
  const int g = e->grid[tsel(threads)];
  if (threads == 64)
    batch_kernel<64><<<g, 64, 0, e->stream>>>(a);
  else if (threads == 128)
    batch_kernel<128><<<g, 128, 0, e->stream>>>(a);
  else
    batch_kernel<256><<<g, 256, 0, e->stream>>>(a);
  return cudaGetLastError();
}

// The resident kernels of the three classes (CTAs of a class with no
// replica leave at once).
cudaError_t launch_resident_kernels(Engine* e) {
  if (!e->resident) return cudaSuccess;
  BatchArgs a{e->d_slots, e->d_states, e->d_ctl, e->d_table, e->log_every, e->spin_limit};
  batch_resident_kernel<128, 1><<<e->grid_res[1], 128, kResBytes1, e->stream>>>(a, e->d_active);
  batch_resident_kernel<256, 2><<<e->grid_res[2], 256, kResBytes2, e->stream>>>(a, e->d_active);
  batch_resident_kernel<1024, 3><<<e->grid_res[3], 1024, e->res_bytes3, e->stream>>>(a, e->d_active);
  return cudaGetLastError();
}

cudaError_t launch_compact(Engine* e) {
  batch_compact_kernel<<<1, kCompactThreads, 0, e->stream>>>(e->d_slots, e->d_states, e->d_ctl, e->d_active,
                                                             e->d_active_tmp, e->d_table, e->d_admit,
                                                             e->log_every);
  return cudaGetLastError();
}

void engine_free(Engine* e) {
  if (e->stream) cudaStreamSynchronize(e->stream);
  if (e->graph) cudaGraphExecDestroy(e->graph);
  cudaFree(e->arena_mem);
  cudaFree(e->d_slots);
  cudaFree(e->d_states);
  cudaFree(e->d_ctl);
  cudaFree(e->d_active);
  cudaFree(e->d_active_tmp);
  cudaFree(e->d_table);
  cudaFree(e->d_admit);
  cudaFree(e->d_maps);
  if (e->h_pinned) cudaFreeHost(e->h_pinned);
  if (e->own_stream && e->stream) cudaStreamDestroy(e->stream);
  e->arena_mem = nullptr;
  e->stream = nullptr;
}

int engine_init(Engine* e, int max_slots, size_t arena_bytes, size_t table_cap, uint32_t log_every,
                int threads, bool use_graph, void* stream) {
  if (threads != 0 && threads != 64 && threads != 128 && threads != 256) {
    set_last_error("threads must be 0, 64, 128 or 256");
    return ESCG_EINVAL;
  }
  e->max_slots = max_slots;
  e->log_every = log_every ? log_every : 10;
  e->threads = threads;
  e->use_graph = use_graph;
  e->table_cap = table_cap;
  cudaError_t err = cudaGetDevice(&e->device);
  if (err == cudaSuccess) {
    if (stream) {
      e->stream = (cudaStream_t)stream;
    } else {
      err = cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking);
      e->own_stream = true;
    }
  }
  if (err == cudaSuccess) err = cudaMalloc(&e->arena_mem, arena_bytes);
  if (err == cudaSuccess) err = cudaMalloc(&e->d_slots, sizeof(SlotDesc) * max_slots);
  if (err == cudaSuccess) err = cudaMalloc(&e->d_states, sizeof(SlotState) * max_slots);
  if (err == cudaSuccess) err = cudaMalloc(&e->d_ctl, sizeof(BatchCtl));
  if (err == cudaSuccess) err = cudaMalloc(&e->d_active, sizeof(uint32_t) * max_slots);
  if (err == cudaSuccess) err = cudaMalloc(&e->d_active_tmp, sizeof(uint32_t) * max_slots);
  if (err == cudaSuccess) err = cudaMalloc(&e->d_table, sizeof(uint32_t) * table_cap);
  if (err == cudaSuccess) err = cudaMalloc(&e->d_admit, sizeof(uint32_t) * (max_slots + 1));
  if (err == cudaSuccess) err = cudaMalloc(&e->d_maps, sizeof(CUtensorMap) * max_slots);
  if (err == cudaSuccess) err = cudaMallocHost(&e->h_pinned, sizeof(uint32_t) * (max_slots + 16));
  if (err == cudaSuccess) err = cudaMemsetAsync(e->d_ctl, 0, sizeof(BatchCtl), e->stream);
  if (err == cudaSuccess) err = cudaMemsetAsync(e->d_states, 0, sizeof(SlotState) * max_slots, e->stream);
  if (err != cudaSuccess) {
    set_last_error("engine allocation failed: %s", cudaGetErrorString(err));
    return ESCG_ENOMEM;
  }
  e->arena.init(arena_bytes);
  e->h_slots.assign(max_slots, SlotDesc{});
  e->slot_off.assign(max_slots, 0);
  e->slot_bytes.assign(max_slots, 0);
  int sms = 0, per = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, e->device);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_kernel<64>, 64, 0);
  e->grid[0] = sms * (per < 1 ? 1 : per);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_kernel<128>, 128, 0);
  e->grid[1] = sms * (per < 1 ? 1 : per);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_kernel<256>, 256, 0);
  e->grid[2] = sms * (per < 1 ? 1 : per);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_tma_kernel<64>, 64 + 32, 0);
  e->grid_tma[0] = sms * (per < 1 ? 1 : per);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_tma_kernel<128>, 128 + 32, 0);
  e->grid_tma[1] = sms * (per < 1 ? 1 : per);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_tma_kernel<256>, 256 + 32, 0);
  e->grid_tma[2] = sms * (per < 1 ? 1 : per);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, e->device);
  e->res_bytes3 = optin - (int)(sizeof(ResidentSmem) + sizeof(SlotDesc)) - 256;
  cudaFuncSetAttribute(batch_resident_kernel<128, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kResBytes1);
  cudaFuncSetAttribute(batch_resident_kernel<256, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kResBytes2);
  if (cudaFuncSetAttribute(batch_resident_kernel<1024, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           e->res_bytes3) != cudaSuccess)
    e->res_bytes3 = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_resident_kernel<128, 1>, 128, kResBytes1);
  e->grid_res[1] = sms * (per < 1 ? 1 : per);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_resident_kernel<256, 2>, 256, kResBytes2);
  e->grid_res[2] = sms * (per < 1 ? 1 : per);
  per = 0;
  if (e->res_bytes3 > 0)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_resident_kernel<1024, 3>, 1024, e->res_bytes3);
  e->grid_res[3] = sms * (per < 1 ? 1 : per);
  cudaGetLastError();
  return ESCG_OK;
}

// Places a replica into `slot`: arena memory, tables, initial lattice and
// counts; it joins the active set at the next chunk.  ESCG_ENOMEM if the
// arena has no room (nothing is changed then).
int engine_add(Engine* e, const escg_replica_spec& sp, const SlotPlan& pl, int slot) {
  size_t off = 0;
  if (!e->arena.alloc(pl.bytes, &off)) {
    set_last_error("device arena full");
    return ESCG_ENOMEM;
  }
  uint8_t* base = e->arena_mem + off;
  const BPartition& p = pl.part;
  std::vector<uint8_t> img(pl.bytes - pl.tab, 0);   // tables | transitions | epochs
  int32_t* tab = reinterpret_cast<int32_t*>(img.data());
  size_t w = 0;
  for (int32_t v : p.cs) tab[w++] = v;
  for (int32_t v : p.fs) tab[w++] = v;
  for (int32_t v : p.fc) tab[w++] = v;
  const double I = sp.rates.interact, Pr = sp.rates.reproduce, X = sp.rates.exchange;
  const double R = (X + I) + Pr;
  const uint64_t tx = (uint64_t)std::floor(std::ldexp(X / R, 32) + 0.5);
  const uint64_t txi = (uint64_t)std::floor(std::ldexp((X + I) / R, 32) + 0.5);
  build_transitions(sp.S, sp.digraph, sp.dominance_prob, tx, txi,
                    reinterpret_cast<uint32_t*>(img.data() + (pl.trans - pl.tab)));
  SlotDesc sd;
  std::memset(&sd, 0, sizeof sd);
  LatticeDesc& d = sd.d;
  d.lat = base + pl.lat;
  d.L = sp.L;
  d.pitch = escg_lattice_pitch(sp.L);
  d.P = p.P;
  d.GQ = p.GQ;
  d.cs = reinterpret_cast<int32_t*>(base + pl.tab);
  d.fs = d.cs + p.cs.size();
  d.fc = d.fs + p.fs.size();
  d.H = sp.L;   // replicas are square
  d.Py = p.P;
  d.csy = d.cs;
  d.fsy = d.fs;
  d.fcy = d.fc;
  d.ax = make_axis_geom(sp.L, p.P);
  d.ay = d.ax;
  d.bits = 8;
  d.trans = base + pl.trans;
  d.key0 = (uint32_t)sp.seed;
  d.key1 = (uint32_t)(sp.seed >> 32);
  for (int r = 0; r < 10; ++r) {
    d.rk[2 * r] = d.key0 + (uint32_t)r * 0x9E3779B9u;
    d.rk[2 * r + 1] = d.key1 + (uint32_t)r * 0xBB67AE85u;
  }
  d.tx = tx >> 32 ? 0xFFFFFFFFu : (uint32_t)tx;
  d.txi = txi >> 32 ? 0xFFFFFFFFu : (uint32_t)txi;
  d.S = sp.S;
  d.uniform64 = 0;
  fill_perm24(d.perm24);
  sd.done = reinterpret_cast<uint32_t*>(base + pl.done);
  sd.max_mcs = (uint32_t)sp.max_mcs;
  sd.stop_at_extinction = sp.stop_at_extinction ? 1 : 0;
  sd.nb4 = p.P * p.P / 4;
  // whole-lattice residency class by the size of the shared-memory image (when
  // enabled)
  if (e->resident && p.P <= 8) {
    const int bytes = resident_dyn_bytes(sp.L, sp.L);
    sd.rclass = bytes <= kResBytes1 ? 1 : (bytes <= kResBytes2 ? 2 : (bytes <= e->res_bytes3 ? 3 : 0));
    if (sd.rclass) sd.nb4 = 0;   // not in the chunk kernel's table
  }
  CUtensorMap map;
  if (!encode_lattice_map(&map, d.lat, d.L, d.pitch, kBSP, kBRows)) {
    e->arena.release(off, pl.bytes);
    set_last_error("cuTensorMapEncodeTiled failed for L=%d", sp.L);
    return ESCG_ECUDA;
  }
  // the slot is idle on the device, so these synchronous copies race nothing
  cudaError_t err = cudaMemcpy(base + pl.tab, img.data(), img.size(), cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemcpy(e->d_maps + slot, &map, sizeof map, cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemcpy(e->d_slots + slot, &sd, sizeof sd, cudaMemcpyHostToDevice);
  if (err == cudaSuccess) err = cudaMemsetAsync(e->d_states + slot, 0, sizeof(SlotState), e->stream);
  if (err == cudaSuccess) err = launch_init(d, pl.TE, e->stream);
  if (err == cudaSuccess) {
    e->h_pinned[0] = (uint32_t)slot;   // consumed by the kernel below before the next use
    err = cudaMemcpyAsync(e->d_admit + e->max_slots, &e->h_pinned[0], sizeof(uint32_t),
                          cudaMemcpyHostToDevice, e->stream);
  }
  if (err == cudaSuccess) {
    batch_count_kernel<<<1, 256, 0, e->stream>>>(e->d_slots, e->d_states, e->d_admit + e->max_slots, 1);
    err = cudaGetLastError();
  }
  if (err == cudaSuccess) err = cudaStreamSynchronize(e->stream);
  if (err != cudaSuccess) {
    e->arena.release(off, pl.bytes);
    set_last_error("replica set-up failed: %s", cudaGetErrorString(err));
    return ESCG_ECUDA;
  }
  e->launches += 2;
  e->h_slots[slot] = sd;
  e->slot_off[slot] = off;
  e->slot_bytes[slot] = pl.bytes;
  e->pending_admit.push_back((uint32_t)slot);
  return ESCG_OK;
}

void engine_release(Engine* e, int slot) {
  if (e->slot_bytes[slot]) e->arena.release(e->slot_off[slot], e->slot_bytes[slot]);
  e->slot_bytes[slot] = 0;
}

int engine_flush_admits(Engine* e) {
  const uint32_t n = (uint32_t)e->pending_admit.size();
  if (!n) return ESCG_OK;
  // the admit list region [0, max_slots-1) and ctl->n_admit are read only by
  // the next compaction, which follows these copies on the stream
  cudaError_t err = cudaStreamSynchronize(e->stream);   // the pinned staging is reused
  for (uint32_t i = 0; i < n && err == cudaSuccess; ++i) e->h_pinned[i] = e->pending_admit[i];
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(e->d_admit, e->h_pinned, sizeof(uint32_t) * n, cudaMemcpyHostToDevice, e->stream);
  if (err == cudaSuccess) {
    e->h_pinned[e->max_slots + 8] = n;
    err = cudaMemcpyAsync(&e->d_ctl->n_admit, &e->h_pinned[e->max_slots + 8], sizeof(uint32_t),
                          cudaMemcpyHostToDevice, e->stream);
  }
  if (err != cudaSuccess) {
    set_last_error("admission upload failed: %s", cudaGetErrorString(err));
    return ESCG_ECUDA;
  }
  e->pending_admit.clear();
  return ESCG_OK;
}

// One chunk: compaction, the resident kernels, then the chunk kernel (whose
// last CTA records how far the launch advanced the replicas).
int engine_chunk(Engine* e, int threads) {
  if (launch_compact(e) != cudaSuccess || launch_resident_kernels(e) != cudaSuccess ||
      launch_batch_kernel(e, threads) != cudaSuccess) {
    set_last_error("chunk launch failed");
    return ESCG_ECUDA;
  }
  e->launches += e->resident ? 5 : 2;
  return ESCG_OK;
}

// Online autotuning of the chunk kernel: its CTA size (64, 128, 256 consumer
// threads) and its staging (the warp-specialised TMA kernel or the plain
// one), one chunk per candidate, timed with events; the physical mapping
// never changes the results, so the tuning chunks are ordinary chunks of the
// run.
int engine_autotune(Engine* e, uint64_t* chunks_left) {
  const int cand[3] = {64, 128, 256};
  float best = 1e30f;
  int best_t = 256;
  bool best_tma = true;
  for (int m = 0; m < 2; ++m)
    for (int c = 0; c < 3 && *chunks_left > 0; ++c) {
      e->tma = (m == 0);
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      cudaEventRecord(e0, e->stream);
      const int rc = engine_chunk(e, cand[c]);
      cudaEventRecord(e1, e->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      if (rc != ESCG_OK) return rc;
      --*chunks_left;
      if (ms < best) {
        best = ms;
        best_t = cand[c];
        best_tma = e->tma;
      }
    }
  e->threads = best_t;
  e->tma = best_tma;
  return ESCG_OK;
}

int engine_build_graph(Engine* e) {
  if (!e->use_graph || e->graph) return ESCG_OK;
  cudaGraph_t g;
  if (cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    set_last_error("CUDA graph capture failed to start");
    return ESCG_ECUDA;
  }
  for (int c = 0; c < Engine::kGraphChunks; ++c) {
    launch_compact(e);
    launch_resident_kernels(e);
    launch_batch_kernel(e, e->threads);
  }
  if (cudaStreamEndCapture(e->stream, &g) != cudaSuccess || cudaGraphInstantiate(&e->graph, g, 0) != cudaSuccess) {
    set_last_error("CUDA graph capture failed");
    return ESCG_ECUDA;
  }
  cudaGraphDestroy(g);
  return ESCG_OK;
}

int engine_active(Engine* e, uint32_t* out) {
  if (cudaMemcpyAsync(&e->h_pinned[e->max_slots + 9], &e->d_ctl->n_active, sizeof(uint32_t),
                      cudaMemcpyDeviceToHost, e->stream) != cudaSuccess ||
      cudaStreamSynchronize(e->stream) != cudaSuccess) {
    set_last_error("reading the active count failed");
    return ESCG_ECUDA;
  }
  *out = e->h_pinned[e->max_slots + 9];
  return ESCG_OK;
}

// Runs up to `chunks` chunks (0: until no replica is active), stopping early
// when the active set empties; ends with a compaction so that every
// replica's MCS number and retirement are settled.
int engine_run(Engine* e, uint64_t chunks, bool until_idle) {
  int rc = engine_flush_admits(e);
  if (rc != ESCG_OK) return rc;
  uint64_t left = chunks;
  if (e->threads == 0) {
    rc = engine_autotune(e, &left);
    if (rc != ESCG_OK) return rc;
  }
  rc = engine_build_graph(e);
  if (rc != ESCG_OK) return rc;
  const uint64_t G = Engine::kGraphChunks;
  while (until_idle || left > 0) {
    bool group = false;
    if (e->graph && (until_idle || left >= G)) {
      if (cudaGraphLaunch(e->graph, e->stream) != cudaSuccess) {
        set_last_error("graph launch failed");
        return ESCG_ECUDA;
      }
      e->launches += (e->resident ? 5 : 2) * G;
      left = left >= G ? left - G : 0;
      group = true;
    } else {
      rc = engine_chunk(e, e->threads);
      if (rc != ESCG_OK) return rc;
      left = left ? left - 1 : 0;
    }
    if (group || left == 0) {   // the host checks after a graph group or the last chunk
      uint32_t n_active = 0;
      rc = engine_active(e, &n_active);
      if (rc != ESCG_OK) return rc;
      if (n_active == 0) break;
    }
  }
  if (launch_compact(e) != cudaSuccess) {
    set_last_error("batch compaction launch failed");
    return ESCG_ECUDA;
  }
  e->launches++;
  return ESCG_OK;
}

int engine_check(Engine* e) {
  if (cudaStreamSynchronize(e->stream) != cudaSuccess) {
    set_last_error("engine stream failed: %s", cudaGetErrorString(cudaGetLastError()));
    return ESCG_ECUDA;
  }
  BatchCtl ctl;
  if (cudaMemcpy(&ctl, e->d_ctl, sizeof ctl, cudaMemcpyDeviceToHost) != cudaSuccess) return ESCG_ECUDA;
  if (ctl.error & kErrTimeout) {
    set_last_error("a bounded device-side wait timed out");
    return ESCG_ETIMEOUT;
  }
  return ESCG_OK;
}

size_t table_capacity(int max_slots, size_t arena_bytes) { return (size_t)max_slots + arena_bytes / 4096 + 64; }

}  // namespace

struct escg_batch {
  Engine e;
  int n = 0;
  uint64_t budget_max = 0;
  std::vector<int> L, S;
};

extern "C" {

void escg_batch_default_options(escg_batch_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof *opt);
  opt->log_every = 10;
  opt->threads = 0;
  opt->use_graph = 1;
  opt->resident = 0;
}

escg_batch_t* escg_batch_create(int32_t n, const escg_replica_spec* specs, const escg_batch_options* opt) {
  if (n < 1 || n > 65535 || !specs) {
    set_last_error("need 1 <= n <= 65535 replicas");
    return nullptr;
  }
  escg_batch_options o;
  escg_batch_default_options(&o);
  if (opt) o = *opt;
  std::vector<SlotPlan> plans(n);
  size_t total = 0;
  for (int i = 0; i < n; ++i) {
    if (plan_slot(specs[i], &plans[i], i) != ESCG_OK) return nullptr;
    total += plans[i].bytes;
  }
  escg_batch* b = new (std::nothrow) escg_batch;
  if (!b) return nullptr;
  b->n = n;
  if (engine_init(&b->e, n, total, table_capacity(n, total), o.log_every, o.threads, o.use_graph != 0,
                  o.cuda_stream) != ESCG_OK) {
    engine_free(&b->e);
    delete b;
    return nullptr;
  }
  b->e.resident = o.resident != 0;
  for (int i = 0; i < n; ++i) {
    if (engine_add(&b->e, specs[i], plans[i], i) != ESCG_OK) {
      engine_free(&b->e);
      delete b;
      return nullptr;
    }
    b->L.push_back(specs[i].L);
    b->S.push_back(specs[i].S);
    if (specs[i].max_mcs > b->budget_max) b->budget_max = specs[i].max_mcs;
  }
  return b;
}

int escg_batch_run(escg_batch_t* b, uint64_t max_mcs) {
  if (!b) return ESCG_EINVAL;
  const uint32_t le = b->e.log_every;
  if (max_mcs == 0) return engine_run(&b->e, (b->budget_max + le - 1) / le + 1, false);
  return engine_run(&b->e, (max_mcs + le - 1) / le, false);
}

int escg_batch_sync(escg_batch_t* b) { return b ? engine_check(&b->e) : ESCG_EINVAL; }

int escg_batch_status(escg_batch_t* b, uint64_t* mcs_out, int32_t* extinct_out, uint64_t* counts16_out) {
  if (!b) return ESCG_EINVAL;
  int rc = engine_check(&b->e);
  if (rc != ESCG_OK) return rc;
  std::vector<SlotState> st(b->n);
  if (cudaMemcpy(st.data(), b->e.d_states, sizeof(SlotState) * b->n, cudaMemcpyDeviceToHost) != cudaSuccess)
    return ESCG_ECUDA;
  for (int i = 0; i < b->n; ++i) {
    if (mcs_out) mcs_out[i] = st[i].mcs;
    if (extinct_out) extinct_out[i] = (int32_t)st[i].stopped;
    if (counts16_out)
      for (int v = 0; v < kMaxStates; ++v) counts16_out[i * kMaxStates + v] = st[i].counts[v];
  }
  return ESCG_OK;
}

int32_t escg_batch_active(escg_batch_t* b) {
  if (!b) return -1;
  uint32_t n = 0;
  if (engine_active(&b->e, &n) != ESCG_OK) return -1;
  return (int32_t)n;
}

int escg_batch_snapshot(escg_batch_t* b, int32_t i, uint8_t* host_out) {
  if (!b || i < 0 || i >= b->n || !host_out) return ESCG_EINVAL;
  int rc = engine_check(&b->e);
  if (rc != ESCG_OK) return rc;
  const LatticeDesc& d = b->e.h_slots[i].d;
  if (cudaMemcpy2D(host_out, d.L, d.lat, d.pitch, d.L, d.L, cudaMemcpyDeviceToHost) != cudaSuccess)
    return ESCG_ECUDA;
  return ESCG_OK;
}

int32_t escg_batch_threads(escg_batch_t* b) { return b ? b->e.threads : 0; }
int32_t escg_batch_uses_tma(escg_batch_t* b) { return b ? (int32_t)b->e.tma : 0; }
uint64_t escg_batch_launch_count(escg_batch_t* b) { return b ? b->e.launches : 0; }

void escg_batch_destroy(escg_batch_t* b) {
  if (!b) return;
  engine_free(&b->e);
  delete b;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Serving: a FIFO request queue over the slot engine.
namespace {

struct Request {
  int64_t id = 0;
  double submitted_s = 0.0;       // host clock, seconds since the server was created
  escg_replica_spec spec{};
  std::vector<uint8_t> digraph;   // owned copies
  std::vector<double> prob;
  SlotPlan plan;
};

struct Result {
  uint64_t mcs = 0;
  int32_t extinct = 0;
  double submitted_s = 0.0, admitted_s = 0.0, finished_s = 0.0;   // host clock (see escg_server_timing)
  uint64_t counts[kMaxStates] = {};
  std::vector<uint8_t> lattice;
};

}  // namespace

struct escg_server {
  Engine e;
  escg_server_options opt{};
  std::deque<Request> queue;
  std::vector<int64_t> slot_req;     // request id resident in each slot, -1 free
  std::vector<int> free_slots;
  std::vector<int> slot_L;
  std::unordered_map<int64_t, Result> results;
  std::vector<int64_t> finished;     // not yet polled
  int64_t next_id = 0;
  int resident = 0;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  std::vector<double> slot_submitted, slot_admitted;   // of the run resident in each slot
  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

extern "C" {

void escg_server_default_options(escg_server_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof *opt);
  opt->arena_bytes = 256ull << 20;
  opt->max_slots = 1024;
  opt->log_every = 10;
  opt->threads = 0;
  opt->chunks_per_step = 4;
  opt->keep_lattice = 0;
}

escg_server_t* escg_server_create(const escg_server_options* opt) {
  escg_server* s = new (std::nothrow) escg_server;
  if (!s) return nullptr;
  escg_server_default_options(&s->opt);
  if (opt) s->opt = *opt;
  if (s->opt.max_slots < 1 || s->opt.max_slots > 65535 || s->opt.arena_bytes < 4096) {
    set_last_error("server needs 1 <= max_slots <= 65535 and a non-trivial arena");
    delete s;
    return nullptr;
  }
  if (s->opt.chunks_per_step == 0) s->opt.chunks_per_step = 4;
  if (engine_init(&s->e, s->opt.max_slots, s->opt.arena_bytes,
                  table_capacity(s->opt.max_slots, s->opt.arena_bytes), s->opt.log_every, s->opt.threads,
                  true, s->opt.cuda_stream) != ESCG_OK) {
    engine_free(&s->e);
    delete s;
    return nullptr;
  }
  s->slot_req.assign(s->opt.max_slots, -1);
  s->slot_L.assign(s->opt.max_slots, 0);
  s->slot_submitted.assign(s->opt.max_slots, 0.0);
  s->slot_admitted.assign(s->opt.max_slots, 0.0);
  for (int i = s->opt.max_slots - 1; i >= 0; --i) s->free_slots.push_back(i);
  return s;
}

int64_t escg_server_submit(escg_server_t* s, const escg_replica_spec* spec) {
  if (!s || !spec) {
    set_last_error("NULL argument");
    return ESCG_EINVAL;
  }
  Request r;
  r.id = s->next_id;
  if (plan_slot(*spec, &r.plan, (int)r.id) != ESCG_OK) return ESCG_EINVAL;
  if (r.plan.bytes > s->e.arena.capacity()) {
    set_last_error("run needs %zu bytes, more than the whole arena", r.plan.bytes);
    return ESCG_ENOMEM;
  }
  r.spec = *spec;
  r.submitted_s = s->now();
  r.digraph.assign(spec->digraph, spec->digraph + spec->S * spec->S);
  if (spec->dominance_prob) r.prob.assign(spec->dominance_prob, spec->dominance_prob + spec->S * spec->S);
  s->queue.push_back(std::move(r));
  Request& q = s->queue.back();
  q.spec.digraph = q.digraph.data();
  q.spec.dominance_prob = q.prob.empty() ? nullptr : q.prob.data();
  return s->next_id++;
}

int escg_server_step(escg_server_t* s, int32_t* finished_out) {
  if (!s) return ESCG_EINVAL;
  // 1. admissions, FIFO, while a slot and arena room are free
  while (!s->queue.empty() && !s->free_slots.empty()) {
    Request& r = s->queue.front();
    const int slot = s->free_slots.back();
    const int rc = engine_add(&s->e, r.spec, r.plan, slot);
    if (rc == ESCG_ENOMEM) break;   // wait for retirements
    if (rc != ESCG_OK) return rc;
    s->free_slots.pop_back();
    s->slot_req[slot] = r.id;
    s->slot_L[slot] = r.spec.L;
    s->slot_submitted[slot] = r.submitted_s;
    s->slot_admitted[slot] = s->now();
    s->resident++;
    s->queue.pop_front();
  }
  int32_t nfin = 0;
  if (s->resident > 0) {
    // 2. advance every resident run
    int rc = engine_run(&s->e, s->opt.chunks_per_step, false);
    if (rc == ESCG_OK) rc = engine_check(&s->e);
    if (rc != ESCG_OK) return rc;
    // 3. retire finished runs
    std::vector<SlotState> st(s->opt.max_slots);
    if (cudaMemcpy(st.data(), s->e.d_states, sizeof(SlotState) * s->opt.max_slots, cudaMemcpyDeviceToHost) !=
        cudaSuccess) {
      set_last_error("reading run states failed");
      return ESCG_ECUDA;
    }
    for (int slot = 0; slot < s->opt.max_slots; ++slot) {
      if (s->slot_req[slot] < 0) continue;
      const SlotState& x = st[slot];
      if (!(x.stopped || x.mcs >= s->e.h_slots[slot].max_mcs)) continue;
      Result res;
      res.mcs = x.mcs;
      res.extinct = (int32_t)x.stopped;
      for (int v = 0; v < kMaxStates; ++v) res.counts[v] = x.counts[v];
      res.submitted_s = s->slot_submitted[slot];
      res.admitted_s = s->slot_admitted[slot];
      res.finished_s = s->now();
      if (s->opt.keep_lattice) {
        const LatticeDesc& d = s->e.h_slots[slot].d;
        res.lattice.resize((size_t)d.L * d.L);
        if (cudaMemcpy2D(res.lattice.data(), d.L, d.lat, d.pitch, d.L, d.L, cudaMemcpyDeviceToHost) !=
            cudaSuccess) {
          set_last_error("copying a finished lattice failed");
          return ESCG_ECUDA;
        }
      }
      const int64_t id = s->slot_req[slot];
      s->results[id] = std::move(res);
      s->finished.push_back(id);
      engine_release(&s->e, slot);
      s->slot_req[slot] = -1;
      s->free_slots.push_back(slot);
      s->resident--;
      nfin++;
    }
  }
  if (finished_out) *finished_out = nfin;
  return ESCG_OK;
}

int escg_server_cancel(escg_server_t* s, int64_t id) {
  if (!s) return ESCG_EINVAL;
  // still queued: drop it; its result is the run not started (MCS 0)
  for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
    if (it->id != id) continue;
    Result res;
    res.submitted_s = it->submitted_s;
    res.admitted_s = res.finished_s = s->now();
    s->queue.erase(it);
    s->results[id] = std::move(res);
    s->finished.push_back(id);
    return ESCG_OK;
  }
  int slot = -1;
  for (int i = 0; i < s->opt.max_slots; ++i)
    if (s->slot_req[i] == id) slot = i;
  if (slot < 0) {
    set_last_error("run %lld is neither queued nor running", (long long)id);
    return ESCG_ESTATE;
  }
  // resident: between steps the device is idle and every replica's MCS is
  // settled.  The run's budget becomes its current MCS and one compaction
  // takes it out of the active list before its slot can be reused.
  SlotState x;
  cudaError_t err = cudaStreamSynchronize(s->e.stream);
  if (err == cudaSuccess) err = cudaMemcpy(&x, s->e.d_states + slot, sizeof x, cudaMemcpyDeviceToHost);
  if (err == cudaSuccess)
    err = cudaMemcpy(&s->e.d_slots[slot].max_mcs, &x.mcs, sizeof(uint32_t), cudaMemcpyHostToDevice);
  s->e.h_slots[slot].max_mcs = x.mcs;
  if (err == cudaSuccess) err = launch_compact(&s->e);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s->e.stream);
  if (err != cudaSuccess) {
    set_last_error("cancelling run %lld failed: %s", (long long)id, cudaGetErrorString(err));
    return ESCG_ECUDA;
  }
  s->e.launches++;
  Result res;
  res.mcs = x.mcs;
  res.extinct = (int32_t)x.stopped;
  for (int v = 0; v < kMaxStates; ++v) res.counts[v] = x.counts[v];
  res.submitted_s = s->slot_submitted[slot];
  res.admitted_s = s->slot_admitted[slot];
  res.finished_s = s->now();
  if (s->opt.keep_lattice) {
    const LatticeDesc& d = s->e.h_slots[slot].d;
    res.lattice.resize((size_t)d.L * d.L);
    if (cudaMemcpy2D(res.lattice.data(), d.L, d.lat, d.pitch, d.L, d.L, cudaMemcpyDeviceToHost) != cudaSuccess) {
      set_last_error("copying a cancelled lattice failed");
      return ESCG_ECUDA;
    }
  }
  s->results[id] = std::move(res);
  s->finished.push_back(id);
  engine_release(&s->e, slot);
  s->slot_req[slot] = -1;
  s->free_slots.push_back(slot);
  s->resident--;
  return ESCG_OK;
}

int escg_server_poll(escg_server_t* s, int64_t* ids_out, int32_t cap, int32_t* n_out) {
  if (!s || (cap > 0 && !ids_out) || cap < 0) return ESCG_EINVAL;
  const int32_t n = (int32_t)std::min<size_t>((size_t)cap, s->finished.size());
  for (int32_t i = 0; i < n; ++i) ids_out[i] = s->finished[i];
  s->finished.erase(s->finished.begin(), s->finished.begin() + n);
  if (n_out) *n_out = n;
  return ESCG_OK;
}

int escg_server_result(escg_server_t* s, int64_t id, uint64_t* mcs_out, int32_t* extinct_out,
                       uint64_t* counts16_out, uint8_t* lattice_out) {
  if (!s) return ESCG_EINVAL;
  auto it = s->results.find(id);
  if (it == s->results.end()) {
    set_last_error("run %lld has not finished", (long long)id);
    return ESCG_ESTATE;
  }
  const Result& r = it->second;
  if (mcs_out) *mcs_out = r.mcs;
  if (extinct_out) *extinct_out = r.extinct;
  if (counts16_out)
    for (int v = 0; v < kMaxStates; ++v) counts16_out[v] = r.counts[v];
  if (lattice_out) {
    if (r.lattice.empty()) {
      set_last_error("lattices are kept only with keep_lattice");
      return ESCG_ESTATE;
    }
    std::memcpy(lattice_out, r.lattice.data(), r.lattice.size());
  }
  return ESCG_OK;
}

int escg_server_timing(escg_server_t* s, int64_t id, double* submitted_s, double* admitted_s, double* finished_s) {
  if (!s) return ESCG_EINVAL;
  auto it = s->results.find(id);
  if (it == s->results.end()) {
    set_last_error("run %lld has not finished", (long long)id);
    return ESCG_ESTATE;
  }
  if (submitted_s) *submitted_s = it->second.submitted_s;
  if (admitted_s) *admitted_s = it->second.admitted_s;
  if (finished_s) *finished_s = it->second.finished_s;
  return ESCG_OK;
}

int escg_server_stats(escg_server_t* s, int32_t* resident, int32_t* queued, uint64_t* bytes_in_use) {
  if (!s) return ESCG_EINVAL;
  if (resident) *resident = s->resident;
  if (queued) *queued = (int32_t)s->queue.size();
  if (bytes_in_use) *bytes_in_use = s->e.arena.used();
  return ESCG_OK;
}

int32_t escg_server_threads(escg_server_t* s) { return s ? s->e.threads : 0; }
int32_t escg_server_uses_tma(escg_server_t* s) { return s ? (int32_t)s->e.tma : 0; }
uint64_t escg_server_launch_count(escg_server_t* s) { return s ? s->e.launches : 0; }

void escg_server_destroy(escg_server_t* s) {
  if (!s) return;
  engine_free(&s->e);
  delete s;
}

}  // extern "C"
