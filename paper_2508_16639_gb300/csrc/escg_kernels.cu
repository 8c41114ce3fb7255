// escg_kernels.cu -- CUDA kernels of the ESCG Monte Carlo step (sm_103a)
// and their host-side launchers.
//
//   init_kernel        site-parallel Philox initialisation (schedule v1)
//   count_kernel       species histogram (warp-reduced, one atomic per warp
//                      per state), the densities() of Alg. 4
//   finalize_kernel    appends a logged count vector, stasis() check
//   phase_kernel       one coarse colour phase: one CTA per active block
//   persistent_kernel  many MCS in one launch: CTAs take (MCS, phase, block)
//                      work items in schedule order from a ticket counter and
//                      start a block once its 8 neighbours have reached the
//                      required epoch (bounded spin; gives up with an error
//                      status instead of hanging); species counts of log
//                      points are fused into the visits
//   persistent_ll_kernel   the same work items with boundary records (a
//                      visit's edge and rim lines, epoch-tagged) in place of
//                      epoch flags and rim loads
//   persistent_own_kernel  each CTA owns one 2x2 group of blocks for the
//                      whole launch, their tiles resident in shared memory;
//                      visits exchange only boundary records
#include <cstdio>

#include "escg_device.cuh"
#include "escg_resident.cuh"
#include "escg_rule8.cuh"
#include "escg_internal.h"
#include "escg_tma.cuh"
#include "escg_sync.cuh"



namespace escg_impl {

// ---------------------------------------------------------------------------
// One thread per group of 4 sites (a 32-bit word, 16-bit word or byte of
// the row, by bits per site); sites past column L (row padding) are 0.
__global__ void init_kernel(LatticeDesc d, uint64_t T_empty) {
  const int L = d.L, bits = d.bits;
  const int groups = d.pitch * 2 / bits;   // groups of 4 sites per row of pitch bytes
  const size_t total = (size_t)d.H * groups;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total;
       k += (size_t)gridDim.x * blockDim.x) {
    const int row = (int)(k / groups), c0 = 4 * (int)(k % groups);
    uint32_t u = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int col = c0 + e;
      if (col < L) {
        const uint32_t i = (uint32_t)row * (uint32_t)L + (uint32_t)col;
        const uint4 x = philox10(make_uint4(i, 0u, 0u, kTagInit), d.key0, d.key1);
        const uint32_t v = ((uint64_t)x.x < T_empty) ? 0u : 1u + __umulhi(x.y, (uint32_t)d.S);
        u |= v << (8 * e);
      }
    }
    store_group(d.lat + (size_t)row * d.pitch, c0, bits, pack4(u, bits));
  }
}

// Packed lattice <-> one byte per site (host transfers of a packed lattice
// go through a byte image with pitch round_up(L, 16)).  One thread per group.
__global__ void pack_kernel(LatticeDesc d, const uint8_t* bytes, int byte_pitch) {
  const int groups = (d.L + 3) / 4;
  const size_t total = (size_t)d.H * groups;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total;
       k += (size_t)gridDim.x * blockDim.x) {
    const int row = (int)(k / groups), c0 = 4 * (int)(k % groups);
    const uint8_t* src = bytes + (size_t)row * byte_pitch + c0;
    uint32_t u = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (c0 + e < d.L) u |= (uint32_t)(src[e] & ((1u << d.bits) - 1u)) << (8 * e);
    store_group(d.lat + (size_t)row * d.pitch, c0, d.bits, pack4(u, d.bits));
  }
}

__global__ void unpack_kernel(LatticeDesc d, uint8_t* bytes, int byte_pitch) {
  const int groups = (d.L + 3) / 4;
  const size_t total = (size_t)d.H * groups;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total;
       k += (size_t)gridDim.x * blockDim.x) {
    const int row = (int)(k / groups), c0 = 4 * (int)(k % groups);
    const uint32_t u = unpack4(load_group(d.lat + (size_t)row * d.pitch, c0, d.bits), d.bits);
    uint8_t* dst = bytes + (size_t)row * byte_pitch + c0;
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (c0 + e < d.L) dst[e] = (uint8_t)(u >> (8 * e));
  }
}

// Flags (*bad = 1) any lattice byte outside 0..S (padding bytes excluded).
// Sets *bad |= flag if any lattice byte is outside 0..S; with stop != null
// also *stop = 1, so that the kernels that follow on the stream leave the
// lattice alone.
__global__ void validate_kernel(LatticeDesc d, uint32_t* bad, uint32_t flag, uint32_t* stop) {
  const int L = d.L, vec_per_row = (L + 15) / 16;
  const uint32_t lim = 0x7Fu - (uint32_t)d.S;  // byte + lim has bit 7 set iff byte > S (byte < 128)
  const size_t total = (size_t)d.H * vec_per_row;
  uint32_t any = 0;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < total;
       k += (size_t)gridDim.x * blockDim.x) {
    const int row = (int)(k / vec_per_row), q = (int)(k % vec_per_row);
    uint4 w = load16(d, (uint32_t)row, (uint32_t)q);
    uint32_t* p = reinterpret_cast<uint32_t*>(&w);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int valid = L - (16 * q + 4 * e);
      uint32_t x = p[e];
      if (valid <= 0)
        x = 0;
      else if (valid < 4)
        x &= 0xFFFFFFFFu >> (8 * (4 - valid));
      any |= (x | ((x & 0x7F7F7F7Fu) + lim * 0x01010101u)) & 0x80808080u;
    }
  }
  if (__any_sync(0xFFFFFFFFu, any != 0) && (threadIdx.x & 31) == 0) {
    atomicOr(bad, flag);
    if (stop) atomicExch(stop, 1u);
  }
}

// Zeroes a RunState and sets its MCS number and first log number.
__global__ void state_reset_kernel(RunState* st, uint32_t mcs, uint32_t log_num0) {
  uint32_t* w = reinterpret_cast<uint32_t*>(st);
  constexpr int n = (int)(sizeof(RunState) / sizeof(uint32_t));
  for (int k = threadIdx.x; k < n; k += blockDim.x) w[k] = 0u;
  __syncthreads();
  if (threadIdx.x == 0) {
    st->mcs = mcs;
    st->log_num0 = log_num0;
  }
}

__global__ void fill_u32_kernel(uint32_t* p, int n, uint32_t value) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) p[k] = value;
}

// Species histogram (count_vectors per thread, per-CTA sums in shared
// memory, one global atomic per CTA and state: per-warp global atomics on the
// S+1 counters serialised and dominated the kernel).
__global__ void __launch_bounds__(256) count_kernel(LatticeDesc d, RunState* st) {
  if (ld_volatile(&st->stopped)) return;
  __shared__ uint32_t part[kMaxStates];
  if (threadIdx.x < kMaxStates) part[threadIdx.x] = 0u;
  __syncthreads();
  count_vectors(d, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x, part);
  __syncthreads();
  if ((int)threadIdx.x <= d.S && part[threadIdx.x])
    atomicAdd(&st->cur[threadIdx.x], (unsigned long long)part[threadIdx.x]);
}

__global__ void finalize_kernel(RunState* st, int S, LogBuffers lb, uint32_t m_end, uint32_t log_every,
                                int log, int stop_at_extinction, unsigned long long check_total) {
  if (st->stopped) return;
  st->mcs = m_end;
  if (!log) return;
  unsigned long long c[kMaxStates], sum = 0;
  for (int v = 0; v < kMaxStates; ++v) {
    c[v] = st->cur[v];
    st->cur[v] = 0;
    sum += (v <= S) ? c[v] : 0ull;
  }
  if (check_total && sum != check_total) {   // some byte is not a state
    st->error |= kErrBadValue;
    st->stopped = 1;
  }
  write_log_entry(st, lb, S, m_end, log_every, c, stop_at_extinction);
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) phase_kernel(LatticeDesc d, RunState* st, uint32_t m, int slot) {
  if (ld_volatile(&st->stopped)) return;
  __shared__ VisitSmem sm;
  __shared__ uint16_t stash[kStashWords];
  load_trans(d, sm.trans);
  const uint4 x = philox10(make_uint4(0u, 0u, m, kTagOrder), d.key0, d.key1);
  const int colour = order_at(colour_order(x.x, d.perm24), slot);
  const int half = d.P >> 1, j = blockIdx.x;
  const int bx = 2 * (j % half) + (colour & 1), by = 2 * (j / half) + (colour >> 1);
  if (d.uniform64 && d.bits != 8)
    visit_uniform<true, true>(d, bx, by, m, sm);
  else if (d.uniform64)
    visit_uniform<true, false>(d, bx, by, m, sm);
  else if (d.bits != 8)
    visit_generic<true, true>(d, bx, by, m, sm, stash);
  else
    visit_generic<true, false>(d, bx, by, m, sm, stash);
}

// ---------------------------------------------------------------------------
constexpr int kPersistentThreads = 256;
// The uniform persistent kernel is compiled for 4 resident CTAs per SM (up
// to 64 registers, no spills) and launched with kUniLaunchPerSM.  Measured at
// L = 3200: 4 per SM beat 2, 3, 5 and 6 -- fewer co-resident visits finish
// each hop of the colour-phase dependency chain sooner, and 4 still hide most
// of the memory latency.
constexpr int kUniMinBlocks = 4;
constexpr int kUniLaunchPerSM = 4;

__device__ __forceinline__ void own_fine_phases(const LatticeDesc& d, int bx, int by, uint32_t m, uint8_t* tile,
                                                uint32_t ord, const uint8_t* trans);

// NT = 256: one quad (2 x 2 sub-blocks) per thread, up to 4 CTAs per SM;
// NT = 128 (uniform geometry, any bits per site): two quads per thread
// stepped pairwise (own_fine_phases), up to 8 CTAs per SM -- twice the
// visits in flight per SM for the same number of threads.
// VAR (uniform geometry, one byte per site): a rule variant on 64 x 64
// blocks -- bit 0 a reflecting boundary, bit 1 the Moore neighbourhood.
template <bool UNI, bool PACKED = false, int NT = kPersistentThreads, int VAR = 0>
__global__ void __launch_bounds__(NT, NT == 128 ? 8 : (UNI ? kUniMinBlocks : 4))
    persistent_kernel(PersistentArgs a) {
  static_assert(NT == kPersistentThreads || (NT == 128 && UNI), "128-thread CTAs: uniform geometry only");
  static_assert(VAR == 0 || (UNI && !PACKED && NT == kPersistentThreads), "variants: uniform bytes, 256 threads");
  __shared__ VisitSmem sm;
  __shared__ uint16_t stash[(UNI || !PACKED) ? 1 : kStashWords];
  __shared__ uint32_t s_ord, s_quit, s_abort;
  __shared__ uint4 s_dec;   // the item's (m, k, bx, by), decoded by the ticket thread
  // Neighbour indices of the polls by a compare-and-wrap instead of the
  // modulo (measured with the per-thread ticket decode this kernel had
  // before: 1.8 % faster on generic lattices at L = 4800, 0.9 % in the
  // 128-thread build at L = 6400, 0.8 % slower in the 256-thread uniform
  // build at L = 3200, which keeps the modulo).
  constexpr bool kCmpWrap = !(UNI && !PACKED && NT == kPersistentThreads && VAR == 0);
  // The uniform 256-thread build steps on the 8-byte-entry transition table
  // (rule8: one shared-memory read off the exchange path; L = 3200 -0.7 %,
  // -1.3 % at M = 1e-5 where more steps leave the exchange path).
  constexpr bool kT8 = UNI && !PACKED && NT == kPersistentThreads && VAR == 0;
  // Generic builds: the epoch is released by a thread of the last warp, and
  // only warps 0 and 1 (the ticket thread and the pollers) meet at the top of
  // the loop, behind a named barrier, so that the release's wait for the
  // tile stores overlaps the next ticket's decode and polls (L = 4800 -2.1 %;
  // +3.2 % in the uniform build at L = 3200, which keeps one CTA barrier).
  constexpr bool kSplitTop = !UNI;
  constexpr int kReleaseThread = kSplitTop ? NT - 32 : 0;
  const LatticeDesc& d = a.d;
  RunState* st = a.st;
  const int tid = threadIdx.x;
  const bool run = !ld_volatile(&st->stopped);
  if (run) {
    if (kT8)
      fill_trans8(reinterpret_cast<uint2*>(sm.trans), d.trans, d.S, tid, NT);
    else
      load_trans(d, sm.trans);
    const int P = d.P, half = P >> 1, Py = d.Py;
    const uint32_t nb = (uint32_t)(P * Py), per = nb >> 2;
    const uint64_t total = (uint64_t)a.n_mcs * nb;
    // Tickets are taken in schedule order from a shared dispenser, one at a
    // time, as the CTA releases the epoch of its previous visit (taking the
    // next one at the start of a visit was measured slower at L = 3200: an
    // item that becomes ready then waits behind a whole visit of its CTA).
    // The ticket thread is in warp 1, not in the warp that releases the
    // epoch, and reads the abort flag together with the ticket, so neither
    // round trip delays the release or each other.
    constexpr int kTicketThread = 32;
    uint32_t c_m = 0xFFFFFFFFu, c_ord = 0;   // ticket thread: coarse order of MCS c_m
    uint32_t t_next = 0, ab_next = 0;        // ticket thread: next ticket, abort flag seen with it
    if (tid == kTicketThread) {
      t_next = atomicAdd(&st->ticket, 1u);
      ab_next = ld_volatile(&st->abort);
    }
    for (;;) {
      if (tid == kTicketThread) {
        const uint32_t t = t_next;
        uint32_t quit = ((uint64_t)t >= total) || ab_next;
        if (!quit) {
          // The ticket's item, decoded here once for the CTA with
          // host-computed reciprocals (div_by_rcp) instead of every thread
          // dividing by run-time counts (0.7-1.1 % faster at L = 3200, 4800
          // and 6400): MCS m, coarse slot k, block j of that slot's colour.
          uint32_t rem, j, jx;
          const uint32_t m = a.m_begin + div_by_rcp(t, nb, a.rcp_nb, rem);
          if (m != c_m) {
            c_m = m;
            c_ord = colour_order(philox10(make_uint4(0u, 0u, m, kTagOrder), d.key0, d.key1).x, d.perm24);
          }
          s_ord = c_ord;
          const uint32_t kk = div_by_rcp(rem, per, a.rcp_per, j);
          const uint32_t jy = div_by_rcp(j, (uint32_t)half, a.rcp_half, jx);
          const uint32_t col = (uint32_t)order_at(c_ord, (int)kk);
          s_dec = make_uint4(m, kk, 2u * jx + (col & 1u), 2u * jy + (col >> 1));
        }
        s_quit = quit;
        s_abort = 0;
      }
      if (tid < kMaxStates) sm.hist[tid] = 0;
      // The ticket's item (s_dec): MCS m, coarse slot k, colour, block (bx, by).
      uint32_t m = 0;
      int k = 0, colour = 0, bx = 0, by = 0;
      auto decode = [&]() {
        const uint4 v = s_dec;
        m = v.x;
        k = (int)v.y;
        bx = (int)v.z;
        by = (int)v.w;
        colour = (bx & 1) | ((by & 1) << 1);
      };
      if (kSplitTop) {
        // Named barrier 1 over 64 threads: warps 0 and 1 (the condition is
        // warp-uniform) reach it exactly once per iteration -- the loop is
        // left only after the CTA barrier below, by every thread alike -- and
        // no other code of this kernel uses barrier 1.
        if (tid < 64) bar_named(1, 64);
      } else {
        __syncthreads();
        if (s_quit) break;
      }
      const bool early = !kSplitTop || tid < 64;
      const bool go = early && !s_quit;
      if (go) decode();
      // Wait until the 8 neighbours (and the block itself) have completed
      // every visit that precedes this one in schedule order; meanwhile
      // warp 1 draws the block's fine colour order.
      if (go && tid == kTicketThread) sm.forder = fine_order(d, bx, by, m);
      if (go && tid < 9) {
        const uint32_t ord = s_ord;
        const int dx = tid % 3 - 1, dy = tid / 3 - 1;
        const int nx = kCmpWrap ? wrap(bx + dx, P) : (bx + dx + P) % P;
        const int ny = kCmpWrap ? wrap(by + dy, Py) : (by + dy + Py) % Py;
        const int ncol = colour ^ ((dx & 1) | ((dy & 1) << 1));
        const uint32_t need = (tid == 4) ? m : (slot_of(ord, ncol) < k ? m + 1u : m);
        const uint32_t* flag = a.done + ny * P + nx;
        uint32_t spins = 0;
        while (ld_acquire(flag) < need) {
          // the abort flag every 16th round, not between every two polls
          if ((spins & 15u) == 15u && ld_volatile(&st->abort)) {
            s_abort = 1;
            break;
          }
          if (++spins > a.spin_limit) {
            atomicOr(&st->error, kErrTimeout);
            atomicExch(&st->abort, 1u);
            s_abort = 1;
            break;
          }
          __nanosleep(64);
        }
      }
      __syncthreads();
      if (s_quit || s_abort) break;  // uniform across the CTA
      if (!early) decode();
      const uint32_t ord = s_ord;
      if (VAR != 0) {
        const int x0 = bx * kUniB, y0 = by * kUniB;
        load_piece_uni(d, x0, y0, sm.tile, tid);
        if (VAR & 2) corner_uni(d, x0, y0, sm.tile, tid, false);
        __syncthreads();
        const uint8_t* trans = reinterpret_cast<const uint8_t*>(sm.trans);
        const bool edge = (VAR & 1) && (bx == 0 || bx == P - 1 || by == 0 || by == Py - 1);
        if (edge)
          fine_phases_var<(VAR & 2) != 0, true>(d, bx, by, m, sm.tile, sm.forder, trans);
        else
          fine_phases_var<(VAR & 2) != 0, false>(d, bx, by, m, sm.tile, sm.forder, trans);
        store_piece_uni(d, x0, y0, sm.tile, tid);
        if (VAR & 2) corner_uni(d, x0, y0, sm.tile, tid, true);
      } else if (NT == 128) {
        const int x0 = bx * kUniB, y0 = by * kUniB;
        uint32_t rim_raw = 0;   // packed: the rim group of piece tid + 128
        if (PACKED) {
          load_piece_uni_packed(d, x0, y0, sm.tile, tid, d.bits);
          rim_raw = load_piece_uni_packed(d, x0, y0, sm.tile, tid + 128, d.bits);
        } else {
          load_piece_uni(d, x0, y0, sm.tile, tid);
          load_piece_uni(d, x0, y0, sm.tile, tid + 128);
        }
        __syncthreads();
        own_fine_phases(d, bx, by, m, sm.tile, sm.forder, reinterpret_cast<const uint8_t*>(sm.trans));
        if (PACKED) {
          store_piece_uni_packed(d, x0, y0, sm.tile, tid, d.bits, 0u);
          store_piece_uni_packed(d, x0, y0, sm.tile, tid + 128, d.bits, rim_raw);
        } else {
          store_piece_uni(d, x0, y0, sm.tile, tid);
          store_piece_uni(d, x0, y0, sm.tile, tid + 128);
        }
      } else if (UNI) {
        if (PACKED)
          visit_uniform<false, PACKED>(d, bx, by, m, sm);
        else
          visit_uniform_x0<kT8>(d, bx, by, m, sm);
      } else {
        visit_generic<false, PACKED>(d, bx, by, m, sm, stash);
      }
      const bool log_point = a.fuse_counts && ((m + 1u) % a.log_every) == 0u;
      if (log_point) {
        const int sV = slot_of(ord, colour ^ 2), sH = slot_of(ord, colour ^ 1),
                  sD = slot_of(ord, colour ^ 3);
        if (NT == 128) {
          count_pieces_uni<kUniSP, kColOff>(sm.tile, sm.hist, d.S, k, sV, sH, sD, tid);
          count_pieces_uni<kUniSP, kColOff>(sm.tile, sm.hist, d.S, k, sV, sH, sD, tid + 128);
        } else if (UNI) {
          count_visit_uni<kUniSP, kColOff>(sm.tile, sm.hist, d.S, k, sV, sH, sD);
        } else {
          count_visit_generic<PACKED>(d, bx, by, sm, k, sV, sH, sD);
        }
      }
      __syncthreads();
      if (tid == kReleaseThread && by * P + bx != a.stall_block) {
        // st.release orders the CTA's tile stores (made before the barrier
        // above) before the new epoch; no separate fence is needed.  The
        // counts of a log point live in shared memory and are published
        // after the release, off the neighbours' critical path.
        st_release(a.done + by * P + bx, m + 1u);
      }
      if (tid == kTicketThread) {
        t_next = atomicAdd(&st->ticket, 1u);
        ab_next = ld_volatile(&st->abort);
      }
      if (log_point) {
        const uint32_t ring = ((m + 1u) / a.log_every) % (uint32_t)kPendRing;
        if (tid <= d.S && sm.hist[tid]) atomicAdd(&st->acc[ring][tid], (unsigned long long)sm.hist[tid]);
        __syncthreads();
        if (tid == 0) {
          __threadfence();
          if (atomicAdd(&st->pend[ring], 1u) == nb - 1u) {
            // last block of this log point: every contribution is in acc
            __threadfence();
            unsigned long long c[kMaxStates];
            for (int v = 0; v < kMaxStates; ++v) c[v] = atomicExch(&st->acc[ring][v], 0ull);
            st->pend[ring] = 0;
            write_log_entry(st, a.lb, d.S, m + 1u, a.log_every, c, a.stop_at_extinction);
          }
        }
      }
    }
  }
  // The last CTA to leave publishes the MCS number and resets the
  // dispensers for the next launch on this stream.
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(&st->exited, 1u) == gridDim.x - 1u) {
      st->exited = 0;
      st->ticket = 0;
      if (!st->stopped && !st->abort) st->mcs = a.m_begin + a.n_mcs;
    }
  }
}

// ---------------------------------------------------------------------------
// Boundary-mailbox persistent kernel (uniform geometry; the default
// persistent path).  Same work items, schedule order and results as
// persistent_kernel; what differs is how a visit learns that its neighbours
// are done and gets their data.
//
// A visit publishes its block's four boundary records -- per side, the
// block's edge line and the rim line beyond it (the strip it wrote into the
// neighbour), after the visit -- as 8-byte words holding 4 lattice bytes in
// the low half and the epoch of the visit (m + 1) in the high half, each
// written with one single-copy-atomic 64-bit store.  A neighbour polls those
// words directly: a word with the expected epoch is also the data, so flag
// and data arrive in one round trip and the writer needs no fence before
// publishing.  The lattice array receives only the block's own interior,
// released by the block's epoch flag, which only the block's next visit
// reads (one MCS later, off the neighbours' critical path).  Rim strips
// reach the lattice array at the end of the launch (ll_merge_kernel), so a
// launch starts from a complete lattice array and needs no record from an
// earlier launch.
//
// Record layout: ob[(block * 4 + side) * 32 + part * 16 + w]; side 0 top,
// 1 bottom, 2 left, 3 right; part 0 the block's edge line, 1 the rim line;
// word w holds positions 4w..4w+3 along the side, byte j = position 4w + j.
//
// Which visit wrote a cell last: the coarse order is drawn afresh every MCS,
// so a neighbour of colour c was last visited (before the visit at slot k of
// MCS m) at (m, slot_m(c)) if slot_m(c) < k, else at (m - 1, slot_m-1(c)),
// and the block itself at (m - 1, slot_m-1(own colour)).  key = 4 + slot_m
// for the former, slot_m-1 for the latter orders all of them.  Every staged
// cell takes the value of its latest writer among the block's own previous
// visit (the interior from the lattice array, the rim lines from the block's
// own records), the edge neighbour across that side and, at the 12 cells
// that two neighbours touch (interior corners: the vertical and the
// horizontal neighbour; rim ends: an edge neighbour and a diagonal one), the
// other neighbour.
constexpr int kLLConsumers = 256, kLLThreads = kLLConsumers + 32;
// 4 CTAs of 9 warps per SM (56 registers); 5 (40 registers, with spills)
// was measured slower at L = 3200.
constexpr int kLLMinBlocks = 4;

// Tile index of position pos (0..63) of line (side, part) of a uniform block.
__device__ __forceinline__ int line_tidx(int side, int part, int pos) {
  const int fixed = (side & 1) ? (part ? kUniB : kUniB - 1) : (part ? -1 : 0);
  return (side < 2) ? tidx(fixed, pos, kUniSP) : tidx(pos, fixed, kUniSP);
}

// Lattice coordinates of position pos of line (side, part) of block (x0, y0).
__device__ __forceinline__ void line_cell(int side, int part, int pos, int x0, int y0, int L, int& y, int& x) {
  const int fixed = (side & 1) ? (part ? kUniB : kUniB - 1) : (part ? -1 : 0);
  y = wrap(y0 + ((side < 2) ? fixed : pos), L);
  x = wrap(x0 + ((side < 2) ? pos : fixed), L);
}

// Shared state of the mailbox kernel: two tiles -- the consumers (warps
// 0..7) visit one while the producer (warp 8) stages the next work item in
// the other -- and the two items' decoded fields.
constexpr int kUniTileBytes = (kUniB + 2) * kUniSP;
struct LLItem {
  uint32_t m, ord, ordp, forder, quit, staged;
  int32_t k, bx, by;
};
struct LLSmem {
  alignas(16) uint8_t tile[2][kUniTileBytes];
  uint32_t trans[kTransWords];
  uint32_t hist[kMaxStates];
  LLItem item[2];
  uint32_t abort;
};

__device__ __forceinline__ void cons_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
__device__ __forceinline__ void cons_hi_sync() { asm volatile("bar.sync 2, 128;" ::: "memory"); }

__device__ __forceinline__ void tile_row16(uint8_t* tile, int r, int c, uint4 v) {
  uint2* dst = reinterpret_cast<uint2*>(tile + tidx(r, c, kUniSP));
  dst[0] = make_uint2(v.x, v.y);
  dst[1] = make_uint2(v.z, v.w);
}

// Producer (one warp): takes the next ticket, decodes it into sm.item[b]
// and, when it can do so without waiting, stages the block's interior in
// sm.tile[b] (and, on the first visit of the launch, its rim lines from the
// lattice array).  Never blocks on another CTA.
struct LLOrders {
  uint32_t m, ord, ordp;
  bool valid;
};
__device__ void ll_produce(const PersistentArgs& a, LLSmem& sm, int b, LLOrders& o) {
  const LatticeDesc& d = a.d;
  RunState* st = a.st;
  const int lane = threadIdx.x & 31;
  const int P = d.P, half = P >> 1, pitch = d.pitch;
  const uint32_t nb = (uint32_t)(P * P), per = nb >> 2;
  const uint64_t total = (uint64_t)a.n_mcs * nb;
  uint32_t t = 0, ab = 0;
  if (lane == 0) {
    t = atomicAdd(&st->ticket, 1u);
    ab = ld_volatile(&st->abort);
  }
  t = __shfl_sync(0xFFFFFFFFu, t, 0);
  ab = __shfl_sync(0xFFFFFFFFu, ab, 0);
  LLItem it{};
  it.quit = ((uint64_t)t >= total) || ab;
  if (!it.quit) {
    const uint32_t mi = t / nb, rem = t - mi * nb, m = a.m_begin + mi;
    if (m != o.m || !o.valid) {
      o.ordp = (o.valid && m == o.m + 1u)
                   ? o.ord
                   : colour_order(philox10(make_uint4(0u, 0u, m - 1u, kTagOrder), d.key0, d.key1).x, d.perm24);
      o.ord = colour_order(philox10(make_uint4(0u, 0u, m, kTagOrder), d.key0, d.key1).x, d.perm24);
      o.m = m;
      o.valid = true;
    }
    it.m = m;
    it.ord = o.ord;
    it.ordp = o.ordp;
    it.k = (int)(rem / per);
    const int j = (int)(rem - (uint32_t)it.k * per);
    const int colour = order_at(o.ord, it.k);
    it.bx = 2 * (j % half) + (colour & 1);
    it.by = 2 * (j / half) + (colour >> 1);
    it.forder = fine_order(d, it.bx, it.by, m);
    const int X = it.by * P + it.bx, x0 = it.bx * kUniB, y0 = it.by * kUniB;
    const bool first = (m == a.m_begin);
    uint32_t ready = first ? 1u : 0u;
    if (!first && lane == 0) ready = ld_acquire(a.done + X) >= m ? 1u : 0u;
    ready = __shfl_sync(0xFFFFFFFFu, ready, 0);   // orders the loads below after the acquire
    it.staged = ready;
    uint8_t* tile = sm.tile[b];
    if (ready) {
#pragma unroll
      for (int h = 0; h < 8; ++h) {
        const int idx = lane + 32 * h, r = idx >> 2, q = idx & 3;
        tile_row16(tile, r, 16 * q,
                   __ldcg(reinterpret_cast<const uint4*>(d.lat + (size_t)(y0 + r) * pitch + x0) + q));
      }
    }
    if (first) {   // rim lines, as the lattice array holds them at launch start
      const int L = d.L;
      if (lane < 8) {
        const int r = (lane < 4) ? -1 : kUniB, q = lane & 3;
        tile_row16(tile, r, 16 * q,
                   __ldcg(reinterpret_cast<const uint4*>(d.lat + (size_t)wrap(y0 + r, L) * pitch + x0) + q));
      }
      const int xl = wrap(x0 - 1, L), xr = wrap(x0 + kUniB, L);
      for (int r = lane; r < kUniB; r += 32) {
        tile[tidx(r, -1, kUniSP)] = __ldcg(d.lat + (size_t)(y0 + r) * pitch + xl);
        tile[tidx(r, kUniB, kUniSP)] = __ldcg(d.lat + (size_t)(y0 + r) * pitch + xr);
      }
    }
  }
  if (lane == 0) sm.item[b] = it;
}

__global__ void __launch_bounds__(kLLThreads, kLLMinBlocks) persistent_ll_kernel(PersistentArgs a) {
  __shared__ LLSmem sm;
  const LatticeDesc& d = a.d;
  RunState* st = a.st;
  unsigned long long* ob = a.ob;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool producer = (warp == kLLConsumers / 32);
  // consumer roles besides the visit: warps 0..3 poll and publish the
  // records of sides 0..3; warp 4 lanes 0..7 poll the diagonal neighbours'
  // rim ends, lane 8 waits for the block's own epoch when the producer could
  // not stage the interior; tid 255 releases the epochs.
  constexpr int kReleaseThread = kLLConsumers - 1;
  const bool run = !ld_volatile(&st->stopped);
  int rel_blk = -1;
  uint32_t rel_epoch = 0;
  if (run) {
    load_trans(d, sm.trans);
    if (tid == 0) sm.abort = 0;
    const int P = d.P, pitch = d.pitch;
    const uint32_t nb = (uint32_t)(P * P);
    LLOrders ords{0u, 0u, 0u, false};
    if (producer) ll_produce(a, sm, 0, ords);
    __syncthreads();
    const uint8_t* trans = reinterpret_cast<const uint8_t*>(sm.trans);
    for (uint32_t n = 0;; ++n) {
      const int b = (int)(n & 1u);
      const LLItem it = sm.item[b];
      if (it.quit || sm.abort) break;   // uniform: read after a barrier
      if (producer) {
        ll_produce(a, sm, b ^ 1, ords);
      } else {
        if (tid == kReleaseThread && rel_blk >= 0) {
          // the previous visit's interior stores all precede the barrier
          st_release(a.done + rel_blk, rel_epoch);
          rel_blk = -1;
        }
        if (tid < kMaxStates) sm.hist[tid] = 0;
        const uint32_t m = it.m, ord = it.ord, ordp = it.ordp;
        const int k = it.k, bx = it.bx, by = it.by, colour = order_at(ord, k);
        const int X = by * P + bx, x0 = bx * kUniB, y0 = by * kUniB;
        uint8_t* tile = sm.tile[b];
        const int sV = slot_of(ord, colour ^ 2), sH = slot_of(ord, colour ^ 1), sD = slot_of(ord, colour ^ 3);
        const int kV0 = sV < k ? sV + 4 : slot_of(ordp, colour ^ 2);
        const int kH0 = sH < k ? sH + 4 : slot_of(ordp, colour ^ 1);
        const int kD0 = sD < k ? sD + 4 : slot_of(ordp, colour ^ 3);
        const uint32_t eV = sV < k ? m + 1u : m, eH = sH < k ? m + 1u : m, eD = sD < k ? m + 1u : m;
        // The first visit of a launch stages its tile from the lattice array
        // (complete at launch start; a neighbour that has not visited yet in
        // this launch cannot write it before this visit publishes) and takes
        // only the neighbours that visited earlier in this launch from their
        // records: their keys (>= 4) beat the lattice's (3), the others' (-1)
        // lose to it.
        const bool first = (m == a.m_begin);
        const int kV = first && sV > k ? -1 : kV0, kH = first && sH > k ? -1 : kH0;
        const int kD = first && sD > k ? -1 : kD0, kXp = first ? 3 : slot_of(ordp, colour);
        unsigned long long word = 0, own = 0;
        bool failed = false;
        if (warp < 4) {
          // edge neighbour on side `warp`: its record of the opposite side;
          // lanes 0..15 also the block's own rim line of that side as its
          // previous visit left it (first visit: already staged)
          const int s = warp;
          const int nx = (s == 2) ? (bx + P - 1) % P : (s == 3) ? (bx + 1) % P : bx;
          const int ny = (s == 0) ? (by + P - 1) % P : (s == 1) ? (by + 1) % P : by;
          const uint32_t e = (s < 2) ? eV : eH;
          const unsigned long long* p = ob + ((size_t)(ny * P + nx) * 4 + (s ^ 1)) * 32 + lane;
          const unsigned long long* q = ob + ((size_t)X * 4 + s) * 32 + 16 + (lane & 15);
          bool got = first && ((s < 2) ? sV : sH) > k, got_own = first || lane >= 16;
          uint32_t spins = 0;
          while (!got || !got_own) {
            if (!got) got = (uint32_t)((word = ld_word(p)) >> 32) == e;
            if (!got_own) got_own = (uint32_t)((own = ld_word(q)) >> 32) == m;
            if (got && got_own) break;
            if ((spins & 15u) == 15u && ld_volatile(&st->abort)) {
              failed = true;
              break;
            }
            if (++spins > a.spin_limit) {
              atomicOr(&st->error, kErrTimeout);
              atomicExch(&st->abort, 1u);
              failed = true;
              break;
            }
            __nanosleep(64);
          }
        } else if (warp == 4 && lane < 8) {
          // rim end of a diagonal neighbour: lanes 0..3 the ends of the top
          // and bottom rim rows, 4..7 those of the left and right rim columns
          const int dx = (lane == 0 || lane == 2 || lane == 4 || lane == 5) ? -1 : 1;
          const int dy = (lane == 0 || lane == 1 || lane == 4 || lane == 6) ? -1 : 1;
          const int rec = (lane < 4) ? (dx < 0 ? 3 : 2) : (dy < 0 ? 1 : 0);
          const int pos = (lane < 4) ? (dy < 0 ? 63 : 0) : (dx < 0 ? 63 : 0);
          const int nx = (bx + P + dx) % P, ny = (by + P + dy) % P;
          const unsigned long long* p = ob + ((size_t)(ny * P + nx) * 4 + rec) * 32 + 16 + (pos >> 2);
          uint32_t spins = 0;
          while (!(first && sD > k) && (uint32_t)((word = ld_word(p)) >> 32) != eD) {
            if ((spins & 15u) == 15u && ld_volatile(&st->abort)) {
              failed = true;
              break;
            }
            if (++spins > a.spin_limit) {
              atomicOr(&st->error, kErrTimeout);
              atomicExch(&st->abort, 1u);
              failed = true;
              break;
            }
            __nanosleep(64);
          }
        }
        if (!it.staged && warp >= 4) {
          // the producer found the block's previous visit unfinished: wait
          // for its epoch here, then stage the interior
          if (tid == 4 * 32 + 8) {
            uint32_t spins = 0;
            while (ld_acquire(a.done + X) < m) {
              if (ld_volatile(&st->abort)) {
                failed = true;
                break;
              }
              if (++spins > a.spin_limit) {
                atomicOr(&st->error, kErrTimeout);
                atomicExch(&st->abort, 1u);
                failed = true;
                break;
              }
              __nanosleep(64);
            }
          }
          cons_hi_sync();
          const int i = tid - 128;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int idx = i + 128 * h, r = idx >> 2, q = idx & 3;
            tile_row16(tile, r, 16 * q,
                       __ldcg(reinterpret_cast<const uint4*>(d.lat + (size_t)(y0 + r) * pitch + x0) + q));
          }
        }
        if (failed) sm.abort = 1u;
        // each staged boundary cell takes the value of its latest writer (the
        // choice depends only on the schedule, so every writer decides alone)
        auto place = [&]() {
          if (warp < 4) {
            const int s = warp, xp = 1 - (lane >> 4), w = lane & 15;
            const int kS = (s < 2) ? kV : kH, kO = (s < 2) ? kH : kV;
            const uint32_t data = (uint32_t)word, mine = (uint32_t)own;
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
              const int pos = 4 * w + jj;
              const bool end = (pos == 0) || (pos == kUniB - 1);
              uint8_t* cell = tile + line_tidx(s, xp, pos);
              if (xp == 0) {
                // edge line: the interior already holds the block's own value
                if (kS > (end ? max(kO, kXp) : kXp)) *cell = (uint8_t)(data >> (8 * jj));
              } else if (kS > (end ? max(kD, kXp) : kXp)) {
                *cell = (uint8_t)(data >> (8 * jj));
              } else if (!first && kXp > (end ? max(kS, kD) : kS)) {
                *cell = (uint8_t)(mine >> (8 * jj));
              }
            }
          } else if (warp == 4 && lane < 8) {
            const int xs = (lane < 4) ? (lane >> 1) : 2 + ((lane - 4) >> 1);
            const int xpos = (lane & 1) ? kUniB - 1 : 0;
            const int dpos = (lane < 4) ? ((lane < 2) ? 63 : 0) : ((lane < 6) ? 63 : 0);
            if (kD > max((xs < 2) ? kV : kH, kXp))
              tile[line_tidx(xs, 1, xpos)] = (uint8_t)((uint32_t)word >> (8 * (dpos & 3)));
          }
        };
        // staged interior: place at once; otherwise after the interior lands
        if (it.staged && !failed) place();
        cons_sync();
        if (!sm.abort) {
          if (!it.staged) {
            place();
            cons_sync();
          }
          fine_phases_tile<1, kLLConsumers>(d, bx, by, m, tile, it.forder, trans);
          if (X != a.stall_block) {
            // publish the records first: they are the neighbours' critical path
            if (warp < 4) {
              const int s = warp, part = lane >> 4, w = lane & 15;
              uint32_t bytes = 0;
#pragma unroll
              for (int jj = 0; jj < 4; ++jj) bytes |= (uint32_t)tile[line_tidx(s, part, 4 * w + jj)] << (8 * jj);
              st_word(ob + ((size_t)X * 4 + s) * 32 + lane, ((unsigned long long)(m + 1u) << 32) | bytes);
            }
            {  // the interior to the lattice array
              const int r = tid >> 2, q = tid & 3;
              const uint2* src = reinterpret_cast<const uint2*>(tile + tidx(r, 16 * q, kUniSP));
              const uint2 u0 = src[0], u1 = src[1];
              reinterpret_cast<uint4*>(d.lat + (size_t)(y0 + r) * pitch + x0)[q] = make_uint4(u0.x, u0.y, u1.x, u1.y);
            }
            if (tid == kReleaseThread) {
              rel_blk = X;
              rel_epoch = m + 1u;
            }
          }
          if (((m + 1u) % a.log_every) == 0u) {
            count_visit_uni<kUniSP, kColOff>(tile, sm.hist, d.S, k, sV, sH, sD);
            cons_sync();
            const uint32_t ring = ((m + 1u) / a.log_every) % (uint32_t)kPendRing;
            if (tid <= d.S && sm.hist[tid]) atomicAdd(&st->acc[ring][tid], (unsigned long long)sm.hist[tid]);
            cons_sync();
            if (tid == 0) {
              __threadfence();
              if (atomicAdd(&st->pend[ring], 1u) == nb - 1u) {
                // last block of this log point: every contribution is in acc
                __threadfence();
                unsigned long long c[kMaxStates];
                for (int v = 0; v < kMaxStates; ++v) c[v] = atomicExch(&st->acc[ring][v], 0ull);
                st->pend[ring] = 0;
                write_log_entry(st, a.lb, d.S, m + 1u, a.log_every, c, a.stop_at_extinction);
              }
            }
          }
        }
      }
      __syncthreads();
    }
    if (tid == kReleaseThread && rel_blk >= 0) st_release(a.done + rel_blk, rel_epoch);
  }
  // The last CTA to leave publishes the MCS number and resets the
  // dispensers for the next launch on this stream.
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(&st->exited, 1u) == gridDim.x - 1u) {
      st->exited = 0;
      st->ticket = 0;
      if (!st->stopped && !st->abort) st->mcs = a.m_begin + a.n_mcs;
    }
  }
}

// One CTA of 256 threads per block: thread (side, pos) settles edge cell pos
// of the block's side `side` (the interior corners by the row threads only).
// Every block was last visited in MCS m_end - 1 (coarse order `ord`); the
// cell's last writer is the block itself or the neighbour across that side
// or, at a corner, the neighbour across the other side -- whichever has the
// latest slot.
__global__ void __launch_bounds__(256) ll_merge_kernel(LatticeDesc d, const unsigned long long* ob,
                                                       const RunState* st, uint32_t m_end, uint32_t ord) {
  // a launch that did not run (the lattice had stopped earlier) left nothing
  // to merge
  if (st->mcs != m_end || st->abort) return;
  const int X = blockIdx.x, P = d.P, bx = X % P, by = X / P;
  const int t = threadIdx.x, s = t >> 6, pos = t & 63;
  const bool end = (pos == 0) || (pos == kUniB - 1);
  if (s >= 2 && end) return;
  const int colour = 2 * (by & 1) + (bx & 1);
  const int kX = slot_of(ord, colour), sV = slot_of(ord, colour ^ 2), sH = slot_of(ord, colour ^ 1);
  // neighbour across side s: its record of the opposite side, rim line
  int best = kX, nbr = -1, rec = 0, npos = pos;
  const int kS = (s < 2) ? sV : sH;
  if (kS > best) {
    best = kS;
    nbr = (s == 0) ? ((by + P - 1) % P) * P + bx : (s == 1) ? ((by + 1) % P) * P + bx
        : (s == 2) ? by * P + (bx + P - 1) % P : by * P + (bx + 1) % P;
    rec = s ^ 1;
  }
  if (end && sH > best) {   // row threads: the horizontal neighbour at the corner
    best = sH;
    nbr = (pos == 0) ? by * P + (bx + P - 1) % P : by * P + (bx + 1) % P;
    rec = (pos == 0) ? 3 : 2;
    npos = (s == 0) ? 0 : kUniB - 1;
  }
  if (nbr < 0) return;  // the block's own value is already in the lattice array
  const unsigned long long wv = ob[((size_t)nbr * 4 + rec) * 32 + 16 + (npos >> 2)];
  int y, x;
  line_cell(s, 0, pos, bx * kUniB, by * kUniB, d.L, y, x);
  d.lat[(size_t)y * d.pitch + x] = (uint8_t)((uint32_t)wv >> (8 * (npos & 3)));
}

// ---------------------------------------------------------------------------
// Block-owner kernel (uniform geometry; one byte per site or packed).  CTA g
// owns coarse group g -- the 2x2 blocks (2 gx + cx, 2 gy + cy), one of each
// colour -- for the whole launch and keeps their four tiles (interior and rim
// lines) in shared memory from visit to visit.  A visit exchanges only the
// mailbox kernel's boundary records: it polls its 4 edge neighbours' records
// and 8 diagonal rim-end words, places each boundary cell from its latest
// writer (the block's own previous visit is already in the tile), runs the
// four fine phases and publishes its 4 records.  There is no ticket, no
// interior load or store and no epoch flag: the lattice array is read when
// the launch starts (nothing writes it during the launch) and written when
// it ends, each block's edge cells settled first from the final records of
// the neighbours that visited after it.  Same schedule, same results.
//
// Every CTA waits for visits that only its neighbours' owners perform, so the
// whole grid must be resident at once: it is a cooperative launch, made only
// when the occupancy allows, with shared memory padded so that the CTAs
// spread over all SMs (at most ceil(groups / SMs) per SM).
// CTAs of 256 threads (one quad per thread) or, where the grid needs more
// than 4 CTAs per SM, 128 (two quads per thread, stepped pairwise).

struct OwnSmem {
  alignas(16) uint8_t tile[4][kUniTileBytes];   // tile[c]: the group's block of colour c
  uint32_t trans[kTransWords];
  uint32_t hist[kMaxStates];
  uint32_t forder;   // fine order of the current visit
  uint32_t abort;
};

// The group's block (bx, by) as the lattice array holds it: interior, top and
// bottom rim rows, left and right rim columns (the corners are not used).
// One byte per site: 16-byte pieces; packed (d.bits 4 or 2): groups of 4
// sites, unpacked into the tile.
template <int NT>
__device__ __forceinline__ void own_stage(const LatticeDesc& d, uint8_t* tile, int bx, int by) {
  const int L = d.L, pitch = d.pitch, bits = d.bits, x0 = bx * kUniB, y0 = by * kUniB;
  if (bits == 8) {
    for (int i = threadIdx.x; i < (kUniB + 2) * 4; i += NT) {
      const int r = (i >> 2) - 1, q = i & 3;
      tile_row16(tile, r, 16 * q,
                 __ldcg(reinterpret_cast<const uint4*>(d.lat + (size_t)wrap(y0 + r, d.H) * pitch + x0) + q));
    }
  } else {
    for (int i = threadIdx.x; i < (kUniB + 2) * (kUniB / 4); i += NT) {
      const int r = i / (kUniB / 4) - 1, k = i % (kUniB / 4);
      const uint32_t raw = load_group(d.lat + (size_t)wrap(y0 + r, d.H) * pitch, x0 + 4 * k, bits);
      *reinterpret_cast<uint32_t*>(tile + tidx(r, 4 * k, kUniSP)) = unpack4(raw, bits);
    }
  }
  const int xl = wrap(x0 - 1, L), xr = wrap(x0 + kUniB, L);
  for (int i = threadIdx.x; i < 2 * kUniB; i += NT) {
    const int r = i & (kUniB - 1), right = i >= kUniB, gx = right ? xr : xl;
    const uint8_t* row = d.lat + (size_t)(y0 + r) * pitch;
    tile[tidx(r, right ? kUniB : -1, kUniSP)] =
        bits == 8 ? __ldcg(row + gx) : (uint8_t)(unpack4(load_group(row, gx & ~3, bits), bits) >> (8 * (gx & 3)));
  }
}

// New values of an attempt's pair (cell a, neighbour b) as one byte (low
// nibble: the cell, high nibble: the neighbour), the transition of
// apply_rule.
__device__ __forceinline__ uint32_t rule_nn(const uint8_t* __restrict__ trans, uint32_t a, uint32_t b, uint32_t u,
                                            uint32_t tx, uint32_t txi, uint32_t s1) {
  if (u < tx) return b | (a << 4);
  const uint32_t pair = a * s1 + b;
  const uint32_t tp = reinterpret_cast<const uint32_t*>(trans)[kTransPairs + pair];
  const uint32_t act = (u >= txi) ? 2u : (u < tp ? 1u : 3u);
  return trans[pair * 4u + act];
}

// Two elementary steps (words wa, wb) on two sub-blocks of the same fine
// colour (first cells at basea, baseb): their cells and neighbours are
// disjoint, so both pairs are read before either is written and the two
// dependency chains overlap.  Each step is attempt_uni's.
template <int SP>
__device__ __forceinline__ void attempt_uni_pair(uint8_t* __restrict__ tile, const uint8_t* __restrict__ trans,
                                                 uint32_t wa, int basea, uint32_t wb, int baseb, uint32_t tx,
                                                 uint32_t txi, uint32_t s1) {
  constexpr uint32_t kTi = 0u | (1u << 8) | ((uint32_t)SP << 16) | ((uint32_t)(SP + 1) << 24);
  constexpr uint32_t kTj = 0u | ((uint32_t)(2 * SP) << 8) | ((uint32_t)(SP - 1) << 16) | ((uint32_t)(SP + 1) << 24);
  const int tia = basea + (int)__byte_perm(kTi, 0u, wa >> 30);
  const int tja = tia - SP + (int)__byte_perm(kTj, 0u, (wa >> 28) & 3u);
  const int tib = baseb + (int)__byte_perm(kTi, 0u, wb >> 30);
  const int tjb = tib - SP + (int)__byte_perm(kTj, 0u, (wb >> 28) & 3u);
  const uint32_t aa = tile[tia], ba = tile[tja], ab = tile[tib], bb = tile[tjb];
  const uint32_t na = rule_nn(trans, aa, ba, wa << 4, tx, txi, s1);
  const uint32_t nb = rule_nn(trans, ab, bb, wb << 4, tx, txi, s1);
  tile[tia] = (uint8_t)(na & 15u);
  tile[tja] = (uint8_t)(na >> 4);
  tile[tib] = (uint8_t)(nb & 15u);
  tile[tjb] = (uint8_t)(nb >> 4);
}

// The four fine colour phases of a uniform visit by 128 threads: thread t
// takes quads t and t + 128 (rows 4 qy..4 qy+3 and 32 rows below) and runs
// their steps pairwise.
__device__ __forceinline__ void own_fine_phases(const LatticeDesc& d, int bx, int by, uint32_t m, uint8_t* tile,
                                                uint32_t ord, const uint8_t* trans) {
  const int t = threadIdx.x, qx = t & 15, qy = t >> 4;
  const uint32_t s1 = (uint32_t)d.S + 1u, tx = d.tx, txi = d.txi;
  const uint32_t GQ = (uint32_t)d.GQ;
  const uint32_t g00 = (uint32_t)(by * (kUniB / 2) + 2 * qy) * GQ + (uint32_t)(bx * (kUniB / 2) + 2 * qx);
  const int base00 = tidx(4 * qy, 4 * qx, kUniSP);
  constexpr uint32_t kRowsB = kUniB / 4;          // quad rows 8.. are 16 sub-block rows below
  constexpr int kBaseB = (kUniB / 2) * kUniSP;    // and 32 tile rows below
#pragma unroll
  for (int fi = 0; fi < 4; ++fi) {
    const uint32_t fcol = (ord >> (2 * fi)) & 3u, cx = fcol & 1u, cy = fcol >> 1;
    const uint32_t g = g00 + cy * GQ + cx;
    const int base = base00 + (int)(cy * (2 * kUniSP) + 2 * cx);
    const uint4 xa = philox10_rk(make_uint4(0u, g, m, kTagStep), d.rk);
    const uint4 xb = philox10_rk(make_uint4(0u, g + kRowsB * GQ, m, kTagStep), d.rk);
    attempt_uni_pair<kUniSP>(tile, trans, xa.x, base, xb.x, base + kBaseB, tx, txi, s1);
    attempt_uni_pair<kUniSP>(tile, trans, xa.y, base, xb.y, base + kBaseB, tx, txi, s1);
    attempt_uni_pair<kUniSP>(tile, trans, xa.z, base, xb.z, base + kBaseB, tx, txi, s1);
    attempt_uni_pair<kUniSP>(tile, trans, xa.w, base, xb.w, base + kBaseB, tx, txi, s1);
    __syncthreads();
  }
}

template <int NT>
__global__ void __launch_bounds__(NT, NT == 128 ? 8 : 4) persistent_own_kernel(PersistentArgs a) {
  extern __shared__ uint8_t own_pad[];   // occupancy padding only
  __shared__ OwnSmem sm;
  (void)own_pad;
  const LatticeDesc& d = a.d;
  RunState* st = a.st;
  unsigned long long* ob = a.ob;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool run = !ld_volatile(&st->stopped);
  if (run) {
    load_trans(d, sm.trans);
    const int P = d.P, Py = d.Py, half = P >> 1, pitch = d.pitch;
    const uint32_t nb = (uint32_t)(P * Py);
    const int gx = (int)blockIdx.x % half, gy = (int)blockIdx.x / half;
    for (int c = 0; c < 4; ++c) own_stage<NT>(d, sm.tile[c], 2 * gx + (c & 1), 2 * gy + (c >> 1));
    const uint8_t* trans = reinterpret_cast<const uint8_t*>(sm.trans);
    const uint32_t m_end = a.m_begin + a.n_mcs;
    uint32_t ordp = colour_order(philox10(make_uint4(0u, 0u, a.m_begin - 1u, kTagOrder), d.key0, d.key1).x,
                                 d.perm24);
    uint32_t ord = colour_order(philox10(make_uint4(0u, 0u, a.m_begin, kTagOrder), d.key0, d.key1).x, d.perm24);
    uint32_t ord_next = ord;
    if (tid == 0) sm.abort = 0;
    __syncthreads();
    bool quit = false;
    for (uint32_t m = a.m_begin; m < m_end && !quit; ++m) {
      if (m != a.m_begin) {
        ordp = ord;
        ord = ord_next;
      }
      for (int k = 0; k < 4; ++k) {
        if (tid < kMaxStates) sm.hist[tid] = 0;
        const int colour = order_at(ord, k);
        const int bx = 2 * gx + (colour & 1), by = 2 * gy + (colour >> 1);
        const int X = by * P + bx;
        uint8_t* tile = sm.tile[colour];
        const int sV = slot_of(ord, colour ^ 2), sH = slot_of(ord, colour ^ 1), sD = slot_of(ord, colour ^ 3);
        const int kV0 = sV < k ? sV + 4 : slot_of(ordp, colour ^ 2);
        const int kH0 = sH < k ? sH + 4 : slot_of(ordp, colour ^ 1);
        const int kD0 = sD < k ? sD + 4 : slot_of(ordp, colour ^ 3);
        const uint32_t eV = sV < k ? m + 1u : m, eH = sH < k ? m + 1u : m, eD = sD < k ? m + 1u : m;
        // first visit of the launch: the tile holds the lattice array as it
        // was at launch start; only neighbours that visited earlier in this
        // launch come from their records (keys >= 4 beat the lattice's 3)
        const bool first = (m == a.m_begin);
        const int kV = first && sV > k ? -1 : kV0, kH = first && sH > k ? -1 : kH0;
        const int kD = first && sD > k ? -1 : kD0, kXp = first ? 3 : slot_of(ordp, colour);
        // warp s < 4: the record of the edge neighbour across side s (its
        // record of the opposite side, one word per lane); lanes 0 and 1 also
        // a diagonal neighbour's rim-end word, dl = 2 s + lane: dl 0..3 the
        // ends of the top and bottom rim rows, 4..7 those of the left and
        // right rim columns
        const bool poller = warp < 4;
        const int s = warp & 3;
        const int nx = (s == 2) ? (bx + P - 1) % P : (s == 3) ? (bx + 1) % P : bx;
        const int ny = (s == 0) ? (by + Py - 1) % Py : (s == 1) ? (by + 1) % Py : by;
        const uint32_t e = (s < 2) ? eV : eH;
        const unsigned long long* p = ob + ((size_t)(ny * P + nx) * 4 + (s ^ 1)) * 32 + lane;
        const int dl = 2 * s + (lane & 1);
        const int ddx = (dl == 0 || dl == 2 || dl == 4 || dl == 5) ? -1 : 1;
        const int ddy = (dl == 0 || dl == 1 || dl == 4 || dl == 6) ? -1 : 1;
        const int drec = (dl < 4) ? (ddx < 0 ? 3 : 2) : (ddy < 0 ? 1 : 0);
        const int dpos = (dl < 4) ? (ddy < 0 ? 63 : 0) : (ddx < 0 ? 63 : 0);
        const unsigned long long* pd =
            ob + ((size_t)(((by + Py + ddy) % Py) * P + (bx + P + ddx) % P) * 4 + drec) * 32 + 16 + (dpos >> 2);
        bool got = !poller || (first && ((s < 2) ? sV : sH) > k);
        bool got_d = !poller || lane >= 2 || (first && sD > k);
        unsigned long long word = 0, dword = 0;
        if (!got) word = ld_word(p);
        if (!got_d) dword = ld_word(pd);
        // while those loads are in flight: the fine order of this visit and
        // the coarse order of the next MCS
        if (tid == NT - 1) sm.forder = fine_order(d, bx, by, m);
        if (k == 3) ord_next = colour_order(philox10(make_uint4(0u, 0u, m + 1u, kTagOrder), d.key0, d.key1).x,
                                            d.perm24);
        bool failed = false;
        uint32_t spins = 0;
        for (;;) {
          if (!got) got = (uint32_t)(word >> 32) == e;
          if (!got_d) got_d = (uint32_t)(dword >> 32) == eD;
          if (got && got_d) break;
          if ((spins & 15u) == 15u && ld_volatile(&st->abort)) {
            failed = true;
            break;
          }
          if (++spins > a.spin_limit) {
            atomicOr(&st->error, kErrTimeout);
            atomicExch(&st->abort, 1u);
            failed = true;
            break;
          }
          __nanosleep(64);
          if (!got) word = ld_word(p);
          if (!got_d) dword = ld_word(pd);
        }
        if (failed) {
          sm.abort = 1u;
        } else if (poller) {
          // each boundary cell takes the value of its latest writer; where
          // that is the block itself, the tile already holds it
          const int xp = 1 - (lane >> 4), w = lane & 15;
          const int kS = (s < 2) ? kV : kH, kO = (s < 2) ? kH : kV;
          const uint32_t data = (uint32_t)word;
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            const int pos = 4 * w + jj;
            const bool end = (pos == 0) || (pos == kUniB - 1);
            const int beat = end ? max(xp == 0 ? kO : kD, kXp) : kXp;
            if (kS > beat) tile[line_tidx(s, xp, pos)] = (uint8_t)(data >> (8 * jj));
          }
          if (lane < 2) {
            const int xs = (dl < 4) ? (dl >> 1) : 2 + ((dl - 4) >> 1);
            const int xpos = (dl & 1) ? kUniB - 1 : 0;
            if (kD > max((xs < 2) ? kV : kH, kXp))
              tile[line_tidx(xs, 1, xpos)] = (uint8_t)((uint32_t)dword >> (8 * (dpos & 3)));
          }
        }
        __syncthreads();
        if (sm.abort) {
          quit = true;
          break;
        }
        if (NT == 128)
          own_fine_phases(d, bx, by, m, tile, sm.forder, trans);
        else
          fine_phases_tile(d, bx, by, m, tile, sm.forder, trans);
        if (poller && X != a.stall_block) {
          const int part = lane >> 4, w = lane & 15;
          uint32_t bytes = 0;
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) bytes |= (uint32_t)tile[line_tidx(s, part, 4 * w + jj)] << (8 * jj);
          st_word(ob + ((size_t)X * 4 + s) * 32 + lane, ((unsigned long long)(m + 1u) << 32) | bytes);
        }
        if (((m + 1u) % a.log_every) == 0u) {
          count_pieces_uni<kUniSP, kColOff>(tile, sm.hist, d.S, k, sV, sH, sD, tid);
          if (NT == 128) count_pieces_uni<kUniSP, kColOff>(tile, sm.hist, d.S, k, sV, sH, sD, tid + 128);
          __syncthreads();
          const uint32_t ring = ((m + 1u) / a.log_every) % (uint32_t)kPendRing;
          if (tid <= d.S && sm.hist[tid]) atomicAdd(&st->acc[ring][tid], (unsigned long long)sm.hist[tid]);
          __syncthreads();
          if (tid == 0) {
            __threadfence();
            if (atomicAdd(&st->pend[ring], 1u) == nb - 1u) {
              // last block of this log point: every contribution is in acc
              __threadfence();
              unsigned long long c[kMaxStates];
              for (int v = 0; v < kMaxStates; ++v) c[v] = atomicExch(&st->acc[ring][v], 0ull);
              st->pend[ring] = 0;
              write_log_entry(st, a.lb, d.S, m + 1u, a.log_every, c, a.stop_at_extinction);
            }
          }
        }
        // the next visit's placement must not overtake this visit's record
        // reads and counts
        __syncthreads();
      }
    }
    // Edge cells that a neighbour changed after the block's last visit (a
    // vertical or horizontal neighbour visiting later in the last MCS) take
    // the value of their latest writer from that neighbour's final record
    // (epoch m_end).  Then the interiors, edge lines included, complete the
    // lattice array: every rim cell is some block's edge cell.
    if (!quit) {
      // item i: block of colour i >> 6, side (i >> 4) & 3, record word i & 15
      constexpr int kPer = 256 / NT;
      unsigned long long wv[kPer];
      const unsigned long long* wp[kPer];
      bool need[kPer];
#pragma unroll
      for (int j = 0; j < kPer; ++j) {
        const int i = tid + j * NT, c = i >> 6, s = (i >> 4) & 3;
        const int bx = 2 * gx + (c & 1), by = 2 * gy + (c >> 1);
        const int nx = (s == 2) ? (bx + P - 1) % P : (s == 3) ? (bx + 1) % P : bx;
        const int ny = (s == 0) ? (by + Py - 1) % Py : (s == 1) ? (by + 1) % Py : by;
        need[j] = slot_of(ord, (s < 2) ? c ^ 2 : c ^ 1) > slot_of(ord, c);
        wp[j] = ob + ((size_t)(ny * P + nx) * 4 + (s ^ 1)) * 32 + 16 + (i & 15);
        wv[j] = need[j] ? ld_word(wp[j]) : 0ull;
      }
      bool failed = false;
      uint32_t spins = 0;
      for (;;) {
        bool all = true;
#pragma unroll
        for (int j = 0; j < kPer; ++j) all = all && (!need[j] || (uint32_t)(wv[j] >> 32) == m_end);
        if (all) break;
        if (ld_volatile(&st->abort)) {
          failed = true;
          break;
        }
        if (++spins > a.spin_limit) {
          atomicOr(&st->error, kErrTimeout);
          atomicExch(&st->abort, 1u);
          failed = true;
          break;
        }
        __nanosleep(64);
#pragma unroll
        for (int j = 0; j < kPer; ++j)
          if (need[j] && (uint32_t)(wv[j] >> 32) != m_end) wv[j] = ld_word(wp[j]);
      }
      if (!failed) {
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
          if (!need[j]) continue;
          const int i = tid + j * NT, c = i >> 6, s = (i >> 4) & 3, w = i & 15;
          const int kX = slot_of(ord, c), kS = slot_of(ord, (s < 2) ? c ^ 2 : c ^ 1);
          const int kO = slot_of(ord, (s < 2) ? c ^ 1 : c ^ 2);
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            const int pos = 4 * w + jj;
            const bool end = (pos == 0) || (pos == kUniB - 1);
            if (kS > (end ? max(kO, kX) : kX))
              sm.tile[c][line_tidx(s, 0, pos)] = (uint8_t)((uint32_t)wv[j] >> (8 * jj));
          }
        }
      }
      __syncthreads();
    }
    if (d.bits == 8) {
      for (int i = tid; i < 4 * kUniB * 4; i += NT) {
        const int c = i >> 8, r = (i >> 2) & (kUniB - 1), q = i & 3;
        const int x0 = (2 * gx + (c & 1)) * kUniB, y0 = (2 * gy + (c >> 1)) * kUniB;
        const uint2* src = reinterpret_cast<const uint2*>(sm.tile[c] + tidx(r, 16 * q, kUniSP));
        const uint2 u0 = src[0], u1 = src[1];
        reinterpret_cast<uint4*>(d.lat + (size_t)(y0 + r) * pitch + x0)[q] = make_uint4(u0.x, u0.y, u1.x, u1.y);
      }
    } else {
      // packed: whole groups of 4 sites (a block starts on a group boundary,
      // so no group is shared with another block)
      for (int i = tid; i < 4 * kUniB * (kUniB / 4); i += NT) {
        const int c = i >> 10, r = (i >> 4) & (kUniB - 1), k = i & 15;
        const int x0 = (2 * gx + (c & 1)) * kUniB, y0 = (2 * gy + (c >> 1)) * kUniB;
        const uint32_t v = *reinterpret_cast<const uint32_t*>(sm.tile[c] + tidx(r, 4 * k, kUniSP));
        store_group(d.lat + (size_t)(y0 + r) * pitch, x0 + 4 * k, d.bits, pack4(v, d.bits));
      }
    }
  }
  // The last CTA to leave publishes the MCS number.
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(&st->exited, 1u) == gridDim.x - 1u) {
      st->exited = 0;
      st->ticket = 0;
      if (!st->stopped && !st->abort) st->mcs = a.m_begin + a.n_mcs;
    }
  }
}

// ---------------------------------------------------------------------------
// Warp-specialised persistent kernel for the uniform geometry (64x64 blocks,
// 2x2 sub-blocks).  Warp 8 is the producer: it takes the next work item from
// the ticket counter, waits for the block's 8 neighbours, and stages the
// block + rim into one of two shared-memory tiles with a single TMA box load
// (112 x 66 bytes from (x0-16, y0-1); the wrap-around rim cells of blocks on
// the lattice edge, which the box fills with zeros, are patched afterwards
// with plain loads).  Warps 0..7 (the consumers) run the four fine colour
// phases on the other tile, write the block back, count log points and
// publish the block's epoch.  The producer's waits and copies overlap the
// consumers' arithmetic.
constexpr int kTmaSP = 112, kTmaColOff = 16, kTmaRows = kUniB + 2;
constexpr uint32_t kTmaBoxBytes = (uint32_t)(kTmaSP * kTmaRows);   // 7392
constexpr int kTmaTileStride = 7424;                               // 128-byte multiple
constexpr int kTmaConsumers = 256, kTmaThreads = kTmaConsumers + 32;
constexpr uint32_t kMbarLimit = 1u << 26;
// The consumers' wait for a staged tile suspends (hint) instead of spinning,
// bounded by about 4 s of SM clock.
constexpr uint32_t kMbarHintNs = 2000;
constexpr long long kMbarMaxCycles = 8000000000ll;
// Work items a producer holds (9 lanes poll each).  Measured at L = 3200: a
// window of 3 was slower than 1 -- dispatching a newer ready item delays the
// globally oldest one behind a whole visit and lengthens the critical path.
constexpr int kLookahead = 1;

struct TmaItem {
  uint32_t m, ord, forder, quit;
  int32_t k, bx, by, colour;
};

struct TmaSmem {
  alignas(128) uint8_t tile[2][kTmaTileStride];
  uint32_t trans[kTransWords];
  alignas(8) uint64_t full[2], empty[2], tma[2];
  TmaItem item[2];
  uint32_t hist[kMaxStates];
};

__device__ __forceinline__ int tix(int r, int c) { return tidx_u<kTmaSP, kTmaColOff>(r, c); }

__device__ __forceinline__ void tma_fail(RunState* st) {
  atomicOr(&st->error, kErrTimeout);
  atomicExch(&st->abort, 1u);
}

// Producer with a lookahead window: it holds up to kLookahead work items
// (taken from the ticket counter in schedule order) and dispatches whichever
// is ready first, oldest first among the ready ones.  An item is ready when
// its 8 neighbours (and the block itself) have completed every visit that
// precedes it in schedule order.  Progress is guaranteed: the oldest
// unfinished item of the whole launch has all its dependencies done, and
// the producer holding it dispatches it as soon as it polls it.
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ void tma_producer(const TmaArgs& a, TmaSmem& sm) {
  const PersistentArgs& p = a.p;
  const LatticeDesc& d = p.d;
  RunState* st = p.st;
  const int lane = threadIdx.x & 31;
  const int P = d.P, half = P >> 1, L = d.L, pitch = d.pitch;
  const uint32_t nb = (uint32_t)(P * P), per = nb >> 2;
  const uint64_t total = (uint64_t)p.n_mcs * nb;
  // held items: ticket (0xFFFFFFFF = empty slot) and decoded fields
  uint32_t h_t = 0xFFFFFFFFu, h_m = 0, h_ord = 0;
  int h_k = 0, h_bx = 0, h_by = 0, h_col = 0;   // lane j < kLookahead holds slot j
  bool exhausted = false, failed = false;
  for (uint32_t n = 0;; ++n) {
    const int b = (int)(n & 1u);
    const uint32_t use = n >> 1;
    // refill empty slots with new tickets
    if (!exhausted && !failed) {
      const bool want = lane < kLookahead && h_t == 0xFFFFFFFFu;
      const uint32_t need_mask = __ballot_sync(0xFFFFFFFFu, want);
      if (need_mask) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(&st->ticket, (uint32_t)__popc(need_mask));
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if (want) {
          const uint32_t t = base + (uint32_t)__popc(need_mask & ((1u << lane) - 1u));
          if ((uint64_t)t < total) {
            h_t = t;
            const uint32_t mi = t / nb, rem = t - mi * nb;
            h_m = p.m_begin + mi;
            h_k = (int)(rem / per);
            const int j = (int)(rem - (uint32_t)h_k * per);
            h_ord = colour_order(philox10_rk(make_uint4(0u, 0u, h_m, kTagOrder), d.rk).x, d.perm24);
            h_col = order_at(h_ord, h_k);
            h_bx = 2 * (j % half) + (h_col & 1);
            h_by = 2 * (j / half) + (h_col >> 1);
          }
        }
        // a ticket past the end means every later one is too
        exhausted = __any_sync(0xFFFFFFFFu, want && h_t == 0xFFFFFFFFu);
      }
    }
    const uint32_t held = __ballot_sync(0xFFFFFFFFu, lane < kLookahead && h_t != 0xFFFFFFFFu);
    bool quit = failed || held == 0u;
    // the consumers must have released this buffer
    if (!quit) {
      uint32_t ok = 1;
      if (lane == 0 && !mbar_wait(&sm.empty[b], (use & 1u) ^ 1u, kMbarLimit)) {
        tma_fail(st);
        ok = 0;
      }
      quit = __shfl_sync(0xFFFFFFFFu, ok, 0) == 0u;
    }
    // poll the held items until one is ready: lane 9j+f checks neighbour f
    // of slot j
    int pick = -1;
    if (!quit) {
      const int j = lane / 9, f = lane % 9;
      const bool mine = lane < 9 * kLookahead;
      const uint32_t jt = __shfl_sync(0xFFFFFFFFu, h_t, mine ? j : 0);
      const uint32_t jm = __shfl_sync(0xFFFFFFFFu, h_m, mine ? j : 0);
      const uint32_t jord = __shfl_sync(0xFFFFFFFFu, h_ord, mine ? j : 0);
      const int jk = __shfl_sync(0xFFFFFFFFu, h_k, mine ? j : 0);
      const int jbx = __shfl_sync(0xFFFFFFFFu, h_bx, mine ? j : 0);
      const int jby = __shfl_sync(0xFFFFFFFFu, h_by, mine ? j : 0);
      const int jcol = __shfl_sync(0xFFFFFFFFu, h_col, mine ? j : 0);
      const uint32_t* flag = p.done;
      uint32_t need = 0;
      const bool active = mine && jt != 0xFFFFFFFFu;
      if (active) {
        const int dx = f % 3 - 1, dy = f / 3 - 1;
        const int nx = (jbx + dx + P) % P, ny = (jby + dy + P) % P;
        const int ncol = jcol ^ ((dx & 1) | ((dy & 1) << 1));
        need = (f == 4) ? jm : (slot_of(jord, ncol) < jk ? jm + 1u : jm);
        flag = p.done + ny * P + nx;
      }
      for (uint32_t spins = 0;; ++spins) {
        const bool not_ready = active && ld_relaxed(flag) < need;
        const uint32_t nr = __ballot_sync(0xFFFFFFFFu, not_ready);
        // slot j is ready when it is held and none of its 9 lanes is waiting
        uint32_t best_t = 0xFFFFFFFFu;
        for (int jj = 0; jj < kLookahead; ++jj) {
          const uint32_t tj = __shfl_sync(0xFFFFFFFFu, h_t, jj);
          const bool ready = tj != 0xFFFFFFFFu && ((nr >> (9 * jj)) & 0x1FFu) == 0u;
          if (ready && tj < best_t) {
            best_t = tj;
            pick = jj;
          }
        }
        if (pick >= 0) break;
        const uint32_t ab = __shfl_sync(0xFFFFFFFFu, lane == 0 ? ld_volatile(&st->abort) : 0u, 0);
        if (ab) {   // uniform across the warp
          quit = true;
          break;
        }
        if (spins > p.spin_limit) {
          if (lane == 0) tma_fail(st);
          quit = true;
          break;
        }
        __nanosleep(32);
      }
      // acquire what the neighbours published, for the async proxy too
      __threadfence();
      fence_proxy_async_global();
    }
    if (quit) {
      failed = true;
      if (lane == 0) sm.item[b].quit = 1;
      __syncwarp();
      mbar_arrive(&sm.full[b]);
      break;
    }
    const uint32_t m = __shfl_sync(0xFFFFFFFFu, h_m, pick);
    const uint32_t ord = __shfl_sync(0xFFFFFFFFu, h_ord, pick);
    const int k = __shfl_sync(0xFFFFFFFFu, h_k, pick);
    const int bx = __shfl_sync(0xFFFFFFFFu, h_bx, pick);
    const int by = __shfl_sync(0xFFFFFFFFu, h_by, pick);
    const int colour = __shfl_sync(0xFFFFFFFFu, h_col, pick);
    if (lane == pick) h_t = 0xFFFFFFFFu;   // slot freed
    uint32_t forder = 0;
    if (lane == 1)
      forder = colour_order(philox10_rk(make_uint4(0u, (uint32_t)(by * P + bx), m, kTagFineOrder), d.rk).x, d.perm24);
    forder = __shfl_sync(0xFFFFFFFFu, forder, 1);
    const int x0 = bx * kUniB, y0 = by * kUniB;
    uint8_t* tile = sm.tile[b];
    uint32_t ok = 1;
    if (lane == 0) {
      fence_proxy_async_smem();  // the consumers' writes to this tile precede the TMA's
      mbar_arrive_expect_tx(&sm.tma[b], kTmaBoxBytes);
      tma_load_2d(tile, &a.map, x0 - kTmaColOff, y0 - 1, &sm.tma[b]);
      if (!mbar_wait(&sm.tma[b], use & 1u, kMbarLimit)) {
        tma_fail(st);
        // do not leave a copy in flight into this CTA's shared memory
        ok = mbar_wait(&sm.tma[b], use & 1u, kMbarLimit) ? 0u : 2u;
      }
    }
    ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
    if (ok == 1u) {
      // wrap-around rim cells the box filled with zeros
      if (by == 0 && lane < 4) {
        const uint4 v = __ldcg(reinterpret_cast<const uint4*>(d.lat + (size_t)(L - 1) * pitch + x0) + lane);
        *reinterpret_cast<uint4*>(tile + tix(-1, 16 * lane)) = v;
      }
      if (by == P - 1 && lane >= 4 && lane < 8) {
        const int q = lane - 4;
        const uint4 v = __ldcg(reinterpret_cast<const uint4*>(d.lat + x0) + q);
        *reinterpret_cast<uint4*>(tile + tix(kUniB, 16 * q)) = v;
      }
      if (bx == 0) {
        tile[tix(lane, -1)] = __ldcg(d.lat + (size_t)(y0 + lane) * pitch + (L - 1));
        tile[tix(lane + 32, -1)] = __ldcg(d.lat + (size_t)(y0 + lane + 32) * pitch + (L - 1));
      }
      if (bx == P - 1) {
        tile[tix(lane, kUniB)] = __ldcg(d.lat + (size_t)(y0 + lane) * pitch);
        tile[tix(lane + 32, kUniB)] = __ldcg(d.lat + (size_t)(y0 + lane + 32) * pitch);
      }
      if (lane == 0) {
        TmaItem& it = sm.item[b];
        it.m = m; it.ord = ord; it.forder = forder; it.quit = 0;
        it.k = k; it.bx = bx; it.by = by; it.colour = colour;
      }
    } else {
      failed = true;
      if (lane == 0) sm.item[b].quit = 1;
    }
    __syncwarp();
    mbar_arrive(&sm.full[b]);   // 32 arrivals complete the phase
    if (failed) break;
  }
}

__device__ void tma_consumer(const TmaArgs& a, TmaSmem& sm) {
  const PersistentArgs& p = a.p;
  const LatticeDesc& d = p.d;
  RunState* st = p.st;
  const int t = threadIdx.x, qx = t & 15, qy = t >> 4;
  const int P = d.P, L = d.L, pitch = d.pitch;
  const uint32_t nb = (uint32_t)(P * P), s1 = (uint32_t)d.S + 1u, tx = d.tx, txi = d.txi;
  const uint8_t* trans = reinterpret_cast<const uint8_t*>(sm.trans);
  for (uint32_t n = 0;; ++n) {
    const int b = (int)(n & 1u);
    const uint32_t use = n >> 1;
    if (!mbar_wait_sleep(&sm.full[b], use & 1u, kMbarHintNs, kMbarMaxCycles)) {
      if (t == 0) tma_fail(st);
      break;
    }
    const TmaItem it = sm.item[b];
    if (it.quit) break;
    uint8_t* tile = sm.tile[b];
    if (t < kMaxStates) sm.hist[t] = 0;
    const uint32_t GQ = (uint32_t)d.GQ;
    const uint32_t g00 = (uint32_t)(it.by * (kUniB / 2) + 2 * qy) * GQ + (uint32_t)(it.bx * (kUniB / 2) + 2 * qx);
    const int base00 = tix(4 * qy, 4 * qx);
#pragma unroll
    for (int fi = 0; fi < 4; ++fi) {
      const uint32_t fcol = (it.forder >> (2 * fi)) & 3u, cx = fcol & 1u, cy = fcol >> 1;
      const uint32_t g = g00 + cy * GQ + cx;
      const int base = base00 + (int)(cy * (2 * kTmaSP) + 2 * cx);
      const uint4 x = philox10_rk(make_uint4(0u, g, it.m, kTagStep), d.rk);
      attempt_uni<kTmaSP>(tile, trans, x.x, base, tx, txi, s1);
      attempt_uni<kTmaSP>(tile, trans, x.y, base, tx, txi, s1);
      attempt_uni<kTmaSP>(tile, trans, x.z, base, tx, txi, s1);
      attempt_uni<kTmaSP>(tile, trans, x.w, base, tx, txi, s1);
      bar_sync_consumers(kTmaConsumers);
    }
    const bool log_point = ((it.m + 1u) % p.log_every) == 0u;
    if (log_point) {
      const int sV = slot_of(it.ord, it.colour ^ 2), sH = slot_of(it.ord, it.colour ^ 1),
                sD = slot_of(it.ord, it.colour ^ 3);
      count_visit_uni<kTmaSP, kTmaColOff>(tile, sm.hist, d.S, it.k, sV, sH, sD);
    }
    // write back interior and rim strips (never the corners)
    const int x0 = it.bx * kUniB, y0 = it.by * kUniB;
    {
      const int r = t >> 2, q = t & 3;
      const uint4 v = *reinterpret_cast<const uint4*>(tile + tix(r, 16 * q));
      reinterpret_cast<uint4*>(d.lat + (size_t)(y0 + r) * pitch + x0)[q] = v;
    }
    if (t < 8) {
      const int r = (t < 4) ? -1 : kUniB, q = t & 3;
      const uint4 v = *reinterpret_cast<const uint4*>(tile + tix(r, 16 * q));
      reinterpret_cast<uint4*>(d.lat + (size_t)wrap(y0 + r, L) * pitch + x0)[q] = v;
    } else if (t >= 128) {
      const int kk = t - 128, c = (kk < 64) ? -1 : kUniB, r = kk & 63;
      d.lat[(size_t)(y0 + r) * pitch + wrap(x0 + c, L)] = tile[tix(r, c)];
    }
    bar_sync_consumers(kTmaConsumers);
    if (log_point) {
      const uint32_t ring = ((it.m + 1u) / p.log_every) % (uint32_t)kPendRing;
      if (t <= d.S && sm.hist[t]) atomicAdd(&st->acc[ring][t], (unsigned long long)sm.hist[t]);
      bar_sync_consumers(kTmaConsumers);
      if (t == 0) {
        __threadfence();
        if (atomicAdd(&st->pend[ring], 1u) == nb - 1u) {
          __threadfence();
          unsigned long long c[kMaxStates];
          for (int v = 0; v < kMaxStates; ++v) c[v] = atomicExch(&st->acc[ring][v], 0ull);
          st->pend[ring] = 0;
          write_log_entry(st, p.lb, d.S, it.m + 1u, p.log_every, c, p.stop_at_extinction);
        }
      }
    }
    if (t == 0) {
      if (it.by * P + it.bx != p.stall_block) {
        // release: the consumers' stores (ordered before by the named
        // barrier) become visible before the new epoch
        st_release(p.done + it.by * P + it.bx, it.m + 1u);
      }
      mbar_arrive(&sm.empty[b]);   // the tile may be refilled
    }
  }
}

__global__ void __launch_bounds__(kTmaThreads, 4) persistent_tma_kernel(const __grid_constant__ TmaArgs a) {
  __shared__ TmaSmem sm;
  RunState* st = a.p.st;
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sm.full[b], 32);
      mbar_init(&sm.empty[b], 1);
      mbar_init(&sm.tma[b], 1);
    }
    fence_mbar_init();
  }
  load_trans(a.p.d, sm.trans);
  __syncthreads();
  if (!ld_volatile(&st->stopped)) {
    if (tid >= kTmaConsumers)
      tma_producer(a, sm);
    else
      tma_consumer(a, sm);
  }
  __syncthreads();
  // The last CTA to leave publishes the MCS number and resets the
  // dispensers for the next launch on this stream.
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(&st->exited, 1u) == gridDim.x - 1u) {
      st->exited = 0;
      st->ticket = 0;
      if (!st->stopped && !st->abort) st->mcs = a.p.m_begin + a.p.n_mcs;
    }
  }
}

// ---------------------------------------------------------------------------
// Whole-lattice residency (escg_resident.cuh): one CTA holds the lattice in
// shared memory for the whole launch; counts of log points and the MCS
// number are written in-kernel.
constexpr int kResThreads = 1024;
__global__ void __launch_bounds__(kResThreads) resident_kernel(PersistentArgs a) {
  extern __shared__ __align__(16) uint8_t res_dyn[];
  __shared__ ResidentSmem rs;
  const LatticeDesc& d = a.d;
  RunState* st = a.st;
  if (ld_volatile(&st->stopped)) return;
  const int sp = resident_pitch(d.L);
  uint8_t* img = res_dyn;
  uint8_t* snap = res_dyn + (d.H + 2) * sp;
  load_trans(d, rs.trans);
  resident_load(d, img, sp);
  __syncthreads();
  const uint32_t m_end = a.m_begin + a.n_mcs;
  resident_run(d, img, sp, snap, rs, a.m_begin, m_end, a.log_every, [&](uint32_t mm, const uint32_t* hist) {
    unsigned long long c[kMaxStates];
    for (int v = 0; v < kMaxStates; ++v) c[v] = hist[v];
    write_log_entry(st, a.lb, d.S, mm, a.log_every, c, a.stop_at_extinction);
    return st->stopped != 0u;
  });
  resident_store(d, img, sp);
  if (threadIdx.x == 0 && !st->stopped) st->mcs = m_end;
}

// Largest dynamic shared memory a resident launch may use on this device.
int resident_max_dyn_bytes(int device) {
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  return optin - (int)sizeof(ResidentSmem) - 256;
}

bool resident_fits(const LatticeDesc& d, int device) {
  return d.P <= 8 && d.Py <= 8 && resident_dyn_bytes(d.L, d.H) <= resident_max_dyn_bytes(device);
}

cudaError_t launch_resident(const PersistentArgs& a, cudaStream_t stream) {
  const int bytes = resident_dyn_bytes(a.d.L, a.d.H);
  cudaError_t e = cudaFuncSetAttribute(resident_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  resident_kernel<<<1, kResThreads, bytes, stream>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
static inline int blocks_for(size_t n, int threads, int cap) {
  size_t b = (n + threads - 1) / threads;
  if (b > (size_t)cap) b = cap;
  return b < 1 ? 1 : (int)b;
}

cudaError_t launch_init(const LatticeDesc& d, uint64_t T_empty, cudaStream_t stream) {
  const size_t n = (size_t)d.H * (d.pitch * 2 / d.bits);
  init_kernel<<<blocks_for(n, 256, 152 * 32), 256, 0, stream>>>(d, T_empty);
  return cudaGetLastError();
}

cudaError_t launch_pack(const LatticeDesc& d, const uint8_t* bytes, int byte_pitch, cudaStream_t stream) {
  const size_t n = (size_t)d.H * ((d.L + 3) / 4);
  pack_kernel<<<blocks_for(n, 256, 152 * 8), 256, 0, stream>>>(d, bytes, byte_pitch);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const LatticeDesc& d, uint8_t* bytes, int byte_pitch, cudaStream_t stream) {
  const size_t n = (size_t)d.H * ((d.L + 3) / 4);
  unpack_kernel<<<blocks_for(n, 256, 152 * 8), 256, 0, stream>>>(d, bytes, byte_pitch);
  return cudaGetLastError();
}

cudaError_t launch_fill_u32(uint32_t* p, int n, uint32_t value, cudaStream_t stream) {
  fill_u32_kernel<<<blocks_for((size_t)n, 256, 152 * 4), 256, 0, stream>>>(p, n, value);
  return cudaGetLastError();
}

cudaError_t launch_validate(const LatticeDesc& d, uint32_t* bad, uint32_t flag, uint32_t* stop,
                            cudaStream_t stream) {
  const size_t n = (size_t)d.H * ((d.L + 15) / 16);
  validate_kernel<<<blocks_for(n, 256, 152 * 8), 256, 0, stream>>>(d, bad, flag, stop);
  return cudaGetLastError();
}

cudaError_t launch_state_reset(RunState* st, uint32_t mcs, uint32_t log_num0, cudaStream_t stream) {
  state_reset_kernel<<<1, 256, 0, stream>>>(st, mcs, log_num0);
  return cudaGetLastError();
}

cudaError_t launch_count(const LatticeDesc& d, RunState* st, cudaStream_t stream) {
  const size_t n = (size_t)d.H * ((d.L + 15) / 16);
  count_kernel<<<blocks_for(n, 256 * 4, 152 * 4), 256, 0, stream>>>(d, st);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const LatticeDesc& d, RunState* st, LogBuffers lb, uint32_t m_end,
                            uint32_t log_every, int log, int stop_at_extinction, cudaStream_t stream,
                            uint64_t check_total) {
  finalize_kernel<<<1, 1, 0, stream>>>(st, d.S, lb, m_end, log_every, log, stop_at_extinction,
                                       (unsigned long long)check_total);
  return cudaGetLastError();
}

cudaError_t launch_phase(const LatticeDesc& d, RunState* st, uint32_t m, int slot, cudaStream_t stream) {
  const int nblocks = (d.P * d.Py) / 4;
  phase_kernel<<<nblocks, 256, 0, stream>>>(d, st, m, slot);
  return cudaGetLastError();
}

cudaError_t launch_persistent_tma(const TmaArgs& a, int grid, cudaStream_t stream) {
  persistent_tma_kernel<<<grid, kTmaThreads, 0, stream>>>(a);
  return cudaGetLastError();
}

int persistent_tma_grid(int device) {
  int sms = 0, per_sm = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_tma_kernel, kTmaThreads, 0);
  if (per_sm < 1) per_sm = 1;
  return sms * per_sm;
}

cudaError_t launch_persistent(const PersistentArgs& args, int grid, cudaStream_t stream) {
  PersistentArgs a = args;
  const uint32_t nb = (uint32_t)(a.d.P * a.d.Py);
  a.rcp_nb = div_rcp32(nb);
  a.rcp_per = div_rcp32(nb >> 2);
  a.rcp_half = div_rcp32((uint32_t)(a.d.P >> 1));
  if (a.d.uniform_var) {
    const int var = (a.d.nbh == 8 ? 2 : 0) | (a.d.reflect ? 1 : 0);
    if (var == 1)
      persistent_kernel<true, false, kPersistentThreads, 1><<<grid, kPersistentThreads, 0, stream>>>(a);
    else if (var == 2)
      persistent_kernel<true, false, kPersistentThreads, 2><<<grid, kPersistentThreads, 0, stream>>>(a);
    else
      persistent_kernel<true, false, kPersistentThreads, 3><<<grid, kPersistentThreads, 0, stream>>>(a);
  } else if (a.threads == 128 && a.d.uniform64 && a.d.bits == 8)
    persistent_kernel<true, false, 128><<<grid, 128, 0, stream>>>(a);
  else if (a.threads == 128 && a.d.uniform64)
    persistent_kernel<true, true, 128><<<grid, 128, 0, stream>>>(a);
  else if (a.d.uniform64 && a.d.bits != 8)
    persistent_kernel<true, true><<<grid, kPersistentThreads, 0, stream>>>(a);
  else if (a.d.uniform64)
    persistent_kernel<true, false><<<grid, kPersistentThreads, 0, stream>>>(a);
  else if (a.d.bits != 8)
    persistent_kernel<false, true><<<grid, kPersistentThreads, 0, stream>>>(a);
  else
    persistent_kernel<false, false><<<grid, kPersistentThreads, 0, stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_persistent_ll(const PersistentArgs& a, int grid, cudaStream_t stream) {
  persistent_ll_kernel<<<grid, kLLThreads, 0, stream>>>(a);
  return cudaGetLastError();
}

int persistent_ll_grid(int device) {
  int sms = 0, per_sm = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_ll_kernel, kLLThreads, 0);
  if (per_sm > kLLMinBlocks) per_sm = kLLMinBlocks;
  if (per_sm < 1) per_sm = 1;
  return sms * per_sm;
}

// Shared-memory padding for NT-thread owner CTAs so that an SM holds at
// most per_sm of them (and at least per_sm fit), or -1.
template <int NT>
static int own_padding(int per_sm, int smem_sm, int reserved, int optin) {
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, persistent_own_kernel<NT>) != cudaSuccess) return -1;
  const int stat = (int)fa.sharedSizeBytes;
  if (optin - stat <= 0 ||
      cudaFuncSetAttribute(persistent_own_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - stat) !=
          cudaSuccess)
    return -1;
  int dyn = smem_sm / per_sm - reserved - stat - 256;
  if (dyn > optin - stat) dyn = optin - stat;
  for (dyn = dyn > 0 ? dyn & ~127 : 0;; dyn -= 1024) {
    if (dyn < 0) dyn = 0;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, persistent_own_kernel<NT>, NT, (size_t)dyn) !=
        cudaSuccess)
      return -1;
    if (occ >= per_sm) return dyn;
    if (dyn == 0) return -1;   // the grid cannot be resident at once
  }
}

int persistent_own_config(const LatticeDesc& d, int device, int* dyn_bytes, int* threads, int* ctas_per_sm,
                          int min_per_sm) {
  const int groups = (d.P / 2) * (d.Py / 2);
  int sms = 0, smem_sm = 0, reserved = 0, optin = 0, coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device);
  if (!coop) return 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, device);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  if (sms <= 0) return 0;
  // the padding spreads the grid over all SMs: at most ceil(groups / SMs)
  // CTAs per SM
  int per_sm = (groups + sms - 1) / sms;
  if (per_sm < min_per_sm) per_sm = min_per_sm;
  // 256 threads while 4 fit an SM (54 registers); beyond, 128 (a 256-thread
  // build for 5 per SM, held to 48 registers, was measured slower)
  const int nt = per_sm <= 4 ? 256 : 128;
  const int dyn = nt == 256 ? own_padding<256>(per_sm, smem_sm, reserved, optin)
                            : own_padding<128>(per_sm, smem_sm, reserved, optin);
  if (dyn < 0) return 0;
  *dyn_bytes = dyn;
  *threads = nt;
  *ctas_per_sm = per_sm;
  return groups;
}

// A cooperative launch: the runtime starts the grid only with every CTA
// resident, also while kernels of other streams hold part of the device.
cudaError_t launch_persistent_own(const PersistentArgs& a, int dyn_bytes, int threads, cudaStream_t stream) {
  const int groups = (a.d.P / 2) * (a.d.Py / 2);
  PersistentArgs arg = a;
  void* params[] = {&arg};
  const void* fn = threads == 256 ? reinterpret_cast<const void*>(&persistent_own_kernel<256>)
                                  : reinterpret_cast<const void*>(&persistent_own_kernel<128>);
  return cudaLaunchCooperativeKernel(fn, dim3(groups), dim3(threads), params, (size_t)dyn_bytes, stream);
}

cudaError_t launch_ll_merge(const LatticeDesc& d, const unsigned long long* ob, const RunState* st,
                            uint32_t m_end, cudaStream_t stream) {
  // coarse order of MCS m_end - 1, as the device draws it
  const uint32_t x = philox10(make_uint4(0u, 0u, m_end - 1u, kTagOrder), d.key0, d.key1).x;
  const uint32_t ord = d.perm24[(uint32_t)(((uint64_t)x * 24u) >> 32)];
  ll_merge_kernel<<<d.P * d.P, 256, 0, stream>>>(d, ob, st, m_end, ord);
  return cudaGetLastError();
}

int persistent_grid128(int device) {
  int sms = 0, per_sm = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  // the same grid for one byte and for 2 or 4 bits per site: the fewer CTAs
  // of the two builds that an SM holds
  int per_sm_packed = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_kernel<true, false, 128>, 128, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_packed, persistent_kernel<true, true, 128>, 128, 0);
  if (per_sm_packed < per_sm) per_sm = per_sm_packed;
  if (per_sm > 8) per_sm = 8;
  if (per_sm < 1) per_sm = 1;
  return sms * per_sm;
}

int persistent_grid(int device, bool uniform) {
  int sms = 0, per_sm = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (uniform) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_kernel<true>, kPersistentThreads, 0);
    if (per_sm > kUniLaunchPerSM) per_sm = kUniLaunchPerSM;
  } else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_kernel<false>, kPersistentThreads, 0);
  if (per_sm < 1) per_sm = 1;
  return sms * per_sm;
}

}  // namespace escg_impl
