// escg_owner.cu -- block owners on any schedule-v1 partition of the von
// Neumann rule: L or H not a multiple of 128, rectangles, a periodic or a
// reflecting boundary, one byte per site or packed.
//
// The design of persistent_own_kernel (escg_kernels.cu) for the generic
// geometry: CTA g owns coarse group g -- the 2x2 blocks (2 gx + cx,
// 2 gy + cy), one of each colour -- for a whole cooperative launch and keeps
// their four tiles (interior and rim lines) in shared memory.  A visit polls
// the boundary records of its edge neighbours and the diagonal neighbours'
// rim-end words, places each boundary cell from its latest writer, runs the
// four fine colour phases and publishes its own records.  The lattice array is
// read when the launch starts and written when it ends, after each block's
// edge cells are settled from the final records of the neighbours that
// visited after it.  Same schedule (Alg. 3 steps in the order of schedule
// version 1), same results.
//
// What the generic geometry adds:
//  * Lines of any length: a block is bw x bh sites (48..96), its top and
//    bottom lines have bw cells, its left and right lines bh; a record line
//    has kGLineWords word slots of 4 cells each.
//  * Random words drawn ahead.  Philox depends on (seed, sub-block, MCS,
//    attempt) only, not on the lattice, so a visit draws every word of its
//    four fine phases into shared memory while its record polls are in
//    flight, and each thread moves its sub-block's words into registers
//    before stepping it.  A fine phase then holds only the dependent chain of
//    its longest sub-block's attempts (9 for a 3 x 3 sub-block).
//  * Quads handed out all-2 x 2 first (the batch kernel's order), so that the
//    warps whose lanes step only 4 attempts per phase are not held to the 6
//    or 9 of a lane at the block's leading rows or columns.
//  * Each owned block's geometry and neighbour ids worked out once per
//    launch (no divisions in a visit).
//  * A reflecting boundary: a side on the lattice edge has no neighbour;
//    nothing is polled or placed across it, and no diagonal block writes a
//    rim end beyond it.
//
// Record layout: ob[(block * 4 + side) * 2 kGLineWords + part * kGLineWords
// + w]; side 0 top, 1 bottom, 2 left, 3 right; part 0 the block's edge line,
// 1 the rim line beyond it; word w: 4 lattice bytes (positions 4w..4w+3
// along the side, byte j = position 4w + j) in the low half and the epoch of
// the visit that wrote them (MCS + 1) in the high half, written with one
// single-copy-atomic 64-bit store.
#include "escg_device.cuh"
#include "escg_internal.h"
#include "escg_rule8.cuh"
#include "escg_sync.cuh"

namespace escg_impl {

constexpr int kGLineWords = 32;         // word slots per record line (a line of 96 cells uses 24)
static_assert(kGRecordWords == 4 * 2 * kGLineWords, "record layout");
constexpr int kGSlots = 9;              // attempts of the largest sub-block (3 x 3)


// Geometry of one coarse block's visit.
struct GBlock {
  BlockSpan X, Y;
  int sp;          // tile pitch
  int hx, nq;      // quads per row, quads
  uint32_t inv_hx;
  QuadMap qm;      // quad order: the all-2 x 2 quads first
};

__device__ __forceinline__ GBlock gblock(const LatticeDesc& d, int bx, int by) {
  GBlock b;
  b.X = block_span(d.ax, bx);
  b.Y = block_span(d.ay, by);
  b.sp = tile_pitch(b.X.w);
  b.hx = b.X.Q >> 1;
  b.nq = b.hx * (b.Y.Q >> 1);
  b.inv_hx = (65536u + (uint32_t)b.hx - 1u) / (uint32_t)b.hx;
  b.qm = quad_map(b.X, b.Y);
  return b;
}

// One owned block, worked out once per launch: its geometry, block id, the
// ids of its 4 edge neighbours (side 0 top, 1 bottom, 2 left, 3 right) and
// 4 diagonal neighbours (0 up-left, 1 up-right, 2 down-left, 3 down-right),
// the heights of the block rows above and below and the widths of the block
// columns left and right (the rim-end positions in the diagonals' records),
// and which sides have a neighbour (all, unless the boundary reflects).
struct GColour {
  GBlock g;
  int32_t id;
  int32_t nbr[4];
  int32_t diag[4];
  int32_t h_up, h_down, w_left, w_right;
  int32_t ex[4];
};

__device__ __forceinline__ void gcolour_init(const LatticeDesc& d, int bx, int by, GColour& c) {
  const int P = d.P, Py = d.Py;
  const int xl = bx == 0 ? P - 1 : bx - 1, xr = bx == P - 1 ? 0 : bx + 1;
  const int yu = by == 0 ? Py - 1 : by - 1, yd = by == Py - 1 ? 0 : by + 1;
  c.g = gblock(d, bx, by);
  c.id = by * P + bx;
  c.nbr[0] = yu * P + bx;
  c.nbr[1] = yd * P + bx;
  c.nbr[2] = by * P + xl;
  c.nbr[3] = by * P + xr;
  c.diag[0] = yu * P + xl;
  c.diag[1] = yu * P + xr;
  c.diag[2] = yd * P + xl;
  c.diag[3] = yd * P + xr;
  c.h_up = block_span(d.ay, yu).w;
  c.h_down = block_span(d.ay, yd).w;
  c.w_left = block_span(d.ax, xl).w;
  c.w_right = block_span(d.ax, xr).w;
  const bool refl = d.reflect != 0;
  c.ex[0] = !refl || by > 0;
  c.ex[1] = !refl || by < Py - 1;
  c.ex[2] = !refl || bx > 0;
  c.ex[3] = !refl || bx < P - 1;
}

// Tile index of position pos of line (side, part) of a bw x bh block.
__device__ __forceinline__ int gline_tidx(int s, int part, int pos, int bw, int bh, int sp) {
  const int n = (s < 2) ? bh : bw;   // extent across the line
  const int fixed = (s & 1) ? (part ? n : n - 1) : (part ? -1 : 0);
  return (s < 2) ? tidx(fixed, pos, sp) : tidx(pos, fixed, sp);
}

struct GownSmem {
  GColour col[4];    // the owned block of each colour
  uint32_t trans[kTransWords];
  uint2 trans2[kTransPairs];   // the same table, one 8-byte entry per pair (rule8)
  uint32_t hist[kMaxStates];
  uint32_t forder;   // fine order of the current visit
  uint32_t abort;
};

// The block's tile as the lattice array holds it: interior, top and bottom
// rim rows, left and right rim columns (not the corners; nothing beyond a
// reflecting edge).
template <int NT>
__device__ __forceinline__ void gown_stage(const LatticeDesc& d, uint8_t* tile, const GBlock& g) {
  const int x0 = g.X.s0, bw = g.X.w, y0 = g.Y.s0, bh = g.Y.w, sp = g.sp;
  if (d.bits == 8) {
    load_tile_generic<false>(d, x0, y0, bw, bh, tile, sp, nullptr);
    return;
  }
  const int cols = bw + 2, n = (bh + 2) * cols;
  for (int i = threadIdx.x; i < n; i += NT) {
    const int r = i / cols - 1, c = i % cols - 1;
    if ((r < 0 || r >= bh) && (c < 0 || c >= bw)) continue;   // corner
    const int gy = tile_row_gy(d, y0, r);
    int gx = x0 + c;
    if (gx < 0 || gx >= d.L) {
      if (d.reflect) continue;
      gx = gx < 0 ? gx + d.L : gx - d.L;
    }
    if (gy < 0) continue;
    const uint32_t raw = load_group(d.lat + (size_t)gy * d.pitch, gx & ~3, d.bits);
    tile[(r + 1) * sp + kColOff + c] = (uint8_t)(unpack4(raw, d.bits) >> (8 * (gx & 3)));
  }
}

// Every Philox word of the visit of block g in MCS m, by quad and fine
// colour: W[(colour * kGSlots + t) * NT + q] is the word of attempt t of the
// quad's sub-block of that colour (t < its cell count).  Thread i (of NT
// drawing threads, i = t here) draws the words of colour i mod 4 for the
// quads i/4 + k NT/4, k = 0..3: the sub-blocks
// with 3 x 3 cells (three Philox calls) sit at the block's leading corner,
// and this spreads them over different threads, each with four independent
// draws in flight.
template <int NT>
__device__ __forceinline__ void gown_words(const LatticeDesc& d, const GBlock& g, uint32_t m,
                                           uint32_t* __restrict__ W, int t) {
  const int c = t & 3;
  uint32_t gid[4];
  int nk[4], q[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    q[k] = (t >> 2) + k * (NT / 4);
    int qx, qy;
    quad_at(g.qm, q[k] < g.nq ? q[k] : 0, qx, qy);
    const int fx = 2 * qx + (c & 1), fy = 2 * qy + (c >> 1);
    nk[k] = q[k] < g.nq ? seg_width(g.X, fx) * seg_width(g.Y, fy) : 0;
    gid[k] = (uint32_t)(g.Y.f0 + fy) * (uint32_t)d.GQ + (uint32_t)(g.X.f0 + fx);
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (4 * j < nk[k]) {
        const uint4 x = philox10_rk(make_uint4((uint32_t)j, gid[k], m, kTagStep), d.rk);
        uint32_t* w = W + (c * kGSlots + 4 * j) * NT + q[k];
        w[0] = x.x;
        if (4 * j + 1 < nk[k]) w[NT] = x.y;
        if (4 * j + 2 < nk[k]) w[2 * NT] = x.z;
        if (4 * j + 3 < nk[k]) w[3 * NT] = x.w;
      }
    }
  }
}

// The four fine colour phases of a visit from the drawn words (fine order
// ord), run by threads 0 .. NT - 1, each ending with a barrier: the CTA's
// (BAR = false) or named barrier 1 over those NT threads (BAR = true).
template <int NT, bool REFLECT, bool BAR = false>
__device__ __forceinline__ void gown_fine_phases(const LatticeDesc& d, const GBlock& g, uint8_t* tile,
                                                 uint32_t ord, const uint8_t* trans, const uint2* t2,
                                                 const uint32_t* __restrict__ W) {
  const uint32_t s1 = (uint32_t)d.S + 1u, tx = d.tx, txi = d.txi;
  const int sp = g.sp;
#pragma unroll 1
  for (int fi = 0; fi < 4; ++fi) {
    const int fcol = order_at(ord, fi), cx = fcol & 1, cy = fcol >> 1;
    for (int q = threadIdx.x; q < g.nq; q += NT) {
      int qx, qy;
      quad_at(g.qm, q, qx, qy);
      const int fx = 2 * qx + cx, fy = 2 * qy + cy;
      const int sx = seg_start(g.X, fx), sy = seg_start(g.Y, fy);
      const int base = tidx(sy, sx, sp);
      // the sub-block's words into registers first: the tile stores of one
      // attempt must not hold up the word loads of the next
      const uint32_t* __restrict__ w = W + (fcol * kGSlots) * NT + q;
      const int wx = seg_width(g.X, fx), wy = seg_width(g.Y, fy);
      const uint32_t nk = (uint32_t)(wx * wy), n4 = 4u * nk;
      const uint32_t inv_wx = wx == 2 ? 32768u : 21846u;   // ceil(65536 / wx), widths 2 and 3
      uint32_t wv[kGSlots];
#pragma unroll
      for (int t = 0; t < kGSlots; ++t) wv[t] = (uint32_t)t < nk ? w[t * NT] : 0u;
      if (REFLECT) {
#pragma unroll
        for (int t = 0; t < kGSlots; ++t)
          if ((uint32_t)t < nk)
            attempt_variant(tile, trans, wv[t], n4, 2, base, wx, inv_wx, sp, tx, txi, s1, true,
                            g.Y.s0 + sy, g.X.s0 + sx, d.H, d.L);
      } else {
        attempts8_ahead<kGSlots>(tile, t2, wv, nk, n4, base, wx, inv_wx, sp, tx, txi, s1);
      }
    }
    if (BAR)
      asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
    else
      __syncthreads();
  }
}

// Writes the interior of a block to the lattice array: whole groups of 4
// sites where the block holds all four; at the row ends the block's sites
// only.  One byte per site: single bytes.  Packed: every group whose 32-bit
// word also holds sites of the horizontally adjacent block (whose owner may
// write them at the same time) is merged in with an atomic clear and set of
// the block's bits, so that no plain store and atomic meet on one word.
template <int NT>
__device__ __forceinline__ void gown_store(const LatticeDesc& d, const uint8_t* tile, const GBlock& g) {
  const int x0 = g.X.s0, bw = g.X.w, y0 = g.Y.s0, bh = g.Y.w, sp = g.sp, bits = d.bits;
  const int g0 = x0 >> 2, ng = ((x0 + bw - 1) >> 2) - g0 + 1;
  for (int i = threadIdx.x; i < bh * ng; i += NT) {
    const int r = i / ng, c0 = 4 * (g0 + i % ng);
    uint8_t* row = d.lat + (size_t)(y0 + r) * d.pitch;
    const uint8_t* src = tile + (r + 1) * sp + kColOff + (c0 - x0);
    uint32_t mask = 0, v = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (c0 + e >= x0 && c0 + e < x0 + bw) {
        mask |= 1u << e;
        v |= (uint32_t)src[e] << (8 * e);
      }
    if (bits == 8) {
      if (mask == 0xFu) {
        *reinterpret_cast<uint32_t*>(row + c0) = v;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if ((mask >> e) & 1u) row[c0 + e] = (uint8_t)(v >> (8 * e));
      }
      continue;
    }
    const int goff = (c0 * bits) >> 3;                  // byte offset of the group in the row
    const int ws0 = ((goff & ~3) << 3) / bits;          // first site of its 32-bit word
    const bool shared = ws0 < x0 || ws0 + 32 / bits > x0 + bw;
    if (!shared) {
      store_group(row, c0, bits, pack4(v, bits));
    } else {
      uint32_t* word = reinterpret_cast<uint32_t*>(row + (goff & ~3));
      const int sh = 8 * (goff & 3);
      uint32_t mb = 0;
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if ((mask >> e) & 1u) mb |= ((1u << bits) - 1u) << (e * bits);
      atomicAnd(word, ~(mb << sh));
      atomicOr(word, (pack4(v, bits) & mb) << sh);
    }
  }
}

// PREF (512 threads, blocks of at most 256 quads): threads 0..255 run the
// fine phases, synchronised by named barrier 1 (executed by exactly those
// 256 threads -- warps 0..7 -- four times per visit, so its count of 256
// always completes), while threads 256..511 draw the next visit's words
// into the other half of a double buffer; a CTA barrier joins them after
// the fine phases.  The first visit of a launch draws its own words.
template <int NT, bool REFLECT, bool PREF>
__global__ void __launch_bounds__(NT, NT == 256 ? 3 : 1) persistent_gown_kernel(const __grid_constant__ GownArgs ga) {
  static_assert(!PREF || NT == 512, "word prefetch: 512-thread CTAs");
  constexpr int kHalf = NT / 2;   // PREF: the fine-phase threads and the drawing threads
  extern __shared__ __align__(16) uint8_t gdyn[];
  __shared__ GownSmem sm;
  const PersistentArgs& a = ga.p;
  const LatticeDesc& d = a.d;
  RunState* st = a.st;
  unsigned long long* ob = a.ob;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tstride = ga.tile_stride;
  uint32_t* W = reinterpret_cast<uint32_t*>(gdyn + 4 * tstride);
  // PREF: the double buffer, half b at W + b * 4 * kGSlots * kHalf
  auto Wb = [W](uint32_t b) { return W + (b & 1u) * (uint32_t)(4 * kGSlots * kHalf); };
  constexpr int kLW = kGLineWords;
  const bool run = !ld_volatile(&st->stopped);
  if (run) {
    load_trans(d, sm.trans);
    fill_trans8(sm.trans2, d.trans, d.S, tid, NT);
    const int P = d.P, half = P >> 1;
    const uint32_t nb = (uint32_t)(P * d.Py);
    const int gx = (int)blockIdx.x % half, gy = (int)blockIdx.x / half;
    if (tid < 4) gcolour_init(d, 2 * gx + (tid & 1), 2 * gy + (tid >> 1), sm.col[tid]);
    if (tid == 0) sm.abort = 0;
    __syncthreads();
    for (int c = 0; c < 4; ++c) gown_stage<NT>(d, gdyn + c * tstride, sm.col[c].g);
    const uint8_t* trans = reinterpret_cast<const uint8_t*>(sm.trans);
    const uint32_t m_end = a.m_begin + a.n_mcs;
    uint32_t ordp = colour_order(philox10(make_uint4(0u, 0u, a.m_begin - 1u, kTagOrder), d.key0, d.key1).x,
                                 d.perm24);
    uint32_t ord = colour_order(philox10(make_uint4(0u, 0u, a.m_begin, kTagOrder), d.key0, d.key1).x, d.perm24);
    uint32_t ord_next = colour_order(philox10(make_uint4(0u, 0u, a.m_begin + 1u, kTagOrder), d.key0, d.key1).x,
                                     d.perm24);
    // the polling role of this thread: warp w < 8 polls side s = w & 3, part
    // w >> 2 of the edge neighbour's record of the opposite side (one word per
    // lane); lanes 24 and 25 of warps 0..3 also a diagonal neighbour's
    // rim-end word, dl = 2 s + (lane & 1): dl 0..3 the ends of the top and
    // bottom rim rows, 4..7 those of the left and right rim columns
    const bool poller = warp < 8;
    const int s = warp & 3, part = (warp >> 2) & 1;
    const int dl = 2 * s + (lane & 1);
    const int ddx = (dl == 0 || dl == 2 || dl == 4 || dl == 5) ? -1 : 1;
    const int ddy = (dl == 0 || dl == 1 || dl == 4 || dl == 6) ? -1 : 1;
    const int oside = (dl < 4) ? (ddx < 0 ? 2 : 3) : (ddy < 0 ? 0 : 1);
    const int dq = (ddy > 0 ? 2 : 0) + (ddx > 0 ? 1 : 0);            // diagonal index
    const int drec = (dl < 4) ? (ddx < 0 ? 3 : 2) : (ddy < 0 ? 1 : 0);  // its record side
    const bool isd = poller && part == 0 && (lane == 24 || lane == 25);
    const int o0 = (s < 2) ? 2 : 0, o1 = (s < 2) ? 3 : 1;   // other-axis sides at the two line ends
    bool quit = false;
    uint32_t v = 0;   // visits so far in this launch
    if (PREF && tid < kHalf) gown_words<kHalf>(d, sm.col[order_at(ord, 0)].g, a.m_begin, Wb(0u), tid);
    for (uint32_t m = a.m_begin; m < m_end && !quit; ++m) {
      if (m != a.m_begin) {
        ordp = ord;
        ord = ord_next;
        ord_next = colour_order(philox10(make_uint4(0u, 0u, m + 1u, kTagOrder), d.key0, d.key1).x, d.perm24);
      }
      for (int k = 0; k < 4; ++k) {
        if (tid < kMaxStates) sm.hist[tid] = 0;
        const int colour = order_at(ord, k);
        const GColour& C = sm.col[colour];
        // a register copy: tile stores (bytes) could otherwise alias it and
        // force reloads inside the fine phases
        const GBlock g = C.g;
        const int bw = g.X.w, bh = g.Y.w, sp = g.sp;
        uint8_t* tile = gdyn + colour * tstride;
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
        const int len = (s < 2) ? bw : bh, nwd = (len + 3) >> 2;
        const bool exs = C.ex[s] != 0;
        const uint32_t e = (s < 2) ? eV : eH;
        const unsigned long long* p = ob + ((size_t)C.nbr[s] * 4 + (s ^ 1)) * (2 * kLW) + part * kLW + lane;
        const bool dex = exs && C.ex[oside] != 0;
        const int dpos = (dl < 4) ? (ddy < 0 ? C.h_up - 1 : 0) : (ddx < 0 ? C.w_left - 1 : 0);
        const unsigned long long* pd = ob + ((size_t)C.diag[dq] * 4 + drec) * (2 * kLW) + kLW + (dpos >> 2);
        const bool skip_s = first && ((s < 2) ? sV : sH) > k;   // that neighbour has not visited yet
        bool got = !poller || !exs || lane >= nwd || skip_s;
        bool got_d = !isd || !dex || (first && sD > k);
        unsigned long long word = 0, dword = 0;
        if (!got) word = ld_word(p);
        if (!got_d) dword = ld_word(pd);
        // while those loads are in flight: every random word and the fine
        // order of this visit (the words of the previous visit are no longer
        // read: its last fine phase ended with a barrier)
        if (!PREF) gown_words<NT>(d, g, m, W, tid);
        if (tid == NT - 1) sm.forder = fine_order(d, 2 * gx + (colour & 1), 2 * gy + (colour >> 1), m);
        bool failed = false;
        uint32_t spins = 0;
        for (;;) {
          if (!got) got = (uint32_t)(word >> 32) == e;
          if (!got_d) got_d = (uint32_t)(dword >> 32) == eD;
          if (got && got_d) break;
          // the abort flag every 16th round: a read of it in every round would
          // put a second L2 round trip between two polls
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
        } else if (poller && exs) {
          // each boundary cell takes the value of its latest writer; where
          // that is the block itself, the tile already holds it
          const int xp = 1 - part;
          const int kS = (s < 2) ? kV : kH, kO = (s < 2) ? kH : kV;
          if (lane < nwd && !skip_s) {
            const uint32_t data = (uint32_t)word;
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
              const int pos = 4 * lane + jj;
              if (pos >= len) break;
              int beat = kXp;
              if (pos == 0 || pos == len - 1) {
                const bool ex_o = C.ex[pos == 0 ? o0 : o1] != 0;
                beat = max(beat, ex_o ? (xp == 0 ? kO : kD) : -1);
              }
              if (kS > beat) tile[gline_tidx(s, xp, pos, bw, bh, sp)] = (uint8_t)(data >> (8 * jj));
            }
          }
          if (isd && dex && !(first && sD > k)) {
            const int xpos = (dl & 1) ? len - 1 : 0;
            if (kD > max((s < 2) ? kV : kH, kXp))
              tile[gline_tidx(s, 1, xpos, bw, bh, sp)] = (uint8_t)((uint32_t)dword >> (8 * (dpos & 3)));
          }
        }
        __syncthreads();
        if (sm.abort) {
          quit = true;
          break;
        }
        if (PREF) {
          if (tid < kHalf) {
            gown_fine_phases<kHalf, REFLECT, true>(d, g, tile, sm.forder, trans, sm.trans2, Wb(v));
          } else {
            // the next visit: slot k + 1 of this MCS, else slot 0 of the next
            const uint32_t mn = k < 3 ? m : m + 1u;
            if (mn < m_end) {
              const GBlock gn = sm.col[order_at(k < 3 ? ord : ord_next, (k + 1) & 3)].g;
              gown_words<kHalf>(d, gn, mn, Wb(v + 1u), tid - kHalf);
            }
          }
          __syncthreads();
        } else {
          gown_fine_phases<NT, REFLECT>(d, g, tile, sm.forder, trans, sm.trans2, W);
        }
        ++v;
        if (poller && exs && lane < nwd && C.id != a.stall_block) {
          uint32_t bytes = 0;
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            const int pos = 4 * lane + jj;
            if (pos < len) bytes |= (uint32_t)tile[gline_tidx(s, part, pos, bw, bh, sp)] << (8 * jj);
          }
          st_word(ob + ((size_t)C.id * 4 + s) * (2 * kLW) + part * kLW + lane,
                  ((unsigned long long)(m + 1u) << 32) | bytes);
        }
        if (a.fuse_counts && ((m + 1u) % a.log_every) == 0u) {
          count_tile_generic(tile, sp, kColOff, bw, bh, sm.hist, NT >> 5, k, sV, sH, sD);
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
        // the next visit's placement and words must not overtake this visit's
        // record reads and counts
        __syncthreads();
      }
    }
    // Edge cells that a neighbour changed after the block's last visit (a
    // vertical or horizontal neighbour visiting later in the last MCS) take
    // the value of their latest writer from that neighbour's final record
    // (epoch m_end).  Then the interiors, edge lines included, complete the
    // lattice array: every rim cell is some block's edge cell.
    if (!quit) {
      // item i: block of colour i >> 7, side (i >> 5) & 3, record word i & 31
      constexpr int kPer = 512 / NT;
      unsigned long long wv[kPer];
      const unsigned long long* wp[kPer];
      bool need[kPer];
#pragma unroll
      for (int j = 0; j < kPer; ++j) {
        const int i = tid + j * NT, c = i >> 7, si = (i >> 5) & 3, w = i & 31;
        const GColour& C = sm.col[c];
        const int len = (si < 2) ? C.g.X.w : C.g.Y.w;
        need[j] = 4 * w < len && C.ex[si] != 0 && slot_of(ord, (si < 2) ? c ^ 2 : c ^ 1) > slot_of(ord, c);
        wp[j] = ob + ((size_t)C.nbr[si] * 4 + (si ^ 1)) * (2 * kLW) + kLW + w;
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
          const int i = tid + j * NT, c = i >> 7, si = (i >> 5) & 3, w = i & 31;
          const GColour& C = sm.col[c];
          const int bw = C.g.X.w, bh = C.g.Y.w;
          const int len = (si < 2) ? bw : bh;
          const int kX = slot_of(ord, c), kS = slot_of(ord, (si < 2) ? c ^ 2 : c ^ 1);
          const int kO = slot_of(ord, (si < 2) ? c ^ 1 : c ^ 2);
          const int e0 = (si < 2) ? 2 : 0, e1 = (si < 2) ? 3 : 1;
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            const int pos = 4 * w + jj;
            if (pos >= len) break;
            int beat = kX;
            if (pos == 0 || pos == len - 1) beat = max(beat, C.ex[pos == 0 ? e0 : e1] ? kO : -1);
            if (kS > beat)
              gdyn[c * tstride + gline_tidx(si, 0, pos, bw, bh, C.g.sp)] = (uint8_t)((uint32_t)wv[j] >> (8 * jj));
          }
        }
      }
      __syncthreads();
    }
    for (int c = 0; c < 4; ++c) gown_store<NT>(d, gdyn + c * tstride, sm.col[c].g);
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
template <int NT, bool REFLECT, bool PREF>
static int gown_padding(int per_sm, int smem_sm, int reserved, int optin, int need_dyn) {
  const void* fn = reinterpret_cast<const void*>(&persistent_gown_kernel<NT, REFLECT, PREF>);
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) return -1;
  const int stat = (int)fa.sharedSizeBytes;
  if (optin - stat < need_dyn ||
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - stat) != cudaSuccess)
    return -1;
  // padding: at most per_sm CTAs fit an SM, so the grid spreads over all SMs
  int dyn = smem_sm / per_sm - reserved - stat - 256;
  if (dyn > optin - stat) dyn = optin - stat;
  for (dyn = dyn > need_dyn ? dyn & ~127 : need_dyn;; dyn -= 1024) {
    if (dyn < need_dyn) dyn = need_dyn;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, NT, (size_t)dyn) != cudaSuccess) return -1;
    if (occ >= per_sm) return dyn;
    if (dyn == need_dyn) return -1;   // the grid cannot be resident at once
  }
}

int persistent_gown_config(const LatticeDesc& d, int device, GownConfig* cfg, int min_per_sm) {
  if (d.nbh != 4 || d.P < 2 || d.Py < 2) return 0;
  // widest block and its fine segments on each axis
  auto axis_ok = [](const AxisGeom& g, int* wmax, int* qmax) {
    const int wa = g.q + (g.r > 0 ? 1 : 0);
    *wmax = wa;
    *qmax = g.r > 0 ? g.Qa : g.Qb;
    const int fmax_a = g.Qa > 0 ? g.fqa + (g.fra > 0 ? 1 : 0) : 99;
    const int fmax_b = g.Qb > 0 ? g.fqb + (g.frb > 0 ? 1 : 0) : 99;
    const int fmax = g.r > 0 ? (fmax_a > fmax_b ? fmax_a : fmax_b) : fmax_b;
    const int fmin_b = g.Qb > 0 ? g.fqb : 0;
    return wa <= kMaxBlock && fmax <= 3 && fmin_b >= 2;
  };
  int wx = 0, qx = 0, wy = 0, qy = 0;
  if (!axis_ok(d.ax, &wx, &qx) || !axis_ok(d.ay, &wy, &qy)) return 0;
  const int nq = (qx / 2) * (qy / 2);
  if (nq > 512) return 0;
  const int groups = (d.P / 2) * (d.Py / 2);
  int sms = 0, smem_sm = 0, reserved = 0, optin = 0, coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device);
  if (!coop) return 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, device);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  if (sms <= 0) return 0;
  int per_sm = (groups + sms - 1) / sms;
  if (per_sm < min_per_sm) per_sm = min_per_sm;
  // one thread per quad (256 or 512); 512 also for blocks of up to 256
  // quads when each SM holds one CTA: the visit's words are then drawn by
  // twice the threads, two quads' worth each instead of four
  const int nt = (nq > 256 || per_sm == 1) ? 512 : 256;
  const int tile_bytes = ((wy + 2) * (((kColOff + wx + 1) + 15) & ~15) + 15) & ~15;
  const int need_dyn = 4 * tile_bytes + 4 * kGSlots * nt * (int)sizeof(uint32_t);
  const bool refl = d.reflect != 0;
  int dyn;
  // 512 threads on blocks of at most 256 quads: the upper half draws the
  // next visit's words during the fine phases (the two buffers take the
  // space of one 512-thread buffer)
  const bool pref = nt == 512 && nq <= 256;
  if (nt == 256)
    dyn = refl ? gown_padding<256, true, false>(per_sm, smem_sm, reserved, optin, need_dyn)
               : gown_padding<256, false, false>(per_sm, smem_sm, reserved, optin, need_dyn);
  else if (pref)
    dyn = refl ? gown_padding<512, true, true>(per_sm, smem_sm, reserved, optin, need_dyn)
               : gown_padding<512, false, true>(per_sm, smem_sm, reserved, optin, need_dyn);
  else
    dyn = refl ? gown_padding<512, true, false>(per_sm, smem_sm, reserved, optin, need_dyn)
               : gown_padding<512, false, false>(per_sm, smem_sm, reserved, optin, need_dyn);
  if (dyn < 0) return 0;
  cfg->dyn_bytes = dyn;
  cfg->threads = nt;
  cfg->ctas_per_sm = per_sm;
  cfg->tile_stride = tile_bytes;
  cfg->prefetch = pref ? 1 : 0;
  return groups;
}

// A cooperative launch: the runtime starts the grid only with every CTA
// resident, also while kernels of other streams hold part of the device.
cudaError_t launch_persistent_gown(const PersistentArgs& a, const GownConfig& cfg, cudaStream_t stream) {
  const int groups = (a.d.P / 2) * (a.d.Py / 2);
  GownArgs arg;
  arg.p = a;
  arg.tile_stride = cfg.tile_stride;
  void* params[] = {&arg};
  const bool refl = a.d.reflect != 0;
  const void* fn;
  if (cfg.threads == 256)
    fn = refl ? reinterpret_cast<const void*>(&persistent_gown_kernel<256, true, false>)
              : reinterpret_cast<const void*>(&persistent_gown_kernel<256, false, false>);
  else if (cfg.prefetch)
    fn = refl ? reinterpret_cast<const void*>(&persistent_gown_kernel<512, true, true>)
              : reinterpret_cast<const void*>(&persistent_gown_kernel<512, false, true>);
  else
    fn = refl ? reinterpret_cast<const void*>(&persistent_gown_kernel<512, true, false>)
              : reinterpret_cast<const void*>(&persistent_gown_kernel<512, false, false>);
  return cudaLaunchCooperativeKernel(fn, dim3(groups), dim3(cfg.threads), params, (size_t)cfg.dyn_bytes, stream);
}

}  // namespace escg_impl
