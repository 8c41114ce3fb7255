// escg_device.cuh -- device-side building blocks of the ESCG Monte Carlo
// step on sm_103a: Philox4x32-10, the elementary step on a shared-memory
// tile, the visit of one coarse block (load block + 1-site rim, four fine
// colour phases, write back) and the fused species count of a visit.
//
// The schedule implemented here (version 1) is the coloured two-level
// sublattice decomposition of the lattice: coarse blocks coloured 2x2, fine
// sub-blocks (2..4 sites per axis) coloured 2x2 inside each block.  Within a
// coarse phase every block of one colour owns its interior and its rim
// strips; within a fine phase every sub-block of one colour owns its cells
// and their von Neumann neighbours.  No two threads ever touch the same site
// in the same phase, so no atomics are needed and the result does not depend
// on thread or block scheduling.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "escg_types.h"

namespace escg_impl {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64-bit multiplies; the high halves are mixed with the other two
// counter words and the round key.  One wide multiply gives both halves.
// Also compiled for the host (launchers that need a draw of the schedule).
__host__ __device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1,
                   (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// Same, with the ten round keys precomputed (rk[2r], rk[2r+1] = key + r *
// Weyl constants); rk points into the kernel's parameter space, so the keys
// are constant-bank operands of the XORs rather than per-thread additions.
__device__ __forceinline__ uint4 philox10_rk(uint4 c, const uint32_t* __restrict__ rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk[2 * r], (uint32_t)p1,
                   (uint32_t)(p0 >> 32) ^ c.w ^ rk[2 * r + 1], (uint32_t)p0);
  }
  return c;
}

// Colour order drawn by x0: entry floor(x0 * 24 / 2^32) of the 24 orders of
// the four colours (lexicographic; d.perm24 holds them as 4 x 2-bit colours,
// first colour in the lowest bits).
__device__ __forceinline__ uint32_t colour_order(uint32_t x0, const uint8_t* perm24) {
  return perm24[__umulhi(x0, 24u)];
}
__device__ __forceinline__ int order_at(uint32_t ord, int k) { return (ord >> (2 * k)) & 3; }
__device__ __forceinline__ int slot_of(uint32_t ord, int colour) {
  int s = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) s = (order_at(ord, k) == colour) ? k : s;
  return s;
}

// Per-CTA shared state of a block visit.
struct VisitSmem {
  uint8_t tile[kMaxTileRows * kMaxTilePitch];
  uint32_t trans[kTransWords];   // LatticeDesc::trans
  uint32_t forder;
  uint32_t hist[kMaxStates];
};

// Transition of the pair (a, b) under the action drawn by u: byte
// (a*(S+1)+b)*4 + action of the table, action = exchange if u < T_X,
// interaction if u < T_XI and u is below the pair's interaction threshold
// (an edge that wins with a probability: Park, Chen and Szolnoki's model),
// no change if only the latter fails, reproduction otherwise.  New a in the
// low nibble, new b in the high nibble.  Thresholds of 2^32 are stored as
// 0xFFFFFFFF, which is exact because u is always a multiple of 4.
// Exchange (u < T_X) is a plain swap and needs no table: with epsilon = 2MN
// it is the action of almost every attempt on large lattices, so it takes a
// short path of its own (identical result: the table entry is the swap).
__device__ __forceinline__ void apply_rule(uint8_t* __restrict__ tile, const uint8_t* __restrict__ trans,
                                           int ti, int tj, uint32_t u, uint32_t tx, uint32_t txi,
                                           uint32_t s1) {
  const uint32_t a = tile[ti], b = tile[tj];
  if (u < tx) {
    tile[ti] = (uint8_t)b;
    tile[tj] = (uint8_t)a;
  } else {
    const uint32_t pair = a * s1 + b;
    const uint32_t tp = reinterpret_cast<const uint32_t*>(trans)[kTransPairs + pair];
    const uint32_t act = (u >= txi) ? 2u : (u < tp ? 1u : 3u);
    const uint32_t nn = trans[pair * 4u + act];
    tile[ti] = (uint8_t)(nn & 15u);
    tile[tj] = (uint8_t)(nn >> 4);
  }
}

// apply_rule on a pair already read from the tile (a at ti, b at tj).
__device__ __forceinline__ void apply_rule_ab(uint8_t* __restrict__ tile, const uint8_t* __restrict__ trans,
                                              int ti, int tj, uint32_t a, uint32_t b, uint32_t u, uint32_t tx,
                                              uint32_t txi, uint32_t s1) {
  if (u < tx) {
    tile[ti] = (uint8_t)b;
    tile[tj] = (uint8_t)a;
  } else {
    const uint32_t pair = a * s1 + b;
    const uint32_t tp = reinterpret_cast<const uint32_t*>(trans)[kTransPairs + pair];
    const uint32_t act = (u >= txi) ? 2u : (u < tp ? 1u : 3u);
    const uint32_t nn = trans[pair * 4u + act];
    tile[ti] = (uint8_t)(nn & 15u);
    tile[tj] = (uint8_t)(nn >> 4);
  }
}

// apply_rule_ab on a transition table kept in shared memory as one 8-byte
// entry per pair (LatticeDesc::trans with its two halves interleaved: .x the
// four new pairs, byte `act` for action act; .y the pair's interaction
// threshold), so that a step off the exchange path reads one entry instead of
// two dependent words (a at ti, b at tj; u the action draw).
__device__ __forceinline__ void rule8(uint8_t* __restrict__ tile, const uint2* __restrict__ t2, int ti, int tj,
                                      uint32_t a, uint32_t b, uint32_t u, uint32_t tx, uint32_t txi, uint32_t s1) {
  if (u < tx) {
    tile[ti] = (uint8_t)b;
    tile[tj] = (uint8_t)a;
  } else {
    const uint2 e = t2[a * s1 + b];
    const uint32_t act = (u >= txi) ? 2u : (u < e.y ? 1u : 3u);
    const uint32_t nn = e.x >> (8u * act);
    tile[ti] = (uint8_t)(nn & 15u);
    tile[tj] = (uint8_t)((nn >> 4) & 15u);
  }
}

// The cell and neighbour tile indices and the action draw of attempt()'s
// step (w, n4 = 4 * cells, base, wx, inv_wx, sp as there).
__device__ __forceinline__ void locate(uint32_t w, uint32_t n4, int base, int wx, uint32_t inv_wx, int sp,
                                       int& ti, int& tj, uint32_t& u) {
  const uint32_t hi = __umulhi(w, n4);
  u = w * n4;
  const uint32_t site = hi >> 2, dir = hi & 3u;
  const uint32_t r = (site * inv_wx) >> 16;
  const uint32_t c = site - r * (uint32_t)wx;
  ti = base + (int)r * sp + (int)c;
  const int mag = (dir & 2u) ? 1 : sp;
  tj = ti + ((dir & 1u) ? mag : -mag);
}

// The steps of a generic sub-block from the words wv[] in registers, each step's cell and neighbour located while the previous
// step's pair is read (the locating arithmetic sits ahead of the branch of
// the previous step's rule instead of behind it).
// Steps t < n run (n <= N).
template <int N>
__device__ __forceinline__ void attempts_ahead(uint8_t* __restrict__ tile, const uint8_t* __restrict__ trans,
                                               const uint32_t* wv, uint32_t n, uint32_t n4, int base, int wx,
                                               uint32_t inv_wx, int sp, uint32_t tx, uint32_t txi, uint32_t s1) {
  int ti, tj;
  uint32_t u;
  locate(wv[0], n4, base, wx, inv_wx, sp, ti, tj, u);
#pragma unroll
  for (int t = 0; t < N; ++t) {
    if ((uint32_t)t >= n) break;
    const uint32_t a = tile[ti], b = tile[tj];
    int ti2 = 0, tj2 = 0;
    uint32_t u2 = 0;
    if (t + 1 < N) locate(wv[t + 1], n4, base, wx, inv_wx, sp, ti2, tj2, u2);
    apply_rule_ab(tile, trans, ti, tj, a, b, u, tx, txi, s1);
    ti = ti2;
    tj = tj2;
    u = u2;
  }
}

// One elementary step (Alg. 3) of a generic sub-block.  w: the attempt's
// 32-bit Philox word; n4 = 4 * cells of the sub-block; base: tile index of
// the sub-block's first cell; wx: its width; inv_wx = ceil(65536 / wx).
__device__ __forceinline__ void attempt(uint8_t* __restrict__ tile, const uint8_t* __restrict__ trans,
                                        uint32_t w, uint32_t n4, int base, int wx, uint32_t inv_wx,
                                        int sp, uint32_t tx, uint32_t txi, uint32_t s1) {
  const uint32_t hi = __umulhi(w, n4);
  const uint32_t u = w * n4;
  const uint32_t site = hi >> 2, dir = hi & 3u;
  const uint32_t r = (site * inv_wx) >> 16;
  const uint32_t c = site - r * (uint32_t)wx;
  const int ti = base + (int)r * sp + (int)c;
  const int mag = (dir & 2u) ? 1 : sp;
  const int tj = ti + ((dir & 1u) ? mag : -mag);
  apply_rule(tile, trans, ti, tj, u, tx, txi, s1);
}

// One elementary step of a generic sub-block under a rule variant (the
// paper's --neighbourhood 4/8 and --flux options): p = w * (nbh * n_k), cell
// = hi >> lg(nbh), direction = hi & (nbh - 1) (0 up, 1 down, 2 left,
// 3 right, 4 up-left, 5 up-right, 6 down-left, 7 down-right); with reflect,
// a step that would leave the lattice is mirrored.  (gy, gx): lattice
// coordinates of the sub-block's first cell.
__device__ __forceinline__ void attempt_variant(uint8_t* __restrict__ tile, const uint8_t* __restrict__ trans,
                                                uint32_t w, uint32_t nn, int lg, int base, int wx,
                                                uint32_t inv_wx, int sp, uint32_t tx, uint32_t txi,
                                                uint32_t s1, bool reflect, int gy, int gx, int H, int L) {
  const uint32_t hi = __umulhi(w, nn);
  const uint32_t u = w * nn;
  const uint32_t site = hi >> lg, dir = hi & ((1u << lg) - 1u);
  const uint32_t r = (site * inv_wx) >> 16;
  const uint32_t c = site - r * (uint32_t)wx;
  // row and column steps of the eight directions, two bits each
  int dr = (int)((0xA058u >> (2 * dir)) & 3u) - 1;   // -1, 1, 0, 0, -1, -1, 1, 1
  int dc = (int)((0x8885u >> (2 * dir)) & 3u) - 1;   //  0, 0, -1, 1, -1, 1, -1, 1
  if (reflect) {
    const int row = gy + (int)r, col = gx + (int)c;
    if (row + dr < 0 || row + dr >= H) dr = -dr;
    if (col + dc < 0 || col + dc >= L) dc = -dc;
  }
  const int ti = base + (int)r * sp + (int)c;
  const int tj = ti + dr * sp + dc;
  apply_rule(tile, trans, ti, tj, u, tx, txi, s1);
}

// Tile index of block-local (row r, col c), r, c in [-1, B].
__device__ __forceinline__ int tidx(int r, int c, int sp) { return (r + 1) * sp + c + kColOff; }
__device__ __forceinline__ int tile_pitch(int bw) { return ((kColOff + bw + 1) + 15) & ~15; }
__device__ __forceinline__ int wrap(int v, int L) { return v < 0 ? v + L : (v >= L ? v - L : v); }

// Bit-packed lattices: site c of a row occupies bits [c b, (c + 1) b) of the
// row's little-endian bit string, b = LatticeDesc::bits (8: one byte per
// site; 4 or 2: packed).  A group of 4 sites that starts at a multiple of 4
// is one 32-bit word (b = 8), one 16-bit word (4) or one byte (2); kernels
// move groups and work on one byte per site in shared memory.
__device__ __forceinline__ uint32_t load_group(const uint8_t* row, int c0, int bits) {
  if (bits == 8) return __ldcg(reinterpret_cast<const uint32_t*>(row + c0));
  if (bits == 4) return __ldcg(reinterpret_cast<const uint16_t*>(row + (c0 >> 1)));
  return __ldcg(row + (c0 >> 2));
}
__device__ __forceinline__ void store_group(uint8_t* row, int c0, int bits, uint32_t raw) {
  if (bits == 8)
    *reinterpret_cast<uint32_t*>(row + c0) = raw;
  else if (bits == 4)
    *reinterpret_cast<uint16_t*>(row + (c0 >> 1)) = (uint16_t)raw;
  else
    row[c0 >> 2] = (uint8_t)raw;
}
// 4 packed sites -> 4 bytes (site e in byte e), and back.
__device__ __forceinline__ uint32_t unpack4(uint32_t raw, int bits) {
  if (bits == 8) return raw;
  if (bits == 4)
    return (raw & 0xFu) | ((raw & 0xF0u) << 4) | ((raw & 0xF00u) << 8) | ((raw & 0xF000u) << 12);
  return (raw & 0x3u) | ((raw & 0xCu) << 6) | ((raw & 0x30u) << 12) | ((raw & 0xC0u) << 18);
}
__device__ __forceinline__ uint32_t pack4(uint32_t v, int bits) {
  if (bits == 8) return v;
  if (bits == 4)
    return (v & 0xFu) | ((v >> 4) & 0xF0u) | ((v >> 8) & 0xF00u) | ((v >> 12) & 0xF000u);
  return (v & 0x3u) | ((v >> 6) & 0xCu) | ((v >> 12) & 0x30u) | ((v >> 18) & 0xC0u);
}

// Uniform geometry: 64x64 blocks, 2x2 sub-blocks, one thread per 2x2 pair of
// sub-blocks ("quad"), 256 threads.
constexpr int kUniB = 64;
constexpr int kUniSP = 80;   // tile_pitch(64)
constexpr int kUniThreads = 256;

// One elementary step on a 2x2 sub-block of a tile with row pitch SP: 4*n_k
// = 16, so the high 4 bits of w are the cell (bit 31 row, bit 30 column) and
// the direction (bits 29..28: 0 up, 1 down, 2 left, 3 right), and u = w << 4.
// The two offsets come from byte tables indexed by those bit pairs: a
// __byte_perm selector below 4 picks that byte into the low byte, and its
// three zero nibbles pick byte 0, which is 0 in both tables.  kTj holds the
// neighbour's offset from the cell plus SP, so that every entry is a byte.
template <int SP>
__device__ __forceinline__ void attempt_uni(uint8_t* __restrict__ tile, const uint8_t* __restrict__ trans,
                                            uint32_t w, int base, uint32_t tx, uint32_t txi, uint32_t s1) {
  static_assert(SP < 128, "offsets must fit the byte tables");
  constexpr uint32_t kTi = 0u | (1u << 8) | ((uint32_t)SP << 16) | ((uint32_t)(SP + 1) << 24);
  constexpr uint32_t kTj = 0u | ((uint32_t)(2 * SP) << 8) | ((uint32_t)(SP - 1) << 16) | ((uint32_t)(SP + 1) << 24);
  const int ti = base + (int)__byte_perm(kTi, 0u, w >> 30);
  const int tj = ti - SP + (int)__byte_perm(kTj, 0u, (w >> 28) & 3u);
  apply_rule(tile, trans, ti, tj, w << 4, tx, txi, s1);
}

// attempt_uni on the 8-byte-entry table (rule8).
template <int SP>
__device__ __forceinline__ void attempt_uni8(uint8_t* __restrict__ tile, const uint2* __restrict__ t2, uint32_t w,
                                             int base, uint32_t tx, uint32_t txi, uint32_t s1) {
  constexpr uint32_t kTi = 0u | (1u << 8) | ((uint32_t)SP << 16) | ((uint32_t)(SP + 1) << 24);
  constexpr uint32_t kTj = 0u | ((uint32_t)(2 * SP) << 8) | ((uint32_t)(SP - 1) << 16) | ((uint32_t)(SP + 1) << 24);
  const int ti = base + (int)__byte_perm(kTi, 0u, w >> 30);
  const int tj = ti - SP + (int)__byte_perm(kTj, 0u, (w >> 28) & 3u);
  rule8(tile, t2, ti, tj, tile[ti], tile[tj], w << 4, tx, txi, s1);
}

template <int SP, int COFF>
__device__ __forceinline__ int tidx_u(int r, int c) { return (r + 1) * SP + c + COFF; }

// A coarse block's span along one axis and its fine segments (AxisGeom).
struct BlockSpan {
  int s0, w;    // first site, width
  int f0, Q;    // global index of the first fine segment, fine segments
  int fq, fr;   // fine segment k: start k fq + min(k, fr), width fq + (k < fr)
};

__device__ __forceinline__ BlockSpan block_span(const AxisGeom& g, int b) {
  BlockSpan s;
  const bool wide = b < g.r;
  const int nw = min(b, g.r);
  s.s0 = b * g.q + nw;
  s.w = g.q + (wide ? 1 : 0);
  s.f0 = nw * g.Qa + (b - nw) * g.Qb;
  s.Q = wide ? g.Qa : g.Qb;
  s.fq = wide ? g.fqa : g.fqb;
  s.fr = wide ? g.fra : g.frb;
  return s;
}
__device__ __forceinline__ int seg_start(const BlockSpan& s, int k) { return k * s.fq + min(k, s.fr); }
__device__ __forceinline__ int seg_width(const BlockSpan& s, int k) { return s.fq + (k < s.fr ? 1 : 0); }

// Generic staging of a block's tile.  A visit uses the block interior and
// the four 1-site rim strips, the corners too in the Moore neighbourhood,
// and nothing beyond the lattice edge with a reflecting boundary.  Every
// tile row is moved by one warp, lane k taking the k-th aligned group of 4
// sites of the row's columns that do not wrap around the lattice edge (at
// most 26 groups); the one column that wraps (a block at the left or right
// edge of a periodic lattice) comes with its group, taken by lane 31 (left)
// or 30 (right).  The per-lane plan is the same for all rows of a kind
// (interior rows, rim rows), so it is worked out once per visit.  Loads go
// through L2 (ld.global.cg: data written by other CTAs of the same launch
// must not be served from a stale L1 line).
struct RowPlan {
  int gcol;       // lattice column of the group's first site (a multiple of 4)
  int tcol;       // tile column of that site
  uint32_t mask;  // sites of the group that belong to the tile (bit e: site e); 0: none
};

__device__ __forceinline__ RowPlan row_plan(const LatticeDesc& d, int x0, int bw, bool rim, int lane) {
  RowPlan p;
  const bool reflect = d.reflect != 0, trim = rim && d.nbh != 8;
  const int c_lo = trim ? 0 : -1, c_hi = trim ? bw - 1 : bw;
  const int g_lo = max(x0 + c_lo, 0), g_hi = min(x0 + c_hi, d.L - 1);
  const int gc0 = (g_lo & ~3) + 4 * lane;
  p.mask = 0;
  p.gcol = 0;
  p.tcol = 0;
  if (gc0 <= g_hi) {
    p.gcol = gc0;
    p.tcol = gc0 - x0;
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (gc0 + e >= g_lo && gc0 + e <= g_hi) p.mask |= 1u << e;
  } else if (lane == 31 && !reflect && x0 + c_lo < 0) {
    const int e = (d.L - 1) & 3;
    p.gcol = (d.L - 1) & ~3;
    p.tcol = -1 - e;
    p.mask = 1u << e;
  } else if (lane == 30 && !reflect && x0 + c_hi >= d.L) {
    p.gcol = 0;
    p.tcol = bw;
    p.mask = 1;
  }
  return p;
}

// Lattice row of tile row r, or -1 beyond a reflecting edge.
__device__ __forceinline__ int tile_row_gy(const LatticeDesc& d, int y0, int r) {
  const int gy = y0 + r;
  if (gy >= 0 && gy < d.H) return gy;
  if (d.reflect) return -1;
  return gy < 0 ? gy + d.H : gy - d.H;
}

// Stash of a packed lattice's partially used groups, one 16-bit entry per
// tile row and lane: the write-back merges the tile's sites into the group
// as it was loaded.  Every group a visit writes holds no site that another
// block of the same colour reads or writes (blocks are at least 32 sites
// wide), and no other block writes its other sites during the visit.
constexpr int kStashLanes = 32;
constexpr int kStashWords = kMaxTileRows * kStashLanes;

// Each warp issues the loads of up to 8 rows before it writes any of them
// to shared memory: a tile costs two L2 round trips.  PACKED = false: one
// byte per site (the packing code is compiled out).
template <bool PACKED = false>
__device__ __forceinline__ void load_tile_generic(const LatticeDesc& d, int x0, int y0, int bw, int bh,
                                                  uint8_t* tile, int sp, uint16_t* stash) {
  constexpr int kRows = 8;
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5, bits = PACKED ? d.bits : 8;
  const RowPlan pi = row_plan(d, x0, bw, false, lane), pr = row_plan(d, x0, bw, true, lane);
  for (int r0 = (int)(threadIdx.x >> 5) - 1; r0 <= bh; r0 += kRows * nw) {
    uint32_t v[kRows];
#pragma unroll
    for (int i = 0; i < kRows; ++i) {
      const int r = r0 + i * nw;
      v[i] = 0;
      const RowPlan& p = (r < 0 || r >= bh) ? pr : pi;
      const int gy = tile_row_gy(d, y0, r);
      if (r > bh || gy < 0 || !p.mask) continue;
      v[i] = load_group(d.lat + (size_t)gy * d.pitch, p.gcol, bits);
    }
#pragma unroll
    for (int i = 0; i < kRows; ++i) {
      const int r = r0 + i * nw;
      const RowPlan& p = (r < 0 || r >= bh) ? pr : pi;
      if (r > bh || tile_row_gy(d, y0, r) < 0) continue;
      if (PACKED && p.mask && p.mask != 0xFu) stash[(r + 1) * kStashLanes + lane] = (uint16_t)v[i];
      const uint32_t u = unpack4(v[i], bits);
      uint8_t* dst = tile + (r + 1) * sp + kColOff + p.tcol;
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if ((p.mask >> e) & 1u) dst[e] = (uint8_t)(u >> (8 * e));
    }
  }
}

// Writes back exactly the sites load_tile_generic loaded (the rims and
// corners belong to blocks of other colours, which no other CTA updates
// during this visit): whole groups where all four sites are the tile's;
// at the ends of a row single bytes (one byte per site) or the loaded group
// with the tile's sites merged in (packed).
// origin: tile offset of block column 0 within a tile row (kColOff for the
// tiles staged here); nw: warps taking part (threads 0 .. 32 nw - 1).
template <bool PACKED = false>
__device__ __forceinline__ void store_tile_generic(const LatticeDesc& d, int x0, int y0, int bw, int bh,
                                                   const uint8_t* tile, int sp, const uint16_t* stash,
                                                   int origin = kColOff, int nw = 0) {
  const int lane = threadIdx.x & 31, bits = PACKED ? d.bits : 8;
  if (nw == 0) nw = blockDim.x >> 5;
  const RowPlan pi = row_plan(d, x0, bw, false, lane), pr = row_plan(d, x0, bw, true, lane);
  for (int r = (int)(threadIdx.x >> 5) - 1; r <= bh; r += nw) {
    const RowPlan& p = (r < 0 || r >= bh) ? pr : pi;
    const int gy = tile_row_gy(d, y0, r);
    if (gy < 0 || !p.mask) continue;
    const uint8_t* src = tile + (r + 1) * sp + origin + p.tcol;
    uint8_t* row = d.lat + (size_t)gy * d.pitch;
    if (p.mask == 0xFu) {
      const uint32_t w = (uint32_t)src[0] | ((uint32_t)src[1] << 8) | ((uint32_t)src[2] << 16) |
                         ((uint32_t)src[3] << 24);
      store_group(row, p.gcol, bits, pack4(w, bits));
    } else if (bits == 8) {
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if ((p.mask >> e) & 1u) row[p.gcol + e] = src[e];
    } else {
      uint32_t u = unpack4(stash[(r + 1) * kStashLanes + lane], bits);
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if ((p.mask >> e) & 1u) u = (u & ~(0xFFu << (8 * e))) | ((uint32_t)src[e] << (8 * e));
      store_group(row, p.gcol, bits, pack4(u, bits));
    }
  }
}

// Generic tiles of one-byte lattices are staged in aligned 8-byte groups.
// The tile's column origin depends on the block, origin = 8 + (x0 mod 8), so
// that every lattice column that is a multiple of 8 sits on an 8-byte
// boundary of the tile; the row pitch round_up(bw + 23, 16) holds the groups
// from the one with the left rim column to the one with the right rim
// column.  The sites these groups bring in beyond the rim columns, and the
// corners, belong to the block's eight neighbours, which no visit updates
// while this one runs, and lie at least a block width (32 sites or more)
// away from every other block's tile; the fine phases never reach them, so
// they go back to the lattice as they came.  Row padding beyond column L is
// neither needed nor written: the lattice's last group of a row is written
// back one byte at a time.
__device__ __forceinline__ int gen_origin(int x0) { return 8 + (x0 & 7); }
__device__ __forceinline__ int gen_pitch(int bw) { return (bw + 23 + 15) & ~15; }

// Rows r = -1 .. bh of a generic tile, two per warp and pass (16 lanes per
// row, one 8-byte group per lane); the periodic rim columns of the blocks at
// the lattice's left and right edges come as single bytes.  The loads of
// kPass passes are issued before any of them is written to the tile.
__device__ __forceinline__ void load_tile_aligned(const LatticeDesc& d, int x0, int y0, int bw, int bh,
                                                  uint8_t* tile, int sp, int origin) {
  constexpr int kPass = 5;
  const int L = d.L, lane = threadIdx.x & 31, l16 = lane & 15, nw = blockDim.x >> 5;
  const int g_lo = max(x0 - 1, 0) >> 3, g_hi = min(x0 + bw, L - 1) >> 3;
  const bool act = l16 <= g_hi - g_lo;
  const int gcol = (g_lo + l16) * 8, tcol = origin + gcol - x0;
  const bool wrap_l = !d.reflect && x0 == 0 && l16 == 0;
  const bool wrap_r = !d.reflect && x0 + bw == L && l16 == g_hi - g_lo;
  for (int r0 = 2 * (int)(threadIdx.x >> 5) + (lane >> 4) - 1; r0 <= bh; r0 += 2 * nw * kPass) {
    uint2 v[kPass];
    uint8_t wl[kPass], wr[kPass];
#pragma unroll
    for (int i = 0; i < kPass; ++i) {
      const int r = r0 + 2 * nw * i;
      const int gy = r <= bh ? tile_row_gy(d, y0, r) : -1;
      v[i] = make_uint2(0u, 0u);
      wl[i] = wr[i] = 0;
      if (!act || gy < 0) continue;
      const uint8_t* row = d.lat + (size_t)gy * d.pitch;
      v[i] = __ldcg(reinterpret_cast<const uint2*>(row + gcol));
      if (wrap_l) wl[i] = __ldcg(row + L - 1);
      if (wrap_r) wr[i] = __ldcg(row);
    }
#pragma unroll
    for (int i = 0; i < kPass; ++i) {
      const int r = r0 + 2 * nw * i;
      if (!act || r > bh || tile_row_gy(d, y0, r) < 0) continue;
      uint8_t* trow = tile + (r + 1) * sp;
      *reinterpret_cast<uint2*>(trow + tcol) = v[i];
      if (wrap_l) trow[origin - 1] = wl[i];
      if (wrap_r) trow[origin + bw] = wr[i];
    }
  }
}

// Writes back what load_tile_aligned staged.
__device__ __forceinline__ void store_tile_aligned(const LatticeDesc& d, int x0, int y0, int bw, int bh,
                                                   const uint8_t* tile, int sp, int origin) {
  const int L = d.L, lane = threadIdx.x & 31, l16 = lane & 15, nw = blockDim.x >> 5;
  const int g_lo = max(x0 - 1, 0) >> 3, g_hi = min(x0 + bw, L - 1) >> 3;
  const bool act = l16 <= g_hi - g_lo;
  const int gcol = (g_lo + l16) * 8, tcol = origin + gcol - x0;
  const bool wrap_l = !d.reflect && x0 == 0 && l16 == 0;
  const bool wrap_r = !d.reflect && x0 + bw == L && l16 == g_hi - g_lo;
  for (int r = 2 * (int)(threadIdx.x >> 5) + (lane >> 4) - 1; r <= bh; r += 2 * nw) {
    const int gy = tile_row_gy(d, y0, r);
    if (!act || gy < 0) continue;
    uint8_t* row = d.lat + (size_t)gy * d.pitch;
    const uint8_t* trow = tile + (r + 1) * sp;
    const uint2 v = *reinterpret_cast<const uint2*>(trow + tcol);
    if (gcol + 8 <= L) {
      *reinterpret_cast<uint2*>(row + gcol) = v;
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e)
        if (gcol + e < L) row[gcol + e] = (uint8_t)(((e < 4) ? v.x : v.y) >> (8 * (e & 3)));
    }
    if (wrap_l) row[L - 1] = trow[origin - 1];
    if (wrap_r) row[0] = trow[origin + bw];
  }
}

// Piece t (0..255) of a uniform one-byte-per-site tile: a 16-byte quarter
// row of the interior and, for t < 8, of the top / bottom rim rows, for
// t >= 128 one cell of the left / right rim columns.  load_tile_uni and
// store_tile_uni run piece threadIdx.x; CTAs of fewer threads run several.
__device__ __forceinline__ void load_piece_uni(const LatticeDesc& d, int x0, int y0, uint8_t* tile, int t) {
  const int L = d.L, pitch = d.pitch;
  {  // interior: 64 rows x 4 x 16 bytes, one 16-byte load per piece
    const int r = t >> 2, q = t & 3;
    const uint4 v = __ldcg(reinterpret_cast<const uint4*>(d.lat + (size_t)(y0 + r) * pitch + x0) + q);
    uint2* dst = reinterpret_cast<uint2*>(tile + tidx(r, 16 * q, kUniSP));
    dst[0] = make_uint2(v.x, v.y);
    dst[1] = make_uint2(v.z, v.w);
  }
  if (t < 8) {  // top / bottom rim rows
    const int r = (t < 4) ? -1 : kUniB, q = t & 3;
    const uint4 v = __ldcg(reinterpret_cast<const uint4*>(d.lat + (size_t)wrap(y0 + r, d.H) * pitch + x0) + q);
    uint2* dst = reinterpret_cast<uint2*>(tile + tidx(r, 16 * q, kUniSP));
    dst[0] = make_uint2(v.x, v.y);
    dst[1] = make_uint2(v.z, v.w);
  } else if (t >= 128) {  // left / right rim columns
    const int k = t - 128, c = (k < 64) ? -1 : kUniB, r = k & 63;
    tile[tidx(r, c, kUniSP)] = __ldcg(d.lat + (size_t)(y0 + r) * pitch + wrap(x0 + c, L));
  }
}

__device__ __forceinline__ void store_piece_uni(const LatticeDesc& d, int x0, int y0, const uint8_t* tile, int t) {
  const int L = d.L, pitch = d.pitch;
  {
    const int r = t >> 2, q = t & 3;
    const uint2* src = reinterpret_cast<const uint2*>(tile + tidx(r, 16 * q, kUniSP));
    const uint2 a = src[0], b = src[1];
    reinterpret_cast<uint4*>(d.lat + (size_t)(y0 + r) * pitch + x0)[q] = make_uint4(a.x, a.y, b.x, b.y);
  }
  if (t < 8) {
    const int r = (t < 4) ? -1 : kUniB, q = t & 3;
    const uint2* src = reinterpret_cast<const uint2*>(tile + tidx(r, 16 * q, kUniSP));
    const uint2 a = src[0], b = src[1];
    reinterpret_cast<uint4*>(d.lat + (size_t)wrap(y0 + r, d.H) * pitch + x0)[q] = make_uint4(a.x, a.y, b.x, b.y);
  } else if (t >= 128) {
    const int k = t - 128, c = (k < 64) ? -1 : kUniB, r = k & 63;
    d.lat[(size_t)(y0 + r) * pitch + wrap(x0 + c, L)] = tile[tidx(r, c, kUniSP)];
  }
}

// Piece t (0..255) of a uniform tile on a packed lattice (2 or 4 bits per
// site), the same pieces as load_piece_uni: a quarter row is one 32-bit
// (2 bits) or 64-bit (4 bits) load, and a rim-column site comes with its
// group of 4, which is returned (0 for the other pieces) for
// store_piece_uni_packed to write the group back whole.  The other three
// sites of that group belong to the neighbouring block, which no visit
// updates while this one runs.
__device__ __forceinline__ uint32_t load_piece_uni_packed(const LatticeDesc& d, int x0, int y0, uint8_t* tile,
                                                          int t, int bits) {
  const int L = d.L, pitch = d.pitch;
  auto quarter = [&](int r, int gy, int q) {
    const uint8_t* row = d.lat + (size_t)gy * pitch;
    uint32_t lo, hi;
    if (bits == 2) {
      const uint32_t w = __ldcg(reinterpret_cast<const uint32_t*>(row + ((x0 + 16 * q) >> 2)));
      lo = w & 0xFFFFu;
      hi = w >> 16;
    } else {
      const uint2 w = __ldcg(reinterpret_cast<const uint2*>(row + ((x0 + 16 * q) >> 1)));
      lo = w.x;
      hi = w.y;
    }
    // lo/hi hold sites 0..7 / 8..15 of the quarter (16 or 32 bits each)
    const int sh = bits == 2 ? 8 : 16;
    uint2* dst = reinterpret_cast<uint2*>(tile + tidx(r, 16 * q, kUniSP));
    dst[0] = make_uint2(unpack4(lo, bits), unpack4(lo >> sh, bits));
    dst[1] = make_uint2(unpack4(hi, bits), unpack4(hi >> sh, bits));
  };
  uint32_t rim_raw = 0;
  quarter(t >> 2, y0 + (t >> 2), t & 3);
  if (t < 8) {
    const int r = (t < 4) ? -1 : kUniB;
    quarter(r, wrap(y0 + r, d.H), t & 3);
  } else if (t >= 128) {
    const int k = t - 128, c = (k < 64) ? -1 : kUniB, r = k & 63;
    const int gx = wrap(x0 + c, L);
    rim_raw = load_group(d.lat + (size_t)(y0 + r) * pitch, gx & ~3, bits);
    tile[tidx(r, c, kUniSP)] = (uint8_t)(unpack4(rim_raw, bits) >> (8 * (gx & 3)));
  }
  return rim_raw;
}

// Writes back piece t as load_piece_uni_packed loaded it; rim_raw is the
// group that call returned for the same piece.
__device__ __forceinline__ void store_piece_uni_packed(const LatticeDesc& d, int x0, int y0, const uint8_t* tile,
                                                       int t, int bits, uint32_t rim_raw) {
  const int L = d.L, pitch = d.pitch;
  auto quarter = [&](int r, int gy, int q) {
    uint8_t* row = d.lat + (size_t)gy * pitch;
    const uint2* src = reinterpret_cast<const uint2*>(tile + tidx(r, 16 * q, kUniSP));
    const uint2 a = src[0], b = src[1];
    const int sh = bits == 2 ? 8 : 16;
    const uint32_t lo = pack4(a.x, bits) | (pack4(a.y, bits) << sh);
    const uint32_t hi = pack4(b.x, bits) | (pack4(b.y, bits) << sh);
    if (bits == 2)
      *reinterpret_cast<uint32_t*>(row + ((x0 + 16 * q) >> 2)) = lo | (hi << 16);
    else
      *reinterpret_cast<uint2*>(row + ((x0 + 16 * q) >> 1)) = make_uint2(lo, hi);
  };
  quarter(t >> 2, y0 + (t >> 2), t & 3);
  if (t < 8) {
    const int r = (t < 4) ? -1 : kUniB;
    quarter(r, wrap(y0 + r, d.H), t & 3);
  } else if (t >= 128) {
    const int k = t - 128, c = (k < 64) ? -1 : kUniB, r = k & 63;
    const int gx = wrap(x0 + c, L), e = gx & 3;
    const uint32_t u = (unpack4(rim_raw, bits) & ~(0xFFu << (8 * e))) |
                       ((uint32_t)tile[tidx(r, c, kUniSP)] << (8 * e));
    store_group(d.lat + (size_t)(y0 + r) * pitch, gx & ~3, bits, pack4(u, bits));
  }
}

// Uniform staging: 64 x 64 interior (64 rows of 16 + 16 + 16 + 16 sites,
// one quarter row per thread), the top and bottom rim rows, and the left and
// right rim columns (threads 128..255, one site each), piece threadIdx.x.
// Packed lattices: the returned rim group goes back to store_tile_uni.
template <bool PACKED = false>
__device__ __forceinline__ uint32_t load_tile_uni(const LatticeDesc& d, int x0, int y0, uint8_t* tile) {
  const int t = threadIdx.x, bits = PACKED ? d.bits : 8;
  if (bits == 8) {
    load_piece_uni(d, x0, y0, tile, t);
    return 0;
  }
  return load_piece_uni_packed(d, x0, y0, tile, t, bits);
}

template <bool PACKED = false>
__device__ __forceinline__ void store_tile_uni(const LatticeDesc& d, int x0, int y0, const uint8_t* tile,
                                               uint32_t rim_raw) {
  const int t = threadIdx.x, bits = PACKED ? d.bits : 8;
  if (bits == 8)
    store_piece_uni(d, x0, y0, tile, t);
  else
    store_piece_uni_packed(d, x0, y0, tile, t, bits, rim_raw);
}

// Loads the transition table (built on the host) and the fine order.
__device__ __forceinline__ void load_trans(const LatticeDesc& d, uint32_t* trans) {
  const int n = (d.S + 1) * (d.S + 1);
  const uint32_t* src = reinterpret_cast<const uint32_t*>(d.trans);
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    trans[k] = src[k];
    trans[kTransPairs + k] = src[kTransPairs + k];
  }
}

// Visit of coarse block (bx, by) in MCS m, uniform geometry.  Must be called
// by all 256 threads; the tile is free for reuse after the caller's next
// __syncthreads().
// Fine colour order of block (bx, by) in MCS m.
__device__ __forceinline__ uint32_t fine_order(const LatticeDesc& d, int bx, int by, uint32_t m) {
  const uint4 x = philox10_rk(make_uint4(0u, (uint32_t)(by * d.P + bx), m, kTagFineOrder), d.rk);
  return colour_order(x.x, d.perm24);
}

// The four fine colour phases of a uniform visit on a staged tile (block
// (bx, by), MCS m, fine order ord), run by threads 0..255; each phase ends
// with a barrier: __syncthreads() when BAR_N == 0, else named barrier
// BAR_ID over BAR_N threads (the threads of the visit).
// X0: the words of the first fine phase are given (xw0, drawn by the caller
// beforehand), else drawn here like the others.
// T8: trans holds the 8-byte-entry table (rule8) instead.
template <int BAR_ID = 0, int BAR_N = 0, bool X0 = false, bool T8 = false>
__device__ __forceinline__ void fine_phases_tile(const LatticeDesc& d, int bx, int by, uint32_t m, uint8_t* tile,
                                                 uint32_t ord, const uint8_t* trans, uint4 xw0 = uint4{}) {
  const int t = threadIdx.x, qx = t & 15, qy = t >> 4;
  const uint32_t s1 = (uint32_t)d.S + 1u, tx = d.tx, txi = d.txi;
  // sub-block (2 qx + cx, 2 qy + cy) of the quad: global index g00 + cy*GQ + cx,
  // first cell at tile index base00 + 2 cy SP + 2 cx
  const uint32_t GQ = (uint32_t)d.GQ;
  const uint32_t g00 = (uint32_t)(by * (kUniB / 2) + 2 * qy) * GQ + (uint32_t)(bx * (kUniB / 2) + 2 * qx);
  const int base00 = tidx(4 * qy, 4 * qx, kUniSP);
#pragma unroll
  for (int fi = 0; fi < 4; ++fi) {
    const uint32_t fcol = (ord >> (2 * fi)) & 3u, cx = fcol & 1u, cy = fcol >> 1;
    const uint32_t g = g00 + cy * GQ + cx;
    const int base = base00 + (int)(cy * (2 * kUniSP) + 2 * cx);
    const uint4 x = (X0 && fi == 0) ? xw0 : philox10_rk(make_uint4(0u, g, m, kTagStep), d.rk);
    if (T8) {
      const uint2* t2 = reinterpret_cast<const uint2*>(trans);
      attempt_uni8<kUniSP>(tile, t2, x.x, base, tx, txi, s1);
      attempt_uni8<kUniSP>(tile, t2, x.y, base, tx, txi, s1);
      attempt_uni8<kUniSP>(tile, t2, x.z, base, tx, txi, s1);
      attempt_uni8<kUniSP>(tile, t2, x.w, base, tx, txi, s1);
    } else {
      attempt_uni<kUniSP>(tile, trans, x.x, base, tx, txi, s1);
      attempt_uni<kUniSP>(tile, trans, x.y, base, tx, txi, s1);
      attempt_uni<kUniSP>(tile, trans, x.z, base, tx, txi, s1);
      attempt_uni<kUniSP>(tile, trans, x.w, base, tx, txi, s1);
    }
    if (BAR_N)
      asm volatile("bar.sync %0, %1;" ::"n"(BAR_ID), "n"(BAR_N) : "memory");
    else
      __syncthreads();
  }
}

// Same on sm.tile with the fine order in sm.forder, all 256 threads.
__device__ __forceinline__ void fine_phases_uni(const LatticeDesc& d, int bx, int by, uint32_t m,
                                                VisitSmem& sm) {
  fine_phases_tile(d, bx, by, m, sm.tile, sm.forder, reinterpret_cast<const uint8_t*>(sm.trans));
}

// OWN_FORDER = false: the caller has stored fine_order(d, bx, by, m) in
// sm.forder before a barrier that precedes the call.
template <bool OWN_FORDER = true, bool PACKED = false>
__device__ __forceinline__ void visit_uniform(const LatticeDesc& d, int bx, int by, uint32_t m,
                                              VisitSmem& sm) {
  const int x0 = bx * kUniB, y0 = by * kUniB;
  if (OWN_FORDER && threadIdx.x == 0) sm.forder = fine_order(d, bx, by, m);
  const uint32_t rim_raw = load_tile_uni<PACKED>(d, x0, y0, sm.tile);
  __syncthreads();
  fine_phases_uni(d, bx, by, m, sm);
  store_tile_uni<PACKED>(d, x0, y0, sm.tile, rim_raw);
}

// visit_uniform on a one-byte lattice with the caller's fine order in
// sm.forder, whose first fine phase draws its Philox words while the tile's
// loads are in flight: the words depend on the schedule only, so they are
// ready when the tile is, and that phase's draw leaves the visit's path
// (L = 3200: 25.84 -> 25.43 us per MCS).  Drawing the second phase's words
// too (into shared memory) measured 25.95, all four 26.88.
template <bool T8 = false>
__device__ __forceinline__ void visit_uniform_x0(const LatticeDesc& d, int bx, int by, uint32_t m,
                                                 VisitSmem& sm) {
  const int x0 = bx * kUniB, y0 = by * kUniB, t = threadIdx.x, L = d.L, pitch = d.pitch;
  // the loads of load_piece_uni, issued first
  const int r = t >> 2, q = t & 3;
  const uint4 v = __ldcg(reinterpret_cast<const uint4*>(d.lat + (size_t)(y0 + r) * pitch + x0) + q);
  const int rr = (t < 4) ? -1 : kUniB;
  const int k = t - 128, cc = (k < 64) ? -1 : kUniB, rc = k & 63;
  uint4 vr = make_uint4(0u, 0u, 0u, 0u);
  uint8_t vc = 0;
  if (t < 8)
    vr = __ldcg(reinterpret_cast<const uint4*>(d.lat + (size_t)wrap(y0 + rr, d.H) * pitch + x0) + q);
  else if (t >= 128)
    vc = __ldcg(d.lat + (size_t)(y0 + rc) * pitch + wrap(x0 + cc, L));
  // the first fine phase's words (fine_phases_tile's sub-block g of that phase)
  const uint32_t ord = sm.forder, fcol = ord & 3u;
  const int qx = t & 15, qy = t >> 4;
  const uint32_t GQ = (uint32_t)d.GQ;
  const uint32_t g = (uint32_t)(by * (kUniB / 2) + 2 * qy + (int)(fcol >> 1)) * GQ +
                     (uint32_t)(bx * (kUniB / 2) + 2 * qx + (int)(fcol & 1u));
  const uint4 xw0 = philox10_rk(make_uint4(0u, g, m, kTagStep), d.rk);
  {
    uint2* dst = reinterpret_cast<uint2*>(sm.tile + tidx(r, 16 * q, kUniSP));
    dst[0] = make_uint2(v.x, v.y);
    dst[1] = make_uint2(v.z, v.w);
  }
  if (t < 8) {
    uint2* dst = reinterpret_cast<uint2*>(sm.tile + tidx(rr, 16 * q, kUniSP));
    dst[0] = make_uint2(vr.x, vr.y);
    dst[1] = make_uint2(vr.z, vr.w);
  } else if (t >= 128) {
    sm.tile[tidx(rc, cc, kUniSP)] = vc;
  }
  __syncthreads();
  fine_phases_tile<0, 0, true, T8>(d, bx, by, m, sm.tile, ord, reinterpret_cast<const uint8_t*>(sm.trans), xw0);
  store_tile_uni<false>(d, x0, y0, sm.tile, 0u);
}

// The step of attempt() for a 2 x 2 sub-block (n_k = 4: p = 16 w, so the
// high 4 bits of w are the cell -- bit 31 row, bit 30 column -- and the
// direction, and u = w << 4), on a tile of row pitch sp.
__device__ __forceinline__ void attempt_2x2(uint8_t* __restrict__ tile, const uint8_t* __restrict__ trans,
                                            uint32_t w, int base, int sp, uint32_t tx, uint32_t txi, uint32_t s1) {
  const uint32_t dir = (w >> 28) & 3u;
  const int ti = base + (int)(w >> 31) * sp + (int)((w >> 30) & 1u);
  const int mag = (dir & 2u) ? 1 : sp;
  const int tj = ti + ((dir & 1u) ? mag : -mag);
  apply_rule(tile, trans, ti, tj, w << 4, tx, txi, s1);
}

// attempt_variant for a 2 x 2 sub-block: p = w (4 nbh), so the cell is
// bits 31..30 of w, the direction the next lg bits and u = w << (2 + lg).
__device__ __forceinline__ void attempt_variant_2x2(uint8_t* __restrict__ tile, const uint8_t* __restrict__ trans,
                                                    uint32_t w, int lg, int base, int sp, uint32_t tx,
                                                    uint32_t txi, uint32_t s1, bool reflect, int gy, int gx,
                                                    int H, int L) {
  const uint32_t r = w >> 31, c = (w >> 30) & 1u;
  const uint32_t dir = (w >> (30 - lg)) & ((1u << lg) - 1u);
  int dr = (int)((0xA058u >> (2 * dir)) & 3u) - 1;
  int dc = (int)((0x8885u >> (2 * dir)) & 3u) - 1;
  if (reflect) {
    const int row = gy + (int)r, col = gx + (int)c;
    if (row + dr < 0 || row + dr >= H) dr = -dr;
    if (col + dc < 0 || col + dc >= L) dc = -dc;
  }
  const int ti = base + (int)r * sp + (int)c;
  apply_rule(tile, trans, ti, ti + dr * sp + dc, w << (2 + lg), tx, txi, s1);
}

// One elementary step on a 2 x 2 sub-block of a uniform tile under a rule
// variant (the step of attempt_variant for n_k = 4): MOORE: p = 32 w, cell =
// bits 31..30 of w (row, column), direction = bits 29..27 (0 up, 1 down,
// 2 left, 3 right, 4 up-left, 5 up-right, 6 down-left, 7 down-right), u =
// w << 5; else the von Neumann step of attempt_uni.  EDGE: the block touches
// the edge of a reflecting lattice, and a step that would leave it is
// mirrored ((gy, gx): lattice coordinates of the sub-block's first cell);
// blocks away from the edge take the plain step, which is then the same.
template <int SP, bool MOORE, bool EDGE>
__device__ __forceinline__ void attempt_uni_var(uint8_t* __restrict__ tile, const uint8_t* __restrict__ trans,
                                                uint32_t w, int base, uint32_t tx, uint32_t txi, uint32_t s1,
                                                int gy, int gx, int H, int L) {
  static_assert(2 * SP + 2 < 256, "offsets must fit the byte tables");
  if (EDGE) {
    attempt_variant_2x2(tile, trans, w, MOORE ? 3 : 2, base, SP, tx, txi, s1, true, gy, gx, H, L);
  } else if (MOORE) {
    // the eight neighbour offsets plus SP + 1, as bytes selected by dir ^ 4
    // (byte 0 holds up-left's 0, so the selector's zero nibbles add nothing)
    constexpr uint32_t kLo = 0u | (2u << 8) | ((uint32_t)(2 * SP) << 16) | ((uint32_t)(2 * SP + 2) << 24);
    constexpr uint32_t kHi = 1u | ((uint32_t)(2 * SP + 1) << 8) | ((uint32_t)SP << 16) | ((uint32_t)(SP + 2) << 24);
    const uint32_t dir = (w >> 27) & 7u;
    const int ti = base + (int)(w >> 31) * SP + (int)((w >> 30) & 1u);
    const int tj = ti - SP - 1 + (int)__byte_perm(kLo, kHi, dir ^ 4u);
    apply_rule(tile, trans, ti, tj, w << 5, tx, txi, s1);
  } else {
    attempt_uni<SP>(tile, trans, w, base, tx, txi, s1);
  }
}

// The four fine colour phases of a uniform visit under a rule variant
// (threads 0..255, a CTA barrier after each).
template <bool MOORE, bool EDGE>
__device__ __forceinline__ void fine_phases_var(const LatticeDesc& d, int bx, int by, uint32_t m, uint8_t* tile,
                                                uint32_t ord, const uint8_t* trans) {
  const int t = threadIdx.x, qx = t & 15, qy = t >> 4;
  const uint32_t s1 = (uint32_t)d.S + 1u, tx = d.tx, txi = d.txi;
  const uint32_t GQ = (uint32_t)d.GQ;
  const uint32_t g00 = (uint32_t)(by * (kUniB / 2) + 2 * qy) * GQ + (uint32_t)(bx * (kUniB / 2) + 2 * qx);
  const int base00 = tidx(4 * qy, 4 * qx, kUniSP);
  const int gy00 = by * kUniB + 4 * qy, gx00 = bx * kUniB + 4 * qx;
#pragma unroll
  for (int fi = 0; fi < 4; ++fi) {
    const uint32_t fcol = (ord >> (2 * fi)) & 3u, cx = fcol & 1u, cy = fcol >> 1;
    const uint32_t g = g00 + cy * GQ + cx;
    const int base = base00 + (int)(cy * (2 * kUniSP) + 2 * cx);
    const int gy = gy00 + 2 * (int)cy, gx = gx00 + 2 * (int)cx;
    const uint4 x = philox10_rk(make_uint4(0u, g, m, kTagStep), d.rk);
    attempt_uni_var<kUniSP, MOORE, EDGE>(tile, trans, x.x, base, tx, txi, s1, gy, gx, d.H, d.L);
    attempt_uni_var<kUniSP, MOORE, EDGE>(tile, trans, x.y, base, tx, txi, s1, gy, gx, d.H, d.L);
    attempt_uni_var<kUniSP, MOORE, EDGE>(tile, trans, x.z, base, tx, txi, s1, gy, gx, d.H, d.L);
    attempt_uni_var<kUniSP, MOORE, EDGE>(tile, trans, x.w, base, tx, txi, s1, gy, gx, d.H, d.L);
    __syncthreads();
  }
}

// The four corner cells of a uniform tile (the Moore rule's diagonal
// neighbours), pieces t = 8..11 of the one-byte staging; corners beyond a
// reflecting edge are loaded wrapped and never stepped into, so writing them
// back leaves their (inactive) block unchanged.
__device__ __forceinline__ void corner_uni(const LatticeDesc& d, int x0, int y0, uint8_t* tile, int t, bool store) {
  if (t < 8 || t >= 12) return;
  const int r = (t & 1) ? kUniB : -1, c = (t & 2) ? kUniB : -1;
  uint8_t* cell = d.lat + (size_t)wrap(y0 + r, d.H) * d.pitch + wrap(x0 + c, d.L);
  if (store)
    *cell = tile[tidx(r, c, kUniSP)];
  else
    tile[tidx(r, c, kUniSP)] = __ldcg(cell);
}


// Order in which a visit hands out the quads (2 x 2 groups of fine
// sub-blocks) of a block: first the rx x ry regular ones (columns qx >= irx,
// rows qy >= iry, all four sub-blocks 2 x 2), then the rows qy < iry, then
// the columns qx < irx of the remaining rows.  irx = ceil(fr / 2) when the
// narrow fine width is 2, else every quad is irregular.
struct QuadMap {
  int hx, irx, iry, rx, n_reg, n_top;
  uint32_t inv_hx, inv_rx, inv_irx;
};

__device__ __forceinline__ QuadMap quad_map(const BlockSpan& X, const BlockSpan& Y) {
  QuadMap m;
  const int hx = X.Q >> 1, hy = Y.Q >> 1;
  m.hx = hx;
  m.irx = X.fq == 2 ? (X.fr + 1) >> 1 : hx;
  m.iry = Y.fq == 2 ? (Y.fr + 1) >> 1 : hy;
  m.rx = hx - m.irx;
  m.n_reg = m.rx * (hy - m.iry);
  m.n_top = m.iry * hx;
  // reciprocals: q / k exact as (q * ceil(65536 / k)) >> 16 for q < 2^16 / k
  m.inv_hx = (65536u + (uint32_t)hx - 1u) / (uint32_t)hx;
  m.inv_rx = m.rx > 0 ? (65536u + (uint32_t)m.rx - 1u) / (uint32_t)m.rx : 0u;
  m.inv_irx = m.irx > 0 ? (65536u + (uint32_t)m.irx - 1u) / (uint32_t)m.irx : 0u;
  return m;
}

__device__ __forceinline__ void quad_at(const QuadMap& m, int q, int& qx, int& qy) {
  if (q < m.n_reg) {
    const int r = (int)(((uint32_t)q * m.inv_rx) >> 16);
    qy = m.iry + r;
    qx = m.irx + (q - r * m.rx);
  } else if (q < m.n_reg + m.n_top) {
    const int i = q - m.n_reg, r = (int)(((uint32_t)i * m.inv_hx) >> 16);
    qy = r;
    qx = i - r * m.hx;
  } else {
    const int i = q - m.n_reg - m.n_top, r = (int)(((uint32_t)i * m.inv_irx) >> 16);
    qy = m.iry + r;
    qx = i - r * m.irx;
  }
}

// Visit of coarse block (bx, by) in MCS m, any geometry of the partition.
// The block's span and fine segments come from the closed-form partition
// (no table loads ahead of the tile load); a thread's quad (2 x 2 fine
// sub-blocks) is found with a reciprocal multiply, exact for the at most
// 24 x 24 quads of a block.
// PACKED: the lattice has 4 or 2 bits per site (d.bits); stash then points
// to kStashWords entries of shared memory.
template <bool OWN_FORDER = true, bool PACKED = false>
__device__ __forceinline__ void visit_generic(const LatticeDesc& d, int bx, int by, uint32_t m,
                                              VisitSmem& sm, uint16_t* stash = nullptr) {
  const BlockSpan X = block_span(d.ax, bx), Y = block_span(d.ay, by);
  const int x0 = X.s0, bw = X.w, y0 = Y.s0, bh = Y.w;
  // packed lattices: the byte staging with the stash; one byte per site:
  // aligned 8-byte groups
  const int sp = PACKED ? tile_pitch(bw) : gen_pitch(bw), org = PACKED ? kColOff : gen_origin(x0);
  const int tid = threadIdx.x, nthr = blockDim.x;
  if (OWN_FORDER && tid == 0) sm.forder = fine_order(d, bx, by, m);
  if (PACKED)
    load_tile_generic<true>(d, x0, y0, bw, bh, sm.tile, sp, stash);
  else
    load_tile_aligned(d, x0, y0, bw, bh, sm.tile, sp, org);
  __syncthreads();
  const uint32_t s1 = (uint32_t)d.S + 1u;
  const uint8_t* trans = reinterpret_cast<const uint8_t*>(sm.trans);
  const int hx = X.Q >> 1, nquads = hx * (Y.Q >> 1);
  const uint32_t inv_hx = (65536u + (uint32_t)hx - 1u) / (uint32_t)hx;
  const uint32_t ord = sm.forder;
  const bool variant = d.nbh == 8 || d.reflect;
  const int lg = d.nbh == 8 ? 3 : 2;
  // Quads in row-major order: a fine phase lasts as long as its largest
  // sub-block (3 x 3 at the block's leading corner), which this order shares
  // out over all warps.  (Handing the all-2 x 2 quads out first, with a
  // shorter 2 x 2 step, was measured 8 % slower here at L = 800 and no
  // faster at L = 3000; the batch chunk kernel, which keeps many blocks in
  // flight per SM, gains from it.)
  for (int fi = 0; fi < 4; ++fi) {
    const int fcol = order_at(ord, fi);
    const int cx = fcol & 1, cy = fcol >> 1;
    for (int q = tid; q < nquads; q += nthr) {
      const int qy = (int)(((uint32_t)q * inv_hx) >> 16), qx = q - qy * hx;
      const int fx = 2 * qx + cx, fy = 2 * qy + cy;
      const int sx = seg_start(X, fx), wx = seg_width(X, fx);
      const int sy = seg_start(Y, fy), wy = seg_width(Y, fy);
      const uint32_t nk = (uint32_t)(wx * wy), n4 = 4u * nk;
      const uint32_t g = (uint32_t)(Y.f0 + fy) * (uint32_t)d.GQ + (uint32_t)(X.f0 + fx);
      // ceil(65536 / wx) for the fine widths 2, 3, 4
      const uint32_t inv_wx = wx == 2 ? 32768u : (wx == 3 ? 21846u : 16384u);
      const int base = (sy + 1) * sp + sx + org;
      for (uint32_t j = 0; 4u * j < nk; ++j) {
        const uint4 x = philox10_rk(make_uint4(j, g, m, kTagStep), d.rk);
        const uint32_t wv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (4u * j + (uint32_t)e < nk) {
            if (variant)
              attempt_variant(sm.tile, trans, wv[e], nk << lg, lg, base, wx, inv_wx, sp, d.tx, d.txi, s1,
                              d.reflect != 0, y0 + sy, x0 + sx, d.H, d.L);
            else
              attempt(sm.tile, trans, wv[e], n4, base, wx, inv_wx, sp, d.tx, d.txi, s1);
          }
      }
    }
    __syncthreads();
  }
  if (PACKED)
    store_tile_generic<true>(d, x0, y0, bw, bh, sm.tile, sp, stash);
  else
    store_tile_aligned(d, x0, y0, bw, bh, sm.tile, sp, org);
}

// ---------------------------------------------------------------------------
// Fused species count of one visit.  After MCS m every site must be counted
// once, by the last block to touch it in that MCS: a site of block X is
// touched by X and by the edge neighbours whose rim strip covers it.  The
// vertical neighbours of a block all have colour c^2, the horizontal ones
// c^1 and the diagonal ones c^3, so the order of the four coarse phases
// decides: a block with slot k counts
//   - its interior sites, except edge rows when the vertical neighbours come
//     later (sV > k) and edge columns when the horizontal ones do (sH > k);
//   - its top/bottom rim sites when sV < k, the end cells also needing
//     sD < k (the diagonal block's rim touches them too);
//   - its left/right rim sites when sH < k, the end cells also needing sD < k.
// The counts are added to sm.hist (zeroed by the caller).

// Number of bytes of w equal to v (v < 128).
__device__ __forceinline__ uint32_t bytes_equal(uint32_t w, uint32_t v) {
  const uint32_t t = w ^ (v * 0x01010101u);
  const uint32_t z = ~(((t & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | t | 0x7F7F7F7Fu);
  return __popc(z);
}

// Sites 16 q .. 16 q + 15 of a row as 16 bytes (any bits per site).
__device__ __forceinline__ uint4 load16(const LatticeDesc& d, uint32_t row, uint32_t q) {
  const uint8_t* p = d.lat + (size_t)row * d.pitch;
  if (d.bits == 8) return __ldcg(reinterpret_cast<const uint4*>(p) + q);
  if (d.bits == 4) {
    const uint2 w = __ldcg(reinterpret_cast<const uint2*>(p) + q);
    return make_uint4(unpack4(w.x, 4), unpack4(w.x >> 16, 4), unpack4(w.y, 4), unpack4(w.y >> 16, 4));
  }
  const uint32_t w = __ldcg(reinterpret_cast<const uint32_t*>(p) + q);
  return make_uint4(unpack4(w, 2), unpack4(w >> 8, 2), unpack4(w >> 16, 2), unpack4(w >> 24, 2));
}

// Adds the species counts of the 16-byte vectors k = start, start + stride,
// ... of a lattice (rows of d.pitch bytes; bytes past column L masked as
// 0xFF, never a state) to a shared histogram part[0..S]: SWAR zero-byte
// counts in registers, one warp reduction and one shared atomic per warp and
// state.  Every lane of the calling warps must call.
__device__ __forceinline__ void count_vectors(const LatticeDesc& d, uint32_t start, uint32_t stride,
                                              uint32_t* part) {
  const int L = d.L, S = d.S;
  const uint32_t vec_per_row = (uint32_t)(L + 15) / 16u;
  const uint32_t total = (uint32_t)d.H * vec_per_row;   // < 2^32 for L, H <= 16384
  uint32_t c[kMaxStates];
#pragma unroll
  for (int v = 0; v < kMaxStates; ++v) c[v] = 0;
  for (uint32_t k = start; k < total; k += stride) {
    const uint32_t row = k / vec_per_row, q = k - row * vec_per_row;
    uint4 w = load16(d, row, q);
    const int col = 16 * (int)q;
    if (col + 16 > L) {
      uint32_t* p = reinterpret_cast<uint32_t*>(&w);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int valid = L - (col + 4 * e);
        if (valid <= 0)
          p[e] = 0xFFFFFFFFu;
        else if (valid < 4)
          p[e] |= 0xFFFFFFFFu << (8 * valid);
      }
    }
#pragma unroll
    for (int v = 0; v < kMaxStates; ++v)
      if (v <= S) c[v] += bytes_equal(w.x, v) + bytes_equal(w.y, v) + bytes_equal(w.z, v) +
                         bytes_equal(w.w, v);
  }
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int v = 0; v < kMaxStates; ++v) {
    if (v <= S) {
      const uint32_t sum = __reduce_add_sync(0xFFFFFFFFu, c[v]);
      if (lane == 0 && sum) atomicAdd(&part[v], sum);
    }
  }
}

__device__ __forceinline__ void hist_add_words(uint32_t* hist, int S, uint32_t w0, uint32_t w1, uint32_t w2,
                                               uint32_t w3) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int v = 0; v < kMaxStates; ++v) {
    if (v <= S) {
      const uint32_t c = bytes_equal(w0, v) + bytes_equal(w1, v) + bytes_equal(w2, v) + bytes_equal(w3, v);
      const uint32_t s = __reduce_add_sync(0xFFFFFFFFu, c);
      if (lane == 0 && s) atomicAdd(&hist[v], s);
    }
  }
}

// Uniform geometry (64x64 blocks): piece t (0..255) is one 16-byte piece of
// the interior and, for t < 24, one rim piece; excluded bytes are set to 0xFF
// (never a state).  hist: per-CTA histogram in shared memory.  All lanes of a
// warp call together.
template <int SP, int COFF>
__device__ __forceinline__ void count_pieces_uni(const uint8_t* tile, uint32_t* hist, int S, int k, int sV,
                                                 int sH, int sD, int t) {
  uint32_t w[4];
  {
    const int r = t >> 2, q = t & 3;
    const uint2* src = reinterpret_cast<const uint2*>(tile + tidx_u<SP, COFF>(r, 16 * q));
    const uint2 a = src[0], b = src[1];
    w[0] = a.x; w[1] = a.y; w[2] = b.x; w[3] = b.y;
    if ((r == 0 || r == kUniB - 1) && sV > k) w[0] = w[1] = w[2] = w[3] = 0xFFFFFFFFu;
    if (q == 0 && sH > k) w[0] |= 0xFFu;
    if (q == 3 && sH > k) w[3] |= 0xFF000000u;
  }
  hist_add_words(hist, S, w[0], w[1], w[2], w[3]);
  // rim pieces: threads 0..7 top/bottom rows (4 x 16 bytes each), threads
  // 8..23 left/right columns (8 x 8 cells each)
  uint32_t x[4] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu};
  if (t < 8 && sV < k) {
    const int r = (t < 4) ? -1 : kUniB, q = t & 3;
    const uint2* src = reinterpret_cast<const uint2*>(tile + tidx_u<SP, COFF>(r, 16 * q));
    const uint2 a = src[0], b = src[1];
    x[0] = a.x; x[1] = a.y; x[2] = b.x; x[3] = b.y;
    if (q == 0 && sD > k) x[0] |= 0xFFu;
    if (q == 3 && sD > k) x[3] |= 0xFF000000u;
  } else if (t >= 8 && t < 24 && sH < k) {
    const int j = t - 8, c = (j < 8) ? -1 : kUniB, r0 = (j & 7) * 8;
    uint32_t p[2] = {0u, 0u};
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int r = r0 + e;
      uint32_t v = tile[tidx_u<SP, COFF>(r, c)];
      if ((r == 0 || r == kUniB - 1) && sD > k) v = 0xFFu;
      p[e >> 2] |= v << (8 * (e & 3));
    }
    x[0] = p[0];
    x[1] = p[1];
  }
  hist_add_words(hist, S, x[0], x[1], x[2], x[3]);
}

// 256 threads, piece t = thread t.
template <int SP, int COFF>
__device__ __forceinline__ void count_visit_uni(const uint8_t* tile, uint32_t* hist, int S, int k, int sV,
                                                int sH, int sD) {
  count_pieces_uni<SP, COFF>(tile, hist, S, k, sV, sH, sD, (int)threadIdx.x);
}

// Any geometry: rows by warps, one site per lane step, shared-memory
// atomics.  The tile has row pitch sp and block column 0 at offset origin;
// nw warps (threads 0 .. 32 nw - 1) take part.
__device__ __forceinline__ void count_tile_generic(const uint8_t* tile, int sp, int origin, int bw, int bh,
                                                   uint32_t* hist, int nw, int k, int sV, int sH, int sD) {
  const int lane = threadIdx.x & 31;
  for (int r = (int)(threadIdx.x >> 5) - 1; r <= bh; r += nw) {
    const bool rim_r = (r < 0 || r >= bh), end_r = (r == 0 || r == bh - 1);
    for (int c = lane - 1; c <= bw; c += 32) {
      const bool rim_c = (c < 0 || c >= bw);
      if (rim_r && rim_c) continue;
      const bool end_c = (c == 0 || c == bw - 1);
      bool count;
      if (rim_r)
        count = sV < k && (!end_c || sD < k);
      else if (rim_c)
        count = sH < k && (!end_r || sD < k);
      else
        count = !(end_r && sV > k) && !(end_c && sH > k);
      if (count) atomicAdd(&hist[tile[(r + 1) * sp + origin + c]], 1u);
    }
  }
}

// The tile as visit_generic<.., PACKED> left it.
template <bool PACKED = false>
__device__ __forceinline__ void count_visit_generic(const LatticeDesc& d, int bx, int by, VisitSmem& sm,
                                                    int k, int sV, int sH, int sD) {
  const BlockSpan X = block_span(d.ax, bx);
  const int bw = X.w, bh = block_span(d.ay, by).w;
  const int sp = PACKED ? tile_pitch(bw) : gen_pitch(bw), org = PACKED ? kColOff : gen_origin(X.s0);
  count_tile_generic(sm.tile, sp, org, bw, bh, sm.hist, blockDim.x >> 5, k, sV, sH, sD);
}

}  // namespace escg_impl
