// escg_device.cuh -- device-side building blocks of the ESCG Monte Carlo
// step on sm_103a: Philox4x32-10, the per-lattice parameter block, the
// elementary step on a shared-memory tile, and the visit of one coarse block
// (load block + 1-site rim, four fine colour phases, write back).
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
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
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

// The 24 orders of the four colours, lexicographic; entry = 4 x 2-bit
// colours, first colour in the lowest bits.
__device__ __constant__ uint8_t c_perm24[24];

__device__ __forceinline__ uint32_t colour_order(uint32_t x0) {
  return c_perm24[__umulhi(x0, 24u)];
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
  uint8_t trans[3 * kMaxStates * kMaxStates];
  int16_t fsx[kMaxFine + 1], fsy[kMaxFine + 1];   // block-local fine starts
  uint32_t forder;
};

// One elementary step (Alg. 3) on the tile.  w: the attempt's 32-bit Philox
// word; n4 = 4 * cells of the sub-block; base: tile index of the sub-block's
// first cell; wx: sub-block width; inv_wx = ceil(65536 / wx).
__device__ __forceinline__ void attempt(uint8_t* __restrict__ tile, const uint8_t* __restrict__ trans,
                                        uint32_t w, uint32_t n4, int base, int wx, uint32_t inv_wx,
                                        int sp, uint32_t tx, uint32_t txi, uint32_t tx_all,
                                        uint32_t txi_all, uint32_t s1, uint32_t ts) {
  const uint32_t hi = __umulhi(w, n4);
  const uint32_t u = w * n4;
  const uint32_t site = hi >> 2, dir = hi & 3u;
  const uint32_t r = (site * inv_wx) >> 16;
  const uint32_t c = site - r * (uint32_t)wx;
  const int ti = base + (int)r * sp + (int)c;
  const int mag = (dir & 2u) ? 1 : sp;
  const int tj = ti + ((dir & 1u) ? mag : -mag);
  const uint32_t a = tile[ti], b = tile[tj];
  const bool ex = tx_all | (u < tx);
  const bool in = txi_all | (u < txi);
  const uint32_t idx = (ex ? 0u : (in ? ts : 2u * ts)) + a * s1 + b;
  const uint32_t nn = trans[idx];
  tile[ti] = (uint8_t)(nn & 15u);
  tile[tj] = (uint8_t)(nn >> 4);
}

// Tile index of block-local (row r, col c), r, c in [-1, B].
__device__ __forceinline__ int tidx(int r, int c, int sp) { return (r + 1) * sp + c + kColOff; }

__device__ __forceinline__ int wrap(int v, int L) { return v < 0 ? v + L : (v >= L ? v - L : v); }

// Loads block interior + the four 1-site rim strips (no corners) into the
// tile through L2 (ld.global.cg: data written by other CTAs of the same
// launch must not be served from a stale L1 line).
__device__ __forceinline__ void load_tile(const LatticeDesc& d, int x0, int y0, int bw, int bh,
                                          uint8_t* tile, int sp) {
  const int L = d.L, pitch = d.pitch;
  const uint8_t* lat = d.lat;
  const int nthr = blockDim.x;
  if (d.uniform64) {
    // interior: 64 rows x 64 bytes as 16-byte loads; rows 16-byte aligned
    for (int k = threadIdx.x; k < 64 * 4; k += nthr) {
      const int r = k >> 2, q = k & 3;
      const uint4 v = __ldcg(reinterpret_cast<const uint4*>(lat + (size_t)(y0 + r) * pitch + x0) + q);
      uint2* dst = reinterpret_cast<uint2*>(tile + tidx(r, 16 * q, sp));
      dst[0] = make_uint2(v.x, v.y);
      dst[1] = make_uint2(v.z, v.w);
    }
    // top / bottom rim rows: 2 x 4 x 16 bytes
    for (int k = threadIdx.x; k < 8; k += nthr) {
      const int top = k < 4, q = k & 3;
      const int r = top ? -1 : 64;
      const int gy = wrap(y0 + r, L);
      const uint4 v = __ldcg(reinterpret_cast<const uint4*>(lat + (size_t)gy * pitch + x0) + q);
      uint2* dst = reinterpret_cast<uint2*>(tile + tidx(r, 16 * q, sp));
      dst[0] = make_uint2(v.x, v.y);
      dst[1] = make_uint2(v.z, v.w);
    }
    // left / right rim columns
    for (int k = threadIdx.x; k < 128; k += nthr) {
      const int left = k < 64, r = k & 63;
      const int c = left ? -1 : 64;
      const int gx = wrap(x0 + c, L);
      tile[tidx(r, c, sp)] = __ldcg(lat + (size_t)(y0 + r) * pitch + gx);
    }
    return;
  }
  const int W = bw + 2, H = bh + 2;
  for (int k = threadIdx.x; k < W * H; k += nthr) {
    const int r = k / W - 1, c = k % W - 1;
    const bool corner = (r < 0 || r >= bh) && (c < 0 || c >= bw);
    if (corner) continue;
    const int gy = wrap(y0 + r, L), gx = wrap(x0 + c, L);
    tile[tidx(r, c, sp)] = __ldcg(lat + (size_t)gy * pitch + gx);
  }
}

// Writes back the block interior and its four rim strips (never the
// corners, which belong to diagonal blocks that may be updated meanwhile).
__device__ __forceinline__ void store_tile(const LatticeDesc& d, int x0, int y0, int bw, int bh,
                                           const uint8_t* tile, int sp) {
  const int L = d.L, pitch = d.pitch;
  uint8_t* lat = d.lat;
  const int nthr = blockDim.x;
  if (d.uniform64) {
    for (int k = threadIdx.x; k < 64 * 4; k += nthr) {
      const int r = k >> 2, q = k & 3;
      const uint2* src = reinterpret_cast<const uint2*>(tile + tidx(r, 16 * q, sp));
      const uint2 a = src[0], b = src[1];
      reinterpret_cast<uint4*>(lat + (size_t)(y0 + r) * pitch + x0)[q] = make_uint4(a.x, a.y, b.x, b.y);
    }
    for (int k = threadIdx.x; k < 8; k += nthr) {
      const int top = k < 4, q = k & 3;
      const int r = top ? -1 : 64;
      const int gy = wrap(y0 + r, L);
      const uint2* src = reinterpret_cast<const uint2*>(tile + tidx(r, 16 * q, sp));
      const uint2 a = src[0], b = src[1];
      reinterpret_cast<uint4*>(lat + (size_t)gy * pitch + x0)[q] = make_uint4(a.x, a.y, b.x, b.y);
    }
    for (int k = threadIdx.x; k < 128; k += nthr) {
      const int left = k < 64, r = k & 63;
      const int c = left ? -1 : 64;
      const int gx = wrap(x0 + c, L);
      lat[(size_t)(y0 + r) * pitch + gx] = tile[tidx(r, c, sp)];
    }
    return;
  }
  const int W = bw + 2, H = bh + 2;
  for (int k = threadIdx.x; k < W * H; k += nthr) {
    const int r = k / W - 1, c = k % W - 1;
    const bool corner = (r < 0 || r >= bh) && (c < 0 || c >= bw);
    if (corner) continue;
    const int gy = wrap(y0 + r, L), gx = wrap(x0 + c, L);
    lat[(size_t)gy * pitch + gx] = tile[tidx(r, c, sp)];
  }
}

__device__ __forceinline__ int tile_pitch(int bw) { return ((kColOff + bw + 1) + 15) & ~15; }

// Loads the transition table of a lattice into shared memory.
__device__ __forceinline__ void load_trans(const LatticeDesc& d, uint8_t* trans) {
  const int n = 3 * (d.S + 1) * (d.S + 1);
  for (int k = threadIdx.x; k < n; k += blockDim.x) trans[k] = d.trans[k];
}

// One visit of coarse block (bx, by) in MCS m: stage, four fine colour
// phases, write back.  Must be called by all threads of the CTA; begins and
// ends with the tile free for reuse.  trans must already be in sm.trans.
__device__ void visit_block(const LatticeDesc& d, int bx, int by, uint32_t m, VisitSmem& sm) {
  const int x0 = d.cs[bx], bw = d.cs[bx + 1] - x0;
  const int y0 = d.cs[by], bh = d.cs[by + 1] - y0;
  const int fx0 = d.fc[bx], Qx = d.fc[bx + 1] - fx0;
  const int fy0 = d.fc[by], Qy = d.fc[by + 1] - fy0;
  const int sp = tile_pitch(bw);
  const int tid = threadIdx.x, nthr = blockDim.x;

  for (int k = tid; k <= Qx; k += nthr) sm.fsx[k] = (int16_t)(d.fs[fx0 + k] - x0);
  for (int k = tid; k <= Qy; k += nthr) sm.fsy[k] = (int16_t)(d.fs[fy0 + k] - y0);
  if (tid == 0) {
    const uint4 x = philox10(make_uint4(0u, (uint32_t)(by * d.P + bx), m, kTagFineOrder), d.key0, d.key1);
    sm.forder = colour_order(x.x);
  }
  load_tile(d, x0, y0, bw, bh, sm.tile, sp);
  __syncthreads();

  const uint32_t s1 = (uint32_t)d.S + 1u, ts = s1 * s1;
  const int hx = Qx >> 1, nquads = hx * (Qy >> 1);
  const uint32_t ord = sm.forder;
  for (int fi = 0; fi < 4; ++fi) {
    const int fcol = order_at(ord, fi);
    const int cx = fcol & 1, cy = fcol >> 1;
    for (int q = tid; q < nquads; q += nthr) {
      const int qy = q / hx, qx = q - qy * hx;
      const int fx = 2 * qx + cx, fy = 2 * qy + cy;
      const int sx = sm.fsx[fx], wx = sm.fsx[fx + 1] - sx;
      const int sy = sm.fsy[fy], wy = sm.fsy[fy + 1] - sy;
      const uint32_t nk = (uint32_t)(wx * wy), n4 = 4u * nk;
      const uint32_t g = (uint32_t)(fy0 + fy) * (uint32_t)d.GQ + (uint32_t)(fx0 + fx);
      const uint32_t inv_wx = (65536u + (uint32_t)wx - 1u) / (uint32_t)wx;
      const int base = tidx(sy, sx, sp);
      for (uint32_t j = 0; 4u * j < nk; ++j) {
        const uint4 x = philox10(make_uint4(j, g, m, kTagStep), d.key0, d.key1);
        const uint32_t wv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (4u * j + (uint32_t)e < nk)
            attempt(sm.tile, sm.trans, wv[e], n4, base, wx, inv_wx, sp, d.tx, d.txi, d.tx_all,
                    d.txi_all, s1, ts);
      }
    }
    __syncthreads();
  }
  store_tile(d, x0, y0, bw, bh, sm.tile, sp);
}

}  // namespace escg_impl
