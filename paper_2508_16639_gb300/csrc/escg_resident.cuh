// escg_resident.cuh -- whole-lattice residency: a lattice small enough for
// one CTA's shared memory stays there for every coarse phase of every MCS of
// a launch (temporal blocking taken to the whole lattice), so its MCS need
// no global memory traffic and no waits on other CTAs.
//
// Shared-memory image: rows -1..H, columns -1..L at tidx(r, c, sp) with
// sp = tile_pitch(L); row/column -1 and H/L are a halo holding copies of the
// opposite edge (the periodic neighbours of the edge sites).  A coarse phase
// of colour c:
//   1. refreshes the halo from the edges and keeps a snapshot of it;
//   2. draws the fine colour order of each block of colour c;
//   3. runs the four fine steps: in step fi every block of colour c performs
//      the sub-blocks of its fi-th fine colour (all blocks of one colour are
//      independent, so their steps run side by side, one CTA barrier apart);
//   4. writes back every halo cell that changed to the site it mirrors.
// A halo cell changes only as the rim of an active block, and the site it
// mirrors then belongs to a block of another colour, which nobody updates
// during the phase; the three copies of a lattice corner (two edges and the
// halo corner) serve blocks of three different colours.  So each visit sees
// and leaves exactly what the one-visit-per-tile kernels stage and write
// back, and the results are bit-identical.  With a reflecting boundary the
// halo is never read or written.
#pragma once

#include "escg_device.cuh"

namespace escg_impl {

// Blocks of one colour a resident lattice may have (P, Py <= 8).
constexpr int kResMaxPhaseBlocks = 16;

struct ResidentSmem {
  uint32_t trans[kTransWords];
  uint32_t forder[kResMaxPhaseBlocks];
  int32_t qstart[kResMaxPhaseBlocks + 1];   // prefix sums of the quads of the phase's blocks
  uint32_t hist[kMaxStates];
  uint32_t stop;
};

__host__ __device__ __forceinline__ int resident_pitch(int L) { return ((kColOff + L + 1) + 15) & ~15; }
// Dynamic shared memory of a resident lattice: image + halo snapshot.
__host__ __device__ __forceinline__ int resident_dyn_bytes(int L, int H) {
  return (H + 2) * resident_pitch(L) + ((2 * (L + H) + 4 + 15) & ~15);
}

// Lattice rows -> image (any bits per site), one group of 4 sites per step.
__device__ __forceinline__ void resident_load(const LatticeDesc& d, uint8_t* img, int sp) {
  const int groups = (d.L + 3) >> 2;
  const int total = d.H * groups;
  for (int k = threadIdx.x; k < total; k += blockDim.x) {
    const int r = k / groups, c0 = 4 * (k - r * groups);
    const uint32_t u = unpack4(load_group(d.lat + (size_t)r * d.pitch, c0, d.bits), d.bits);
    uint8_t* dst = img + tidx(r, c0, sp);
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (c0 + e < d.L) dst[e] = (uint8_t)(u >> (8 * e));
  }
}

// Image -> lattice rows (sites past column L written as 0).
__device__ __forceinline__ void resident_store(const LatticeDesc& d, const uint8_t* img, int sp) {
  const int groups = (d.L + 3) >> 2;
  const int total = d.H * groups;
  for (int k = threadIdx.x; k < total; k += blockDim.x) {
    const int r = k / groups, c0 = 4 * (k - r * groups);
    const uint8_t* src = img + tidx(r, c0, sp);
    uint32_t u = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (c0 + e < d.L) u |= (uint32_t)src[e] << (8 * e);
    store_group(d.lat + (size_t)r * d.pitch, c0, d.bits, pack4(u, d.bits));
  }
}

// Halo cell h (0 <= h < 2L + 2H + 4) and the site it mirrors, as image indices.
__device__ __forceinline__ void halo_cell(int L, int H, int sp, int h, int& halo, int& site) {
  if (h < L) {
    halo = tidx(-1, h, sp);
    site = tidx(H - 1, h, sp);
  } else if (h < 2 * L) {
    halo = tidx(H, h - L, sp);
    site = tidx(0, h - L, sp);
  } else if (h < 2 * L + H) {
    halo = tidx(h - 2 * L, -1, sp);
    site = tidx(h - 2 * L, L - 1, sp);
  } else if (h < 2 * L + 2 * H) {
    halo = tidx(h - 2 * L - H, L, sp);
    site = tidx(h - 2 * L - H, 0, sp);
  } else {
    const int q = h - 2 * L - 2 * H;   // corners: (-1,-1) (-1,L) (H,-1) (H,L)
    const int hr = (q & 2) ? H : -1, hc = (q & 1) ? L : -1;
    halo = tidx(hr, hc, sp);
    site = tidx((q & 2) ? 0 : H - 1, (q & 1) ? 0 : L - 1, sp);
  }
}

__device__ __forceinline__ void halo_refresh(int L, int H, int sp, uint8_t* img, uint8_t* snap) {
  const int nh = 2 * (L + H) + 4;
  for (int h = threadIdx.x; h < nh; h += blockDim.x) {
    int halo, site;
    halo_cell(L, H, sp, h, halo, site);
    const uint8_t v = img[site];
    img[halo] = v;
    snap[h] = v;
  }
}

__device__ __forceinline__ void halo_writeback(int L, int H, int sp, uint8_t* img, const uint8_t* snap) {
  const int nh = 2 * (L + H) + 4;
  for (int h = threadIdx.x; h < nh; h += blockDim.x) {
    int halo, site;
    halo_cell(L, H, sp, h, halo, site);
    const uint8_t v = img[halo];
    if (v != snap[h]) img[site] = v;
  }
}

// Species histogram of the image's sites into rs.hist (zeroed here).
__device__ __forceinline__ void resident_count(const LatticeDesc& d, const uint8_t* img, int sp,
                                               ResidentSmem& rs) {
  if (threadIdx.x < kMaxStates) rs.hist[threadIdx.x] = 0;
  __syncthreads();
  const int words = (d.L + 3) >> 2, total = d.H * words, S = d.S;
  uint32_t c[kMaxStates];
#pragma unroll
  for (int v = 0; v < kMaxStates; ++v) c[v] = 0;
  for (int k = threadIdx.x; k < total; k += blockDim.x) {
    const int r = k / words, w = k - r * words;
    uint32_t x = *reinterpret_cast<const uint32_t*>(img + tidx(r, 4 * w, sp));
    const int valid = d.L - 4 * w;
    if (valid < 4) x |= 0xFFFFFFFFu << (8 * valid);   // not a state
#pragma unroll
    for (int v = 0; v < kMaxStates; ++v)
      if (v <= S) c[v] += bytes_equal(x, (uint32_t)v);
  }
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int v = 0; v < kMaxStates; ++v) {
    if (v <= S) {
      const uint32_t s = __reduce_add_sync(0xFFFFFFFFu, c[v]);
      if (lane == 0 && s) atomicAdd(&rs.hist[v], s);
    }
  }
  __syncthreads();
}

// MCS [m_begin, m_end) on the resident image.  At every MCS m + 1 that is a
// multiple of log_every the species counts are taken and on_log(m + 1,
// hist) is called by thread 0; it returns true to stop there.  Returns the
// MCS reached.  All threads of the CTA must call; blockDim.x a multiple of 32.
template <class OnLog>
__device__ uint32_t resident_run(const LatticeDesc& d, uint8_t* img, int sp, uint8_t* snap, ResidentSmem& rs,
                                 uint32_t m_begin, uint32_t m_end, uint32_t log_every, OnLog on_log) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int L = d.L, H = d.H, half = d.P >> 1;
  const int nb4 = (d.P >> 1) * (d.Py >> 1);
  const bool periodic = !d.reflect, variant = d.nbh == 8 || d.reflect;
  const int lg = d.nbh == 8 ? 3 : 2;
  const uint32_t s1 = (uint32_t)d.S + 1u;
  const uint8_t* trans = reinterpret_cast<const uint8_t*>(rs.trans);
  uint32_t m = m_begin;
  for (; m < m_end; ++m) {
    const uint32_t ord = colour_order(philox10_rk(make_uint4(0u, 0u, m, kTagOrder), d.rk).x, d.perm24);
    for (int k = 0; k < 4; ++k) {
      const int colour = order_at(ord, k);
      if (periodic) halo_refresh(L, H, sp, img, snap);
      if (tid < nb4) {
        const int bx = 2 * (tid % half) + (colour & 1), by = 2 * (tid / half) + (colour >> 1);
        rs.forder[tid] = fine_order(d, bx, by, m);
      }
      if (tid == 0) {
        int acc = 0;
        for (int j = 0; j < nb4; ++j) {
          const int bx = 2 * (j % half) + (colour & 1), by = 2 * (j / half) + (colour >> 1);
          rs.qstart[j] = acc;
          acc += (block_span(d.ax, bx).Q >> 1) * (block_span(d.ay, by).Q >> 1);
        }
        rs.qstart[nb4] = acc;
      }
      __syncthreads();
      const int nq = rs.qstart[nb4];
      for (int fi = 0; fi < 4; ++fi) {
        int j = 0;
        for (int it = tid; it < nq; it += nthr) {
          while (it >= rs.qstart[j + 1]) ++j;   // items ascend per thread
          const int bx = 2 * (j % half) + (colour & 1), by = 2 * (j / half) + (colour >> 1);
          const BlockSpan X = block_span(d.ax, bx), Y = block_span(d.ay, by);
          const int hx = X.Q >> 1, q = it - rs.qstart[j];
          const int qy = q / hx, qx = q - qy * hx;
          const int fcol = order_at(rs.forder[j], fi);
          const int fx = 2 * qx + (fcol & 1), fy = 2 * qy + (fcol >> 1);
          const int sx = X.s0 + seg_start(X, fx), wx = seg_width(X, fx);
          const int sy = Y.s0 + seg_start(Y, fy), wy = seg_width(Y, fy);
          const uint32_t nk = (uint32_t)(wx * wy), n4 = 4u * nk;
          const uint32_t g = (uint32_t)(Y.f0 + fy) * (uint32_t)d.GQ + (uint32_t)(X.f0 + fx);
          const uint32_t inv_wx = wx == 2 ? 32768u : (wx == 3 ? 21846u : 16384u);
          const int base = tidx(sy, sx, sp);
          for (uint32_t jj = 0; 4u * jj < nk; ++jj) {
            const uint4 x = philox10_rk(make_uint4(jj, g, m, kTagStep), d.rk);
            const uint32_t wv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int e = 0; e < 4; ++e)
              if (4u * jj + (uint32_t)e < nk) {
                if (variant)
                  attempt_variant(img, trans, wv[e], nk << lg, lg, base, wx, inv_wx, sp, d.tx, d.txi, s1,
                                  d.reflect != 0, sy, sx, H, L);
                else
                  attempt(img, trans, wv[e], n4, base, wx, inv_wx, sp, d.tx, d.txi, s1);
              }
          }
        }
        __syncthreads();
      }
      if (periodic) {
        halo_writeback(L, H, sp, img, snap);
        __syncthreads();
      }
    }
    if (((m + 1u) % log_every) == 0u) {
      resident_count(d, img, sp, rs);
      if (tid == 0) rs.stop = on_log(m + 1u, rs.hist) ? 1u : 0u;
      __syncthreads();
      if (rs.stop) {
        ++m;
        break;
      }
    }
  }
  return m;
}

}  // namespace escg_impl
