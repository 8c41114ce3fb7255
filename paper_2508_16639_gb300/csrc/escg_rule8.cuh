// escg_rule8.cuh -- the elementary step (Alg. 3) on a transition table kept
// in shared memory as one 8-byte entry per pair: .x the four new pairs (byte
// `act` for action act: 0 exchange, 1 interaction, 2 reproduction, 3 no
// change; new pair a' | b' << 4), .y the pair's interaction threshold (an
// interaction draw u >= it does not take place).  It is LatticeDesc::trans
// with its two halves interleaved, so that a step off the exchange path reads
// one entry instead of two dependent words.  Used by the generic block owners
// and the batch engine's TMA chunk kernel.
#pragma once

#include <cstdint>

#include "escg_device.cuh"

namespace escg_impl {

// t2[p] for the pairs p < (S + 1)^2 from the table `trans` (LatticeDesc
// layout), threads t0, t0 + n, ... of the caller.
__device__ __forceinline__ void fill_trans8(uint2* t2, const uint8_t* trans, int S, int t0, int n) {
  const uint32_t* src = reinterpret_cast<const uint32_t*>(trans);
  for (int k = t0; k < (S + 1) * (S + 1); k += n) t2[k] = make_uint2(src[k], src[kTransPairs + k]);
}

// attempt_2x2 on the 8-byte table.
__device__ __forceinline__ void attempt8_2x2(uint8_t* __restrict__ tile, const uint2* __restrict__ t2, uint32_t w,
                                             int base, int sp, uint32_t tx, uint32_t txi, uint32_t s1) {
  const uint32_t dir = (w >> 28) & 3u;
  const int ti = base + (int)(w >> 31) * sp + (int)((w >> 30) & 1u);
  const int mag = (dir & 2u) ? 1 : sp;
  const int tj = ti + ((dir & 1u) ? mag : -mag);
  rule8(tile, t2, ti, tj, tile[ti], tile[tj], w << 4, tx, txi, s1);
}

// attempt (a generic sub-block's step) on the 8-byte table.
__device__ __forceinline__ void attempt8(uint8_t* __restrict__ tile, const uint2* __restrict__ t2, uint32_t w,
                                         uint32_t n4, int base, int wx, uint32_t inv_wx, int sp, uint32_t tx,
                                         uint32_t txi, uint32_t s1) {
  int ti, tj;
  uint32_t u;
  locate(w, n4, base, wx, inv_wx, sp, ti, tj, u);
  rule8(tile, t2, ti, tj, tile[ti], tile[tj], u, tx, txi, s1);
}

// Steps t < n of a generic sub-block from the words wv[] in registers, each
// step's cell and neighbour located while the previous step's pair is read.
template <int N>
__device__ __forceinline__ void attempts8_ahead(uint8_t* __restrict__ tile, const uint2* __restrict__ t2,
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
    rule8(tile, t2, ti, tj, a, b, u, tx, txi, s1);
    ti = ti2;
    tj = tj2;
    u = u2;
  }
}

}  // namespace escg_impl
