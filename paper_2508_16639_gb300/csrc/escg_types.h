// escg_types.h -- plain data types and constants shared by the host and
// device code of libescg (no device functions here).
#pragma once

#include <cstdint>

namespace escg_impl {

// Philox counter tags (word 3 of the counter).
constexpr uint32_t kTagInit = 1, kTagOrder = 2, kTagFineOrder = 3, kTagStep = 4;

// Largest coarse block edge the partition rule produces (L in [64,192) gives
// two blocks of up to 96 sites), the tile's column offset of the block
// interior (keeps interior rows 8-byte aligned), and the largest tile pitch.
constexpr int kMaxBlock = 96;
constexpr int kColOff = 8;
constexpr int kMaxTilePitch = 128;   // round_up(kMaxBlock + 23, 16): the aligned generic tile
constexpr int kMaxTileRows = kMaxBlock + 2;
constexpr int kMaxFine = kMaxBlock / 2;  // fine segments per block axis
constexpr int kMaxStates = 16;           // S <= 15
// Transition table: kMaxStates^2 words of action bytes, then kMaxStates^2
// words of interaction thresholds (see LatticeDesc::trans).
constexpr int kTransPairs = kMaxStates * kMaxStates;
constexpr int kTransWords = 2 * kTransPairs;

// Division of any 32-bit n by a divisor d >= 1 known before the launch,
// without the device's division sequence: rcp = floor(2^32 / d) (2^32 - 1
// for d = 1) makes q = floor(n * rcp / 2^32) fall short of floor(n / d) by
// less than n / 2^32 < 1, i.e. by 0 or 1, which one comparison of the
// remainder corrects.
inline uint32_t div_rcp32(uint32_t d) {
  return d <= 1 ? 0xFFFFFFFFu : (uint32_t)((1ull << 32) / d);
}
#if defined(__CUDACC__)
__host__ __device__
#endif
inline uint32_t div_by_rcp(uint32_t n, uint32_t d, uint32_t rcp, uint32_t& rem) {
#if defined(__CUDA_ARCH__)
  uint32_t q = __umulhi(n, rcp);
#else
  uint32_t q = (uint32_t)(((uint64_t)n * rcp) >> 32);
#endif
  uint32_t r = n - q * d;
  if (r >= d) {
    ++q;
    r -= d;
  }
  rem = r;
  return q;
}

// Closed form of one axis's schedule-v1 partition, so that a kernel finds a
// block's span and its fine segments by arithmetic instead of table loads:
// n sites split evenly into P coarse parts (the first r parts q + 1 sites
// wide, the rest q), a part of width w into Q = 2 floor(w/4) fine segments
// split evenly the same way (the first fr segments fq + 1 wide, the rest
// fq).  Suffix a: a wide part (q + 1), b: a narrow one (q).
struct AxisGeom {
  int32_t q, r;
  int32_t Qa, Qb;
  int32_t fqa, fra, fqb, frb;
};

inline AxisGeom make_axis_geom(int n, int P) {
  AxisGeom g;
  g.q = n / P;
  g.r = n % P;
  const int wa = g.q + 1, wb = g.q;
  g.Qa = 2 * (wa / 4);
  g.Qb = 2 * (wb / 4);
  g.fqa = g.Qa > 0 ? wa / g.Qa : 0;
  g.fra = g.Qa > 0 ? wa % g.Qa : 0;
  g.fqb = g.Qb > 0 ? wb / g.Qb : 0;
  g.frb = g.Qb > 0 ? wb % g.Qb : 0;
  return g;
}

// Everything a kernel needs to know about one lattice.
struct LatticeDesc {
  uint8_t* lat;         // H rows of `pitch` bytes, site values 0..S
  int32_t L, pitch;     // columns, row stride in bytes
  int32_t H;            // rows (L for a square lattice)
  int32_t P, GQ;        // coarse and fine segments along the columns
  const int32_t* cs;    // [P+1] coarse segment starts (columns)
  const int32_t* fs;    // [GQ+1] fine segment starts (global column coordinates)
  const int32_t* fc;    // [P+1] first global fine index of each coarse segment
  int32_t Py;           // coarse segments along the rows; block id = by * P + bx,
                        // sub-block id = gy * GQ + gx
  const int32_t* csy;   // the row axis's tables, as cs, fs, fc (the same
  const int32_t* fsy;   // arrays when H = L)
  const int32_t* fcy;
  AxisGeom ax, ay;      // the same partitions in closed form (columns, rows)
  const uint8_t* trans; // kTransWords words: byte (a*(S+1)+b)*4 + action of
                        // the first half holds the new pair (a' | b' << 4),
                        // actions 0 exchange, 1 interaction, 2 reproduction,
                        // 3 no change; word kTransPairs + a*(S+1)+b holds the
                        // pair's interaction threshold (an interaction draw
                        // u >= it does not take place; 0xFFFFFFFF: always)
  uint32_t key0, key1;  // Philox key (seed)
  uint32_t rk[20];      // Philox round keys: rk[2r] = key0 + r*0x9E3779B9,
                        // rk[2r+1] = key1 + r*0xBB67AE85
  uint32_t tx, txi;     // thresholds; 2^32 stored as 0xFFFFFFFF (exact: the
                        // action draw u is always a multiple of 4)
  int32_t S;
  int32_t uniform64;    // all blocks 64x64 and all sub-blocks 2x2
  int32_t nbh;          // neighbourhood: 4 (von Neumann) or 8 (Moore)
  int32_t reflect;      // 1: reflecting boundary, 0: periodic
  int32_t bits;         // bits per site in `lat`: 8 (one byte) or 4, 2 (packed
                        // rows: site c at bits [c*bits, (c+1)*bits), little endian)
  uint8_t perm24[24];   // the 24 colour orders, lexicographic (4 x 2 bits)
  int32_t uniform_var;  // all blocks 64x64 with 2x2 sub-blocks, one byte per site,
                        // and a rule variant (Moore and/or reflecting): the flag
                        // kernel's uniform variant visit
};

// Fills perm24 with the 24 orders of the colours {0,1,2,3} in lexicographic
// order, each packed as 4 x 2 bits (first colour in the lowest bits).
inline void fill_perm24(uint8_t* perm24) {
  int n = 0;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b)
      for (int c = 0; c < 4; ++c)
        for (int e = 0; e < 4; ++e) {
          if (a == b || a == c || a == e || b == c || b == e || c == e) continue;
          perm24[n++] = (uint8_t)(a | (b << 2) | (c << 4) | (e << 6));
        }
}

}  // namespace escg_impl
