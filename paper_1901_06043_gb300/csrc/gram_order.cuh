// K-block geometry and visiting order of a Gram over a slab view (internal;
// shared by the Gram kernels).
#pragma once
#include <cstdint>

namespace tk {

// Geometry of the K (contraction) dimension of a slab view.  K runs over
// (r, l) pairs.  With L == 1 a K-block is BK consecutive slabs (column mode,
// contiguous along i).  Otherwise a K-block is up to BK consecutive l of one
// slab (row mode, contiguous along l) that never cross a multiple of L0, the
// fastest sub-index of l: when the modes below n are already truncated, l0
// is an eigen-sorted index whose energy falls along it, and a block confined
// to one run of l0 can be summed smallest-first (see the Gram kernels).  A
// row of L0 l holds nL0B blocks (the last one partial); a slab holds
// nLB = (L / L0) nL0B blocks.
struct KGeom {
  int64_t L, I, Rt;
  int64_t L0;    // block alignment of l (divides L)
  int64_t nL0B;  // K-blocks per run of L0 l
  int64_t nLB;   // K-blocks per slab in row mode
  int64_t NKB;   // total K-blocks
};

__host__ __device__ inline KGeom make_kgeom(int64_t L, int64_t I, int64_t Rt, int bk,
                                             int64_t L0 = 0) {
  KGeom g{L, I, Rt, L, 1, 1, 0};
  if (L == 1) {
    g.NKB = (Rt + bk - 1) / bk;
  } else {
    if (L0 >= 1 && L0 <= L && L % L0 == 0) g.L0 = L0;
    g.nL0B = (g.L0 + bk - 1) / bk;
    g.nLB = (L / g.L0) * g.nL0B;
    g.NKB = Rt * g.nLB;
  }
  return g;
}

// Row mode: the l range [l_begin, l_end) of l-block lb of a slab.
__host__ __device__ inline void lblock_range(const KGeom& g, int64_t lb, int bk, int64_t& l_begin,
                                             int64_t& l_end) {
  const int64_t row = lb / g.nL0B, sub = lb - row * g.nL0B;
  l_begin = row * g.L0 + sub * bk;
  const int64_t e = row * g.L0 + g.L0;
  l_end = (l_begin + bk < e) ? l_begin + bk : e;
}

// Order in which one CTA (split ks of ksplit) visits its K-blocks, and where
// its FP32 chunks end.  FP32 rounding of a running sum only stays unbiased
// when the terms added to it have comparable size; the l index of a row-mode
// view runs over already-truncated modes, whose energy decays with the index
// (their eigenvalues are in descending order), so summing one slab's l-run
// into one FP32 accumulator drops the small terms systematically.
//   column mode (L == 1):  blocks kb0..kb1-1 (BK slabs each, unordered
//                          energies); a chunk is CHUNK blocks.
//   row mode, Rt >= ksplit: the CTA owns slabs [r0, r0+nr) and visits l-block
//                          lb of all of them before lb+1; a chunk never mixes
//                          l-blocks.
//   row mode, Rt < ksplit:  blocks kb0..kb1-1 (lb fastest); every block is
//                          its own chunk.
struct KOrder {
  int mode;
  int64_t kb0, r0, nr, count;
};

constexpr int GCHUNK = 16;

__device__ __forceinline__ KOrder make_korder(const KGeom& g, int ks, int ksplit) {
  KOrder o{0, 0, 0, 1, 0};
  if (g.L == 1) {
    o.mode = 0;
    o.kb0 = g.NKB * ks / ksplit;
    o.count = g.NKB * (ks + 1) / ksplit - o.kb0;
  } else if (g.Rt >= ksplit) {
    o.mode = 1;
    o.r0 = g.Rt * ks / ksplit;
    o.nr = g.Rt * (ks + 1) / ksplit - o.r0;
    o.count = o.nr * g.nLB;
  } else {
    o.mode = 2;
    o.kb0 = g.NKB * ks / ksplit;
    o.count = g.NKB * (ks + 1) / ksplit - o.kb0;
  }
  return o;
}

__device__ __forceinline__ int64_t korder_block(const KGeom& g, const KOrder& o, int64_t idx,
                                                bool& chunk_end) {
  if (o.mode == 1) {
    const int64_t lb = idx / o.nr, rr = idx - lb * o.nr;
    chunk_end = (rr == o.nr - 1) || ((rr + 1) % GCHUNK == 0);
    return (o.r0 + rr) * g.nLB + lb;
  }
  chunk_end = (o.mode == 2) || ((idx + 1) % GCHUNK == 0);
  return o.kb0 + idx;
}

}  // namespace tk
