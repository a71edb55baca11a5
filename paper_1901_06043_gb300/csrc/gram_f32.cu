// FP32-product Gram of a slab view (Section 5.1, Alg. 2: S = sum over slabs r
// of Y_r Y_r^T, Y_r the I x L slab r).  Column mode (L == 1, the first mode of
// the natural-descending layout): every slab is one column, contiguous in i.
// Row mode (L > 1): a K-block is 16 consecutive l of one slab (contiguous in
// l), transposed into shared memory by 4-byte copies, and the blocks are
// visited in the l-block-major order of gram_order.cuh.
//
// Tile 128 x 128 of the lower triangle per CTA, 256 threads with 8 x 8
// outputs each (float4 shared-memory operands: 4 loads per 64 FMAs), K staged
// 16 slabs at a time by a 3-deep cp.async pipeline, split-K over CTAs with a
// fixed-order FP64 reduction of the partial tiles.
//
// Summation (the rank cut compares a tail of ~1e-9 of the trace, so a biased
// rounding in the diagonal would move the cut): the 16 products of a K-block
// are summed into a fresh register, the block sums are added in FP32
// (round-to-nearest, unbiased for these smoothly distributed terms) over a
// chunk of CHUNK blocks, and every chunk sum enters an exact FP32 pair
// (TwoSum: hi + lo) kept in shared memory.  Nothing on the FP64 pipe runs in
// the main loop.
#include <cstdio>

#include "common.cuh"
#include "gram_order.cuh"
#include "kernels.h"

namespace tk {
namespace {

constexpr int BT = 128;     // output tile
constexpr int BK = 16;      // slabs per stage (= the fresh-register K-block)
constexpr int NST = 3;      // pipeline stages
constexpr int CHUNK = 32;   // K-blocks per FP32 chunk sum
constexpr int NTHR = 256;

// Operand loaders: column mode with 16-byte copies (I % 4 == 0, aligned y),
// column mode with 4-byte copies, row mode (4-byte copies, transposing).
enum { LD_COL16 = 0, LD_COL4 = 1, LD_ROW = 2 };

// Operand row stride in floats: padded in row mode, where 16 consecutive l of
// one row i land in 16 different operand rows (bank spread for the copies).
template <int LD> struct Stride { static constexpr int v = (LD == LD_ROW) ? BT + 4 : BT; };

template <int LD>
struct Smem {
  float a[NST][BK][Stride<LD>::v];
  float b[NST][BK][Stride<LD>::v];
  float hi[BT * BT];
  float lo[BT * BT];
};

__device__ __forceinline__ void cp_async16(float* dst, const float* src, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(src),
               "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(s), "l"(src),
               "r"(valid ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Rows [i0, i0+128) of K-block kb into dst[kk][ii]; zero outside the view.
// Column mode: slabs kb*16 .. kb*16+15.  Row mode: l = l0 .. l0+15 of slab r.
template <int LD>
__device__ __forceinline__ void load_panel(float (*dst)[Stride<LD>::v], const float* __restrict__ y,
                                           const KGeom& g, int64_t i0, int64_t kb) {
  const int tid = threadIdx.x;
  if constexpr (LD == LD_COL16) {
#pragma unroll
    for (int e = 0; e < (BK * BT / 4) / NTHR; ++e) {
      const int c = tid + NTHR * e;
      const int kk = c >> 5, q = c & 31;
      const int64_t r = kb * BK + kk, i = i0 + 4 * q;
      const bool valid = (r < g.Rt) && (i < g.I);
      cp_async16(&dst[kk][4 * q], valid ? y + i + g.I * r : y, valid);
    }
  } else if constexpr (LD == LD_COL4) {
#pragma unroll
    for (int e = 0; e < (BK * BT) / NTHR; ++e) {
      const int c = tid + NTHR * e;
      const int kk = c >> 7, q = c & 127;
      const int64_t r = kb * BK + kk, i = i0 + q;
      const bool valid = (r < g.Rt) && (i < g.I);
      cp_async4(&dst[kk][q], valid ? y + i + g.I * r : y, valid);
    }
  } else {
    const int64_t r = kb / g.nLB;
    int64_t lbeg, lend;
    lblock_range(g, kb - r * g.nLB, BK, lbeg, lend);
    const float* base = y + g.L * g.I * r;
#pragma unroll
    for (int e = 0; e < (BK * BT) / NTHR; ++e) {
      const int c = tid + NTHR * e;
      const int kk = c & 15, q = c >> 4;   // 16 threads read 16 consecutive l of row i
      const int64_t l = lbeg + kk, i = i0 + q;
      const bool valid = (l < lend) && (i < g.I);
      cp_async4(&dst[kk][q], valid ? base + l + g.L * i : y, valid);
    }
  }
}

// Column mode, 16-byte copies, with the per-thread address arithmetic hoisted
// out of the K loop: thread chunk e covers kk = c >> 5, i = i0 + 4 (c & 31)
// (c = tid + 256 e); off[e] = i + I kk, iok[e] = i < I.  Only the last
// K-block of the view can run past Rt.
struct ColPanel {
  int64_t off[2];
  bool iok[2];
};
__device__ __forceinline__ ColPanel col_panel(const KGeom& g, int64_t i0) {
  ColPanel p;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int c = threadIdx.x + NTHR * e;
    const int kk = c >> 5, q = c & 31;
    p.off[e] = i0 + 4 * q + g.I * kk;
    p.iok[e] = i0 + 4 * q < g.I;
  }
  return p;
}
__device__ __forceinline__ void load_col16(float (*dst)[BT], const float* __restrict__ y,
                                           const KGeom& g, const ColPanel& p, int64_t kb) {
  const float* base = y + kb * BK * g.I;
  const bool full = (kb + 1) * BK <= g.Rt;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int c = threadIdx.x + NTHR * e;
    const int kk = c >> 5, q = c & 31;
    const bool valid = p.iok[e] && (full || kb * BK + kk < g.Rt);
    cp_async16(&dst[kk][4 * q], valid ? base + p.off[e] : y, valid);
  }
}

// Row mode, with the block sequence of make_korder / korder_block produced
// incrementally (no divisions in the K loop; the same blocks in the same
// order): the slab r, the l-block lb = run * nL0B + sub of the slab, and the
// split-local slab index rr (order mode 1: lb-major over the split's slabs;
// mode 2: lb fastest).
struct RowPos {
  int64_t r;
  int64_t rr;
  int64_t lb, run, sub;
};
__device__ __forceinline__ RowPos row_pos(const KGeom& g, const KOrder& o, int64_t idx) {
  bool unused;
  const int64_t kb = korder_block(g, o, idx, unused);
  RowPos p;
  p.r = kb / g.nLB;
  p.lb = kb - p.r * g.nLB;
  p.run = p.lb / g.nL0B;
  p.sub = p.lb - p.run * g.nL0B;
  p.rr = p.r - o.r0;
  return p;
}
__device__ __forceinline__ void row_advance(const KGeom& g, const KOrder& o, RowPos& p) {
  auto next_lb = [&]() {
    ++p.lb;
    if (++p.sub == g.nL0B) { p.sub = 0; ++p.run; }
  };
  if (o.mode == 1) {
    if (++p.rr == o.nr) {
      p.rr = 0;
      next_lb();
    }
    p.r = o.r0 + p.rr;
  } else {
    next_lb();
    if (p.lb == g.nLB) { p.lb = 0; p.run = 0; p.sub = 0; ++p.r; }
  }
}
// this thread's fixed part of the row-mode copy addresses: element c = tid +
// 256 e goes to dst[c & 15][c >> 4] from l = lbeg + (c & 15), i = i0 + (c >> 4)
struct RowPanel {
  int64_t off[(BK * BT) / NTHR];
  bool iok[(BK * BT) / NTHR];
};
__device__ __forceinline__ RowPanel row_panel(const KGeom& g, int64_t i0) {
  RowPanel p;
#pragma unroll
  for (int e = 0; e < (BK * BT) / NTHR; ++e) {
    const int c = threadIdx.x + NTHR * e;
    const int kk = c & 15, q = c >> 4;
    p.off[e] = kk + g.L * (i0 + q);
    p.iok[e] = i0 + q < g.I;
  }
  return p;
}
__device__ __forceinline__ void load_row(float (*dst)[Stride<LD_ROW>::v], const float* __restrict__ y,
                                         const KGeom& g, const RowPanel& pp, const RowPos& pos) {
  const int64_t lbeg = pos.run * g.L0 + pos.sub * BK;
  const int64_t rem = (pos.run + 1) * g.L0 - lbeg;   // l left in this run of L0
  const float* base = y + g.L * g.I * pos.r + lbeg;
  const int kk = threadIdx.x & 15;
  const bool lok = kk < rem;
#pragma unroll
  for (int e = 0; e < (BK * BT) / NTHR; ++e) {
    const int c = threadIdx.x + NTHR * e;
    const bool valid = lok && pp.iok[e];
    cp_async4(&dst[kk][c >> 4], valid ? base + pp.off[e] : y, valid);
  }
}

// The 16 K-steps of one stage into the fresh per-block sums, then into acc.
// UPPER == false leaves out the thread's (rows 0-63, columns 64-127)
// quadrant, which lies above the diagonal of a diagonal tile.
// The steps run from the last K of the block to the first: in row mode the
// 16 l of a block are consecutive indices of an already-truncated mode,
// whose energy falls with l, so this adds the products in increasing size
// and no square is added to a sum that dwarfs it (round-to-nearest drops
// the small part of such a square one-sidedly: a negative bias of ~5e-10 of
// the trace with the ascending order).  Column-mode blocks have no order.
template <int SA, bool UPPER>
__device__ __forceinline__ void stage_fma(const float (*A)[SA], const float (*B)[SA], int tx, int ty,
                                          float (&acc)[8][8]) {
  float t[8][8];
#pragma unroll
  for (int kq = 0; kq < BK; ++kq) {
    const int kk = BK - 1 - kq;
    const float4 a0 = *reinterpret_cast<const float4*>(&A[kk][ty * 4]);
    const float4 a1 = *reinterpret_cast<const float4*>(&A[kk][64 + ty * 4]);
    const float4 b0 = *reinterpret_cast<const float4*>(&B[kk][tx * 4]);
    const float4 b1 = *reinterpret_cast<const float4*>(&B[kk][64 + tx * 4]);
    const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int v = 0; v < 8; ++v) {
        if (!UPPER && u < 4 && v >= 4) continue;
        t[u][v] = (kq == 0) ? a[u] * b[v] : fmaf(a[u], b[v], t[u][v]);
      }
  }
#pragma unroll
  for (int u = 0; u < 8; ++u)
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      if (!UPPER && u < 4 && v >= 4) continue;
      acc[u][v] += t[u][v];
    }
}

// CTAs are laid out tile-major over the lower triangle of tiles (row ta,
// then tb <= ta); an off-diagonal tile has ko K-splits, a diagonal tile kd
// (its upper quadrants are skipped, so it gets fewer, longer splits and all
// CTAs finish together).  First CTA of tile row ta:
__host__ __device__ __forceinline__ int64_t row_start(int ta, int ko, int kd) {
  return (int64_t)ko * ta * (ta - 1) / 2 + (int64_t)kd * ta;
}

// Compensated form of stage_fma: t + c is the block's sum of products to
// ~2^-48 relative (t and c are overwritten).  Each product's rounding error is exact (p + ep = a b,
// ep = fma(a, b, -p)) and each addition's is exact (TwoSum); the
// round-to-nearest intrinsics keep the compiler from fusing them.  Used for
// row-mode views with few slabs: after the earlier modes are truncated the
// energy sits in a few l, a few block sums dominate every entry, and their
// FP32 rounding (~6e-8 each) does not average out -- 0.3 of the eps = 1e-4
// threshold on the discarded subspace of a 500x500x500x11x8 tensor's third
// mode.  About 10 FP32 operations per product.
template <int SA, bool UPPER>
__device__ __forceinline__ void stage_fma_comp(const float (*A)[SA], const float (*B)[SA], int tx,
                                               int ty, float (&t)[8][8], float (&c)[8][8]) {
#pragma unroll
  for (int kq = 0; kq < BK; ++kq) {
    const int kk = BK - 1 - kq;
    const float4 a0 = *reinterpret_cast<const float4*>(&A[kk][ty * 4]);
    const float4 a1 = *reinterpret_cast<const float4*>(&A[kk][64 + ty * 4]);
    const float4 b0 = *reinterpret_cast<const float4*>(&B[kk][tx * 4]);
    const float4 b1 = *reinterpret_cast<const float4*>(&B[kk][64 + tx * 4]);
    const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int v = 0; v < 8; ++v) {
        if (!UPPER && u < 4 && v >= 4) continue;
        const float p = __fmul_rn(a[u], b[v]);
        const float ep = fmaf(a[u], b[v], -p);
        if (kq == 0) {
          t[u][v] = p;
          c[u][v] = ep;
        } else {
          const float sum = __fadd_rn(t[u][v], p);
          const float bb = __fsub_rn(sum, t[u][v]);
          const float es = __fadd_rn(__fsub_rn(t[u][v], __fsub_rn(sum, bb)), __fsub_rn(p, bb));
          t[u][v] = sum;
          c[u][v] = __fadd_rn(c[u][v], __fadd_rn(ep, es));
        }
      }
  }
}

// One CTA: tile (ta, tb), ta >= tb, over the K-blocks of its split ks in the
// order of make_korder (column mode: a contiguous run, chunks of CHUNK
// blocks; row mode: l-block-major over the split's slabs, chunk ends from
// korder_block).  Writes its FP64 partial tile
// part[blockIdx.x * BT * BT + row * BT + col].
template <int LD, bool COMP>
__global__ void __launch_bounds__(NTHR, 1)
    k_gram_f32(const float* __restrict__ y, KGeom g, int T, int ko, int kd,
               double* __restrict__ part) {
  constexpr int SA = Stride<LD>::v;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<LD>& sm = *reinterpret_cast<Smem<LD>*>(smem_raw);
  int ta = 0;
  while (ta + 1 < T && row_start(ta + 1, ko, kd) <= (int64_t)blockIdx.x) ++ta;
  const int off = (int)((int64_t)blockIdx.x - row_start(ta, ko, kd));
  const bool diag = off >= ta * ko;
  const int tb = diag ? ta : off / ko;
  const int ks = diag ? off - ta * ko : off % ko;
  const int ksplit = diag ? kd : ko;
  const int64_t ia0 = (int64_t)ta * BT, ib0 = (int64_t)tb * BT;
  const KOrder ord = make_korder(g, ks, ksplit);
  const int64_t count = ord.count;

  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  // this thread's rows ty*4 + {0..3} and 64 + ty*4 + {0..3}; columns likewise with tx
  for (int u = 0; u < 8; ++u) {
    const int row = (u < 4) ? ty * 4 + u : 64 + ty * 4 + (u - 4);
    *reinterpret_cast<float4*>(&sm.hi[row * BT + tx * 4]) = make_float4(0.f, 0.f, 0.f, 0.f);
    *reinterpret_cast<float4*>(&sm.hi[row * BT + 64 + tx * 4]) = make_float4(0.f, 0.f, 0.f, 0.f);
    *reinterpret_cast<float4*>(&sm.lo[row * BT + tx * 4]) = make_float4(0.f, 0.f, 0.f, 0.f);
    *reinterpret_cast<float4*>(&sm.lo[row * BT + 64 + tx * 4]) = make_float4(0.f, 0.f, 0.f, 0.f);
  }

  ColPanel cpa, cpb;
  if constexpr (LD == LD_COL16) {
    cpa = col_panel(g, ia0);
    cpb = col_panel(g, ib0);
  }
  RowPanel rpa, rpb;
  RowPos pre{}, cur{};   // row mode: the block to prefetch next, the block being summed
  if constexpr (LD == LD_ROW) {
    rpa = row_panel(g, ia0);
    rpb = row_panel(g, ib0);
    cur = row_pos(g, ord, 0);
    pre = cur;
  }
  // K-block of position idx in this split's order
  auto block_at = [&](int64_t idx) -> int64_t {
    if constexpr (LD == LD_ROW) {
      bool unused;
      return korder_block(g, ord, idx, unused);
    } else {
      return ord.kb0 + idx;
    }
  };
  auto load_stage = [&](int slot, int64_t kb) {
    if constexpr (LD == LD_COL16) {
      load_col16(sm.a[slot], y, g, cpa, kb);
      if (!diag) load_col16(sm.b[slot], y, g, cpb, kb);
    } else {
      load_panel<LD>(sm.a[slot], y, g, ia0, kb);
      if (!diag) load_panel<LD>(sm.b[slot], y, g, ib0, kb);
    }
  };
  auto load_row_stage = [&](int slot, const RowPos& p) {
    if constexpr (LD == LD_ROW) {
      load_row(sm.a[slot], y, g, rpa, p);
      if (!diag) load_row(sm.b[slot], y, g, rpb, p);
    }
  };
#pragma unroll
  for (int s = 0; s < NST - 1; ++s) {
    if (s < count) {
      if constexpr (LD == LD_ROW) {
        load_row_stage(s, pre);
        row_advance(g, ord, pre);
      } else {
        load_stage(s, block_at(s));
      }
    }
    cp_commit();
  }

  float acc[8][8];
#pragma unroll
  for (int u = 0; u < 8; ++u)
#pragma unroll
    for (int v = 0; v < 8; ++v) acc[u][v] = 0.f;

  int st = 0, sn = NST - 1;   // stage slot of idx, and of idx + NST - 1
  for (int64_t idx = 0; idx < count; ++idx) {
    cp_wait<NST - 2>();
    __syncthreads();
    {
      const int64_t nxt = idx + NST - 1;
      if (nxt < count) {
        if constexpr (LD == LD_ROW) {
          load_row_stage(sn, pre);
          row_advance(g, ord, pre);
        } else {
          load_stage(sn, block_at(nxt));
        }
      }
      cp_commit();
    }
    const float(*A)[SA] = sm.a[st];
    if constexpr (COMP) {
      // every block goes straight into the exact (hi, lo) pair; the first
      // l-block of each run of L0 (l0 < 16: where the energy of the earlier,
      // truncated modes sits) is summed exactly, the others plainly
      float t[8][8], c[8][8];
      bool exact;
      if constexpr (LD == LD_ROW) {
        exact = cur.sub == 0;
        row_advance(g, ord, cur);
      } else {
        const int64_t kbc = block_at(idx);
        exact = ((kbc % g.nLB) % g.nL0B) == 0;
      }
      if (exact) {
        if (diag) stage_fma_comp<SA, false>(A, A, tx, ty, t, c);
        else stage_fma_comp<SA, true>(A, sm.b[st], tx, ty, t, c);
      } else {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
          for (int v = 0; v < 8; ++v) { t[u][v] = 0.f; c[u][v] = 0.f; }
        if (diag) stage_fma<SA, false>(A, A, tx, ty, t);
        else stage_fma<SA, true>(A, sm.b[st], tx, ty, t);
      }
      st = (st + 1 == NST) ? 0 : st + 1;
      sn = (sn + 1 == NST) ? 0 : sn + 1;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int row = (u < 4) ? ty * 4 + u : 64 + ty * 4 + (u - 4);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (diag && u < 4 && h == 1) continue;   // above the diagonal: not computed
          float* ph = &sm.hi[row * BT + h * 64 + tx * 4];
          float* pl = &sm.lo[row * BT + h * 64 + tx * 4];
          float4 vh = *reinterpret_cast<float4*>(ph);
          float4 vl = *reinterpret_cast<float4*>(pl);
          float s2, e2;
          two_sum_f(vh.x, t[u][4 * h + 0], s2, e2); vh.x = s2; vl.x += e2 + c[u][4 * h + 0];
          two_sum_f(vh.y, t[u][4 * h + 1], s2, e2); vh.y = s2; vl.y += e2 + c[u][4 * h + 1];
          two_sum_f(vh.z, t[u][4 * h + 2], s2, e2); vh.z = s2; vl.z += e2 + c[u][4 * h + 2];
          two_sum_f(vh.w, t[u][4 * h + 3], s2, e2); vh.w = s2; vl.w += e2 + c[u][4 * h + 3];
          *reinterpret_cast<float4*>(ph) = vh;
          *reinterpret_cast<float4*>(pl) = vl;
        }
      }
      continue;
    }
    if (diag) stage_fma<SA, false>(A, A, tx, ty, acc);
    else stage_fma<SA, true>(A, sm.b[st], tx, ty, acc);
    st = (st + 1 == NST) ? 0 : st + 1;
    sn = (sn + 1 == NST) ? 0 : sn + 1;

    bool chunk_end;
    if constexpr (LD == LD_ROW) {
      // korder_block's chunk ends, from the position of block idx
      chunk_end = (ord.mode == 2) || (cur.rr == ord.nr - 1) || (((cur.rr + 1) % GCHUNK) == 0);
      row_advance(g, ord, cur);
    } else {
      chunk_end = ((idx + 1) % CHUNK) == 0;
    }
    if (chunk_end || idx + 1 == count) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int row = (u < 4) ? ty * 4 + u : 64 + ty * 4 + (u - 4);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float* ph = &sm.hi[row * BT + h * 64 + tx * 4];
          float* pl = &sm.lo[row * BT + h * 64 + tx * 4];
          float4 vh = *reinterpret_cast<float4*>(ph);
          float4 vl = *reinterpret_cast<float4*>(pl);
          float s, e;
          two_sum_f(vh.x, acc[u][4 * h + 0], s, e); vh.x = s; vl.x += e;
          two_sum_f(vh.y, acc[u][4 * h + 1], s, e); vh.y = s; vl.y += e;
          two_sum_f(vh.z, acc[u][4 * h + 2], s, e); vh.z = s; vl.z += e;
          two_sum_f(vh.w, acc[u][4 * h + 3], s, e); vh.w = s; vl.w += e;
          *reinterpret_cast<float4*>(ph) = vh;
          *reinterpret_cast<float4*>(pl) = vl;
        }
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[u][v] = 0.f;
      }
    }
  }
  cp_wait<0>();

  double* out = part + (int64_t)blockIdx.x * BT * BT;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int row = (u < 4) ? ty * 4 + u : 64 + ty * 4 + (u - 4);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int col = h * 64 + tx * 4;
      const float4 vh = *reinterpret_cast<const float4*>(&sm.hi[row * BT + col]);
      const float4 vl = *reinterpret_cast<const float4*>(&sm.lo[row * BT + col]);
      double2* o = reinterpret_cast<double2*>(out + row * BT + col);
      o[0] = make_double2((double)vh.x + (double)vl.x, (double)vh.y + (double)vl.y);
      o[1] = make_double2((double)vh.z + (double)vl.z, (double)vh.w + (double)vl.w);
    }
  }
}

// S[i][j] = S[j][i] = sum over the tile's K-splits (fixed order) of its
// partial tiles.
__global__ void k_gram_f32_reduce(const double* __restrict__ part, int T, int ko, int kd,
                                  int64_t I, double* __restrict__ S) {
  const int64_t ntiles = (int64_t)T * (T + 1) / 2;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ntiles * BT * BT) return;
  const int tile = (int)(idx / (BT * BT));
  const int e = (int)(idx % (BT * BT));
  int ta = (int)((sqrtf(8.f * tile + 1.f) - 1.f) * 0.5f);
  while ((ta + 1) * (ta + 2) / 2 <= tile) ++ta;
  while (ta * (ta + 1) / 2 > tile) --ta;
  const int tb = tile - ta * (ta + 1) / 2;
  const int64_t i = (int64_t)ta * BT + e / BT, j = (int64_t)tb * BT + e % BT;
  if (i >= I || j >= I) return;
  if (ta == tb && j > i) return;   // diagonal tile: its lower half (mirrored below)
  const int64_t first = row_start(ta, ko, kd) + (int64_t)tb * ko;
  const int nk = (ta == tb) ? kd : ko;
  double s = 0.0;
  for (int k = 0; k < nk; ++k) s += part[(first + k) * BT * BT + e];
  S[i * I + j] = s;
  S[j * I + i] = s;
}

}  // namespace

GramPlan plan_gram_f32(int64_t L, int64_t I, int64_t Rt, int num_sms, int64_t L0) {
  GramPlan p;
  if (I < 64 || Rt < 1 || L < 1) return p;   // ntiles == 0: not applicable
  const KGeom g = make_kgeom(L, I, Rt, BK, L0);
  const int64_t T = (I + BT - 1) / BT;
  p.ntiles = (int)(T * (T + 1) / 2);
  const int64_t noff = T * (T - 1) / 2;
  // one wave of one CTA per SM; a diagonal tile costs ~3/4 of an
  // off-diagonal one per K-block (one quadrant skipped, one panel loaded)
  int64_t ko = 1, kd = 1;
  for (int64_t k = 1; k <= num_sms; ++k) {
    const int64_t d = (3 * k + 2) / 4 > 0 ? (3 * k + 2) / 4 : 1;
    if (noff * k + T * d > num_sms) break;
    ko = k;
    kd = d;
  }
  if (noff == 0) kd = num_sms;   // a single diagonal tile
  const int64_t cap = (int64_t)(256ll << 20) / ((int64_t)BT * BT * 8);
  while (noff * ko + T * kd > cap && (ko > 1 || kd > 1)) {
    if (ko > 1) --ko;
    if (kd > 1) --kd;
  }
  if (ko > g.NKB) ko = g.NKB;
  if (kd > g.NKB) kd = g.NKB;
  p.ksplit = (int)ko;
  p.ksplit_diag = (int)kd;
  p.nctas = (int)(noff * ko + T * kd);
  p.scratch_bytes = (size_t)p.nctas * BT * BT * sizeof(double);
  return p;
}

template <int LD, bool COMP>
static cudaError_t launch_ld(const float* y, const KGeom& g, const GramPlan& p, double* scratch,
                             cudaStream_t st) {
  const int smem = (int)sizeof(Smem<LD>);
  cudaError_t e =
      cudaFuncSetAttribute(k_gram_f32<LD, COMP>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int T = (int)((g.I + BT - 1) / BT);
  k_gram_f32<LD, COMP><<<p.nctas, NTHR, smem, st>>>(y, g, T, p.ksplit, p.ksplit_diag, scratch);
  return cudaGetLastError();
}

int gram_f32_compensated(int64_t L, int64_t Rt) { return L > 1 && Rt < 4096; }

cudaError_t launch_gram_f32(const float* y, int64_t L, int64_t I, int64_t Rt, int64_t L0,
                            const GramPlan& p, double* scratch, double* S, cudaStream_t st) {
  const KGeom g = make_kgeom(L, I, Rt, BK, L0);
  cudaError_t e;
  if (L > 1) {
    e = gram_f32_compensated(L, Rt) ? launch_ld<LD_ROW, true>(y, g, p, scratch, st)
                                    : launch_ld<LD_ROW, false>(y, g, p, scratch, st);
  } else if ((I % 4 == 0) && ((((uintptr_t)y) & 15) == 0)) {
    e = launch_ld<LD_COL16, false>(y, g, p, scratch, st);
  } else {
    e = launch_ld<LD_COL4, false>(y, g, p, scratch, st);
  }
  if (e != cudaSuccess) return e;
  const int64_t tot = (int64_t)p.ntiles * BT * BT;
  k_gram_f32_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(
      scratch, (int)((I + BT - 1) / BT), p.ksplit, p.ksplit_diag, I, S);
  count_launches(2);
  return cudaGetLastError();
}

}  // namespace tk
