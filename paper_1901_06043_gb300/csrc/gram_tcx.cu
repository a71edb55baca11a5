// Tensor-core Gram of the column-major mode-0 view (Algorithm 2, n = 0) with
// exact digit products: S = X X^T for the I x K matrix X of FP32 columns.
//
// Arithmetic.  Row i of X is scaled by a power of two s_i with max_k |x_ik s_i|
// in [32, 64) (s_i from the row maxima the norm pass records), and every
// scaled value is split exactly into three integer digits in base 2^7,
//     x s_i = d0 + d1 / 2^7 + d2 / 2^14 + r,   |d0|, |d1|, |d2| <= 64,
// by two rounds of "round to the nearest integer, subtract, scale by 2^7"
// (each subtraction and scaling is exact; r, the last rounding, is the only
// error: |r| <= 2^-15 in these units, 2^-20 of the row maximum).  Digits, and
// d2 / 2^7, are exact in FP16.  The tensor cores (kind::f16, FP32
// accumulators in tensor memory) form all nine digit products, grouped by
// weight:
//     D0 = sum d0 d0'                                      (weight 1)
//     D1 = sum (d0 d1' + d1 d0')                          (2^-7)
//     D2 = sum (d0 d2' + d1 d1' + d2 d0')                 (2^-14)
//     D3 = sum (d1 d2' + d2 d1' + (d2 / 2^7) d2')         (2^-21)
// D0..D2 sum integers of at most 2^12 each (three per column for D2); over a
// window of 1024 columns every partial sum stays an integer below 2^24, so
// those accumulators are exact and the accumulator's truncation never acts
// (it is what moves the eps cut for the rounded-product tensor-core Gram of
// tc.cu).  D3 is not integral: at weight 2^-21 its rounding is ~2^-45 of an
// entry, zero-mean off the diagonal, but on the diagonal it measured a
// systematic +1 % of sum_k r_ik^2, enough to move the sum of the small
// eigenvalues by ~2 % of an eps = 1e-5 threshold; so each diagonal entry's D3
// is summed exactly by the producers (as integers, 2 d1 d2 and d2^2) and the
// tensor cores' D3 is left out there.  Leaving D3 out everywhere is not an
// option: its terms have nonzero mean (d2^2 > 0; and when d1 rounds to +-64
// the remainder d2 takes the opposite sign), measured as a +1e-8 relative
// bias on a trace.  After each window the epilogue warps drain the four sums
// and add D0, D1 / 2^7, D2 / 2^14 and D3 / 2^21 one by one into an exact FP32
// pair (TwoSum, hi + lo) in shared memory (a combined value rounded to FP32
// first measured a +1e-8 trace bias).  The pairs go out as FP64 per-CTA
// partial tiles; a second kernel sums the K splits in a fixed order and
// removes the scales, S_ij = D_ij / (s_i s_j).
//
// The remainders.  The digits give G = sum_k d_ik d_jk with d = x - r, and
// r is correlated with x (it is x's own low part): for a row whose
// neighbours are linear in it, E[x_ik r_jk] = rho_j S_ij / K with rho_j =
// E[r^2] / E[x_j^2] (~2^-40).  So E[G] = S - (S diag(rho) + diag(rho) S) +
// diag(sum_k r_ik^2): every direction is scaled by 1 - O(rho) except for
// the diagonal term, which adds v' diag(sum r^2) v to each eigenvalue and
// so lifts each of the I - R discarded ones by about K E[r^2].  Each diagonal
// entry therefore gets minus its row's sum of r^2 (exact FP64 sums from the
// producers): in an emulation of the digit arithmetic on a 256 x 90112
// view of the benchmarks' recipe (rank 40 plus noise), the sum of the 216
// small eigenvalues lands within 3e-4 of an eps = 1e-5 threshold of its exact
// value this way, and half a threshold off without the term.
//
// The digit split and the TwoSums run on packed FP32 pairs (f32x2
// instructions, two values per instruction, each rounded as the scalar op);
// rounding to an integer is the add-and-subtract of 1.5 * 2^23.
//
// Work split.  Tiles of 128 x 128 over the lower triangle (ta >= tb), times K
// splits sized to one wave of the SMs; the CTAs of a split are adjacent in
// launch order so their shared columns are served from L2.
//
// Roles (24 warps, 80 registers each): warps 0-15 load X (16-byte loads;
// four 4-byte loads in row mode or when I % 4 != 0), split it into the digit
// planes of the A (rows 128 ta..) and B (rows
// 128 tb..) operands, MN-major SW128 (three-stage ring); warps 16-23 drain
// tensor memory, two per lane quarter, 64 columns each, and one thread of
// warp 16 issues each window's MMAs before its drain.  Every wait
// is bounded: one that gives up sets DEV_ERR_MBAR_TIMEOUT and the kernel winds
// down; tensor memory is always released.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace tk {
namespace {

using namespace tc;

constexpr int BK = 16;                          // columns (K) per stage: one MMA step
constexpr int NPROD = 16;                       // one column of the stage each
constexpr int EPI_WARP0 = 16;
constexpr int MMA_WARP = EPI_WARP0;             // the first drain warp also issues the MMAs
constexpr int NEPI = 8;
constexpr int NTHREADS = (EPI_WARP0 + NEPI) * 32;   // 768: 24 warps, 80 registers each
// Stage layout, MN-major SW128 FP16: atoms of 64 mn x 8 k (1 KB).  Each
// operand region is [k group of 8][atom], the digit planes side by side along
// mn (plane q = atoms 2q, 2q + 1), so consecutive planes form one operand of
// 256 rows.
constexpr uint32_t ATOM = 1024;
constexpr uint32_t PLANE_STEP = 2 * ATOM;       // plane q starts at atom 2q
constexpr uint32_t PAIR_BYTES = 128 * 128 * 4;  // hi or lo tile, [col / 2][row][col % 2]
constexpr uint32_t DCORR_BYTES = 128 * 8;      // diagonal corrections per row (FP64)
constexpr int TILE_ELEMS = 128 * 128;
// time per column of a diagonal tile's CTA relative to an off-diagonal one's
// (the producers split 128 rows instead of 256, but also keep the diagonal
// sums).  With the diagonal sums moved into FP64 every 256 stages, a
// 500-row view with 15 splits of each tile took 6.84 against 7.25 ms per
// CTA, and 16 splits per off-diagonal tile with 14 per diagonal one made the
// Gram 3 % faster (6.99 against 7.20 ms).  Equal splits are kept: with
// unequal ones a diagonal CTA reads a column up to half a run apart from
// the off-diagonal CTAs that read it too, far longer than the L2 keeps it,
// so the input would be read from DRAM about twice.
constexpr double kDiagCost = 1.0;

// Per digit count: three 7-bit digits (all nine products, four weight
// classes, windows of 1024 columns) or two (four products, three classes,
// windows of 2048 columns: D1 sums two products of at most 2^12 per column,
// 2048 of them stay within 2^24).  A (rows 128 ta..) holds the digit planes
// and, with three digits, d2 / 2^7 as a fourth; B (rows 128 tb..) the digit
// planes.
template <int NDIG>
struct Dig {
  static constexpr int NPA = NDIG == 3 ? 4 : 2;              // planes of A
  static constexpr int NPB = NDIG;                           // planes of B
  static constexpr int NACC = NDIG == 3 ? 4 : 3;             // accumulators (weight classes)
  static constexpr int NSTAGE = NDIG == 3 ? 3 : 5;
  static constexpr int WIN = NDIG == 3 ? 64 : 128;           // stages per exact window
  static constexpr uint32_t KG_A = 2 * NPA * ATOM, KG_B = 2 * NPB * ATOM;   // k-group strides
  static constexpr uint32_t OFF_A = 0, OFF_B = 2 * KG_A;
  static constexpr uint32_t STAGE_BYTES = 2 * KG_A + 2 * KG_B;   // 28 KB / 16 KB
  static constexpr uint32_t SMEM_BYTES =
      NSTAGE * STAGE_BYTES + 2 * PAIR_BYTES + DCORR_BYTES + 1024;
};

// Byte offset of (mn, k) (mn < 128, k < 16) in plane 0 of an operand region
// with k-group stride kg.
__device__ __forceinline__ uint32_t mn_off(int mn, int k, uint32_t kg) {
  return (uint32_t)(k >> 3) * kg + (uint32_t)(mn >> 6) * ATOM + (uint32_t)(k & 7) * 128u +
         ((uint32_t)(((mn & 63) >> 3) ^ (k & 7)) << 4) + (uint32_t)(mn & 7) * 2u;
}

__device__ __forceinline__ uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (1u << 15) | (1u << 16) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// NA 8-column loads (one per accumulator), then one wait.
template <int NA>
__device__ __forceinline__ void tmem_ld8xn(uint32_t taddr, uint32_t (&r)[4][8]) {
#pragma unroll
  for (int q = 0; q < NA; ++q)
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(r[q][0]), "=r"(r[q][1]), "=r"(r[q][2]), "=r"(r[q][3]), "=r"(r[q][4]),
          "=r"(r[q][5]), "=r"(r[q][6]), "=r"(r[q][7])
        : "r"(taddr + 128u * (uint32_t)q));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 16-byte load that does not allocate in L1 (each value is read once per
// CTA) and keeps the normal L2 policy (the other tiles of the split re-read it).
__device__ __forceinline__ float4 ld_nl1(const float4* p) {
  float4 v;
  asm("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}

// Packed FP32 pair arithmetic (f32x2), each lane rounded to nearest.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {    // a - b, one rounding
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}

// Per-row sums a diagonal tile's producers keep for its diagonal entries,
// two rows per float2 (FP32, exact or short; moved into FP64 every 32
// stages): r2 = sum r^2 (r the last rounding's remainder, in units of the
// last digit) and, with three digits, the diagonal's D3 terms as integers,
// a3 = sum 2 d1 d2 and b3 = sum d2^2 (at most 2^18 and 2^17 over 32 stages).
// The move is ~30 FP64 instructions per lane, each holding its
// sub-partition's FP64 pipe for ~64 cycles, ~8,000 cycles every 32 stages.
// That keeps a diagonal tile's CTA at the pace of the off-diagonal CTAs of
// its K split, which read the same columns: moved every 256 stages, the
// diagonal CTAs ran 6 % faster, drifted ahead and read their columns after
// these had left the L2 (DRAM traffic 1.40x the input instead of 1.00x),
// while the Gram took as long as before (the off-diagonal CTAs set it).
struct DiagAcc {
  float2 r2[2], a3[2], b3[2];
  __device__ void zero() {
#pragma unroll
    for (int u = 0; u < 2; ++u) r2[u] = a3[u] = b3[u] = make_float2(0.f, 0.f);
  }
};

// The digits of two scaled values x (|x| < 64): d0, d1 and (NDIG == 3) d2
// and d2 / 2^7.  x + 1.5 * 2^23 lies in [2^23, 2^24), where the FP32 spacing
// is 1, so the add rounds x to the nearest integer and the subtraction of the
// constant is exact.  R: also add to the diagonal sums (u = 0, 1: which pair
// of rows) r^2, r the exact remainder of the last rounding in units of the
// last digit (|r| <= 1/2): r = 2^14 (x - d0 - d1 / 2^7 - d2 / 2^14), or
// 2^7 (x - d0 - d1 / 2^7); with three digits also 2 d1 d2 and d2^2.
template <int NDIG, bool R>
__device__ __forceinline__ void digits2(float2 x, float2 (&d)[4], DiagAcc& acc, int u) {
  const float2 M = make_float2(0x1.8p23f, 0x1.8p23f), NM = make_float2(-0x1.8p23f, -0x1.8p23f);
  const float2 B = make_float2(128.f, 128.f);
  const float2 d0 = add2(add2(x, M), NM);
  const float2 e = sub2(x, d0);                  // |e| <= 1/2, exact
  const float2 t1 = fma2(e, B, M);
  const float2 d1 = add2(t1, NM);                // round(128 e)
  const float2 f = fma2(e, B, sub2(M, t1));      // 128 e - d1, exact, |f| <= 1/2
  d[0] = d0;
  d[1] = d1;
  if (NDIG == 2) {
    if (R) acc.r2[u] = fma2(f, f, acc.r2[u]);
    return;
  }
  const float2 t2 = fma2(f, B, M);
  const float2 d2 = add2(t2, NM);                // round(128 f)
  if (R) {
    const float2 r = fma2(f, B, sub2(M, t2));    // 128 f - d2, exact, |r| <= 1/2
    acc.r2[u] = fma2(r, r, acc.r2[u]);
    acc.a3[u] = fma2(mul2(d1, d2), make_float2(2.f, 2.f), acc.a3[u]);   // integers: exact
    acc.b3[u] = fma2(d2, d2, acc.b3[u]);
  }
  d[2] = d2;
  d[3] = mul2(d2, make_float2(0x1p-7f, 0x1p-7f));
}

// The digit planes of four values (scaled by s) as FP16 pairs: the first NP
// of d0, d1, d2, d2 / 2^7; R: the diagonal sums of the four rows grow.
template <int NP, int NDIG, bool R>
__device__ __forceinline__ void digits4(float4 v, const float2 (&s)[2], uint2 (&p)[4],
                                        DiagAcc& acc) {
  float2 a[4], b[4];
  digits2<NDIG, R>(mul2(make_float2(v.x, v.y), s[0]), a, acc, 0);
  digits2<NDIG, R>(mul2(make_float2(v.z, v.w), s[1]), b, acc, 1);
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    const __half2 lo = __float22half2_rn(a[q]);
    const __half2 hi = __float22half2_rn(b[q]);
    p[q].x = *reinterpret_cast<const uint32_t*>(&lo);
    p[q].y = *reinterpret_cast<const uint32_t*>(&hi);
  }
}

// The FP32 diagonal sums of the lane's four rows into the FP64 totals of
// their diagonal correction, in scaled units: + D3's diagonal terms
// (2 d1 d2) / 2^21 + d2^2 / 2^28 (three digits), - r^2 times the last
// digit's squared weight.
template <int NDIG>
__device__ __forceinline__ void flush_diag(DiagAcc& acc, double (&tot)[4]) {
  constexpr double W = NDIG == 3 ? 0x1p-28 : 0x1p-14;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float2 r2 = acc.r2[j >> 1];
    double v = -(double)((j & 1) ? r2.y : r2.x);
    if (NDIG == 3) {
      const float2 a3 = acc.a3[j >> 1], b3 = acc.b3[j >> 1];
      v += (double)((j & 1) ? b3.y : b3.x);
      v = fma((double)((j & 1) ? a3.y : a3.x), 0x1p-21, v * W);
    } else {
      v *= W;
    }
    tot[j] += v;
  }
  acc.zero();
}

// (h, l) += v exactly for two entries (TwoSum; l collects the rounding errors).
__device__ __forceinline__ void two_sum2(float2& h, float2& l, float2 v) {
  const float2 s = add2(h, v);
  const float2 bb = sub2(s, h);
  const float2 err = add2(sub2(h, sub2(s, bb)), sub2(v, bb));
  l = add2(l, err);
  h = s;
}

// Column mode (L == 1): X is the column-major I x K matrix, a stage is 16
// consecutive columns.  Row mode (L > 1): element (l, i, r) of the slab view
// at x[l + L (i + I r)]; a stage is 16 consecutive l of one slab r (the last
// l-block of a slab zero-filled past L), K = Rt slabs of nlb blocks each.
struct GramTcxArgs {
  const float* x;
  int64_t L, I, K;         // K: columns (column mode) or slabs (row mode)
  int nlb;                 // row mode: l-blocks per slab, ceil(L / 16)
  int ntiles, nkg, T;      // tiles of the lower triangle, K splits of an off-diagonal tile, row blocks
  int nkg_diag;            // K splits of a diagonal tile
  int noff;                // off-diagonal tiles: CTAs [0, noff * nkg) hold them, the
                           // diagonal ones follow
  const float* scale;      // I power-of-two row scales s_i
  double* part;            // gridDim.x partial tiles, [col][row], FP64 (scaled units)
  unsigned* err;
};

// The j-th off-diagonal tile (ta > tb) of the lower triangle, row by row.
__device__ __forceinline__ void offdiag_tile(int j, int& ta, int& tb) {
  int a = 1;
  while (j >= a) { j -= a; ++a; }
  ta = a;
  tb = j;
}

// Tile t of the lower triangle in row order: (ta, tb) with t = ta (ta + 1) / 2 + tb.
__device__ __forceinline__ void tile_of(int t, int& ta, int& tb) {
  int a = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
  while ((a + 1) * (a + 2) / 2 <= t) ++a;
  while (a * (a + 1) / 2 > t) --a;
  ta = a;
  tb = t - a * (a + 1) / 2;
}

// This CTA's tile and K split.  Equal splits (the planner's choice): split
// by split, all tiles of a split adjacent in launch order, so the CTAs that
// read the same columns at the same time sit side by side (same die, same
// L2 partition).  Measured on a 500 x 440000 view: DRAM traffic 1.00x the
// input in this order, 1.59x with the diagonal tiles' CTAs moved behind the
// off-diagonal ones (the same columns then read by CTAs far apart).  Unequal
// splits: the off-diagonal tiles first (g.nkg splits each, the tiles of a
// split adjacent), then the diagonal ones (g.nkg_diag splits each).
__device__ __forceinline__ void cta_work(const GramTcxArgs& g, int b, int& ta, int& tb, int& kg,
                                         int& nkg) {
  if (g.nkg == g.nkg_diag) {
    tile_of(b % g.ntiles, ta, tb);
    kg = b / g.ntiles;
    nkg = g.nkg;
  } else if (b < g.noff * g.nkg) {
    offdiag_tile(b % g.noff, ta, tb);
    kg = b / g.noff;
    nkg = g.nkg;
  } else {
    b -= g.noff * g.nkg;
    ta = tb = b % g.T;
    kg = b / g.T;
    nkg = g.nkg_diag;
  }
}

// Producer warp (one of NPROD): loads its share of every stage (rows
// 128 ta.. for A and, NOPS == 2, rows 128 tb.. for B), splits it into digit
// planes and hands the stage to the MMA thread.  Each lane holds four
// consecutive rows of one stage column, as four floats:
//   column mode: rows 4 lane .. 4 lane + 3 of column k0 + 16 s + warp, one
//     16-byte load per operand (the column exists for s < nvalid);
//   row mode: rows 8 warp + 4 h .. + 3 (h = lane / 16) at l = 16 lb + lane % 16
//     of the stage's block (r, lb), four 4-byte loads L apart per operand.
// Loads run PF stages ahead of the conversion (register ring), so each warp
// keeps PF + 1 stages of loads in flight (PF = 3 in column mode, where 4
// spills; 2 in row mode, measured faster than 3 there).  (An L2
// prefetch PD stages ahead changed nothing in column mode and cost 30 % in row
// mode, where the extra instructions outweighed the latency they hid.)  NOPS == 1 (diagonal tile):
// the lane's rows' diagonal corrections (flush_diag) are added into
// dcorr[row] (FP64, shared by the CTA's producers).
template <int NOPS, bool ROW, int NDIG, bool VEC>
__device__ __forceinline__ void produce(const GramTcxArgs& g, uint8_t* smem, uint64_t* bar_full,
                                        uint64_t* bar_empty, const float* s_scale, int ta,
                                        int tb, int64_t k0, int64_t k1, int64_t gs0, int nst,
                                        int warp, int lane, double* dcorr) {
  // diagonal sums: FP32 over 32 stages (exact for the integer sums; for r^2
  // a short sum, where small terms are not lost against a large total),
  // then FP64 per row
  DiagAcc acc;
  acc.zero();
  double dtot[4] = {0.0, 0.0, 0.0, 0.0};
  const int mn = ROW ? 8 * warp + 4 * (lane >> 4) : 4 * lane;   // first row of the lane
  const int kcol = ROW ? (lane & 15) : warp;                     // stage column of the lane
  const int64_t row0[2] = {(int64_t)ta * 128 + mn, (int64_t)tb * 128 + mn};
  float2 sc[NOPS][2];
#pragma unroll
  for (int o = 0; o < NOPS; ++o)
#pragma unroll
    for (int u = 0; u < 2; ++u)
      sc[o][u] = make_float2(s_scale[128 * o + mn + 2 * u], s_scale[128 * o + mn + 2 * u + 1]);
  constexpr int PF = ROW ? 2 : 3;
  float4 ring[PF + 1][NOPS];
  int ls = 0;                                   // next stage to load
  // column mode
  const int64_t kfirst = k0 + warp;
  const int nvalid = ROW ? 0 : (kfirst < k1 ? (int)((k1 - kfirst + BK - 1) / BK) : 0);
  bool rok[NOPS];
  const float* lp[NOPS];
  const int64_t step = (int64_t)BK * g.I;
  // row mode: rows valid per operand and row, this lane's pointer at slab 0,
  // block 0, and the block of the next load
  unsigned rmask[NOPS];
  int64_t rl = 0;
  int lbl = 0;
  const int64_t LI = g.L * g.I;
  if (ROW) {
#pragma unroll
    for (int o = 0; o < NOPS; ++o) {
      rmask[o] = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) rmask[o] |= (row0[o] + j < g.I) ? (1u << j) : 0u;
      lp[o] = g.x + (rmask[o] ? g.L * row0[o] : 0) + kcol;
    }
    rl = gs0 / g.nlb;
    lbl = (int)(gs0 % g.nlb);
  } else {
#pragma unroll
    for (int o = 0; o < NOPS; ++o) {
      rok[o] = row0[o] < g.I;
      rmask[o] = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) rmask[o] |= (row0[o] + j < g.I) ? (1u << j) : 0u;
      lp[o] = g.x + kfirst * g.I + (rok[o] ? row0[o] : 0);
    }
  }
  auto load_next = [&](float4 (&v)[NOPS]) {
    if (ROW) {
      const bool lok = ls < nst && 16 * lbl + kcol < g.L;
      const int64_t off = rl * LI + 16 * lbl;
#pragma unroll
      for (int o = 0; o < NOPS; ++o) {
        const float* q = lp[o] + off;
        const unsigned m = lok ? rmask[o] : 0u;
        v[o].x = (m & 1u) ? __ldg(q) : 0.f;
        v[o].y = (m & 2u) ? __ldg(q + g.L) : 0.f;
        v[o].z = (m & 4u) ? __ldg(q + 2 * g.L) : 0.f;
        v[o].w = (m & 8u) ? __ldg(q + 3 * g.L) : 0.f;
      }
      if (++lbl == g.nlb) { lbl = 0; ++rl; }
    } else {
      const bool kok = ls < nvalid;
#pragma unroll
      for (int o = 0; o < NOPS; ++o) {
        if (VEC) {
          v[o] = (kok && rok[o]) ? ld_nl1(reinterpret_cast<const float4*>(lp[o]))
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
          // I % 4 != 0: the lane's four rows start anywhere in the column;
          // four 4-byte loads, rows past I read as zero
          const unsigned m = kok ? rmask[o] : 0u;
          v[o].x = (m & 1u) ? __ldg(lp[o]) : 0.f;
          v[o].y = (m & 2u) ? __ldg(lp[o] + 1) : 0.f;
          v[o].z = (m & 4u) ? __ldg(lp[o] + 2) : 0.f;
          v[o].w = (m & 8u) ? __ldg(lp[o] + 3) : 0.f;
        }
        lp[o] += step;
      }
    }
    ++ls;
  };
  using D = Dig<NDIG>;
  constexpr int NSTAGE = D::NSTAGE;
  const uint32_t o_a = D::OFF_A + mn_off(mn, kcol, D::KG_A);
  const uint32_t o_b = D::OFF_B + mn_off(mn, kcol, D::KG_B);
#pragma unroll
  for (int u = 0; u < PF; ++u) load_next(ring[u]);
  bool go = true;
  int slot = 0;
  uint32_t eph = 1;                              // parity of the next empty-slot wait
  for (int s0 = 0; s0 < nst && go; s0 += PF + 1) {
#pragma unroll
    for (int u = 0; u <= PF; ++u) {
      const int s = s0 + u;
      if (s >= nst || !go) break;
      load_next(ring[(u + PF) % (PF + 1)]);
      const float4 (&v)[NOPS] = ring[u];
      // split first, then wait for the slot: a freed slot only waits for
      // the stores (the split is off the MMA -> producer -> MMA hand-off)
      uint2 p[4], pb[4];
      digits4<D::NPA, NDIG, NOPS == 1>(v[0], sc[0], p, acc);
      if (NOPS == 2) digits4<D::NPB, NDIG, false>(v[NOPS - 1], sc[NOPS - 1], pb, acc);
      if (s >= NSTAGE) {
        if (!mbar_wait(smem_u32(&bar_empty[slot]), eph, g.err)) { go = false; break; }
      }
      uint8_t* st = smem + (size_t)slot * D::STAGE_BYTES;
#pragma unroll
      for (int q = 0; q < D::NPA; ++q) *reinterpret_cast<uint2*>(st + o_a + q * PLANE_STEP) = p[q];
      if (NOPS == 2) {
#pragma unroll
        for (int q = 0; q < D::NPB; ++q)
          *reinterpret_cast<uint2*>(st + o_b + q * PLANE_STEP) = pb[q];
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bar_full[slot]));
      if (++slot == NSTAGE) { slot = 0; eph ^= 1u; }
      if (NOPS == 1 && (s & 31) == 31) flush_diag<NDIG>(acc, dtot);
    }
  }
  if (NOPS == 1) {
    // the lane's rows, over all its columns, into the CTA's per-row totals
    flush_diag<NDIG>(acc, dtot);
#pragma unroll
    for (int j = 0; j < 4; ++j) atomicAdd(dcorr + mn + j, dtot[j]);
  }
}

// VEC (column mode): I % 4 == 0 and x 16-byte aligned, one 16-byte load per
// lane and operand; otherwise four 4-byte loads (a runtime switch between
// the two in the loop cost 14 %, so each is its own kernel).
template <bool ROW, int NDIG, bool VEC>
__global__ void __launch_bounds__(NTHREADS, 1) k_gram_tcx(GramTcxArgs g) {
  using D = Dig<NDIG>;
  constexpr int NSTAGE = D::NSTAGE;
  constexpr int WIN = D::WIN;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float* hi = reinterpret_cast<float*>(smem + NSTAGE * D::STAGE_BYTES);
  float* lo = hi + TILE_ELEMS;
  float2* hi2 = reinterpret_cast<float2*>(hi);
  float2* lo2 = reinterpret_cast<float2*>(lo);
  double* dcorr = reinterpret_cast<double*>(lo + TILE_ELEMS);
  __shared__ uint64_t bar_full[NSTAGE], bar_empty[NSTAGE], bar_accf, bar_acce, bar_done;
  __shared__ uint32_t tmem_base_sh;
  __shared__ float s_scale[256];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int ta, tb, kg, nkg;
  cta_work(g, (int)blockIdx.x, ta, tb, kg, nkg);
  const bool diag = ta == tb;
  // this CTA's K range: columns [k0, k1) (column mode) or stages [gs0, gs1)
  const int64_t ku = ROW ? g.K * g.nlb : g.K;
  const int64_t k0 = ku * kg / nkg, k1 = ku * (kg + 1) / nkg;
  const int nst = ROW ? (int)(k1 - k0) : (int)((k1 - k0 + BK - 1) / BK);
  const int nwin = (nst + WIN - 1) / WIN;

  for (int t = threadIdx.x; t < 256; t += NTHREADS) {
    const int64_t row = (t < 128) ? (int64_t)ta * 128 + t : (int64_t)tb * 128 + (t - 128);
    s_scale[t] = row < g.I ? g.scale[row] : 1.f;
  }
  for (int t = threadIdx.x; t < 2 * TILE_ELEMS; t += NTHREADS) hi[t] = 0.f;   // hi and lo
  for (int t = threadIdx.x; t < 128; t += NTHREADS) dcorr[t] = 0.0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(smem_u32(&bar_full[s]), NPROD);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    mbar_init(smem_u32(&bar_accf), 1);
    mbar_init(smem_u32(&bar_acce), NEPI);
    mbar_init(smem_u32(&bar_done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
        smem_u32(&tmem_base_sh)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base_sh;
  // Diagonal tiles: each diagonal entry gets the producers' correction
  // (flush_diag) before the tile goes out: its D3 terms summed exactly, and
  // minus sum_k r_ik^2, which matches the diagonal to the off-diagonal
  // entries (see the file comment).

  if (warp < NPROD) {
    // ---------------- producers: X -> digit planes of A (and B)
    if (diag)
      produce<1, ROW, NDIG, VEC>(g, smem, bar_full, bar_empty, s_scale, ta, tb, k0, k1, k0, nst, warp,
                            lane, dcorr);
    else
      produce<2, ROW, NDIG, VEC>(g, smem, bar_full, bar_empty, s_scale, ta, tb, k0, k1, k0, nst, warp,
                            lane, dcorr);
  } else {
    // ---------------- drain warps: exact window sums -> FP32 pairs.  Lane 0
    // of warp MMA_WARP first issues the window's MMAs (nine per stage, one
    // thread); the next window cannot start before this drain ends anyway.
    const int e = warp - EPI_WARP0;
    const int q = warp & 3;                  // lane quarter this warp may access
    const int c0 = (e >> 2) * 64;            // this warp's 64 columns
    const int row = 32 * q + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
    const bool issuer = warp == MMA_WARP && lane == 0;
    bool ok = true, done = false;
    int slot = 0;
    uint32_t fph = 0;                        // parity of the next full-slot wait
    for (int w = 0; w < nwin; ++w) {
      if (warp == MMA_WARP) {
        if (issuer && ok) {
          const uint32_t id128 = instr_desc(128, 128), id256 = instr_desc(128, 256);
          const uint32_t sbase = smem_u32(smem);
          const uint32_t boff = diag ? D::OFF_A : D::OFF_B, bkg = diag ? D::KG_A : D::KG_B;
          const int s_end = min(nst, (w + 1) * WIN);
          if (w >= 1) ok = mbar_wait(smem_u32(&bar_acce), (w - 1) & 1, g.err);
          for (int s = w * WIN; s < s_end && ok; ++s) {
            ok = mbar_wait(smem_u32(&bar_full[slot]), fph, g.err);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t st = sbase + (uint32_t)slot * D::STAGE_BYTES;
            uint64_t a[4], b[3];
#pragma unroll
            for (int u = 0; u < D::NPA; ++u)
              a[u] = smem_desc(st + D::OFF_A + u * PLANE_STEP, ATOM, D::KG_A);
#pragma unroll
            for (int u = 0; u < D::NPB; ++u) b[u] = smem_desc(st + boff + u * PLANE_STEP, ATOM, bkg);
            // b[0] spans planes d0, d1 as one 256-row operand; tensor memory
            // holds D0 | D1 | D2 (| D3) at columns 0 | 128 | 256 (| 384), so
            // a_q x [d0 | d1] lands on two adjacent accumulators.  Each
            // accumulator's first product of a window overwrites (fresh).
            const uint32_t fresh = s == w * WIN ? 0u : 1u;
            if (NDIG == 3) {
              tc_mma(tmem + 0u, a[0], b[0], id256, fresh);      // D0 += a0 d0', D1 += a0 d1'
              tc_mma(tmem + 256u, a[0], b[2], id128, fresh);    // D2 += a0 d2'
              tc_mma(tmem + 128u, a[1], b[0], id256, 1u);       // D1 += a1 d0', D2 += a1 d1'
              tc_mma(tmem + 384u, a[1], b[2], id128, fresh);    // D3 += a1 d2'
              tc_mma(tmem + 256u, a[2], b[0], id256, 1u);       // D2 += a2 d0', D3 += a2 d1'
              tc_mma(tmem + 384u, a[3], b[2], id128, 1u);       // D3 += (d2 / 2^7) d2'
            } else if (fresh) {
              tc_mma(tmem + 0u, a[0], b[0], id256, 1u);         // D0 += a0 d0', D1 += a0 d1'
              tc_mma(tmem + 128u, a[1], b[0], id256, 1u);       // D1 += a1 d0', D2 += a1 d1'
            } else {                                            // first stage of a window
              tc_mma(tmem + 0u, a[0], b[0], id256, 0u);         // D0 = a0 d0', D1 = a0 d1'
              tc_mma(tmem + 256u, a[1], b[1], id128, 0u);       // D2 = a1 d1'
              tc_mma(tmem + 128u, a[1], b[0], id128, 1u);       // D1 += a1 d0'
            }
            tc_commit(smem_u32(&bar_empty[slot]));
            if (++slot == NSTAGE) { slot = 0; fph ^= 1u; }
          }
          if (ok) tc_commit(smem_u32(&bar_accf));
          if (!ok || w == nwin - 1) {
            tc_commit(smem_u32(&bar_done));
            done = true;
          }
        }
        __syncwarp();
      }
      if (!mbar_wait(smem_u32(&bar_accf), w & 1, g.err)) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      for (int cc = 0; cc < 64; cc += 8) {
        uint32_t r[4][8];
        const uint32_t col = (uint32_t)(c0 + cc);
        tmem_ld8xn<D::NACC>(lane_base + col, r);
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
          // the parts D0, D1 / 2^7, D2 / 2^14 (, D3 / 2^21) (each scaling
          // exact) enter the pair one by one (TwoSum each): nothing is
          // rounded before the compensated sum; columns j, j + 1 packed
          const int idx = ((c0 + cc + j) >> 1) * 128 + row;
          float2 h = hi2[idx], l = lo2[idx];
          const float2 p0 = make_float2(__uint_as_float(r[0][j]), __uint_as_float(r[0][j + 1]));
          const float2 p1 = mul2(make_float2(__uint_as_float(r[1][j]), __uint_as_float(r[1][j + 1])),
                                 make_float2(0x1p-7f, 0x1p-7f));
          const float2 p2 = mul2(make_float2(__uint_as_float(r[2][j]), __uint_as_float(r[2][j + 1])),
                                 make_float2(0x1p-14f, 0x1p-14f));
          two_sum2(h, l, p0);
          two_sum2(h, l, p1);
          two_sum2(h, l, p2);
          if (D::NACC == 4) {
            float2 p3 = mul2(make_float2(__uint_as_float(r[3][j]), __uint_as_float(r[3][j + 1])),
                             make_float2(0x1p-21f, 0x1p-21f));
            // a diagonal entry's D3 comes from the producers' exact sums
            if (diag && c0 + cc + j == row) p3.x = 0.f;
            if (diag && c0 + cc + j + 1 == row) p3.y = 0.f;
            two_sum2(h, l, p3);
          }
          hi2[idx] = h;
          lo2[idx] = l;
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bar_acce));
    }
    // a drain that gave up early still lets the issued MMAs retire first
    if (issuer && !done) tc_commit(smem_u32(&bar_done));
  }
  // every tcgen05 op issued by the MMA thread has completed once bar_done fires
  mbar_wait(smem_u32(&bar_done), 0, g.err);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
  }
  // partial tile out (FP64, scaled units)
  double* pt = g.part + (size_t)blockIdx.x * TILE_ELEMS;
  for (int idx = threadIdx.x; idx < TILE_ELEMS; idx += NTHREADS) {
    const int c = idx >> 7, rr = idx & 127;
    const int sidx = ((c >> 1) * 128 + rr) * 2 + (c & 1);
    double v = (double)hi[sidx] + (double)lo[sidx];
    if (diag && c == rr) v += dcorr[rr];
    pt[idx] = v;
  }
}

// S[i][j] = S[j][i] = (sum over the K splits of tile (ta, tb) at [col][row])
// / (s_i s_j), i >= j, splits in order; partial tiles in cta_work's order.
__global__ void k_gram_tcx_reduce(const double* __restrict__ part, int noff, int nkg, int T,
                                  int nkg_diag, int64_t I, const float* __restrict__ scale,
                                  double* __restrict__ S) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= I * I) return;
  const int64_t i = idx / I, j = idx % I;
  if (j > i) return;
  const int ta = (int)(i / 128), tb = (int)(j / 128);
  const size_t off = (size_t)(j - 128 * tb) * 128 + (size_t)(i - 128 * ta);
  double s = 0.0;
  if (nkg == nkg_diag) {
    const int t = ta * (ta + 1) / 2 + tb;
    const int ntiles = T * (T + 1) / 2;
    for (int k = 0; k < nkg; ++k) s += part[(size_t)(t + ntiles * k) * TILE_ELEMS + off];
  } else if (ta == tb) {
    const size_t first = (size_t)noff * nkg + ta;
    for (int k = 0; k < nkg_diag; ++k) s += part[(first + (size_t)T * k) * TILE_ELEMS + off];
  } else {
    const int jo = ta * (ta - 1) / 2 + tb;        // off-diagonal tile index
    for (int k = 0; k < nkg; ++k) s += part[((size_t)jo + (size_t)noff * k) * TILE_ELEMS + off];
  }
  s /= (double)scale[i] * (double)scale[j];
  S[i * I + j] = s;
  S[j * I + i] = s;
}

// Power-of-two row scales from the row maxima (as FP32 bit patterns): the
// largest |x s| in [32, 64); a zero row gets 1; exponents are clamped to the
// FP32 range.
__global__ void k_gram_tcx_scales(const unsigned* __restrict__ rowmax_bits, int64_t I,
                                  float* __restrict__ scale) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= I) return;
  const unsigned b = rowmax_bits[i] & 0x7fffffffu;
  int e = (int)(b >> 23) - 127;              // floor(log2 max) for normal values
  if (b == 0u) e = 5;
  int se = 5 - e;
  if (se > 126) se = 126;
  if (se < -126) se = -126;
  scale[i] = __uint_as_float((unsigned)(se + 127) << 23);
}

// Row maxima of a row-mode slab view, max over (l, r) of |x(l, i, r)|, as
// FP32 bits (non-negative floats order as unsigned integers; rowmax starts at
// 0).  One warp per (row i, run of slabs): lanes stride over l, four slabs at
// a time, and the warp's maximum enters rowmax[i] by one atomicMax.
__global__ void k_rowmax_slab(const float* __restrict__ y, int64_t L, int64_t I, int64_t Rt,
                              int nck, unsigned* __restrict__ rowmax) {
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gw >= I * nck) return;
  const int64_t i = gw % I, ck = gw / I;
  const int64_t r0 = Rt * ck / nck, r1 = Rt * (ck + 1) / nck;
  float m = 0.f;
  const int64_t LI = L * I;
  int64_t r = r0;
  for (; r + 4 <= r1; r += 4) {                 // four slabs' loads in flight
    const float* row = y + L * (i + I * r);
    for (int64_t l = lane; l < L; l += 32) {
      const float a = __ldg(row + l), b = __ldg(row + LI + l);
      const float c = __ldg(row + 2 * LI + l), d = __ldg(row + 3 * LI + l);
      m = fmaxf(m, fmaxf(fmaxf(fabsf(a), fabsf(b)), fmaxf(fabsf(c), fabsf(d))));
    }
  }
  for (; r < r1; ++r) {
    const float* row = y + L * (i + I * r);
    for (int64_t l = lane; l < L; l += 32) m = fmaxf(m, fabsf(__ldg(row + l)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) atomicMax(rowmax + i, __float_as_uint(m));
}

}  // namespace

// Row-mode views whose last l-block is mostly padding stay on the FP32 Gram:
// the l-blocks of a slab may hold at most 25 % zero fill.  Column-mode views
// from 64 rows up (one diagonal tile, its rows past I zero), row-mode views
// from 128.
GramPlan plan_gram_tcx(int64_t L, int64_t I, int64_t Rt, int num_sms) {
  GramPlan p;
  if (I < (L == 1 ? 64 : 128) || I > 4096 || L < 1 || Rt < 1) return p;
  int64_t stages;
  if (L == 1) {
    if (Rt < 4 * BK) return p;
    stages = (Rt + BK - 1) / BK;
  } else {
    const int64_t nlb = (L + BK - 1) / BK;
    if (4 * nlb * BK > 5 * L || L * I >= ((int64_t)1 << 31)) return p;
    stages = Rt * nlb;
    if (stages < 4) return p;
  }
  const int T = (int)((I + 127) / 128);
  const int ntiles = T * (T + 1) / 2, noff = ntiles - T;
  const int64_t maxkg = std::max<int64_t>(1, stages / 4);
  // one wave of CTAs; a diagonal tile splits only its own 128 rows (an
  // off-diagonal one 256), so its CTAs cover kDiagCost / 1 of the columns per
  // unit time and get that share of the splits, and all CTAs finish together
  int ko = 1, kd = 1;
  if (noff == 0) {
    kd = num_sms;
  } else {
    for (int k = 1; k <= num_sms; ++k) {
      const int d = std::max(1, (int)std::ceil(kDiagCost * k - 1e-9));
      if (noff * k + T * d > num_sms) break;
      ko = k;
      kd = d;
    }
  }
  ko = (int)std::min<int64_t>(ko, maxkg);
  kd = (int)std::min<int64_t>(kd, maxkg);
  p.ntiles = ntiles;
  p.ksplit = ko;
  p.ksplit_diag = kd;
  p.nctas = noff * ko + T * kd;
  p.scratch_bytes = (size_t)p.nctas * TILE_ELEMS * sizeof(double) + sizeof(float) * (size_t)I;
  return p;
}

template <bool ROW, int NDIG, bool VEC>
cudaError_t run_gram_tcx(const GramTcxArgs& a, int nctas, cudaStream_t st) {
  constexpr uint32_t smem = Dig<NDIG>::SMEM_BYTES;
  cudaError_t e = cudaFuncSetAttribute(k_gram_tcx<ROW, NDIG, VEC>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_gram_tcx<ROW, NDIG, VEC><<<(unsigned)nctas, NTHREADS, smem, st>>>(a);
  return cudaSuccess;
}

cudaError_t launch_gram_tcx(const float* y, int64_t L, int64_t I, int64_t Rt, const GramPlan& p,
                            const unsigned* rowmax_bits, void* scratch, unsigned* err, double* S,
                            cudaStream_t st, int ndig) {
  if (p.nctas <= 0 || ((uintptr_t)y & 3) != 0 || (ndig != 2 && ndig != 3))
    return cudaErrorInvalidValue;
  cudaError_t e;
  double* part = static_cast<double*>(scratch);
  float* scale = reinterpret_cast<float*>(part + (size_t)p.nctas * TILE_ELEMS);
  k_gram_tcx_scales<<<(unsigned)((I + 255) / 256), 256, 0, st>>>(rowmax_bits, I, scale);
  GramTcxArgs a;
  a.x = y;
  a.L = L;
  a.I = I;
  a.K = Rt;
  a.nlb = (int)((L + BK - 1) / BK);
  a.ntiles = p.ntiles;
  a.nkg = p.ksplit;
  a.nkg_diag = p.ksplit_diag;
  a.T = (int)((I + 127) / 128);
  a.noff = p.ntiles - a.T;
  a.scale = scale;
  a.part = part;
  a.err = err;
  const bool vec = (I % 4) == 0 && ((uintptr_t)y & 15) == 0;
  if (L == 1 && vec)
    e = ndig == 3 ? run_gram_tcx<false, 3, true>(a, p.nctas, st)
                  : run_gram_tcx<false, 2, true>(a, p.nctas, st);
  else if (L == 1)
    e = ndig == 3 ? run_gram_tcx<false, 3, false>(a, p.nctas, st)
                  : run_gram_tcx<false, 2, false>(a, p.nctas, st);
  else
    e = ndig == 3 ? run_gram_tcx<true, 3, true>(a, p.nctas, st)
                  : run_gram_tcx<true, 2, true>(a, p.nctas, st);
  if (e != cudaSuccess) return e;
  const int64_t tot = I * I;
  k_gram_tcx_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(
      part, a.noff, p.ksplit, a.T, p.ksplit_diag, I, scale, S);
  count_launches(3);
  return cudaGetLastError();
}

cudaError_t launch_rowmax_slab(const float* y, int64_t L, int64_t I, int64_t Rt, int num_sms,
                               unsigned* rowmax_bits, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(rowmax_bits, 0, sizeof(unsigned) * (size_t)I, st);
  if (e != cudaSuccess) return e;
  int64_t nck = ((int64_t)num_sms * 64 + I - 1) / I;     // ~64 warps per SM
  if (nck > Rt) nck = Rt;
  if (nck < 1) nck = 1;
  const int64_t warps = I * nck;
  k_rowmax_slab<<<(unsigned)((warps + 7) / 8), 256, 0, st>>>(y, L, I, Rt, (int)nck, rowmax_bits);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace tk
