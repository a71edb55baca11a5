// Tensor-core (tcgen05) TTM of the column-major mode-0 view (Algorithm 3,
// n = 0): Z (K x Rt) = A (K x I) Y (I x Rt), where slab m of the mode-0 view
// is column m of Y (contiguous in i) and A = U_0^T (or any K x I operator of
// the multi-TTM), K <= 128.  Z is written column-major: the K outputs of one
// slab are contiguous, which is the natural-descending layout of the result;
// or transposed (zt), slab fastest, which puts the new mode last.
//
// Arithmetic.  Y and A are scaled by powers of two (max|y s_y| <= 2^14,
// max|a s_a| <= 2^14) and split into two FP16 numbers each, x s = h + l with
// |x s - h - l| <= 2^-22 |x s|.  D = A_h Y_h + A_h Y_l + A_l Y_h runs on the
// tensor cores (kind::f16, FP32 accumulators in tensor memory) and
// Z = D / (s_a s_y).  The dropped A_l Y_l term (<= 2^-22 relative per
// product) and the accumulator's truncation (a shrink of ~1e-6 relative over
// I ~ 500 products) perturb the data of the next mode far below eps; unlike
// the Gram, no tail sum accumulates them.
//
// Work split.  A tile is 128 consecutive slabs (MMA N = 128) over all of I;
// one persistent CTA per SM walks tiles blockIdx.x, blockIdx.x + gridDim.x,
// ...; a stage is 64 i of the tile.  The kernel is bound by reading Y, a
// stream of 256-byte pieces (64 i of one slab) at the slab pitch, which needs
// ~100 KB of reads in flight per SM to approach the HBM rate.  So Y goes
// through its own ring: one loader thread issues a 2D tiled TMA load of the
// stage's box (64 i x 128 slabs, 32 KB, zero-filled outside the view) into
// one of the raw FP32 slots (three, 96 KB in flight; four, 128 KB, when
// K <= 64 lets the MMA run with M = 64 and the A images halve), completing
// on an mbarrier by byte count; eight converter warps split a raw slot into the
// K-major SW128 FP16 hi/lo B operand of one of two operand slots, and one of
// them bulk-copies the stage's pre-split A chunk next to it; warp 9 issues the
// MMAs; warps 10-13 drain the double-buffered accumulators (2 x 128
// tensor-memory columns) and write Z.  Every wait is bounded: a wait that
// gives up sets DEV_ERR_MBAR_TIMEOUT and the kernel winds down.
#include <cuda.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace tk {
namespace {

using namespace tc;

constexpr int TN = 128;                        // slabs per tile (MMA N)
constexpr uint32_t TMEM_COLS = 2 * TN;         // two accumulator buffers
constexpr int TM = 128;                        // largest MMA M (rows of A; K <= TM)
constexpr int SK = 64;                         // i per stage
constexpr int NOP = 2;                         // operand slots
constexpr int LOAD_WARP = 0;
constexpr int NCONV = 8;                       // converter warps 1..8
constexpr int MMA_WARP = 9;
constexpr int NTHREADS = 14 * 32;              // + epilogue warps 10..13
constexpr uint32_t B_BYTES = TN * SK * 2;      // 16 KB
constexpr uint32_t RAW_BYTES = TN * SK * 4;                  // 32 KB
constexpr int CV4 = (TN * SK / 4) / (NCONV * 32);            // float4 per converter thread (8)

// Shapes per MMA M: with K <= 64 outputs an M = 64 MMA halves the A operand
// (8 KB instead of 16 KB per hi / lo image), which frees a fourth raw Y slot:
// 128 KB of reads in flight per SM instead of 96 KB.  Tensor memory holds
// row r of an M = 64 accumulator in lane 32 (r / 16) + r % 16 (measured).
template <int M>
struct ColCfg {
  static constexpr uint32_t A_BYTES = M * SK * 2;
  static constexpr uint32_t OFF_AH = 0, OFF_AL = A_BYTES, OFF_BH = 2 * A_BYTES,
                            OFF_BL = 2 * A_BYTES + B_BYTES;
  static constexpr uint32_t OP_BYTES = 2 * A_BYTES + 2 * B_BYTES;   // 64 or 48 KB
  static constexpr int NRAW = M == 64 ? 4 : 3;                       // raw Y slots
  static constexpr uint32_t SMEM_BYTES = NOP * OP_BYTES + NRAW * RAW_BYTES + 1024;
  static constexpr int RPQ = M / 4;                                  // accumulator rows per lane quarter
};

// Byte offset of (row, k) in a K-major SW128 FP16 tile with 64 k per row:
// 1024-byte atoms of 8 rows x 128 bytes, 16-byte chunks XOR-swizzled by
// row % 8; atoms 1024 bytes apart along the rows.
__host__ __device__ __forceinline__ uint32_t kmaj_off(int row, int k) {
  return (uint32_t)(row >> 3) * 1024u + (uint32_t)(row & 7) * 128u +
         ((uint32_t)((k >> 3) ^ (row & 7)) << 4) + (uint32_t)(k & 7) * 2u;
}

// Instruction descriptor: kind::f16, FP16 A and B, FP32 D, both K-major.
__device__ __forceinline__ uint32_t instr_desc_kk(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// (a, b) = (h_a + l_a, h_b + l_b): FP16 pairs of the round-to-nearest hi part
// and of the remainder.  Pair conversions (two values per instruction) keep
// the split off the scalar conversion pipe, which bounded the kernel.
__device__ __forceinline__ void split_pack(float a, float b, uint32_t& h, uint32_t& l) {
  const __half2 h2 = __float22half2_rn(make_float2(a, b));
  const float2 hf = __half22float2(h2);
  const __half2 l2 = __float22half2_rn(make_float2(a - hf.x, b - hf.y));
  h = *reinterpret_cast<const uint32_t*>(&h2);
  l = *reinterpret_cast<const uint32_t*>(&l2);
}

// A (K x I, FP64: element (k, i) at A[k*lda + i] if arow else A[k + lda*i])
// -> per stage: [A_h tile | A_l tile] as shared-memory images (K-major SW128,
// tm rows x 64 i, zero outside K x I), scaled by s_a; *sa_out = s_a.
// One CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_ttm_tc_prep(const double* __restrict__ A, int K,
                                                      int64_t I, int64_t lda, int arow, int nks,
                                                      int tm, uint8_t* __restrict__ out,
                                                      float* __restrict__ sa_out) {
  const uint32_t a_bytes = (uint32_t)tm * SK * 2;
  __shared__ double red[32];
  __shared__ float s_sa;
  double mx = 0.0;
  for (int64_t e = threadIdx.x; e < (int64_t)K * I; e += blockDim.x) {
    const int64_t k = e / I, i = e % I;
    const double a = arow ? A[k * lda + i] : A[k + lda * i];
    mx = fmax(mx, fabs(a));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = red[threadIdx.x];
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) {
      int ex = 0;
      frexp(v, &ex);                       // v < 2^ex
      int e2 = 14 - ex;
      e2 = e2 > 100 ? 100 : (e2 < -100 ? -100 : e2);
      s_sa = (v > 0.0) ? ldexpf(1.f, e2) : 1.f;
      *sa_out = s_sa;
    }
  }
  __syncthreads();
  const double sa = s_sa;
  const int64_t tot = (int64_t)nks * tm * (SK / 2);   // element pairs (k, k+1)
  for (int64_t e = threadIdx.x; e < tot; e += blockDim.x) {
    const int ks = (int)(e / (tm * (SK / 2)));
    const int rem = (int)(e % (tm * (SK / 2)));
    const int row = rem / (SK / 2), kp = 2 * (rem % (SK / 2));
    float v2[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int64_t i = (int64_t)ks * SK + kp + t;
      double a = 0.0;
      if (row < K && i < I) a = arow ? A[(int64_t)row * lda + i] : A[row + lda * i];
      v2[t] = (float)(a * sa);
    }
    uint32_t h, l;
    split_pack(v2[0], v2[1], h, l);
    uint8_t* base = out + (size_t)ks * 2 * a_bytes;
    const uint32_t o = kmaj_off(row, kp);
    *reinterpret_cast<uint32_t*>(base + o) = h;
    *reinterpret_cast<uint32_t*>(base + a_bytes + o) = l;
  }
}

struct TtmTcArgs {
  const float* y;        // I x Rt column-major, 16-byte aligned, I % 4 == 0
  int64_t I, Rt;
  int K;                 // rows of A = outputs per slab (<= 128)
  int nks;               // stages per tile = ceil(I / 64)
  int64_t ntiles;        // ceil(Rt / 128)
  float sy;              // power of two
  const uint8_t* aprep;  // nks x [A_h | A_l] images
  const float* sa;       // the power-of-two scale of A (device)
  float* z;              // K x Rt column-major, or (zt) Rt x K column-major
  int zt;                // transposed output: z[r * Rt + slab]
  unsigned* err;
};

template <int M>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_ttm_tc_col(TtmTcArgs g, const __grid_constant__ CUtensorMap ymap) {
  using C = ColCfg<M>;
  constexpr int NRAW = C::NRAW;
  constexpr uint32_t A_BYTES = C::A_BYTES, OP_BYTES = C::OP_BYTES;
  constexpr uint32_t OFF_AH = C::OFF_AH, OFF_AL = C::OFF_AL, OFF_BH = C::OFF_BH,
                     OFF_BL = C::OFF_BL;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* raw = smem + NOP * OP_BYTES;
  __shared__ uint64_t raw_full[NRAW], raw_empty[NRAW], op_full[NOP], op_empty[NOP];
  __shared__ uint64_t bar_accf[2], bar_acce[2], bar_done;
  __shared__ uint32_t tmem_base_sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NRAW; ++s) {
      mbar_init(smem_u32(&raw_full[s]), 1);
      mbar_init(smem_u32(&raw_empty[s]), NCONV);
    }
    for (int s = 0; s < NOP; ++s) {
      mbar_init(smem_u32(&op_full[s]), NCONV);
      mbar_init(smem_u32(&op_empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&bar_accf[b]), 1);
      mbar_init(smem_u32(&bar_acce[b]), 4);
    }
    mbar_init(smem_u32(&bar_done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
        smem_u32(&tmem_base_sh)), "n"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base_sh;
  const int64_t my_tiles =
      (g.ntiles > (int64_t)blockIdx.x) ? (g.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t nstages = my_tiles * g.nks;

  if (warp == LOAD_WARP) {
    // ---------------- loader: Y boxes -> raw slots (TMA)
    if (lane == 0) {
      for (int64_t gs = 0; gs < nstages; ++gs) {
        const int r = (int)(gs % NRAW);
        if (gs >= NRAW &&
            !mbar_wait(smem_u32(&raw_empty[r]), (uint32_t)(((gs / NRAW) - 1) & 1), g.err))
          break;
        const int64_t j = gs / g.nks;
        const int ks = (int)(gs - j * g.nks);
        const int64_t m0 = ((int64_t)blockIdx.x + j * gridDim.x) * TN;
        mbar_arrive_expect_tx(smem_u32(&raw_full[r]), RAW_BYTES);
        tma_load_2d(smem_u32(raw + (size_t)r * RAW_BYTES), &ymap, ks * SK, (int)m0,
                    smem_u32(&raw_full[r]));
      }
    }
    __syncwarp();
  } else if (warp <= NCONV) {
    // ---------------- converters: raw FP32 -> FP16 hi/lo B operand; A chunk
    const int ct = threadIdx.x - 32;   // 0..255
    for (int64_t gs = 0; gs < nstages; ++gs) {
      const int r = (int)(gs % NRAW), o = (int)(gs % NOP);
      const int64_t j = gs / g.nks;
      const int ks = (int)(gs - j * g.nks);
      const int64_t m0 = ((int64_t)blockIdx.x + j * gridDim.x) * TN;
      if (!mbar_wait(smem_u32(&raw_full[r]), (uint32_t)((gs / NRAW) & 1), g.err)) break;
      if (gs >= NOP &&
          !mbar_wait(smem_u32(&op_empty[o]), (uint32_t)(((gs / NOP) - 1) & 1), g.err))
        break;
      uint8_t* st = smem + (size_t)o * OP_BYTES;
      if (ct == 0) {
        mbar_expect_tx(smem_u32(&op_full[o]), 2 * A_BYTES);
        bulk_g2s(smem_u32(st + OFF_AH), g.aprep + (size_t)ks * 2 * A_BYTES, 2 * A_BYTES,
                 smem_u32(&op_full[o]));
      }
      const uint8_t* src = raw + (size_t)r * RAW_BYTES;
      float4 v[CV4];
#pragma unroll
      for (int e = 0; e < CV4; ++e) {
        const int c = ct + NCONV * 32 * e;
        const int m = c >> 4, q = c & 15;
        const bool ok = (m0 + m < g.Rt) && ((int64_t)ks * SK + 4 * q < g.I);
        v[e] = ok ? *reinterpret_cast<const float4*>(src + (size_t)m * (SK * 4) + 16 * q)
                  : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&raw_empty[r]));   // raw slot read
#pragma unroll
      for (int e = 0; e < CV4; ++e) {
        const int c = ct + NCONV * 32 * e;
        const int m = c >> 4, q = c & 15;
        uint2 hp, lp;
        split_pack(v[e].x * g.sy, v[e].y * g.sy, hp.x, lp.x);
        split_pack(v[e].z * g.sy, v[e].w * g.sy, hp.y, lp.y);
        const uint32_t off = kmaj_off(m, 4 * q);
        *reinterpret_cast<uint2*>(st + OFF_BH + off) = hp;
        *reinterpret_cast<uint2*>(st + OFF_BL + off) = lp;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&op_full[o]));
    }
  } else if (warp == MMA_WARP) {
    // ---------------- MMA issue (one thread)
    if (lane == 0) {
      const uint32_t idesc = instr_desc_kk(M, TN);
      const uint32_t sbase = smem_u32(smem);
      bool ok = true;
      for (int64_t j = 0; j < my_tiles && ok; ++j) {
        const int buf = (int)(j & 1);
        if (j >= 2) ok = mbar_wait(smem_u32(&bar_acce[buf]), (uint32_t)(((j / 2) - 1) & 1), g.err);
        for (int ks = 0; ks < g.nks && ok; ++ks) {
          const int64_t gs = j * g.nks + ks;
          const int o = (int)(gs % NOP);
          ok = mbar_wait(smem_u32(&op_full[o]), (uint32_t)((gs / NOP) & 1), g.err);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t st = sbase + (uint32_t)o * OP_BYTES;
          const uint32_t d = tmem + (uint32_t)buf * (uint32_t)TN;
          // a K step of 16 FP16 is 32 bytes along the swizzled row: +2 in the
          // descriptor's address field (addr >> 4)
          const uint64_t ah0 = smem_desc(st + OFF_AH, 16, 1024), al0 = smem_desc(st + OFF_AL, 16, 1024);
          const uint64_t bh0 = smem_desc(st + OFF_BH, 16, 1024), bl0 = smem_desc(st + OFF_BL, 16, 1024);
#pragma unroll
          for (int kk = 0; kk < SK / 16; ++kk) {
            const uint64_t ah = ah0 + 2u * kk, al = al0 + 2u * kk;
            const uint64_t bh = bh0 + 2u * kk, bl = bl0 + 2u * kk;
            const uint32_t acc0 = (ks > 0 || kk > 0) ? 1u : 0u;
            tc_mma(d, ah, bh, idesc, acc0);
            tc_mma(d, ah, bl, idesc, 1u);
            tc_mma(d, al, bh, idesc, 1u);
          }
          tc_commit(smem_u32(&op_empty[o]));
        }
        if (ok) tc_commit(smem_u32(&bar_accf[buf]));
      }
      tc_commit(smem_u32(&bar_done));
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: tensor memory -> Z
    const int q = warp & 3;          // the lane quarter this warp may access
    // output row (index of the K outputs) of this lane: M = 128 rows 32 q +
    // lane; M = 64 rows 16 q + lane in lanes 0-15 of the quarter
    const int r = C::RPQ * q + lane;
    const bool rl = lane < C::RPQ;
    const float inv = (float)(1.0 / ((double)g.sy * (double)*g.sa));   // powers of two: exact
    for (int64_t j = 0; j < my_tiles; ++j) {
      const int buf = (int)(j & 1);
      if (!mbar_wait(smem_u32(&bar_accf[buf]), (uint32_t)((j / 2) & 1), g.err)) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int64_t m0 = ((int64_t)blockIdx.x + j * gridDim.x) * TN;
      if (C::RPQ * q < g.K) {
        for (int c0 = 0; c0 < TN; c0 += 32) {
          uint32_t rr[32];
          tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)buf * (uint32_t)TN + (uint32_t)c0, rr);
          if (rl && r < g.K) {
            if (!g.zt) {
#pragma unroll
              for (int jj = 0; jj < 32; ++jj) {
                const int64_t slab = m0 + c0 + jj;
                if (slab < g.Rt) g.z[slab * g.K + r] = __uint_as_float(rr[jj]) * inv;
              }
            } else if ((g.Rt & 3) == 0) {
              // transposed: this lane's 32 slabs are contiguous in its row of
              // Z; 16-byte stores (Rt % 4 == 0: the row starts are aligned)
              float* zr = g.z + (int64_t)r * g.Rt;
#pragma unroll
              for (int jj = 0; jj < 32; jj += 4) {
                const int64_t slab = m0 + c0 + jj;
                if (slab < g.Rt)
                  *reinterpret_cast<float4*>(zr + slab) =
                      make_float4(__uint_as_float(rr[jj]) * inv, __uint_as_float(rr[jj + 1]) * inv,
                                  __uint_as_float(rr[jj + 2]) * inv, __uint_as_float(rr[jj + 3]) * inv);
              }
            } else {
              float* zr = g.z + (int64_t)r * g.Rt;
#pragma unroll
              for (int jj = 0; jj < 32; ++jj) {
                const int64_t slab = m0 + c0 + jj;
                if (slab < g.Rt) zr[slab] = __uint_as_float(rr[jj]) * inv;
              }
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bar_acce[buf]));
    }
  }
  // every tcgen05 op issued by the MMA thread has completed once bar_done fires
  mbar_wait(smem_u32(&bar_done), 0, g.err);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == MMA_WARP) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TMEM_COLS));
  }
}

// ------------------------------------------------------------------------
// Row-mode views (L > 1, L % 4 == 0, I <= 64): per slab r,
// Z_r (L x K, l fastest) = Y_r (L x I) A^T, i.e. Z(l, k, r) = sum_i A(k, i)
// Y(l, i, r) -- the expansions of the multi-TTM reconstruction, where I is a
// core rank.  The MMA's M is l: a work item is 128 consecutive l of one slab
// against an N-tile of 256 outputs k.  Y comes through a three-slot raw ring
// (3D TMA box of 128 l x 64 i, zero-filled outside the view) and eight
// converter warps split it into the MN-major SW128 FP16 hi/lo A operand (l
// contiguous, as loaded).  B = A^T of the CTA's N-tile (K-major SW128 hi/lo
// images, split by a prep kernel) stays resident.  Three products per
// K step, as in the column kernel; double-buffered 2 x 256 accumulator
// columns; eight epilogue warps (two per tensor-memory lane quarter, 128
// columns each, two 32-column loads per wait: with one warp per quarter and
// one load per wait the tensor-memory reads bounded the kernel) write Z
// coalesced along l.  Each CTA serves
// one N-tile (blockIdx.x % NT) and walks the items (slab, l-tile)
// blockIdx.x / NT, + gridDim.x / NT, ...; the NT CTAs of an item run side by
// side, so Y is read from HBM about once.
constexpr int RN = 256;                        // MMA N: outputs per N-tile
constexpr int RM = 128;                        // MMA M: l per item
constexpr uint32_t RA_BYTES = RM * SK * 2;     // 16 KB: one of A hi / lo
constexpr uint32_t RB_BYTES = RN * SK * 2;     // 32 KB: one of B hi / lo
constexpr uint32_t ROP_BYTES = 2 * RA_BYTES;   // A operand slot (hi | lo)
constexpr uint32_t RRAW_BYTES = RM * SK * 4;   // 32 KB raw FP32 box
constexpr int RNOP = 2, RNRAW = 3;
constexpr int RNEPI = 8;                       // epilogue warps 10..17, two per lane quarter
constexpr int RNTHREADS = (MMA_WARP + 1 + RNEPI) * 32;
constexpr uint32_t RSMEM_BYTES = 2 * RB_BYTES + RNOP * ROP_BYTES + RNRAW * RRAW_BYTES + 1024;
constexpr uint32_t RKG = 2 * 1024;             // k-group stride of the MN-major A operand

// Byte offset of (l, i) (l < 128, i < 64) in the MN-major SW128 A operand:
// atoms of 64 l x 8 i (1 KB), [k group of 8 i][atom].
__device__ __forceinline__ uint32_t rmn_off(int l, int i) {
  return (uint32_t)(i >> 3) * RKG + (uint32_t)(l >> 6) * 1024u + (uint32_t)(i & 7) * 128u +
         ((uint32_t)(((l & 63) >> 3) ^ (i & 7)) << 4) + (uint32_t)(l & 7) * 2u;
}

// Instruction descriptor: kind::f16, FP16 A and B, FP32 D, A MN-major, B K-major.
__device__ __forceinline__ uint32_t instr_desc_mk(int M, int N) {
  return (1u << 4) | (1u << 15) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// B images of A^T: N-tile t holds rows k = 256 t + row (row < 256) and
// columns i < 64 of A scaled by s_a, K-major SW128, [B_h | B_l] (64 KB per
// tile, zero outside K x I); *sa_out = s_a.  One CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_ttm_tc_prep_rows(const double* __restrict__ A, int K,
                                                           int64_t I, int64_t lda, int arow,
                                                           int ntile, uint8_t* __restrict__ out,
                                                           float* __restrict__ sa_out) {
  __shared__ double red[32];
  __shared__ float s_sa;
  double mx = 0.0;
  for (int64_t e = threadIdx.x; e < (int64_t)K * I; e += blockDim.x) {
    const int64_t k = e / I, i = e % I;
    const double a = arow ? A[k * lda + i] : A[k + lda * i];
    mx = fmax(mx, fabs(a));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = red[threadIdx.x];
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) {
      int ex = 0;
      frexp(v, &ex);                       // v < 2^ex
      int e2 = 14 - ex;
      e2 = e2 > 100 ? 100 : (e2 < -100 ? -100 : e2);
      s_sa = (v > 0.0) ? ldexpf(1.f, e2) : 1.f;
      *sa_out = s_sa;
    }
  }
  __syncthreads();
  const double sa = s_sa;
  const int64_t tot = (int64_t)ntile * RN * (SK / 2);   // element pairs (i, i + 1)
  for (int64_t e = threadIdx.x; e < tot; e += blockDim.x) {
    const int t = (int)(e / (RN * (SK / 2)));
    const int rem = (int)(e % (RN * (SK / 2)));
    const int row = rem / (SK / 2), kp = 2 * (rem % (SK / 2));
    const int64_t k = (int64_t)t * RN + row;
    float v2[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int64_t i = kp + u;
      double a = 0.0;
      if (k < K && i < I) a = arow ? A[k * lda + i] : A[k + lda * i];
      v2[u] = (float)(a * sa);
    }
    uint32_t h, l;
    split_pack(v2[0], v2[1], h, l);
    uint8_t* base = out + (size_t)t * 2 * RB_BYTES;
    const uint32_t o = kmaj_off(row, kp);
    *reinterpret_cast<uint32_t*>(base + o) = h;
    *reinterpret_cast<uint32_t*>(base + RB_BYTES + o) = l;
  }
}

struct TtmTcRowArgs {
  int64_t L, I, Rt;
  int K;                   // outputs per slab
  int NT;                  // N-tiles of 256 outputs
  int64_t ntl;             // l-tiles per slab, ceil(L / 128)
  int64_t nitems;          // Rt * ntl
  float sy;                // power of two
  const uint8_t* bprep;    // NT x [B_h | B_l]
  const float* sa;         // the power-of-two scale of A (device)
  float* z;                // z[l + L (k + K r)]
  unsigned* err;
};

__global__ void __launch_bounds__(RNTHREADS, 1)
    k_ttm_tc_row(TtmTcRowArgs g, const __grid_constant__ CUtensorMap ymap) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* bimg = smem;                                  // [B_h | B_l], resident
  uint8_t* ops = smem + 2 * RB_BYTES;                    // RNOP A slots
  uint8_t* raw = ops + RNOP * ROP_BYTES;                 // RNRAW raw slots
  __shared__ uint64_t raw_full[RNRAW], raw_empty[RNRAW], op_full[RNOP], op_empty[RNOP];
  __shared__ uint64_t bar_b, bar_accf[2], bar_acce[2], bar_done;
  __shared__ uint32_t tmem_base_sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nt = (int)(blockIdx.x % g.NT);
  const int64_t c0 = blockIdx.x / g.NT, cstep = gridDim.x / g.NT;

  if (threadIdx.x == 0) {
    for (int s = 0; s < RNRAW; ++s) {
      mbar_init(smem_u32(&raw_full[s]), 1);
      mbar_init(smem_u32(&raw_empty[s]), NCONV);
    }
    for (int s = 0; s < RNOP; ++s) {
      mbar_init(smem_u32(&op_full[s]), NCONV);
      mbar_init(smem_u32(&op_empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&bar_accf[b]), 1);
      mbar_init(smem_u32(&bar_acce[b]), RNEPI);
    }
    mbar_init(smem_u32(&bar_b), 1);
    mbar_init(smem_u32(&bar_done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
        smem_u32(&tmem_base_sh)), "n"(2 * RN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base_sh;
  const int64_t my_items = (g.nitems > c0) ? (g.nitems - 1 - c0) / cstep + 1 : 0;

  if (warp == LOAD_WARP) {
    // ---------------- loader: B images once, then Y boxes -> raw slots (TMA)
    if (lane == 0) {
      mbar_arrive_expect_tx(smem_u32(&bar_b), 2 * RB_BYTES);   // bar_b counts this one arrival
      bulk_g2s(smem_u32(bimg), g.bprep + (size_t)nt * 2 * RB_BYTES, 2 * RB_BYTES, smem_u32(&bar_b));
      for (int64_t j = 0; j < my_items; ++j) {
        const int r = (int)(j % RNRAW);
        if (j >= RNRAW &&
            !mbar_wait(smem_u32(&raw_empty[r]), (uint32_t)(((j / RNRAW) - 1) & 1), g.err))
          break;
        const int64_t it = c0 + j * cstep;
        const int64_t slab = it / g.ntl, lt = it - slab * g.ntl;
        mbar_arrive_expect_tx(smem_u32(&raw_full[r]), RRAW_BYTES);
        tma_load_3d(smem_u32(raw + (size_t)r * RRAW_BYTES), &ymap, (int)(lt * RM), 0, (int)slab,
                    smem_u32(&raw_full[r]));
      }
    }
    __syncwarp();
  } else if (warp <= NCONV) {
    // ---------------- converters: raw [i][l] FP32 -> MN-major FP16 hi/lo A
    const int ct = threadIdx.x - 32;   // 0..255
    for (int64_t j = 0; j < my_items; ++j) {
      const int r = (int)(j % RNRAW), o = (int)(j % RNOP);
      if (!mbar_wait(smem_u32(&raw_full[r]), (uint32_t)((j / RNRAW) & 1), g.err)) break;
      if (j >= RNOP &&
          !mbar_wait(smem_u32(&op_empty[o]), (uint32_t)(((j / RNOP) - 1) & 1), g.err))
        break;
      uint8_t* st = ops + (size_t)o * ROP_BYTES;
      const uint8_t* src = raw + (size_t)r * RRAW_BYTES;
      float4 v[CV4];
#pragma unroll
      for (int e = 0; e < CV4; ++e) {
        const int c = ct + NCONV * 32 * e;          // i = c / 32, l = 4 (c % 32)
        v[e] = *reinterpret_cast<const float4*>(src + (size_t)c * 16);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&raw_empty[r]));   // raw slot read
#pragma unroll
      for (int e = 0; e < CV4; ++e) {
        const int c = ct + NCONV * 32 * e;
        const int i = c >> 5, l = 4 * (c & 31);
        uint2 hp, lp;
        split_pack(v[e].x * g.sy, v[e].y * g.sy, hp.x, lp.x);
        split_pack(v[e].z * g.sy, v[e].w * g.sy, hp.y, lp.y);
        const uint32_t off = rmn_off(l, i);
        *reinterpret_cast<uint2*>(st + off) = hp;
        *reinterpret_cast<uint2*>(st + RA_BYTES + off) = lp;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&op_full[o]));
    }
  } else if (warp == MMA_WARP) {
    // ---------------- MMA issue (one thread)
    if (lane == 0) {
      const uint32_t idesc = instr_desc_mk(RM, RN);
      bool ok = mbar_wait(smem_u32(&bar_b), 0, g.err);
      const uint64_t bh0 = smem_desc(smem_u32(bimg), 16, 1024);
      const uint64_t bl0 = smem_desc(smem_u32(bimg + RB_BYTES), 16, 1024);
      for (int64_t j = 0; j < my_items && ok; ++j) {
        const int buf = (int)(j & 1), o = (int)(j % RNOP);
        if (j >= 2) ok = mbar_wait(smem_u32(&bar_acce[buf]), (uint32_t)(((j / 2) - 1) & 1), g.err);
        if (ok) ok = mbar_wait(smem_u32(&op_full[o]), (uint32_t)((j / RNOP) & 1), g.err);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t st = smem_u32(ops + (size_t)o * ROP_BYTES);
        const uint32_t d = tmem + (uint32_t)buf * (uint32_t)RN;
#pragma unroll
        for (int kk = 0; kk < SK / 16; ++kk) {
          // A: a K step of 16 i is two k groups (2 x RKG bytes); B: 32 bytes
          // along its swizzled rows (+2 in the address field)
          const uint64_t ah = smem_desc(st + (uint32_t)kk * 2u * RKG, 1024, RKG);
          const uint64_t al = smem_desc(st + RA_BYTES + (uint32_t)kk * 2u * RKG, 1024, RKG);
          const uint64_t bh = bh0 + 2u * kk, bl = bl0 + 2u * kk;
          const uint32_t acc0 = kk > 0 ? 1u : 0u;
          tc_mma(d, ah, bh, idesc, acc0);
          tc_mma(d, ah, bl, idesc, 1u);
          tc_mma(d, al, bh, idesc, 1u);
        }
        tc_commit(smem_u32(&op_empty[o]));
        tc_commit(smem_u32(&bar_accf[buf]));
      }
      tc_commit(smem_u32(&bar_done));
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: tensor memory -> Z, coalesced along l
    const int q = warp & 3;                          // the lane quarter this warp may access
    const int half = (warp - MMA_WARP - 1) >> 2;     // columns [128 half, 128 half + 128)
    const float inv = (float)(1.0 / ((double)g.sy * (double)*g.sa));   // powers of two: exact
    const int kbase = nt * RN + 128 * half;
    for (int64_t j = 0; j < my_items; ++j) {
      const int buf = (int)(j & 1);
      if (!mbar_wait(smem_u32(&bar_accf[buf]), (uint32_t)((j / 2) & 1), g.err)) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int64_t it = c0 + j * cstep;
      const int64_t slab = it / g.ntl, lt = it - slab * g.ntl;
      const int64_t l = lt * RM + 32 * q + lane;
      float* zl = g.z + l + g.L * g.K * slab;
      const uint32_t tbase = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)buf * (uint32_t)RN +
                             128u * (uint32_t)half;
      for (int cb = 0; cb < 128 && kbase + cb < g.K; cb += 64) {
        uint32_t rr[64];
        tmem_ld32x2(tbase + (uint32_t)cb, rr);
        if (l < g.L) {
#pragma unroll
          for (int jj = 0; jj < 64; ++jj) {
            const int k = kbase + cb + jj;
            if (k < g.K) zl[g.L * (int64_t)k] = __uint_as_float(rr[jj]) * inv;
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bar_acce[buf]));
    }
  }
  mbar_wait(smem_u32(&bar_done), 0, g.err);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == MMA_WARP) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(2 * RN));
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, looked up once through the runtime (no
// link-time dependency on the driver library); the first caller of any
// thread initialises it.
EncodeTiledFn encode_tiled() {
  static const EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return (EncodeTiledFn)p;
    return (EncodeTiledFn) nullptr;
  }();
  return fn;
}

}  // namespace

int ttm_tc_supported(int64_t L, int64_t I, int64_t Rt, int64_t K) {
  return L == 1 && I >= 64 && I <= 65536 && (I % 4) == 0 && K >= 1 && K <= TM && Rt >= 1 &&
         Rt < (1ll << 31);
}

size_t ttm_tc_scratch_bytes(int64_t I, int64_t K) {
  (void)K;
  const size_t nks = (size_t)((I + SK - 1) / SK);
  return nks * 2 * ColCfg<TM>::A_BYTES + 256;
}

template <int M>
cudaError_t run_ttm_tc_col(const TtmTcArgs& a, const CUtensorMap& ymap, int grid,
                           cudaStream_t st) {
  {
    cudaError_t e = allow_max_dyn_smem((const void*)k_ttm_tc_col<M>);
    if (e != cudaSuccess) return e;
  }
  k_ttm_tc_col<M><<<grid, NTHREADS, ColCfg<M>::SMEM_BYTES, st>>>(a, ymap);
  return cudaSuccess;
}

cudaError_t launch_ttm_tc(const float* y, int64_t L, int64_t I, int64_t Rt, const double* A,
                          int64_t K, int64_t lda, int a_rowmajor, float sy, float* z, bool zt,
                          void* scratch, unsigned* err, int num_sms, cudaStream_t st) {
  if (!ttm_tc_supported(L, I, Rt, K) || ((uintptr_t)y & 15) != 0) return cudaErrorInvalidValue;
  if (zt && (Rt & 3) == 0 && ((uintptr_t)z & 15) != 0) return cudaErrorInvalidValue;
  const int nks = (int)((I + SK - 1) / SK);
  const int tm = K <= 64 ? 64 : TM;
  uint8_t* aprep = (uint8_t*)scratch;
  float* sa = (float*)(aprep + (size_t)nks * 2 * ColCfg<TM>::A_BYTES);
  k_ttm_tc_prep<<<1, 1024, 0, st>>>(A, (int)K, I, lda, a_rowmajor, nks, tm, aprep, sa);
  TtmTcArgs a;
  a.y = y;
  a.I = I;
  a.Rt = Rt;
  a.K = (int)K;
  a.nks = nks;
  a.ntiles = (Rt + TN - 1) / TN;
  a.sy = sy;
  a.aprep = aprep;
  a.sa = sa;
  a.z = z;
  a.zt = zt ? 1 : 0;
  a.err = err;
  // Y as a 2D tensor: x = i (contiguous), y = slab; boxes of 64 i x 128 slabs
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return cudaErrorNotSupported;
  alignas(64) CUtensorMap ymap;
  const cuuint64_t gdim[2] = {(cuuint64_t)I, (cuuint64_t)Rt};
  const cuuint64_t gstride[1] = {(cuuint64_t)I * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)SK, (cuuint32_t)TN};
  const cuuint32_t estride[2] = {1, 1};
  if (enc(&ymap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)y, gdim, gstride, box, estride,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  const int grid = (int)(a.ntiles < num_sms ? a.ntiles : num_sms);
  cudaError_t e = tm == 64 ? run_ttm_tc_col<64>(a, ymap, grid, st)
                           : run_ttm_tc_col<TM>(a, ymap, grid, st);
  if (e != cudaSuccess) return e;
  count_launches(2);
  return cudaGetLastError();
}

int ttm_tc_row_supported(int64_t L, int64_t I, int64_t Rt, int64_t K) {
  return L > 1 && (L % 4) == 0 && L < (1ll << 31) && I >= 1 && I <= SK && K >= 1 &&
         K <= 4 * RN && Rt >= 1 && Rt < (1ll << 31) && L * I * Rt < (1ll << 40);
}

size_t ttm_tc_row_scratch_bytes(int64_t K) {
  return (size_t)((K + RN - 1) / RN) * 2 * RB_BYTES + 256;
}

cudaError_t launch_ttm_tc_row(const float* y, int64_t L, int64_t I, int64_t Rt, const double* A,
                              int64_t K, int64_t lda, int a_rowmajor, float sy, float* z,
                              void* scratch, unsigned* err, int num_sms, cudaStream_t st) {
  if (!ttm_tc_row_supported(L, I, Rt, K) || ((uintptr_t)y & 15) != 0) return cudaErrorInvalidValue;
  {
    cudaError_t e = allow_max_dyn_smem((const void*)k_ttm_tc_row);
    if (e != cudaSuccess) return e;
  }
  const int NT = (int)((K + RN - 1) / RN);
  uint8_t* bprep = (uint8_t*)scratch;
  float* sa = (float*)(bprep + (size_t)NT * 2 * RB_BYTES);
  k_ttm_tc_prep_rows<<<1, 1024, 0, st>>>(A, (int)K, I, lda, a_rowmajor, NT, bprep, sa);
  TtmTcRowArgs a;
  a.L = L;
  a.I = I;
  a.Rt = Rt;
  a.K = (int)K;
  a.NT = NT;
  a.ntl = (L + RM - 1) / RM;
  a.nitems = Rt * a.ntl;
  a.sy = sy;
  a.bprep = bprep;
  a.sa = sa;
  a.z = z;
  a.err = err;
  // Y as a 3D tensor: x = l (contiguous), y = i, z = slab; boxes of 128 l x 64 i x 1
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return cudaErrorNotSupported;
  alignas(64) CUtensorMap ymap;
  const cuuint64_t gdim[3] = {(cuuint64_t)L, (cuuint64_t)I, (cuuint64_t)Rt};
  const cuuint64_t gstride[2] = {(cuuint64_t)L * sizeof(float), (cuuint64_t)(L * I) * sizeof(float)};
  const cuuint32_t box[3] = {(cuuint32_t)RM, (cuuint32_t)SK, 1};
  const cuuint32_t estride[3] = {1, 1, 1};
  if (enc(&ymap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)y, gdim, gstride, box, estride,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  int64_t per = num_sms / NT;
  if (per < 1) per = 1;
  if (per > a.nitems) per = a.nitems;
  const int grid = (int)(per * NT);
  k_ttm_tc_row<<<grid, RNTHREADS, RSMEM_BYTES, st>>>(a, ymap);
  count_launches(2);
  return cudaGetLastError();
}

}  // namespace tk
