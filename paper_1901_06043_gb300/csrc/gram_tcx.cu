// Tensor-core Gram of the column-major mode-0 view (Algorithm 2, n = 0) with
// exact digit products: S = X X^T for the I x K matrix X of FP32 columns.
//
// Arithmetic.  Row i of X is scaled by a power of two s_i with max_k |x_ik s_i|
// in [64, 128) (s_i from the row maxima the norm pass records), and every
// scaled value is split exactly into three integer digits,
//     x s_i = d0 + d1 / 2^8 + d2 / 2^16,   |d0|, |d1|, |d2| <= 128,
// by two rounds of "round to the nearest integer, subtract, scale by 2^8"
// (each subtraction and scaling is exact; the last rounding, for values below
// half the row maximum, is the only one: <= 2^-17 in these units, unbiased
// and independent of the value).  Digits are integers below 2^11, exact in
// FP16, and so is d2 / 2^8.  The tensor cores (kind::f16, FP32 accumulators in
// tensor memory) form all nine digit products, grouped by weight:
//     D0 = sum d0 d0'                                      (weight 1)
//     D1 = sum (d0 d1' + d1 d0')                          (2^-8)
//     D2 = sum (d0 d2' + d1 d1' + d2 d0')                 (2^-16)
//     D3 = sum (d1 d2' + d2 d1' + (d2 / 2^8) d2')         (2^-24)
// D0..D2 sum integers below 2^14 each; over a window of 256 columns every
// partial sum stays an integer below 2^24, so those accumulators are exact and
// the accumulator's truncation never acts (it is what moves the eps cut for
// the rounded-product tensor-core Gram of tc.cu).  D3 is not integral, but at
// weight 2^-24 its truncation is ~2^-48 of an entry.  Leaving D3 out is not
// an option: its terms have nonzero mean (d2^2 > 0; and when d1 rounds to
// +-128 the remainder d2 takes the opposite sign) and measured as a +1e-8
// relative bias on a trace and -0.1 threshold on a discarded eigenvalue sum.
// After each window the epilogue warps drain the four sums and add D0, D1 /
// 2^8, D2 / 2^16 and D3 / 2^24 one by one into an exact FP32 pair (TwoSum,
// hi + lo) in shared memory (a combined value rounded to FP32 first measured a
// +1e-8 trace bias).  The pairs go out as FP64 per-CTA partial tiles; a second
// kernel sums the K splits in a fixed order and removes the scales,
// S_ij = D_ij / (s_i s_j).
//
// Work split.  Tiles of 128 x 128 over the lower triangle (ta >= tb), times K
// splits sized to one wave of the SMs; the CTAs of a split are adjacent in
// launch order so their shared columns are served from L2.
//
// Roles (25 warps): warps 0-15 load X with 16-byte loads, split it into the
// digit planes of the A (rows 128 ta..) and B (rows 128 tb..) operands,
// MN-major SW128 (three-stage ring); warp 16 issues the MMAs (one thread);
// warps 17-24 drain tensor memory, two per lane quarter, 64 columns each.  Every wait
// is bounded: one that gives up sets DEV_ERR_MBAR_TIMEOUT and the kernel winds
// down; tensor memory is always released.
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace tk {
namespace {

using namespace tc;

constexpr int BK = 16;                          // columns (K) per stage: one MMA step
constexpr int NSTAGE = 3;
constexpr int WIN = 16;                         // stages per exact window (256 columns)
constexpr int NPROD = 16;                       // one column of the stage each
constexpr int MMA_WARP = 16;
constexpr int EPI_WARP0 = 17;
constexpr int NEPI = 8;
constexpr int NTHREADS = (EPI_WARP0 + NEPI) * 32;   // 800
constexpr uint32_t SK = 2048;                   // atom stride along K (128 mn x 8 k per 2 atoms)
constexpr uint32_t ATOM_MN = 1024;
constexpr uint32_t PLANE = 128 * BK * 2;        // one digit plane of one operand: 4 KB
constexpr uint32_t OFF_A = 0, OFF_B = 4 * PLANE;  // A: d0, d1, d2, d2 / 2^8; B: d0, d1, d2
constexpr uint32_t STAGE_BYTES = 7 * PLANE;     // 28 KB
constexpr uint32_t PAIR_BYTES = 128 * 128 * 4;  // hi or lo tile, [col][row]
constexpr uint32_t SMEM_BYTES = NSTAGE * STAGE_BYTES + 2 * PAIR_BYTES + 1024;
constexpr int TILE_ELEMS = 128 * 128;

// Byte offset of (mn, k) in an MN-major SW128 FP16 tile (as in tc.cu).
__device__ __forceinline__ uint32_t mn_off(int mn, int k) {
  return (uint32_t)(mn >> 6) * ATOM_MN + (uint32_t)(k >> 3) * SK + (uint32_t)(k & 7) * 128u +
         ((uint32_t)(((mn & 63) >> 3) ^ (k & 7)) << 4) + (uint32_t)(mn & 7) * 2u;
}

__device__ __forceinline__ uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (1u << 15) | (1u << 16) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// Four 8-column loads (one per accumulator), then one wait.
__device__ __forceinline__ void tmem_ld8x4(uint32_t taddr, uint32_t (&r)[4][8]) {
#pragma unroll
  for (int q = 0; q < 4; ++q)
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(r[q][0]), "=r"(r[q][1]), "=r"(r[q][2]), "=r"(r[q][3]), "=r"(r[q][4]),
          "=r"(r[q][5]), "=r"(r[q][6]), "=r"(r[q][7])
        : "r"(taddr + 128u * (uint32_t)q));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// The digits of four scaled values, packed as FP16 pairs per plane: d0, d1,
// d2 and (NP == 4) d2 / 2^8.
template <int NP>
__device__ __forceinline__ void digits4(float4 v, const float* s, uint2 (&p)[4]) {
  const float x[4] = {v.x * s[0], v.y * s[1], v.z * s[2], v.w * s[3]};
  float d[4][4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float d0 = rintf(x[j]);
    const float r1 = (x[j] - d0) * 256.f;
    const float d1 = rintf(r1);
    const float d2 = rintf((r1 - d1) * 256.f);
    d[0][j] = d0;
    d[1][j] = d1;
    d[2][j] = d2;
    d[3][j] = d2 * 0x1p-8f;
  }
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    const __half2 a = __floats2half2_rn(d[q][0], d[q][1]);
    const __half2 b = __floats2half2_rn(d[q][2], d[q][3]);
    p[q].x = *reinterpret_cast<const uint32_t*>(&a);
    p[q].y = *reinterpret_cast<const uint32_t*>(&b);
  }
}

struct GramTcxArgs {
  const float* x;          // column-major I x K
  int64_t I, K;
  int ntiles, nkg, T;      // tiles of the lower triangle, K splits, row blocks
  const float* scale;      // I power-of-two row scales s_i
  double* part;            // gridDim.x partial tiles, [col][row], FP64 (scaled units)
  unsigned* err;
};

__device__ __forceinline__ void tile_of(int t, int& ta, int& tb) {
  int a = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
  while ((a + 1) * (a + 2) / 2 <= t) ++a;
  while (a * (a + 1) / 2 > t) --a;
  ta = a;
  tb = t - a * (a + 1) / 2;
}

__global__ void __launch_bounds__(NTHREADS, 1) k_gram_tcx_col(GramTcxArgs g) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float* hi = reinterpret_cast<float*>(smem + NSTAGE * STAGE_BYTES);
  float* lo = hi + TILE_ELEMS;
  __shared__ uint64_t bar_full[NSTAGE], bar_empty[NSTAGE], bar_accf, bar_acce, bar_done;
  __shared__ uint32_t tmem_base_sh;
  __shared__ float s_scale[256];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile = blockIdx.x % g.ntiles, kg = blockIdx.x / g.ntiles;
  int ta, tb;
  tile_of(tile, ta, tb);
  const bool diag = ta == tb;
  const int64_t k0 = g.K * kg / g.nkg, k1 = g.K * (kg + 1) / g.nkg;
  const int nst = (int)((k1 - k0 + BK - 1) / BK);
  const int nwin = (nst + WIN - 1) / WIN;

  for (int t = threadIdx.x; t < 256; t += NTHREADS) {
    const int64_t row = (t < 128) ? (int64_t)ta * 128 + t : (int64_t)tb * 128 + (t - 128);
    s_scale[t] = row < g.I ? g.scale[row] : 1.f;
  }
  for (int t = threadIdx.x; t < 2 * TILE_ELEMS; t += NTHREADS) hi[t] = 0.f;   // hi and lo
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

  if (warp < NPROD) {
    // ---------------- producers: X -> digit planes of A (and B)
    const int nops = diag ? 1 : 2;
    const int64_t row0[2] = {(int64_t)ta * 128 + 4 * lane, (int64_t)tb * 128 + 4 * lane};
    float sc[2][4];
#pragma unroll
    for (int o = 0; o < 2; ++o)
#pragma unroll
      for (int u = 0; u < 4; ++u) sc[o][u] = s_scale[128 * o + 4 * lane + u];
    // loads run PF stages ahead of the conversion (register ring), so each
    // warp keeps PF + 1 stages of 16-byte loads in flight (~80 KB per SM)
    constexpr int PF = 4;
    float4 ring[PF + 1][2][1];
    auto load_stage = [&](int s, float4 (&v)[2][1]) {
#pragma unroll
      for (int j = 0; j < 1; ++j) {
        const int kl = warp + NPROD * j;
        const int64_t kc = k0 + (int64_t)s * BK + kl;
        const bool kok = (s < nst) && kc < k1;
        const float* col = g.x + kc * g.I;
#pragma unroll
        for (int o = 0; o < 2; ++o) {
          const bool ok = kok && (o < nops) && row0[o] < g.I;
          v[o][j] = ok ? __ldcs(reinterpret_cast<const float4*>(col + row0[o]))
                       : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
    };
#pragma unroll
    for (int u = 0; u < PF; ++u) load_stage(u, ring[u]);
    bool go = true;
    for (int s0 = 0; s0 < nst && go; s0 += PF + 1) {
#pragma unroll
      for (int u = 0; u <= PF; ++u) {
        const int s = s0 + u;
        if (s >= nst || !go) break;
        load_stage(s + PF, ring[(u + PF) % (PF + 1)]);
        const float4 (&v)[2][1] = ring[u];
        const int slot = s % NSTAGE;
        if (s >= NSTAGE) {
          if (!mbar_wait(smem_u32(&bar_empty[slot]), ((s / NSTAGE) - 1) & 1, g.err)) { go = false; break; }
        }
        uint8_t* st = smem + (size_t)slot * STAGE_BYTES;
#pragma unroll
        for (int j = 0; j < 1; ++j) {
          const int kl = warp + NPROD * j;
          const uint32_t o = mn_off(4 * lane, kl);
          uint2 p[4];
          digits4<4>(v[0][j], sc[0], p);
#pragma unroll
          for (int q = 0; q < 4; ++q) *reinterpret_cast<uint2*>(st + OFF_A + o + q * PLANE) = p[q];
          if (nops == 2) {
            digits4<3>(v[1][j], sc[1], p);
#pragma unroll
            for (int q = 0; q < 3; ++q) *reinterpret_cast<uint2*>(st + OFF_B + o + q * PLANE) = p[q];
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bar_full[slot]));
      }
    }
  } else if (warp == MMA_WARP) {
    // ---------------- MMA issue (one thread)
    if (lane == 0) {
      const uint32_t idesc = instr_desc(128, 128);
      const uint32_t sbase = smem_u32(smem);
      const uint32_t boff = diag ? OFF_A : OFF_B;
      bool ok = true;
      for (int s = 0; s < nst && ok; ++s) {
        const int slot = s % NSTAGE;
        const int w = s / WIN;
        const bool first = (s % WIN) == 0;
        if (first && w >= 1) ok = mbar_wait(smem_u32(&bar_acce), (w - 1) & 1, g.err);
        if (ok) ok = mbar_wait(smem_u32(&bar_full[slot]), (s / NSTAGE) & 1, g.err);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t st = sbase + (uint32_t)slot * STAGE_BYTES;
        uint64_t a[4], b[3];
#pragma unroll
        for (int q = 0; q < 4; ++q) a[q] = smem_desc(st + OFF_A + q * PLANE, ATOM_MN, SK);
#pragma unroll
        for (int q = 0; q < 3; ++q) b[q] = smem_desc(st + boff + q * PLANE, ATOM_MN, SK);
        const uint32_t fresh = first ? 0u : 1u;
        tc_mma(tmem + 0u, a[0], b[0], idesc, fresh);
        tc_mma(tmem + 128u, a[0], b[1], idesc, fresh);
        tc_mma(tmem + 128u, a[1], b[0], idesc, 1u);
        tc_mma(tmem + 256u, a[0], b[2], idesc, fresh);
        tc_mma(tmem + 256u, a[1], b[1], idesc, 1u);
        tc_mma(tmem + 256u, a[2], b[0], idesc, 1u);
        tc_mma(tmem + 384u, a[1], b[2], idesc, fresh);
        tc_mma(tmem + 384u, a[2], b[1], idesc, 1u);
        tc_mma(tmem + 384u, a[3], b[2], idesc, 1u);
        tc_commit(smem_u32(&bar_empty[slot]));
        if ((s % WIN) == WIN - 1 || s == nst - 1) tc_commit(smem_u32(&bar_accf));
      }
      tc_commit(smem_u32(&bar_done));
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: exact window sums -> FP32 pairs
    const int e = warp - EPI_WARP0;
    const int q = warp & 3;                  // lane quarter this warp may access
    const int c0 = (e >> 2) * 64;            // this warp's 64 columns
    const int row = 32 * q + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
    for (int w = 0; w < nwin; ++w) {
      if (!mbar_wait(smem_u32(&bar_accf), w & 1, g.err)) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      for (int cc = 0; cc < 64; cc += 8) {
        uint32_t r[4][8];
        const uint32_t col = (uint32_t)(c0 + cc);
        tmem_ld8x4(lane_base + col, r);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          // the four parts D0, D1 / 2^8, D2 / 2^16, D3 / 2^24 (each scaling
          // exact) enter the pair one by one (TwoSum each): nothing is
          // rounded before the compensated sum
          const int idx = (c0 + cc + j) * 128 + row;
          float h = hi[idx], l = lo[idx];
          const float parts[4] = {__uint_as_float(r[0][j]), __uint_as_float(r[1][j]) * 0x1p-8f,
                                  __uint_as_float(r[2][j]) * 0x1p-16f,
                                  __uint_as_float(r[3][j]) * 0x1p-24f};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float v = parts[q];
            const float s2 = h + v;
            const float bb = s2 - h;
            l += (h - (s2 - bb)) + (v - bb);
            h = s2;
          }
          hi[idx] = h;
          lo[idx] = l;
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bar_acce));
    }
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
  for (int idx = threadIdx.x; idx < TILE_ELEMS; idx += NTHREADS)
    pt[idx] = (double)hi[idx] + (double)lo[idx];
}

// S[i][j] = S[j][i] = (sum over the K splits of tile (ta, tb) at [col][row])
// / (s_i s_j), i >= j, splits in order.
__global__ void k_gram_tcx_reduce(const double* __restrict__ part, int ntiles, int nkg,
                                  int64_t I, const float* __restrict__ scale,
                                  double* __restrict__ S) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= I * I) return;
  const int64_t i = idx / I, j = idx % I;
  if (j > i) return;
  const int ta = (int)(i / 128), tb = (int)(j / 128);
  const int t = ta * (ta + 1) / 2 + tb;
  const size_t off = (size_t)(j - 128 * tb) * 128 + (size_t)(i - 128 * ta);
  double s = 0.0;
  for (int k = 0; k < nkg; ++k) s += part[(size_t)(t + ntiles * k) * TILE_ELEMS + off];
  s /= (double)scale[i] * (double)scale[j];
  S[i * I + j] = s;
  S[j * I + i] = s;
}

// Power-of-two row scales from the row maxima (as FP32 bit patterns): the
// largest |x s| in [64, 128); a zero row gets 1; exponents are clamped to the
// FP32 range.
__global__ void k_gram_tcx_scales(const unsigned* __restrict__ rowmax_bits, int64_t I,
                                  float* __restrict__ scale) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= I) return;
  const unsigned b = rowmax_bits[i] & 0x7fffffffu;
  int e = (int)(b >> 23) - 127;              // floor(log2 max) for normal values
  if (b == 0u) e = 6;
  int se = 6 - e;
  if (se > 126) se = 126;
  if (se < -126) se = -126;
  scale[i] = __uint_as_float((unsigned)(se + 127) << 23);
}

}  // namespace

GramPlan plan_gram_tcx(int64_t L, int64_t I, int64_t Rt, int num_sms) {
  GramPlan p;
  if (L != 1 || I < 128 || I > 2048 || (I % 4) != 0 || Rt < 4 * BK) return p;
  const int T = (int)((I + 127) / 128);
  const int ntiles = T * (T + 1) / 2;
  int nkg = num_sms / ntiles;
  if (nkg < 1) nkg = 1;
  const int64_t maxkg = Rt / (4 * BK);
  if (nkg > maxkg) nkg = (int)(maxkg < 1 ? 1 : maxkg);
  p.ntiles = ntiles;
  p.ksplit = nkg;
  p.nctas = ntiles * nkg;
  p.scratch_bytes = (size_t)p.nctas * TILE_ELEMS * sizeof(double) + sizeof(float) * (size_t)I;
  return p;
}

cudaError_t launch_gram_tcx(const float* y, int64_t I, int64_t Rt, const GramPlan& p,
                            const unsigned* rowmax_bits, void* scratch, unsigned* err, double* S,
                            cudaStream_t st) {
  if (p.nctas <= 0 || ((uintptr_t)y & 15) != 0) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_gram_tcx_col, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)SMEM_BYTES);
  if (e != cudaSuccess) return e;
  double* part = static_cast<double*>(scratch);
  float* scale = reinterpret_cast<float*>(part + (size_t)p.nctas * TILE_ELEMS);
  k_gram_tcx_scales<<<(unsigned)((I + 255) / 256), 256, 0, st>>>(rowmax_bits, I, scale);
  GramTcxArgs a;
  a.x = y;
  a.I = I;
  a.K = Rt;
  a.ntiles = p.ntiles;
  a.nkg = p.ksplit;
  a.T = (int)((I + 127) / 128);
  a.scale = scale;
  a.part = part;
  a.err = err;
  k_gram_tcx_col<<<(unsigned)p.nctas, NTHREADS, SMEM_BYTES, st>>>(a);
  const int64_t tot = I * I;
  k_gram_tcx_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(part, p.ntiles, p.ksplit, I,
                                                                   scale, S);
  count_launches(3);
  return cudaGetLastError();
}

}  // namespace tk
