// Tensor-core (tcgen05) Gram for the column-major mode-0 view (Algorithm 2,
// n = 0: one product on the column-major I_0 x J^/0 matrix).
//
// Arithmetic.  Every FP32 value x is scaled by a power of two s (so that
// max|x s| <= 2^14) and split into two FP16 numbers, x s = h + l + r with
// |r| <= 2^-22 |x s|.  S s^2 = (H + L)(H + L)^T is accumulated with all four
// products HH^T, HL^T, LH^T, LL^T on the tensor cores (kind::f16, FP32
// accumulators in tensor memory).  Dropping LL^T (the usual three-product
// trick) would leave a positive semidefinite error ||L||_F^2 ~ 2^-24 ||X||^2
// on the discarded eigenvalues -- about 10x the eps = 1e-4 threshold of a
// 5-way tensor -- so it is kept.  The tensor-core accumulator truncates; its
// error stays roughly proportional to the accumulated sum (harmless for the
// signed tail sums of the rank cut) as long as a chunk is short, so every
// CHUNK stages the accumulator is drained, unscaled and added in FP64 into
// a per-CTA partial tile in global memory.  A final kernel sums the partial
// tiles in a fixed order.
//
// Work split.  S is covered by tiles (a, h): rows 128a..128a+127 (one M=128
// MMA operand) x columns 256h..256h+255 (one N=256 operand), for every tile
// that touches the lower triangle.  One CTA owns one tile over one K range;
// the CTAs of a K range are adjacent in launch order so their identical X
// columns are served from L2.
//
// Roles (13 warps): warps 0-7 load X with 16-byte loads, split and write the
// MN-major SW128 operand tiles (two-stage ring); warp 8 issues the MMAs; warps
// 9-12 drain tensor memory (double-buffered accumulators, 2 x 256 columns).
// Every wait is bounded: a wait that gives up sets DEV_ERR_MBAR_TIMEOUT and
// the kernel winds down without touching memory it does not own.
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace tk {
namespace {

using namespace tc;

constexpr int BK = 64;                 // columns (K) per stage
constexpr int NSTAGE = 2;
constexpr int CHUNK = 32;              // stages per tensor-memory accumulation chunk
constexpr int NPROD = 8;               // producer warps
constexpr int MMA_WARP = 8;
constexpr int EPI_WARP0 = 9;
constexpr int NTHREADS = 13 * 32;
constexpr uint32_t A_SK = 2048;        // A tile: 128 m x 64 k, atom stride along K
constexpr uint32_t B_SK = 4096;        // B tile: 256 n x 64 k
constexpr uint32_t ATOM_MN = 1024;     // atom stride along M / N
constexpr uint32_t A_BYTES = 128 * BK * 2;
constexpr uint32_t B_BYTES = 256 * BK * 2;
constexpr uint32_t OFF_HA = 0, OFF_LA = A_BYTES, OFF_HB = 2 * A_BYTES, OFF_LB = 2 * A_BYTES + B_BYTES;
constexpr uint32_t STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;   // 96 KB
constexpr uint32_t SMEM_BYTES = NSTAGE * STAGE_BYTES + 1024;
constexpr int TILE_ELEMS = 128 * 256;

// Byte offset of (mn, k) in an MN-major SW128 FP16 tile: 1024-byte atoms of
// 8 k-rows x 64 mn, 16-byte chunks XOR-swizzled by k%8; atoms ATOM_MN apart
// along MN and sK apart along K.
__device__ __forceinline__ uint32_t mn_off(int mn, int k, uint32_t sK) {
  return (uint32_t)(mn >> 6) * ATOM_MN + (uint32_t)(k >> 3) * sK + (uint32_t)(k & 7) * 128u +
         ((uint32_t)(((mn & 63) >> 3) ^ (k & 7)) << 4) + (uint32_t)(mn & 7) * 2u;
}

// Instruction descriptor: kind::f16, FP16 A and B, FP32 D, both MN-major.
__device__ __forceinline__ uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (0u << 7) | (0u << 10) | (1u << 15) | (1u << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// x s = h + l: FP16 hi part, FP16 part of the remainder.
__device__ __forceinline__ void split4(float4 v, float s, uint2& hp, uint2& lp) {
  const float x[4] = {v.x * s, v.y * s, v.z * s, v.w * s};
  __half h[4], l[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    h[j] = __float2half_rn(x[j]);
    l[j] = __float2half_rn(x[j] - __half2float(h[j]));
  }
  hp.x = (uint32_t)__half_as_ushort(h[0]) | ((uint32_t)__half_as_ushort(h[1]) << 16);
  hp.y = (uint32_t)__half_as_ushort(h[2]) | ((uint32_t)__half_as_ushort(h[3]) << 16);
  lp.x = (uint32_t)__half_as_ushort(l[0]) | ((uint32_t)__half_as_ushort(l[1]) << 16);
  lp.y = (uint32_t)__half_as_ushort(l[2]) | ((uint32_t)__half_as_ushort(l[3]) << 16);
}

struct GramTcArgs {
  const float* x;     // column-major I x K
  int64_t I, K;
  int ntypes, nkg;    // tile types (a, h) and K groups; grid = ntypes * nkg
  int TA;             // row blocks of 128
  float scale;        // power of two, max|x scale| <= 2^14
  double inv_scale2;  // 1 / scale^2
  double* part;       // gridDim.x partial tiles, [col][row] = 256 x 128 FP64, zeroed
  unsigned* err;
};

__device__ __forceinline__ void type_to_tile(int t, int TA, int& a, int& h) {
  int acc = 0;
  for (int aa = 0; aa < TA; ++aa) {
    const int n = aa / 2 + 1;
    if (t < acc + n) { a = aa; h = t - acc; return; }
    acc += n;
  }
  a = TA - 1;
  h = 0;
}

__global__ void __launch_bounds__(NTHREADS, 1) k_gram_tc_col(GramTcArgs g) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t bar_full[NSTAGE], bar_empty[NSTAGE], bar_accf[2], bar_acce[2], bar_done;
  __shared__ uint32_t tmem_base_sh;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int type = blockIdx.x % g.ntypes, kg = blockIdx.x / g.ntypes;
  int ta, th;
  type_to_tile(type, g.TA, ta, th);
  const int64_t k0 = g.K * kg / g.nkg, k1 = g.K * (kg + 1) / g.nkg;
  const int nst = (int)((k1 - k0 + BK - 1) / BK);
  const int nchunks = (nst + CHUNK - 1) / CHUNK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(smem_u32(&bar_full[s]), NPROD);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&bar_accf[b]), 1);
      mbar_init(smem_u32(&bar_acce[b]), 4);
    }
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
    // ---------------- producers: X -> FP16 hi/lo operand tiles
    const int64_t rowA = (int64_t)ta * 128 + 4 * lane;
    const int64_t rowB0 = (int64_t)th * 256 + 4 * lane;
    for (int s = 0; s < nst; ++s) {
      const int slot = s % NSTAGE;
      float4 v[24];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int kl = warp + NPROD * j;
        const int64_t kc = k0 + (int64_t)s * BK + kl;
        const bool kok = kc < k1;
        const float* col = g.x + kc * g.I;
#pragma unroll
        for (int gi = 0; gi < 3; ++gi) {
          const int64_t row = gi == 0 ? rowA : rowB0 + 128 * (gi - 1);
          v[3 * j + gi] = (kok && row < g.I) ? __ldcs(reinterpret_cast<const float4*>(col + row))
                                             : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
      if (s >= NSTAGE) {
        if (!mbar_wait(smem_u32(&bar_empty[slot]), ((s / NSTAGE) - 1) & 1, g.err)) break;
      }
      uint8_t* st = smem + (size_t)slot * STAGE_BYTES;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int kl = warp + NPROD * j;
#pragma unroll
        for (int gi = 0; gi < 3; ++gi) {
          uint2 hp, lp;
          split4(v[3 * j + gi], g.scale, hp, lp);
          uint32_t oh, ol;
          if (gi == 0) {
            const uint32_t o = mn_off(4 * lane, kl, A_SK);
            oh = OFF_HA + o;
            ol = OFF_LA + o;
          } else {
            const uint32_t o = mn_off(128 * (gi - 1) + 4 * lane, kl, B_SK);
            oh = OFF_HB + o;
            ol = OFF_LB + o;
          }
          *reinterpret_cast<uint2*>(st + oh) = hp;
          *reinterpret_cast<uint2*>(st + ol) = lp;
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bar_full[slot]));
    }
  } else if (warp == MMA_WARP) {
    // ---------------- MMA issue (one thread)
    if (lane == 0) {
      const uint32_t idesc = instr_desc(128, 256);
      const uint32_t sbase = smem_u32(smem);
      bool ok = true;
      for (int s = 0; s < nst && ok; ++s) {
        const int slot = s % NSTAGE;
        const int c = s / CHUNK, buf = c & 1;
        const bool first = (s % CHUNK) == 0;
        if (first && c >= 2) ok = mbar_wait(smem_u32(&bar_acce[buf]), ((c / 2) - 1) & 1, g.err);
        if (ok) ok = mbar_wait(smem_u32(&bar_full[slot]), (s / NSTAGE) & 1, g.err);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t st = sbase + (uint32_t)slot * STAGE_BYTES;
        const uint32_t d = tmem + (uint32_t)buf * 256u;
#pragma unroll
        for (int ks = 0; ks < BK / 16; ++ks) {
          const uint64_t ha = smem_desc(st + OFF_HA + ks * 2 * A_SK, ATOM_MN, A_SK);
          const uint64_t la = smem_desc(st + OFF_LA + ks * 2 * A_SK, ATOM_MN, A_SK);
          const uint64_t hb = smem_desc(st + OFF_HB + ks * 2 * B_SK, ATOM_MN, B_SK);
          const uint64_t lb = smem_desc(st + OFF_LB + ks * 2 * B_SK, ATOM_MN, B_SK);
          const uint32_t acc0 = (first && ks == 0) ? 0u : 1u;
          tc_mma(d, ha, hb, idesc, acc0);
          tc_mma(d, ha, lb, idesc, 1u);
          tc_mma(d, la, hb, idesc, 1u);
          tc_mma(d, la, lb, idesc, 1u);
        }
        tc_commit(smem_u32(&bar_empty[slot]));
        if ((s % CHUNK) == CHUNK - 1 || s == nst - 1) tc_commit(smem_u32(&bar_accf[buf]));
      }
      tc_commit(smem_u32(&bar_done));
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: tensor memory -> FP64 partial tile
    const int q = warp & 3;                 // lane quarter this warp may access
    const int row = 32 * q + lane;
    double* pt = g.part + (size_t)blockIdx.x * TILE_ELEMS;
    for (int c = 0; c < nchunks; ++c) {
      const int buf = c & 1;
      if (!mbar_wait(smem_u32(&bar_accf[buf]), (c / 2) & 1, g.err)) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      for (int c0 = 0; c0 < 256; c0 += 32) {
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)buf * 256u + (uint32_t)c0, r);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          double* p = pt + (size_t)(c0 + j) * 128 + row;
          *p += (double)__uint_as_float(r[j]) * g.inv_scale2;
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
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
  }
}

// S[i][j] = S[j][i] = sum over K groups of tile (a, h) at (row = hi - 128a,
// col = lo - 256h), hi = max(i, j), lo = min(i, j).
__global__ void k_gram_tc_reduce(const double* __restrict__ part, int ntypes, int nkg, int TA,
                                 int64_t I, double* __restrict__ S) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= I * I) return;
  const int64_t i = idx / I, j = idx % I;
  if (j > i) return;
  const int a = (int)(i / 128), h = (int)(j / 256);
  int t = 0;
  for (int aa = 0; aa < a; ++aa) t += aa / 2 + 1;
  t += h;
  const size_t off = (size_t)(j - 256 * h) * 128 + (size_t)(i - 128 * a);
  double s = 0.0;
  for (int k = 0; k < nkg; ++k) s += part[(size_t)(t + ntypes * k) * TILE_ELEMS + off];
  S[i * I + j] = s;
  S[j * I + i] = s;
}

int count_types(int TA) {
  int n = 0;
  for (int a = 0; a < TA; ++a) n += a / 2 + 1;
  return n;
}

}  // namespace

TcGramPlan plan_gram_tc(int64_t L, int64_t I, int64_t Rt, int num_sms) {
  TcGramPlan p;
  if (L != 1 || I < 64 || I > 4096 || (I % 4) != 0 || Rt < BK) return p;
  const int TA = (int)((I + 127) / 128);
  p.ntiles = count_types(TA);
  int nkg = num_sms / (int)p.ntiles;
  if (nkg < 1) nkg = 1;
  const int64_t maxkg = (Rt + BK - 1) / BK;
  if (nkg > maxkg) nkg = (int)maxkg;
  p.nsplit = nkg;
  p.scratch_bytes = (size_t)p.ntiles * nkg * TILE_ELEMS * sizeof(double);
  p.ok = 1;
  return p;
}

cudaError_t launch_gram_tc(const float* y, int64_t L, int64_t I, int64_t Rt, const TcGramPlan& p,
                           float scale, double* scratch, unsigned* err, double* S, cudaStream_t st) {
  if (!p.ok || L != 1) return cudaErrorInvalidValue;
  if (((uintptr_t)y & 15) != 0) return cudaErrorInvalidValue;
  {
    cudaError_t e = allow_max_dyn_smem((const void*)k_gram_tc_col);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaMemsetAsync(scratch, 0, p.scratch_bytes, st);
  if (e != cudaSuccess) return e;
  GramTcArgs a;
  a.x = y;
  a.I = I;
  a.K = Rt;
  a.ntypes = (int)p.ntiles;
  a.nkg = (int)p.nsplit;
  a.TA = (int)((I + 127) / 128);
  a.scale = scale;
  a.inv_scale2 = 1.0 / ((double)scale * (double)scale);
  a.part = scratch;
  a.err = err;
  count_launches(2);
  k_gram_tc_col<<<(unsigned)(p.ntiles * p.nsplit), NTHREADS, SMEM_BYTES, st>>>(a);
  const int64_t tot = I * I;
  k_gram_tc_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(scratch, a.ntypes, a.nkg, a.TA, I, S);
  return cudaGetLastError();
}

}  // namespace tk
