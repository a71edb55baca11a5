// Tensor-core (tcgen05) TTM of the column-major mode-0 view (Algorithm 3,
// n = 0): Z (K x Rt) = A (K x I) Y (I x Rt), where slab m of the mode-0 view
// is column m of Y (contiguous in i) and A = U_0^T (or any K x I operator of
// the multi-TTM), K <= 128.  Z is written column-major: the K outputs of one
// slab are contiguous, which is the natural-descending layout of the result.
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
// Work split.  A tile is 256 consecutive slabs (MMA N = 256) over all of I;
// one persistent CTA per SM walks tiles blockIdx.x, blockIdx.x + gridDim.x,
// ...  Stages of 64 i flow through a two-slot ring.  Roles (13 warps): warps
// 0-7 load Y with 16-byte streaming loads, split it into the K-major SW128 B
// operand, and copy the stage's pre-split A chunk; warp 8 issues the MMAs;
// warps 9-12 drain the double-buffered accumulators (2 x 256 tensor-memory
// columns) and write Z.  Every wait is bounded: a wait that gives up sets
// DEV_ERR_MBAR_TIMEOUT and the kernel winds down.
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace tk {
namespace {

using namespace tc;

constexpr int TN = 256;                        // slabs per tile (MMA N)
constexpr int TM = 128;                        // MMA M (rows of A; K <= TM)
constexpr int SK = 64;                         // i per stage
constexpr int NSTAGE = 2;
constexpr int NPROD = 8;
constexpr int MMA_WARP = 8;
constexpr int NTHREADS = 13 * 32;
constexpr uint32_t A_BYTES = TM * SK * 2;      // 16 KB
constexpr uint32_t B_BYTES = TN * SK * 2;      // 32 KB
constexpr uint32_t OFF_AH = 0, OFF_AL = A_BYTES, OFF_BH = 2 * A_BYTES,
                   OFF_BL = 2 * A_BYTES + B_BYTES;
constexpr uint32_t STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;   // 96 KB
constexpr uint32_t SMEM_BYTES = NSTAGE * STAGE_BYTES + 1024;

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

__device__ __forceinline__ void split_pack(float a, float b, uint32_t& h, uint32_t& l) {
  const __half ha = __float2half_rn(a), hb = __float2half_rn(b);
  const __half la = __float2half_rn(a - __half2float(ha));
  const __half lb = __float2half_rn(b - __half2float(hb));
  h = (uint32_t)__half_as_ushort(ha) | ((uint32_t)__half_as_ushort(hb) << 16);
  l = (uint32_t)__half_as_ushort(la) | ((uint32_t)__half_as_ushort(lb) << 16);
}

// A (K x I, FP64: element (k, i) at A[k*lda + i] if arow else A[k + lda*i])
// -> per stage: [A_h tile | A_l tile] as shared-memory images (K-major SW128,
// 128 rows x 64 i, zero outside K x I), scaled by s_a; *sa_out = s_a.
// One CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_ttm_tc_prep(const double* __restrict__ A, int K,
                                                      int64_t I, int64_t lda, int arow, int nks,
                                                      uint8_t* __restrict__ out,
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
  const int64_t tot = (int64_t)nks * TM * (SK / 2);   // element pairs (k, k+1)
  for (int64_t e = threadIdx.x; e < tot; e += blockDim.x) {
    const int ks = (int)(e / (TM * (SK / 2)));
    const int rem = (int)(e % (TM * (SK / 2)));
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
    uint8_t* base = out + (size_t)ks * 2 * A_BYTES;
    const uint32_t o = kmaj_off(row, kp);
    *reinterpret_cast<uint32_t*>(base + o) = h;
    *reinterpret_cast<uint32_t*>(base + A_BYTES + o) = l;
  }
}

struct TtmTcArgs {
  const float* y;        // I x Rt column-major, 16-byte aligned, I % 4 == 0
  int64_t I, Rt;
  int K;                 // rows of A = outputs per slab (<= 128)
  int nks;               // stages per tile = ceil(I / 64)
  int64_t ntiles;        // ceil(Rt / 256)
  float sy;              // power of two
  const uint8_t* aprep;  // nks x [A_h | A_l] images
  const float* sa;       // the power-of-two scale of A (device)
  float* z;              // K x Rt column-major
  unsigned* err;
};

__global__ void __launch_bounds__(NTHREADS, 1) k_ttm_tc_col(TtmTcArgs g) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t bar_full[NSTAGE], bar_empty[NSTAGE], bar_accf[2], bar_acce[2], bar_done;
  __shared__ uint32_t tmem_base_sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

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
  const int64_t my_tiles =
      (g.ntiles > (int64_t)blockIdx.x) ? (g.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

  if (warp < NPROD) {
    // ---------------- producers: Y -> FP16 hi/lo B operand; A chunk copy
    const int ptid = threadIdx.x;   // 0..255
    bool ok = true;
    for (int64_t j = 0; j < my_tiles && ok; ++j) {
      const int64_t m0 = ((int64_t)blockIdx.x + j * gridDim.x) * TN;
      for (int ks = 0; ks < g.nks; ++ks) {
        const int64_t gs = j * g.nks + ks;
        const int slot = (int)(gs % NSTAGE);
        float4 v[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int c = ptid + 256 * e;
          const int m = c >> 4, q = c & 15;
          const int64_t slab = m0 + m, i = (int64_t)ks * SK + 4 * q;
          v[e] = (slab < g.Rt && i < g.I)
                     ? __ldcs(reinterpret_cast<const float4*>(g.y + slab * g.I + i))
                     : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        uint4 av[8];
        const uint4* asrc = reinterpret_cast<const uint4*>(g.aprep + (size_t)ks * 2 * A_BYTES);
#pragma unroll
        for (int e = 0; e < 8; ++e) av[e] = asrc[ptid + 256 * e];
        if (gs >= NSTAGE) {
          if (!mbar_wait(smem_u32(&bar_empty[slot]), (uint32_t)(((gs / NSTAGE) - 1) & 1), g.err)) {
            ok = false;
            break;
          }
        }
        uint8_t* st = smem + (size_t)slot * STAGE_BYTES;
#pragma unroll
        for (int e = 0; e < 8; ++e) reinterpret_cast<uint4*>(st + OFF_AH)[ptid + 256 * e] = av[e];
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int c = ptid + 256 * e;
          const int m = c >> 4, q = c & 15;
          uint2 hp, lp;
          split_pack(v[e].x * g.sy, v[e].y * g.sy, hp.x, lp.x);
          split_pack(v[e].z * g.sy, v[e].w * g.sy, hp.y, lp.y);
          const uint32_t o = kmaj_off(m, 4 * q);
          *reinterpret_cast<uint2*>(st + OFF_BH + o) = hp;
          *reinterpret_cast<uint2*>(st + OFF_BL + o) = lp;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bar_full[slot]));
      }
    }
  } else if (warp == MMA_WARP) {
    // ---------------- MMA issue (one thread)
    if (lane == 0) {
      const uint32_t idesc = instr_desc_kk(TM, TN);
      const uint32_t sbase = smem_u32(smem);
      bool ok = true;
      for (int64_t j = 0; j < my_tiles && ok; ++j) {
        const int buf = (int)(j & 1);
        if (j >= 2) ok = mbar_wait(smem_u32(&bar_acce[buf]), (uint32_t)(((j / 2) - 1) & 1), g.err);
        for (int ks = 0; ks < g.nks && ok; ++ks) {
          const int64_t gs = j * g.nks + ks;
          const int slot = (int)(gs % NSTAGE);
          ok = mbar_wait(smem_u32(&bar_full[slot]), (uint32_t)((gs / NSTAGE) & 1), g.err);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t st = sbase + (uint32_t)slot * STAGE_BYTES;
          const uint32_t d = tmem + (uint32_t)buf * 256u;
#pragma unroll
          for (int kk = 0; kk < SK / 16; ++kk) {
            const uint64_t ah = smem_desc(st + OFF_AH + 32u * kk, 16, 1024);
            const uint64_t al = smem_desc(st + OFF_AL + 32u * kk, 16, 1024);
            const uint64_t bh = smem_desc(st + OFF_BH + 32u * kk, 16, 1024);
            const uint64_t bl = smem_desc(st + OFF_BL + 32u * kk, 16, 1024);
            const uint32_t acc0 = (ks > 0 || kk > 0) ? 1u : 0u;
            tc_mma(d, ah, bh, idesc, acc0);
            tc_mma(d, ah, bl, idesc, 1u);
            tc_mma(d, al, bh, idesc, 1u);
          }
          tc_commit(smem_u32(&bar_empty[slot]));
        }
        if (ok) tc_commit(smem_u32(&bar_accf[buf]));
      }
      tc_commit(smem_u32(&bar_done));
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: tensor memory -> Z
    const int q = warp & 3;          // the lane quarter this warp may access
    const int r = 32 * q + lane;     // output row (index of the K outputs)
    const float inv = (float)(1.0 / ((double)g.sy * (double)*g.sa));   // powers of two: exact
    for (int64_t j = 0; j < my_tiles; ++j) {
      const int buf = (int)(j & 1);
      if (!mbar_wait(smem_u32(&bar_accf[buf]), (uint32_t)((j / 2) & 1), g.err)) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int64_t m0 = ((int64_t)blockIdx.x + j * gridDim.x) * TN;
      if (32 * q < g.K) {
        for (int c0 = 0; c0 < TN; c0 += 32) {
          uint32_t rr[32];
          tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)buf * 256u + (uint32_t)c0, rr);
          if (r < g.K) {
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
              const int64_t slab = m0 + c0 + jj;
              if (slab < g.Rt) g.z[slab * g.K + r] = __uint_as_float(rr[jj]) * inv;
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
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
  }
}

}  // namespace

int ttm_tc_supported(int64_t L, int64_t I, int64_t Rt, int64_t K) {
  return L == 1 && I >= 64 && I <= 65536 && (I % 4) == 0 && K >= 1 && K <= TM && Rt >= 1;
}

size_t ttm_tc_scratch_bytes(int64_t I, int64_t K) {
  (void)K;
  const size_t nks = (size_t)((I + SK - 1) / SK);
  return nks * 2 * A_BYTES + 256;
}

cudaError_t launch_ttm_tc(const float* y, int64_t L, int64_t I, int64_t Rt, const double* A,
                          int64_t K, int64_t lda, int a_rowmajor, float sy, float* z, void* scratch,
                          unsigned* err, int num_sms, cudaStream_t st) {
  if (!ttm_tc_supported(L, I, Rt, K) || ((uintptr_t)y & 15) != 0) return cudaErrorInvalidValue;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_ttm_tc_col, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SMEM_BYTES);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int nks = (int)((I + SK - 1) / SK);
  uint8_t* aprep = (uint8_t*)scratch;
  float* sa = (float*)(aprep + (size_t)nks * 2 * A_BYTES);
  k_ttm_tc_prep<<<1, 1024, 0, st>>>(A, (int)K, I, lda, a_rowmajor, nks, aprep, sa);
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
  a.err = err;
  const int grid = (int)(a.ntiles < num_sms ? a.ntiles : num_sms);
  k_ttm_tc_col<<<grid, NTHREADS, SMEM_BYTES, st>>>(a);
  count_launches(2);
  return cudaGetLastError();
}

}  // namespace tk
