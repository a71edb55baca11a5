// Gram of a slab view with a small mode (I < 64): S = sum over slabs of
// Y_r Y_r^T (Section 5.1, Alg. 2), with FP64 products and FP64 sums for
// every input precision.
//
// Why FP64 here.  Such modes come last in an ST-HOSVD, after the others are
// truncated: the l index of the view then runs over a few eigen-sorted
// components, a few K-blocks carry most of each entry, and the ~6e-8
// relative rounding of an FP32 block sum no longer averages out over many
// slabs.  Projected on the discarded subspace it reached half the eps = 1e-4
// threshold on a 256x256x256x11x32 tensor.  The work is I(I+1)/2 FP64 FMAs
// per K element (products of FP32 inputs are exact in FP64), which for
// I < 64 is a small fraction of the mode's reads even at this part's FP64
// rate.
//
// Layout: one thread per entry (i <= j) of the lower triangle (several per
// thread when I(I+1)/2 > 256); a CTA stages K-blocks of 64 (the K geometry of
// gram_order.cuh) in shared memory as FP64 and walks K-blocks blockIdx.x,
// blockIdx.x + gridDim.x, ...; each CTA writes its partial triangle and a
// second kernel sums the partials (a fixed order, see k_gram_small_reduce).
#include "common.cuh"
#include "gram_order.cuh"
#include "kernels.h"

namespace tk {
namespace {

constexpr int SBK = 64;          // K per block (64: 22-29 % faster than 16 on 55 MB views)
constexpr int SNT = 256;         // threads per CTA
constexpr int SMAXI = 63;
constexpr int SMAXP = SMAXI * (SMAXI + 1) / 2;              // 2016 entries
constexpr int SPPT = (SMAXP + SNT - 1) / SNT;               // entries per thread (8)

template <typename TIn>
__global__ void __launch_bounds__(SNT) k_gram_small(const TIn* __restrict__ y, KGeom g,
                                                    double* __restrict__ part) {
  __shared__ double ys[SBK][SMAXI + 2];   // odd row stride in doubles: the l-major staging spreads over banks
  const int I = (int)g.I;
  const int npair = I * (I + 1) / 2;
  // this thread's entries: p = threadIdx.x + SNT * e  ->  (i, j), j <= i
  int pi[SPPT], pj[SPPT];
#pragma unroll
  for (int e = 0; e < SPPT; ++e) {
    const int p = threadIdx.x + SNT * e;
    int i = (int)((sqrtf(8.f * (float)p + 1.f) - 1.f) * 0.5f);
    while ((i + 1) * (i + 2) / 2 <= p) ++i;
    while (i * (i + 1) / 2 > p) --i;
    pi[e] = (p < npair) ? i : 0;
    pj[e] = (p < npair) ? p - i * (i + 1) / 2 : 0;
  }
  double acc[SPPT];
#pragma unroll
  for (int e = 0; e < SPPT; ++e) acc[e] = 0.0;

  for (int64_t kb = blockIdx.x; kb < g.NKB; kb += gridDim.x) {
    __syncthreads();
    // stage the block: SBK K x I values
    if (g.L == 1) {
      for (int c = threadIdx.x; c < SBK * I; c += SNT) {
        const int kk = c / I, i = c - kk * I;
        const int64_t r = kb * SBK + kk;
        ys[kk][i] = (r < g.Rt) ? (double)y[i + g.I * r] : 0.0;
      }
    } else {
      const int64_t r = kb / g.nLB;
      int64_t lbeg, lend;
      lblock_range(g, kb - r * g.nLB, SBK, lbeg, lend);
      const TIn* base = y + g.L * g.I * r;
      for (int c = threadIdx.x; c < SBK * I; c += SNT) {
        const int i = c / SBK, kk = c - i * SBK;   // consecutive threads: consecutive l
        const int64_t l = lbeg + kk;
        ys[kk][i] = (l < lend) ? (double)base[l + g.L * i] : 0.0;
      }
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < SPPT; ++e) {
      if (threadIdx.x + SNT * e >= npair) break;
      const int i = pi[e], j = pj[e];
      double a = acc[e];
#pragma unroll
      for (int kk = 0; kk < SBK; ++kk) a = fma(ys[kk][i], ys[kk][j], a);
      acc[e] = a;
    }
  }
  double* out = part + (int64_t)blockIdx.x * npair;
#pragma unroll
  for (int e = 0; e < SPPT; ++e) {
    const int p = threadIdx.x + SNT * e;
    if (p < npair) out[p] = acc[e];
  }
}

// S[i][j] = S[j][i] = sum over CTAs of the partial triangles: one warp per
// entry, lane l summing parts l, l + 32, ... in order, then a fixed butterfly
// across the lanes (a chain of ~nparts / 32 FP64 additions instead of nparts).
__global__ void k_gram_small_reduce(const double* __restrict__ part, int nparts, int I,
                                    double* __restrict__ S) {
  const int npair = I * (I + 1) / 2;
  const int p = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (p >= npair) return;
  int i = (int)((sqrtf(8.f * (float)p + 1.f) - 1.f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= p) ++i;
  while (i * (i + 1) / 2 > p) --i;
  const int j = p - i * (i + 1) / 2;
  double s = 0.0;
  for (int k = lane; k < nparts; k += 32) s += part[(int64_t)k * npair + p];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    S[(int64_t)i * I + j] = s;
    S[(int64_t)j * I + i] = s;
  }
}

}  // namespace

GramPlan plan_gram_small(int64_t L, int64_t I, int64_t Rt, int num_sms, int64_t L0) {
  GramPlan p;
  if (I < 1 || I > SMAXI || L < 1 || Rt < 1) return p;   // nctas == 0: not applicable
  const KGeom g = make_kgeom(L, I, Rt, SBK, L0);
  int64_t n = (int64_t)num_sms * 8;
  if (n > g.NKB) n = g.NKB;
  if (n < 1) n = 1;
  p.nctas = (int)n;
  p.ntiles = 1;
  p.scratch_bytes = (size_t)n * (size_t)(I * (I + 1) / 2) * sizeof(double);
  return p;
}

cudaError_t launch_gram_small(const void* y, tucker_dtype dt, int64_t L, int64_t I, int64_t Rt,
                              int64_t L0, const GramPlan& p, double* scratch, double* S,
                              cudaStream_t st) {
  const KGeom g = make_kgeom(L, I, Rt, SBK, L0);
  if (dt == TUCKER_F64)
    k_gram_small<double><<<p.nctas, SNT, 0, st>>>((const double*)y, g, scratch);
  else
    k_gram_small<float><<<p.nctas, SNT, 0, st>>>((const float*)y, g, scratch);
  const int npair = (int)(I * (I + 1) / 2);
  k_gram_small_reduce<<<(npair + 7) / 8, 256, 0, st>>>(scratch, p.nctas, (int)I, S);
  count_launches(2);
  return cudaGetLastError();
}

}  // namespace tk
