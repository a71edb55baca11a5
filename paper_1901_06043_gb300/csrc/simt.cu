// SIMT kernels of the ST-HOSVD path: FP64 sum of squares (Section 2.2.2),
// slab-batched Gram (Algorithm 2) and slab TTM (Algorithm 3) in FP64 or
// FP32 arithmetic, over the unfolding-free strided view (Rt, I, L) of
// Section 4.2: element (l, i, r) of the mode-n view sits at l + L*(i + I*r).
#include <algorithm>
#include <cstdio>

#include "common.cuh"
#include "kernels.h"
#include "gram_order.cuh"

namespace tk {

// ------------------------------------------------------------ sum of squares

// Block reduction of a thread's (sum, max|x|): partial[b] = sum of block b,
// partial[gridDim.x + b] = max of block b.  Any block size up to 1024.
__device__ __forceinline__ void block_store_sum_max(double acc, double mx, double* partial,
                                                    unsigned* nonfinite, bool bad) {
  for (int o = 16; o > 0; o >>= 1) {
    acc += __shfl_xor_sync(0xffffffffu, acc, o);
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  __shared__ double s[32], m[32];
  if ((threadIdx.x & 31) == 0) {
    s[threadIdx.x >> 5] = acc;
    m[threadIdx.x >> 5] = mx;
  }
  if (bad) atomicOr(nonfinite, 1u);
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0, tm = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      t += s[w];
      tm = fmax(tm, m[w]);
    }
    partial[blockIdx.x] = t;
    partial[gridDim.x + blockIdx.x] = tm;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_sumsq(const T* __restrict__ y, int64_t n,
                                               double* __restrict__ partial,
                                               unsigned* __restrict__ nonfinite) {
  double acc = 0.0, mx = 0.0;
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    double v = (double)y[i];
    bad |= !isfinite(v);
    acc = fma(v, v, acc);
    mx = fmax(mx, fabs(v));
  }
  block_store_sum_max(acc, mx, partial, nonfinite, bad);
}

// Fixed-order reduction of `count` (sum, max) partials into out[0] (sum)
// and out[1] (max), one block.
__global__ void __launch_bounds__(256) k_reduce_sum(const double* __restrict__ partial, int count,
                                                    double* __restrict__ out) {
  double acc = 0.0, mx = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    acc += partial[i];
    mx = fmax(mx, partial[count + i]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    acc += __shfl_xor_sync(0xffffffffu, acc, o);
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  __shared__ double s[8], m[8];
  if ((threadIdx.x & 31) == 0) {
    s[threadIdx.x >> 5] = acc;
    m[threadIdx.x >> 5] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0, tm = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      t += s[w];
      tm = fmax(tm, m[w]);
    }
    out[0] = t;
    out[1] = tm;
  }
}

// Error-free FP32 sum: s + e == a + b exactly (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// FP32 input: x^2 = p + e exactly (p = fl(x*x), e = fma(x, x, -p)); the p
// are summed as an FP32 pair (hi, lo) with TwoSum and the pair is moved into
// the FP64 sum every 128 elements, so the result matches an FP64 sum of the
// exact squares to ~1e-15 while the kernel stays on the FP32 pipe and the
// HBM roofline.  Every FP64 instruction costs a sub-partition's FP64 pipe 64
// cycles per warp, so the per-element path has none: the moves into FP64
// convert on integer bits, max |x| and the non-finite test are integer
// maxima of the bit patterns, and a group of 16 whose largest |x| is at
// least 2^64 (an FP32 square could overflow) or nonzero and below 2^-60 (its
// squares would underflow FP32) is squared in FP64 on a warp-uniform branch
// (in a group with a larger value, squares below 2^-120 are ~2^-96 of it).
__device__ __forceinline__ double f32_bits_to_f64(float x) {
  // exact for normal x; zero and subnormals (below 1.2e-38) become 0
  const unsigned u = __float_as_uint(x);
  const unsigned ex = (u >> 23) & 0xffu;
  const unsigned long long b = (unsigned long long)(u >> 31) << 63 |
                               (unsigned long long)(ex + 1023u - 127u) << 52 |
                               (unsigned long long)(u & 0x7fffffu) << 29;
  return ex == 0u ? 0.0 : __longlong_as_double((long long)b);
}

struct SumSqF32 {
  double acc = 0.0;
  float hi = 0.f, lo = 0.f;
  unsigned mxb = 0;     // max |x| as bits; >= 0x7f800000: NaN or Inf seen
  __device__ __forceinline__ void add_fast(float x) {
    const float p = x * x;
    const float e = fmaf(x, x, -p);
    float s, err;
    two_sum(hi, p, s, err);
    hi = s;
    lo += err + e;
  }
  __device__ __forceinline__ void add(float x) {   // tails: per-element test
    const unsigned b = __float_as_uint(x) & 0x7fffffffu;
    mxb = max(mxb, b);
    if (b >= 0x5f800000u || (b != 0u && b < 0x21800000u)) acc = fma((double)x, (double)x, acc);
    else add_fast(x);
  }
  __device__ __forceinline__ void flush() {
    acc += f32_bits_to_f64(hi) + f32_bits_to_f64(lo);
    hi = lo = 0.f;
  }
};

__global__ void __launch_bounds__(256) k_sumsq_f32(const float* __restrict__ y, int64_t n,
                                                   double* __restrict__ partial,
                                                   unsigned* __restrict__ nonfinite) {
  SumSqF32 s;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t head = (int64_t)(((16 - ((uintptr_t)y & 15)) & 15) / 4);
  if (head > n) head = n;
  const int64_t nv = (n - head) / 4;
  const float4* yv = reinterpret_cast<const float4*>(y + head);
  // four independent 16-byte loads in flight per thread per iteration
  int64_t v = tid;
  int groups = 0;
  for (; v + 3 * stride < nv; v += 4 * stride) {
    float4 q[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) q[u] = __ldcs(yv + v + u * stride);
    unsigned gm = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      gm = max(gm, __float_as_uint(q[u].x) & 0x7fffffffu);
      gm = max(gm, __float_as_uint(q[u].y) & 0x7fffffffu);
      gm = max(gm, __float_as_uint(q[u].z) & 0x7fffffffu);
      gm = max(gm, __float_as_uint(q[u].w) & 0x7fffffffu);
    }
    s.mxb = max(s.mxb, gm);
    if (__any_sync(__activemask(), gm >= 0x5f800000u || (gm != 0u && gm < 0x21800000u))) {
#pragma unroll
      for (int u = 0; u < 4; ++u) { s.add(q[u].x); s.add(q[u].y); s.add(q[u].z); s.add(q[u].w); }
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        s.add_fast(q[u].x); s.add_fast(q[u].y); s.add_fast(q[u].z); s.add_fast(q[u].w);
      }
    }
    if (++groups == 8) { s.flush(); groups = 0; }
  }
  for (; v < nv; v += stride) {
    const float4 q = __ldcs(yv + v);
    s.add(q.x); s.add(q.y); s.add(q.z); s.add(q.w);
  }
  for (int64_t i = tid; i < head; i += stride) s.add(y[i]);
  for (int64_t i = head + 4 * nv + tid; i < n; i += stride) s.add(y[i]);
  s.flush();
  const bool bad = s.mxb >= 0x7f800000u;
  block_store_sum_max(s.acc, bad ? 0.0 : (double)__uint_as_float(s.mxb), partial, nonfinite, bad);
}

// The same sum of squares over the column-major I0 x ncols view (mode 0),
// recording also each row's max |x| (as FP32 bits, atomicMax into
// rowmax_bits[I0], zeroed by the caller): thread t owns rows 4t..4t+3 (and
// 4(t + blockDim.x).., ... when I0 / 4 exceeds the block: `passes` rounds over
// the block's columns, one per row quad) and walks the columns blockIdx.x,
// blockIdx.x + gridDim.x, ..., eight columns per iteration in flight.  VEC:
// one 16-byte load per quad (I0 % 4 == 0, 16-byte aligned y); otherwise four
// 4-byte loads, rows past I0 read as zero.  I0 <= 8192.
template <bool VEC>
__device__ __forceinline__ float4 load_quad(const float* p, int64_t r4, int64_t I0) {
  if (VEC) return __ldcs(reinterpret_cast<const float4*>(p));
  float4 q;
  q.x = (r4 < I0) ? __ldcs(p) : 0.f;
  q.y = (r4 + 1 < I0) ? __ldcs(p + 1) : 0.f;
  q.z = (r4 + 2 < I0) ? __ldcs(p + 2) : 0.f;
  q.w = (r4 + 3 < I0) ? __ldcs(p + 3) : 0.f;
  return q;
}

template <bool VEC>
__global__ void __launch_bounds__(512) k_sumsq_rowmax_f32(const float* __restrict__ y, int64_t I0,
                                                           int64_t ncols, int passes,
                                                           double* __restrict__ partial,
                                                           unsigned* __restrict__ nonfinite,
                                                           unsigned* __restrict__ rowmax_bits) {
  SumSqF32 s;
  int groups = 0;
  for (int pass = 0; pass < passes; ++pass) {
    const int64_t r4 = 4 * ((int64_t)threadIdx.x + (int64_t)pass * blockDim.x);
    const bool active = r4 < I0;
    unsigned rm[4] = {0u, 0u, 0u, 0u};
    int64_t c = blockIdx.x;
    constexpr int U = 8;
    for (; c + (U - 1) * (int64_t)gridDim.x < ncols; c += U * (int64_t)gridDim.x) {
      float4 q[U];
#pragma unroll
      for (int u = 0; u < U; ++u)
        q[u] = active ? load_quad<VEC>(y + r4 + I0 * (c + u * (int64_t)gridDim.x), r4, I0)
                      : make_float4(0.f, 0.f, 0.f, 0.f);
      unsigned gm = 0;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const unsigned b0 = __float_as_uint(q[u].x) & 0x7fffffffu, b1 = __float_as_uint(q[u].y) & 0x7fffffffu;
        const unsigned b2 = __float_as_uint(q[u].z) & 0x7fffffffu, b3 = __float_as_uint(q[u].w) & 0x7fffffffu;
        rm[0] = max(rm[0], b0); rm[1] = max(rm[1], b1); rm[2] = max(rm[2], b2); rm[3] = max(rm[3], b3);
        gm = max(gm, max(max(b0, b1), max(b2, b3)));
      }
      s.mxb = max(s.mxb, gm);
      if (__any_sync(__activemask(), gm >= 0x5f800000u || (gm != 0u && gm < 0x21800000u))) {
#pragma unroll
        for (int u = 0; u < U; ++u) { s.add(q[u].x); s.add(q[u].y); s.add(q[u].z); s.add(q[u].w); }
      } else {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          s.add_fast(q[u].x); s.add_fast(q[u].y); s.add_fast(q[u].z); s.add_fast(q[u].w);
        }
      }
      if (++groups == 4) { s.flush(); groups = 0; }
    }
    for (; c < ncols; c += gridDim.x) {
      if (!active) continue;
      const float4 q = load_quad<VEC>(y + r4 + I0 * c, r4, I0);
      rm[0] = max(rm[0], __float_as_uint(q.x) & 0x7fffffffu);
      rm[1] = max(rm[1], __float_as_uint(q.y) & 0x7fffffffu);
      rm[2] = max(rm[2], __float_as_uint(q.z) & 0x7fffffffu);
      rm[3] = max(rm[3], __float_as_uint(q.w) & 0x7fffffffu);
      s.add(q.x); s.add(q.y); s.add(q.z); s.add(q.w);
    }
    if (active) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (rm[u] && r4 + u < I0) atomicMax(rowmax_bits + r4 + u, rm[u]);
    }
  }
  s.flush();
  const bool bad = s.mxb >= 0x7f800000u;
  block_store_sum_max(s.acc, bad ? 0.0 : (double)__uint_as_float(s.mxb), partial, nonfinite, bad);
}

cudaError_t launch_sumsq_rowmax(const float* y, int64_t I0, int64_t ncols, double* partial,
                                int nblocks, unsigned* nonfinite, unsigned* rowmax_bits, double* out,
                                cudaStream_t st) {
  if (I0 > 8192 || I0 < 1 || ((uintptr_t)y & 3) != 0) return cudaErrorInvalidValue;
  const bool vec = I0 % 4 == 0 && ((uintptr_t)y & 15) == 0;
  // row quads per thread: as few passes as a 512-thread block allows, the
  // quads spread evenly over them
  const int64_t quads = (I0 + 3) / 4;
  const int passes = (int)((quads + 511) / 512);
  const int threads = (int)(((quads + passes - 1) / passes + 31) / 32 * 32);
  count_launches(2);
  if (vec)
    k_sumsq_rowmax_f32<true><<<nblocks, threads, 0, st>>>(y, I0, ncols, passes, partial, nonfinite,
                                                        rowmax_bits);
  else
    k_sumsq_rowmax_f32<false><<<nblocks, threads, 0, st>>>(y, I0, ncols, passes, partial,
                                                         nonfinite, rowmax_bits);
  k_reduce_sum<<<1, 256, 0, st>>>(partial, nblocks, out);
  return cudaGetLastError();
}

cudaError_t launch_sumsq(const void* y, tucker_dtype dt, int64_t n, double* partial, int nblocks,
                         unsigned* nonfinite, double* out, cudaStream_t st) {
  count_launches(2);
  if (dt == TUCKER_F64)
    k_sumsq<double><<<nblocks, 256, 0, st>>>((const double*)y, n, partial, nonfinite);
  else
    k_sumsq_f32<<<nblocks, 256, 0, st>>>((const float*)y, n, partial, nonfinite);
  k_reduce_sum<<<1, 256, 0, st>>>(partial, nblocks, out);
  return cudaGetLastError();
}

// b[i] += a[i] (FP64), grid-stride.
__global__ void k_add_f64(const double* __restrict__ a, double* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] += a[i];
}

cudaError_t launch_add_f64(const double* a, double* b, int64_t n, int num_sms, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int nb = (int)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms * 4);
  count_launches(1);
  k_add_f64<<<nb, 256, 0, st>>>(a, b, n);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ Gram

constexpr int GT = 64;    // Gram output tile
constexpr int GBK = 16;   // K-block

// Loads the (GBK x GT) panel of rows [i0, i0+GT) for K-block kb into regs.
template <typename TIn, typename TC>
__device__ __forceinline__ void gram_load(const TIn* __restrict__ y, const KGeom& g, int64_t kb,
                                          int64_t i0, TC (&reg)[4]) {
  const int tid = threadIdx.x;
  if (g.L == 1) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int idx = tid + 256 * e;
      int ii = idx % GT, kk = idx / GT;
      int64_t r = kb * GBK + kk, i = i0 + ii;
      reg[e] = (r < g.Rt && i < g.I) ? (TC)y[i + g.I * r] : (TC)0;
    }
  } else {
    int64_t r = kb / g.nLB;
    int64_t lbeg, lend;
    lblock_range(g, kb - r * g.nLB, GBK, lbeg, lend);
    const TIn* base = y + g.L * g.I * r;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int idx = tid + 256 * e;
      int kk = idx % GBK, ii = idx / GBK;
      int64_t l = lbeg + kk, i = i0 + ii;
      reg[e] = (l < lend && i < g.I) ? (TC)base[l + g.L * i] : (TC)0;
    }
  }
}

template <typename TC>
__device__ __forceinline__ void gram_store(TC (*sm)[GT + 1], const KGeom& g, const TC (&reg)[4]) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    int idx = tid + 256 * e;
    int ii, kk;
    if (g.L == 1) { ii = idx % GT; kk = idx / GT; }
    else { kk = idx % GBK; ii = idx / GBK; }
    sm[kk][ii] = reg[e];
  }
}

// One CTA: lower-triangle tile (ta >= tb) of S over its K-blocks.  TC is the
// product type.  FP64 products are summed in FP64.  FP32 products are summed
// by FMA in FP32 within a chunk, and the chunk sums are combined as an exact
// FP32 pair (TwoSum), which keeps the FP64 pipe (1/62 of the FP32 rate on
// this part) out of the inner loop.  Writes the FP64 partial tile to
// part[(ks * ntiles + tile) * GT * GT].
template <typename TIn, typename TC>
__global__ void __launch_bounds__(256) k_gram_simt(const TIn* __restrict__ y, KGeom g, int ntiles,
                                                   int ksplit, double* __restrict__ part) {
  __shared__ TC As[GBK][GT + 1];
  __shared__ TC Bs[GBK][GT + 1];
  const int tile = blockIdx.x;
  const int ks = blockIdx.y;
  // tile -> (ta, tb), ta >= tb, row-major over the lower triangle
  int ta = (int)((sqrtf(8.f * tile + 1.f) - 1.f) * 0.5f);
  while ((ta + 1) * (ta + 2) / 2 <= tile) ++ta;
  while (ta * (ta + 1) / 2 > tile) --ta;
  const int tb = tile - ta * (ta + 1) / 2;
  const bool diag = (ta == tb);
  const int64_t ia0 = (int64_t)ta * GT, ib0 = (int64_t)tb * GT;
  const KOrder ord = make_korder(g, ks, ksplit);

  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  TC acc[4][4];
  float hi[4][4], lo[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) { acc[u][v] = (TC)0; hi[u][v] = 0.f; lo[u][v] = 0.f; }

  TC ra[4], rb[4];
  bool end_cur = false, end_next = false;
  int64_t kb = 0;
  if (ord.count > 0) {
    kb = korder_block(g, ord, 0, end_cur);
    gram_load<TIn, TC>(y, g, kb, ia0, ra);
    if (!diag) gram_load<TIn, TC>(y, g, kb, ib0, rb);
  }
  for (int64_t idx = 0; idx < ord.count; ++idx) {
    gram_store<TC>(As, g, ra);
    if (!diag) gram_store<TC>(Bs, g, rb);
    __syncthreads();
    if (idx + 1 < ord.count) {
      const int64_t kbn = korder_block(g, ord, idx + 1, end_next);
      gram_load<TIn, TC>(y, g, kbn, ia0, ra);
      if (!diag) gram_load<TIn, TC>(y, g, kbn, ib0, rb);
    }
    TC (*Bp)[GT + 1] = diag ? As : Bs;
    // FP32: the 16 products of a K-block are summed into a fresh register
    // first and only that block sum enters the chunk accumulator.  Squares
    // x^2 pile up near zero (chi-square), and adding them one by one to a
    // large FP32 sum rounds with a negative bias ~ (terms in the sum)^1.5;
    // 16-term block sums have a smooth density and round without bias.  The
    // block runs from its last K to its first: in row mode its 16 l are
    // consecutive indices of a truncated mode whose energy falls with l, so
    // the products are added in increasing size.
    TC t[4][4];
#pragma unroll
    for (int kq = 0; kq < GBK; ++kq) {
      const int kk = GBK - 1 - kq;
      TC a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = As[kk][ty + 16 * u];
#pragma unroll
      for (int v = 0; v < 4; ++v) b[v] = Bp[kk][tx + 16 * v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          if constexpr (sizeof(TC) == 4)
            t[u][v] = (kq == 0) ? a[u] * b[v] : fma(a[u], b[v], t[u][v]);
          else
            acc[u][v] = fma(a[u], b[v], acc[u][v]);
        }
    }
    if constexpr (sizeof(TC) == 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] += t[u][v];
    }
    __syncthreads();
    if constexpr (sizeof(TC) == 4) {
      if (end_cur) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            float s, e;
            two_sum(hi[u][v], (float)acc[u][v], s, e);
            hi[u][v] = s;
            lo[u][v] += e;
            acc[u][v] = (TC)0;
          }
      }
    }
    end_cur = end_next;
  }
  double* out = part + ((int64_t)ks * ntiles + tile) * GT * GT;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v)
      out[(ty + 16 * u) * GT + tx + 16 * v] =
          (double)hi[u][v] + (double)lo[u][v] + (double)acc[u][v];
}

// S[i][j] = S[j][i] = sum over ks (fixed order) of the partial tiles.
__global__ void k_gram_reduce(const double* __restrict__ part, int ntiles, int ksplit, int64_t I,
                              double* __restrict__ S) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)ntiles * GT * GT) return;
  int tile = (int)(idx / (GT * GT));
  int e = (int)(idx % (GT * GT));
  int ta = (int)((sqrtf(8.f * tile + 1.f) - 1.f) * 0.5f);
  while ((ta + 1) * (ta + 2) / 2 <= tile) ++ta;
  while (ta * (ta + 1) / 2 > tile) --ta;
  int tb = tile - ta * (ta + 1) / 2;
  int64_t i = (int64_t)ta * GT + e / GT, j = (int64_t)tb * GT + e % GT;
  if (i >= I || j >= I) return;
  if (ta == tb && j > i) return;  // diagonal tile: write its lower half (and mirror)
  double s = 0.0;
  for (int k = 0; k < ksplit; ++k) s += part[((int64_t)k * ntiles + tile) * GT * GT + e];
  S[i * I + j] = s;
  S[j * I + i] = s;
}

GramPlan plan_gram_simt(int64_t L, int64_t I, int64_t Rt, int num_sms, int64_t L0) {
  GramPlan p;
  KGeom g = make_kgeom(L, I, Rt, GBK, L0);
  int T = (int)((I + GT - 1) / GT);
  p.ntiles = T * (T + 1) / 2;
  int64_t want = ((int64_t)num_sms * 4 + p.ntiles - 1) / p.ntiles;
  int64_t cap = (int64_t)(256ll << 20) / ((int64_t)p.ntiles * GT * GT * 8);
  if (want > cap) want = cap;
  if (want > g.NKB) want = g.NKB;
  if (want < 1) want = 1;
  p.ksplit = (int)want;
  p.scratch_bytes = (size_t)p.ksplit * p.ntiles * GT * GT * sizeof(double);
  return p;
}

// Same split as plan_gram_simt, with the partial-tile scratch held to at most
// max_bytes (fewer K-splits).  ok == 0 when even one split does not fit.
GramPlan plan_gram_simt_capped(int64_t L, int64_t I, int64_t Rt, int num_sms, size_t max_bytes,
                               int* ok, int64_t L0) {
  GramPlan p = plan_gram_simt(L, I, Rt, num_sms, L0);
  const size_t per_split = (size_t)p.ntiles * GT * GT * sizeof(double);
  *ok = per_split <= max_bytes;
  if (!*ok) return p;
  if (p.scratch_bytes > max_bytes) {
    p.ksplit = (int)(max_bytes / per_split);
    p.scratch_bytes = (size_t)p.ksplit * per_split;
  }
  return p;
}

cudaError_t launch_gram_simt(const void* y, tucker_dtype dt, bool fp64, int64_t L, int64_t I,
                             int64_t Rt, int64_t L0, const GramPlan& p, double* scratch, double* S,
                             cudaStream_t st) {
  KGeom g = make_kgeom(L, I, Rt, GBK, L0);
  dim3 grid(p.ntiles, p.ksplit);
  count_launches(2);
  if (dt == TUCKER_F64) {
    if (fp64) k_gram_simt<double, double><<<grid, 256, 0, st>>>((const double*)y, g, p.ntiles, p.ksplit, scratch);
    else k_gram_simt<double, float><<<grid, 256, 0, st>>>((const double*)y, g, p.ntiles, p.ksplit, scratch);
  } else {
    if (fp64) k_gram_simt<float, double><<<grid, 256, 0, st>>>((const float*)y, g, p.ntiles, p.ksplit, scratch);
    else k_gram_simt<float, float><<<grid, 256, 0, st>>>((const float*)y, g, p.ntiles, p.ksplit, scratch);
  }
  int64_t tot = (int64_t)p.ntiles * GT * GT;
  k_gram_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(scratch, p.ntiles, p.ksplit, I, S);
  return cudaGetLastError();
}

// ------------------------------------------------------------------- TTM

constexpr int TT = 64;    // output tile (k and m)
constexpr int TBI = 16;   // contraction step

// Z (K x M) = A (K x I) * Y (I x M), M = the (r, l) pairs of the slab view.
// Row mode (L > 1): an m-tile is 64 consecutive l of one slab.  Column mode
// (L == 1): an m-tile is 64 consecutive slabs; zt writes Z transposed
// (z[r + Rt k], slab fastest: the new mode last).
template <typename TIn, typename TOut, typename TC>
__global__ void __launch_bounds__(256) k_ttm_simt(const TIn* __restrict__ y, int64_t L, int64_t I,
                                                  int64_t Rt, int64_t nLT,
                                                  const double* __restrict__ A, int64_t K,
                                                  int64_t lda, int a_rowmajor,
                                                  const float* __restrict__ A32,
                                                  TOut* __restrict__ z, int zt) {
  __shared__ TC As[TBI][TT + 1];   // As[i][k]
  __shared__ TC Ys[TBI][TT + 1];   // Ys[i][m]
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  // output coordinates of this thread: the index that is contiguous in Z goes
  // to consecutive threads (k in column mode, l in row mode)
  const bool kfast = (L == 1) && !zt;
  const int kq = kfast ? tx : ty, mq = kfast ? ty : tx;
  const int64_t mt = blockIdx.x;
  const int64_t k0 = (int64_t)blockIdx.y * TT;
  int64_t r0, l0;
  if (L == 1) { r0 = mt * TT; l0 = 0; }
  else { r0 = mt / nLT; l0 = (mt - r0 * nLT) * TT; }
  const TIn* ybase = (L == 1) ? y : y + L * I * r0;

  TC acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = (TC)0;

  for (int64_t i0 = 0; i0 < I; i0 += TBI) {
    // A tile: 64 k x 16 i
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int idx = tid + 256 * e;
      int ii, kk;
      if (a_rowmajor) { ii = idx % TBI; kk = idx / TBI; }
      else { kk = idx % TT; ii = idx / TT; }
      int64_t k = k0 + kk, i = i0 + ii;
      TC v = (TC)0;
      if (k < K && i < I) {
        if (A32) v = (TC)A32[k * I + i];   // FP32 operator converted once (k_ttm_a32)
        else v = (TC)(a_rowmajor ? A[k * lda + i] : A[k + lda * i]);
      }
      As[ii][kk] = v;
    }
    // Y tile: 16 i x 64 m
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int idx = tid + 256 * e;
      int ii, mm;
      TC v = (TC)0;
      if (L == 1) {
        ii = idx % TBI; mm = idx / TBI;
        int64_t i = i0 + ii, r = r0 + mm;
        if (i < I && r < Rt) v = (TC)ybase[i + I * r];
      } else {
        mm = idx % TT; ii = idx / TT;
        int64_t i = i0 + ii, l = l0 + mm;
        if (i < I && l < L) v = (TC)ybase[l + L * i];
      }
      Ys[ii][mm] = v;
    }
    __syncthreads();
#pragma unroll
    for (int ii = 0; ii < TBI; ++ii) {
      TC a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = As[ii][kq + 16 * u];
#pragma unroll
      for (int v = 0; v < 4; ++v) b[v] = Ys[ii][mq + 16 * v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
  // write Z: (k, m) -> l + L*(k + K*r)
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    int64_t k = k0 + kq + 16 * u;
    if (k >= K) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      int mm = mq + 16 * v;
      if (L == 1) {
        int64_t r = r0 + mm;
        if (r < Rt) {
          if (zt) z[r + Rt * k] = (TOut)acc[u][v];
          else z[k + K * r] = (TOut)acc[u][v];
        }
      } else {
        int64_t l = l0 + mm;
        if (l < L) z[l + L * (k + K * r0)] = (TOut)acc[u][v];
      }
    }
  }
}

// A (K x I, FP64, either layout) -> FP32 row-major K x I.  An FP64 -> FP32
// conversion runs on the FP64 pipe (64 cycles per warp instruction), so the
// FP32 TTM converts its operator once here instead of in every tile.
__global__ void k_ttm_a32(const double* __restrict__ A, int64_t K, int64_t I, int64_t lda,
                          int a_rowmajor, float* __restrict__ A32) {
  const int64_t n = K * I;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = e / I, i = e - k * I;
    A32[e] = (float)(a_rowmajor ? A[k * lda + i] : A[k + lda * i]);
  }
}

template <typename TIn, typename TOut>
static void ttm_dispatch_c(bool fp64, dim3 grid, cudaStream_t st, const void* y, int64_t L, int64_t I,
                           int64_t Rt, int64_t nLT, const double* A, int64_t K, int64_t lda,
                           int arow, const float* A32, void* z, int zt) {
  if (fp64)
    k_ttm_simt<TIn, TOut, double><<<grid, 256, 0, st>>>((const TIn*)y, L, I, Rt, nLT, A, K, lda, arow,
                                                        nullptr, (TOut*)z, zt);
  else
    k_ttm_simt<TIn, TOut, float><<<grid, 256, 0, st>>>((const TIn*)y, L, I, Rt, nLT, A, K, lda, arow,
                                                       A32, (TOut*)z, zt);
}

cudaError_t launch_ttm_simt(const void* y, tucker_dtype ydt, bool fp64, int64_t L, int64_t I,
                            int64_t Rt, const double* A, int64_t K, int64_t lda, int a_rowmajor,
                            float* a32_scratch, void* z, tucker_dtype zdt, cudaStream_t st,
                            bool zt) {
  if (zt && L != 1) return cudaErrorInvalidValue;
  int64_t nLT = 1, nMT;
  if (L == 1) nMT = (Rt + TT - 1) / TT;
  else { nLT = (L + TT - 1) / TT; nMT = Rt * nLT; }
  if (nMT <= 0 || K <= 0) return cudaSuccess;
  if (nMT > 0x7fffffffll) return cudaErrorInvalidConfiguration;
  dim3 grid((unsigned)nMT, (unsigned)((K + TT - 1) / TT));
  const float* A32 = nullptr;
  if (!fp64 && a32_scratch) {
    const int64_t n = K * I;
    k_ttm_a32<<<(unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024), 256, 0, st>>>(
        A, K, I, lda, a_rowmajor, a32_scratch);
    count_launches(1);
    A32 = a32_scratch;
  }
  count_launches(1);
  if (ydt == TUCKER_F64) {
    if (zdt == TUCKER_F64) ttm_dispatch_c<double, double>(fp64, grid, st, y, L, I, Rt, nLT, A, K, lda, a_rowmajor, A32, z, zt);
    else ttm_dispatch_c<double, float>(fp64, grid, st, y, L, I, Rt, nLT, A, K, lda, a_rowmajor, A32, z, zt);
  } else {
    if (zdt == TUCKER_F64) ttm_dispatch_c<float, double>(fp64, grid, st, y, L, I, Rt, nLT, A, K, lda, a_rowmajor, A32, z, zt);
    else ttm_dispatch_c<float, float>(fp64, grid, st, y, L, I, Rt, nLT, A, K, lda, a_rowmajor, A32, z, zt);
  }
  return cudaGetLastError();
}

}  // namespace tk
