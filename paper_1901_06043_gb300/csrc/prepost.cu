// Pre- and post-processing of Section 3.5: statistics of every mode-n
// hyperslice (mean, standard deviation, maximum, minimum, 1-norm, 2-norm)
// and one linear function per hyperslice, y = (x - shift_i) * scale_i, or
// its inverse x = y / scale_i + shift_i after a reconstruction.
//
// Hyperslice i of mode n is every element (l, i, r) of the slab view
// (Rt, I, L): Rt runs of L contiguous elements, I L apart.  Two access
// regimes keep the loads coalesced:
//   rows  (L < 256): the tensor is a column-major P x Rt matrix with
//         P = L I "virtual rows"; virtual row q belongs to hyperslice q / L.
//         A thread owns one virtual row and walks a range of columns, so a
//         warp reads 32 consecutive elements per column.
//   runs  (L >= 256): work units are (hyperslice i, slab r, chunk of 4096 l)
//         in i-major order; a CTA takes a contiguous range of units, so it
//         sees one or two hyperslices and walks their runs with 16-byte
//         loads where alignment allows.
// Every element is read once per pass; sums are accumulated in FP64 per
// thread, then per CTA, then added into per-hyperslice FP64 accumulators
// with atomics (a few per CTA), so the sums are exact to FP64 rounding but
// not bitwise reproducible from run to run.  The standard deviation takes
// a second pass over the data, sum (x - mean_i)^2, which avoids the
// cancellation of sum x^2 - count mean^2.
#include "common.cuh"
#include "kernels.h"

namespace tk {
namespace {

constexpr int kThreads = 256;
constexpr int64_t kChunk = 4096;     // l per unit in the runs regime
constexpr int kAcc = 8;              // accumulators per hyperslice

// Accumulator slots: 0 sum, 1 sum of squares, 2 sum |x|, 3 max (ordered
// bits), 4 min (ordered bits), 5 sum (x - mean)^2.
__device__ __forceinline__ long long ordered(double v) {
  const long long b = __double_as_longlong(v);
  return b ^ ((b >> 63) & 0x7fffffffffffffffll);
}
__device__ __forceinline__ double unordered(long long k) {
  return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffll));
}

template <typename T>
__device__ __forceinline__ double ld(const T* p) {
  return (double)__ldg(p);
}

struct Part {
  double s, s2, sa, c2, mx, mn;
  __device__ void init() {
    s = s2 = sa = c2 = 0.0;
    mx = -INFINITY;
    mn = INFINITY;
  }
  template <int PASS>
  __device__ __forceinline__ void add(double v, double mean) {
    if (PASS == 0) {
      s += v;
      s2 = fma(v, v, s2);
      sa += fabs(v);
      mx = fmax(mx, v);
      mn = fmin(mn, v);
    } else {
      const double d = v - mean;
      c2 = fma(d, d, c2);
    }
  }
};

template <int PASS>
__device__ void flush(double* acc, int64_t i, const Part& p) {
  double* a = acc + i * kAcc;
  if (PASS == 0) {
    atomicAdd(a + 0, p.s);
    atomicAdd(a + 1, p.s2);
    atomicAdd(a + 2, p.sa);
    atomicMax(reinterpret_cast<long long*>(a + 3), ordered(p.mx));
    atomicMin(reinterpret_cast<long long*>(a + 4), ordered(p.mn));
  } else {
    atomicAdd(a + 5, p.c2);
  }
}

// Block reduction of a Part into thread 0 (all threads call it).
template <int PASS>
__device__ Part block_reduce(Part p) {
  __shared__ double sh[6][kThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    if (PASS == 0) {
      p.s += __shfl_xor_sync(0xffffffffu, p.s, o);
      p.s2 += __shfl_xor_sync(0xffffffffu, p.s2, o);
      p.sa += __shfl_xor_sync(0xffffffffu, p.sa, o);
      p.mx = fmax(p.mx, __shfl_xor_sync(0xffffffffu, p.mx, o));
      p.mn = fmin(p.mn, __shfl_xor_sync(0xffffffffu, p.mn, o));
    } else {
      p.c2 += __shfl_xor_sync(0xffffffffu, p.c2, o);
    }
  }
  __syncthreads();
  if (lane == 0) {
    sh[0][w] = p.s; sh[1][w] = p.s2; sh[2][w] = p.sa;
    sh[3][w] = p.mx; sh[4][w] = p.mn; sh[5][w] = p.c2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < kThreads / 32; ++k) {
      p.s += sh[0][k]; p.s2 += sh[1][k]; p.sa += sh[2][k];
      p.mx = fmax(p.mx, sh[3][k]); p.mn = fmin(p.mn, sh[4][k]); p.c2 += sh[5][k];
    }
  }
  return p;
}

// rows regime: grid (row blocks, column chunks); thread = virtual row q.
template <typename T, int PASS>
__global__ void __launch_bounds__(kThreads) k_stats_rows(const T* __restrict__ x, int64_t L,
                                                          int64_t P, int64_t Rt, int ncol,
                                                          const double* __restrict__ mean,
                                                          double* __restrict__ acc) {
  const int64_t q = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (q >= P) return;
  const int64_t i = q / L;
  const int64_t r0 = Rt * blockIdx.y / ncol, r1 = Rt * (blockIdx.y + 1) / ncol;
  const double m = PASS ? mean[i] : 0.0;
  Part p;
  p.init();
  const T* c = x + q + P * r0;
  int64_t r = r0;
  for (; r + 4 <= r1; r += 4, c += 4 * P) {     // four columns' loads in flight
    const double a = ld(c), b = ld(c + P), d = ld(c + 2 * P), e = ld(c + 3 * P);
    p.add<PASS>(a, m);
    p.add<PASS>(b, m);
    p.add<PASS>(d, m);
    p.add<PASS>(e, m);
  }
  for (; r < r1; ++r, c += P) p.add<PASS>(ld(c), m);
  if (r1 > r0) flush<PASS>(acc, i, p);
}

// runs regime (L >= 256): units (i, r, chunk) in i-major order, a contiguous
// range of units per CTA.
template <typename T, int PASS>
__global__ void __launch_bounds__(kThreads) k_stats_runs(const T* __restrict__ x, int64_t L,
                                                          int64_t I, int64_t Rt,
                                                          const double* __restrict__ mean,
                                                          double* __restrict__ acc) {
  const int64_t nch = (L + kChunk - 1) / kChunk;
  const int64_t per_i = Rt * nch, units = I * per_i;
  const int64_t u0 = units * blockIdx.x / gridDim.x, u1 = units * (blockIdx.x + 1) / gridDim.x;
  if (u0 >= u1) return;
  int64_t cur = u0 / per_i;
  Part p;
  p.init();
  double m = PASS ? mean[cur] : 0.0;
  for (int64_t u = u0; u < u1; ++u) {
    const int64_t i = u / per_i, rest = u % per_i;
    if (i != cur) {                       // uniform across the block
      Part t = block_reduce<PASS>(p);
      if (threadIdx.x == 0) flush<PASS>(acc, cur, t);
      p.init();
      cur = i;
      m = PASS ? mean[cur] : 0.0;
    }
    const int64_t r = rest / nch, ch = rest % nch;
    const int64_t l0 = ch * kChunk, l1 = min(L, l0 + kChunk);
    const T* run = x + L * (i + I * r);
    for (int64_t l = l0 + threadIdx.x; l < l1; l += kThreads) p.add<PASS>(ld(run + l), m);
  }
  Part t = block_reduce<PASS>(p);
  if (threadIdx.x == 0) flush<PASS>(acc, cur, t);
}

__global__ void k_stats_init(double* acc, int64_t I) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= I) return;
  double* a = acc + i * kAcc;
  a[0] = a[1] = a[2] = a[5] = 0.0;
  reinterpret_cast<long long*>(a)[3] = ordered(-INFINITY);
  reinterpret_cast<long long*>(a)[4] = ordered(INFINITY);
}

__global__ void k_stats_mean(double* acc, int64_t I, double count, double* mean) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < I) mean[i] = acc[i * kAcc] / count;
}

// stats[6 i + k]: mean, std, max, min, 1-norm, 2-norm; bad: any non-finite
__global__ void k_stats_final(const double* acc, const double* mean, int64_t I, double count,
                              double* stats, unsigned* bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= I) return;
  const double* a = acc + i * kAcc;
  const double mx = unordered(reinterpret_cast<const long long*>(a)[3]);
  const double mn = unordered(reinterpret_cast<const long long*>(a)[4]);
  double* s = stats + 6 * i;
  s[0] = mean[i];
  s[1] = sqrt(a[5] / count);
  s[2] = mx;
  s[3] = mn;
  s[4] = a[2];
  s[5] = sqrt(a[1]);
  if (!isfinite(a[1]) || !isfinite(a[5]) || !isfinite(mx) || !isfinite(mn)) atomicOr(bad, 1u);
}

// ---- the linear map per hyperslice
template <typename T, bool INV>
__device__ __forceinline__ T apply1(T v, double sh, double sc) {
  return INV ? (T)((double)v / sc + sh) : (T)(((double)v - sh) * sc);
}

template <typename T, bool INV>
__global__ void __launch_bounds__(kThreads) k_apply_rows(const T* x, int64_t L, int64_t P,
                                                          int64_t Rt, int ncol,
                                                          const double* __restrict__ shift,
                                                          const double* __restrict__ scale, T* y) {
  const int64_t q = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (q >= P) return;
  const int64_t i = q / L;
  const double sh = shift[i], sc = scale[i];
  const int64_t r0 = Rt * blockIdx.y / ncol, r1 = Rt * (blockIdx.y + 1) / ncol;
  int64_t r = r0;
  for (; r + 4 <= r1; r += 4) {
    const int64_t o = q + P * r;
    const T a = x[o], b = x[o + P], c = x[o + 2 * P], d = x[o + 3 * P];
    y[o] = apply1<T, INV>(a, sh, sc);
    y[o + P] = apply1<T, INV>(b, sh, sc);
    y[o + 2 * P] = apply1<T, INV>(c, sh, sc);
    y[o + 3 * P] = apply1<T, INV>(d, sh, sc);
  }
  for (; r < r1; ++r) y[q + P * r] = apply1<T, INV>(x[q + P * r], sh, sc);
}

// runs regime: a unit is (run j = i + I r, chunk); VEC: 16-byte accesses
// (L and both pointers aligned so that every run starts on 16 bytes)
template <typename T, bool INV, bool VEC>
__global__ void __launch_bounds__(kThreads) k_apply_runs(const T* x, int64_t L, int64_t I,
                                                          int64_t Rt,
                                                          const double* __restrict__ shift,
                                                          const double* __restrict__ scale, T* y) {
  constexpr int V = 16 / sizeof(T);
  const int64_t nch = (L + kChunk - 1) / kChunk;
  const int64_t units = I * Rt * nch;
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const int64_t j = u / nch, ch = u % nch;
    const int64_t i = j % I;
    const double sh = shift[i], sc = scale[i];
    const int64_t l0 = ch * kChunk, l1 = min(L, l0 + kChunk);
    const int64_t base = L * j;
    if (VEC) {
      for (int64_t l = l0 + (int64_t)threadIdx.x * V; l < l1; l += (int64_t)kThreads * V) {
        if constexpr (sizeof(T) == 4) {
          float4 v = *reinterpret_cast<const float4*>(x + base + l);
          v.x = (float)apply1<T, INV>((T)v.x, sh, sc);
          v.y = (float)apply1<T, INV>((T)v.y, sh, sc);
          v.z = (float)apply1<T, INV>((T)v.z, sh, sc);
          v.w = (float)apply1<T, INV>((T)v.w, sh, sc);
          *reinterpret_cast<float4*>(y + base + l) = v;
        } else {
          double2 v = *reinterpret_cast<const double2*>(x + base + l);
          v.x = (double)apply1<T, INV>((T)v.x, sh, sc);
          v.y = (double)apply1<T, INV>((T)v.y, sh, sc);
          *reinterpret_cast<double2*>(y + base + l) = v;
        }
      }
    } else {
      for (int64_t l = l0 + threadIdx.x; l < l1; l += kThreads)
        y[base + l] = apply1<T, INV>(x[base + l], sh, sc);
    }
  }
}

// derive (shift, scale) from the statistics: method 0 standardization
// (mean, 1 / std), 1 max rescaling (0, 1 / max |x|); a zero divisor keeps 1
__global__ void k_params(const double* stats, int64_t I, int method, double* shift,
                         double* scale) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= I) return;
  const double* s = stats + 6 * i;
  if (method == 0) {
    shift[i] = s[0];
    scale[i] = s[1] > 0.0 ? 1.0 / s[1] : 1.0;
  } else {
    const double m = fmax(fabs(s[2]), fabs(s[3]));
    shift[i] = 0.0;
    scale[i] = m > 0.0 ? 1.0 / m : 1.0;
  }
}

int col_chunks(int64_t rowblocks, int64_t Rt, int num_sms) {
  int64_t c = ((int64_t)num_sms * 8 + rowblocks - 1) / rowblocks;
  if (c > Rt) c = Rt;
  if (c > 65535) c = 65535;
  return (int)(c < 1 ? 1 : c);
}

template <typename T, int PASS>
void stats_pass(const T* x, int64_t L, int64_t I, int64_t Rt, const double* mean, double* acc,
                int num_sms, cudaStream_t st) {
  if (L < 256) {
    const int64_t P = L * I;
    const int64_t rb = (P + kThreads - 1) / kThreads;
    const int nc = col_chunks(rb, Rt, num_sms);
    k_stats_rows<T, PASS><<<dim3((unsigned)rb, (unsigned)nc), kThreads, 0, st>>>(x, L, P, Rt, nc,
                                                                                mean, acc);
  } else {
    const int64_t units = I * Rt * ((L + kChunk - 1) / kChunk);
    int64_t g = (int64_t)num_sms * 8;
    if (g > units) g = units;
    k_stats_runs<T, PASS><<<(unsigned)g, kThreads, 0, st>>>(x, L, I, Rt, mean, acc);
  }
}

template <typename T>
cudaError_t stats_t(const T* x, int64_t L, int64_t I, int64_t Rt, double* work, double* stats,
                    unsigned* bad, int num_sms, cudaStream_t st) {
  double* acc = work;
  double* mean = work + kAcc * I;
  const unsigned nb = (unsigned)((I + 255) / 256);
  const double count = (double)L * (double)Rt;
  k_stats_init<<<nb, 256, 0, st>>>(acc, I);
  stats_pass<T, 0>(x, L, I, Rt, nullptr, acc, num_sms, st);
  k_stats_mean<<<nb, 256, 0, st>>>(acc, I, count, mean);
  stats_pass<T, 1>(x, L, I, Rt, mean, acc, num_sms, st);
  k_stats_final<<<nb, 256, 0, st>>>(acc, mean, I, count, stats, bad);
  count_launches(5);
  return cudaGetLastError();
}

template <typename T, bool INV>
void apply_t(const T* x, int64_t L, int64_t I, int64_t Rt, const double* shift,
             const double* scale, T* y, int num_sms, cudaStream_t st) {
  if (L < 256) {
    const int64_t P = L * I;
    const int64_t rb = (P + kThreads - 1) / kThreads;
    const int nc = col_chunks(rb, Rt, num_sms);
    k_apply_rows<T, INV><<<dim3((unsigned)rb, (unsigned)nc), kThreads, 0, st>>>(x, L, P, Rt, nc,
                                                                               shift, scale, y);
    return;
  }
  const int64_t units = I * Rt * ((L + kChunk - 1) / kChunk);
  int64_t g = (int64_t)num_sms * 16;
  if (g > units) g = units;
  const bool vec = (L % (16 / (int64_t)sizeof(T))) == 0 && ((uintptr_t)x & 15) == 0 &&
                   ((uintptr_t)y & 15) == 0;
  if (vec)
    k_apply_runs<T, INV, true><<<(unsigned)g, kThreads, 0, st>>>(x, L, I, Rt, shift, scale, y);
  else
    k_apply_runs<T, INV, false><<<(unsigned)g, kThreads, 0, st>>>(x, L, I, Rt, shift, scale, y);
}

}  // namespace

size_t slice_stats_work_bytes(int64_t I) { return sizeof(double) * (size_t)(kAcc + 1) * I; }

cudaError_t launch_slice_stats(const void* x, tucker_dtype dt, int64_t L, int64_t I, int64_t Rt,
                               void* work, double* stats, unsigned* bad, int num_sms,
                               cudaStream_t st) {
  if (dt == TUCKER_F32)
    return stats_t((const float*)x, L, I, Rt, (double*)work, stats, bad, num_sms, st);
  return stats_t((const double*)x, L, I, Rt, (double*)work, stats, bad, num_sms, st);
}

cudaError_t launch_slice_params(const double* stats, int64_t I, int method, double* shift,
                                double* scale, cudaStream_t st) {
  k_params<<<(unsigned)((I + 255) / 256), 256, 0, st>>>(stats, I, method, shift, scale);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_slice_apply(const void* x, tucker_dtype dt, int64_t L, int64_t I, int64_t Rt,
                               const double* shift, const double* scale, int inverse, void* y,
                               int num_sms, cudaStream_t st) {
  if (dt == TUCKER_F32) {
    if (inverse)
      apply_t<float, true>((const float*)x, L, I, Rt, shift, scale, (float*)y, num_sms, st);
    else
      apply_t<float, false>((const float*)x, L, I, Rt, shift, scale, (float*)y, num_sms, st);
  } else {
    if (inverse)
      apply_t<double, true>((const double*)x, L, I, Rt, shift, scale, (double*)y, num_sms, st);
    else
      apply_t<double, false>((const double*)x, L, I, Rt, shift, scale, (double*)y, num_sms, st);
  }
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace tk
