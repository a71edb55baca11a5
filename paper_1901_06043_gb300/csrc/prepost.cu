// Pre- and post-processing of Section 3.5: statistics of every mode-n
// hyperslice (mean, standard deviation, maximum, minimum, 1-norm, 2-norm)
// and one linear function per hyperslice, y = (x - shift_i) * scale_i, or
// its inverse x = y / scale_i + shift_i after a reconstruction.
//
// Hyperslice i of mode n is every element (l, i, r) of the slab view
// (Rt, I, L): Rt runs of L contiguous elements, I L apart.  Two access
// regimes keep the loads coalesced:
//   rows  (L < 4096): the tensor is a column-major P x Rt matrix with
//         P = L I "virtual rows"; virtual row q belongs to hyperslice q / L.
//         A thread owns one virtual row and walks a range of columns; when
//         P < 256 a block covers 256 / P columns at a time, so consecutive
//         threads always read consecutive elements.
//   runs  (L >= 4096): work units are (hyperslice i, slab r, chunk of 4096 l)
//         in i-major order; a CTA takes a contiguous range of units, so it
//         sees one or two hyperslices.
//
// Arithmetic.  The FP64 pipe of this part runs at 1/64 of the FP32 rate, so
// FP32 data is reduced and transformed on the FP32 pipe with error-free
// transformations: each sum is an FP32 pair (hi, lo) grown by TwoSum (a new
// term may exceed the running sum, so never the cheaper Fast2Sum), squares are exact
// (TwoProduct by FMA).  Every 16 elements of a thread the pair is merged
// exactly into a second-level pair that is renormalised (|lo| <= ulp(hi) / 2,
// so its later roundings stay at 2^-48 of hi), and every 1024 elements that
// pair moves into FP64; the result is the FP64 sum to ~1e-14 of sum |x|.  The
// standard deviation takes a second pass over the data, sum (x - mean)^2 with
// the mean as an FP32 pair and x - mean_hi exact by TwoSum, which avoids the
// cancellation of sum x^2 - count mean^2.  The transform evaluates
// (x - shift) * scale (inverse: x * (1 / scale) + shift) in FP32-pair
// arithmetic and rounds once to FP32.  FP64 data is handled in FP64.
// Per-thread sums are combined per CTA, then added into per-hyperslice FP64
// accumulators with atomics (a few per CTA): exact to FP64 rounding, not
// bitwise reproducible from run to run.
#include "common.cuh"
#include "kernels.h"

namespace tk {
namespace {

constexpr int kThreads = 256;
constexpr int64_t kChunk = 4096;     // l per unit in the runs regime
constexpr int kAcc = 8;              // accumulators per hyperslice
constexpr int kGroup = 16;           // FP32 pairs merged into the second level
constexpr int kGroups = 64;          // second-level pairs moved into FP64
constexpr int64_t kRowsMaxL = 4096;  // rows regime below this run length

// Accumulator slots: 0 sum, 1 sum of squares, 2 sum |x|, 3 max (ordered
// bits), 4 min (ordered bits), 5 sum (x - mean)^2.
__device__ __forceinline__ long long ordered(double v) {
  const long long b = __double_as_longlong(v);
  return b ^ ((b >> 63) & 0x7fffffffffffffffll);
}
__device__ __forceinline__ double unordered(long long k) {
  return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffll));
}

// (h, l) += v exactly (TwoSum, any magnitudes); l collects the errors.
__device__ __forceinline__ void two_sum(float& h, float& l, float v) {
  const float s = __fadd_rn(h, v);
  const float bb = __fsub_rn(s, h);
  const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(v, bb));
  h = s;
  l = __fadd_rn(l, err);
}
// Per-thread partial sums of one hyperslice.  PASS 0: sum, sum of squares,
// sum |x|, max, min; PASS 1: sum (x - mean)^2.
template <typename T, int PASS> struct Part;

template <int PASS> struct Part<double, PASS> {
  double s, s2, sa, c2, mx, mn, mean;
  __device__ void init(double m) {
    s = s2 = sa = c2 = 0.0;
    mx = -INFINITY;
    mn = INFINITY;
    mean = m;
  }
  __device__ __forceinline__ void add(double v) {
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
  __device__ void flush() {}
};

template <int PASS> struct Part<float, PASS> {
  double s, s2, sa, c2, mx, mn;           // FP64 totals
  float sh, sl, qh, ql, ah, al;           // level 1: FP32 pairs of the current group
  float SH, SL, QH, QL, AH, AL;           // level 2: renormalised pairs of the groups
  float mh, ml;                           // the mean as an FP32 pair (PASS 1)
  float fmx, fmn;
  int n, g;
  __device__ void init(double m) {
    s = s2 = sa = c2 = 0.0;
    mx = -INFINITY;
    mn = INFINITY;
    sh = sl = qh = ql = ah = al = 0.f;
    SH = SL = QH = QL = AH = AL = 0.f;
    fmx = -INFINITY;
    fmn = INFINITY;
    mh = (float)m;
    ml = (float)(m - (double)mh);
    n = g = 0;
  }
  __device__ __forceinline__ void add(float v) {
    if (PASS == 0) {
      two_sum(sh, sl, v);
      const float p = __fmul_rn(v, v);
      const float pe = __fmaf_rn(v, v, -p);            // v^2 = p + pe exactly
      two_sum(qh, ql, p);
      ql = __fadd_rn(ql, pe);
      two_sum(ah, al, fabsf(v));
      fmx = fmaxf(fmx, v);
      fmn = fminf(fmn, v);
    } else {
      // d = v - mean = (s + e) - ml with s + e = v - mh exactly
      float s_ = v, e = 0.f;
      two_sum(s_, e, -mh);
      const float t = __fsub_rn(e, ml);
      const float p = __fmul_rn(s_, s_);
      const float pe = __fmaf_rn(s_, s_, -p);
      // d^2 = p + pe + t (2 s + t); |t| can be a sizeable part of |s| when
      // the slice varies little around its mean, so t^2 stays
      two_sum(qh, ql, p);
      ql = __fadd_rn(ql, __fmaf_rn(__fadd_rn(2.f * s_, t), t, pe));
    }
    if (++n == kGroup) merge();
  }
  // (H, L) += (h, l) exactly up to the rounding of L, then renormalised so
  // that |L| <= ulp(H) / 2 (its later roundings stay at 2^-48 of H)
  __device__ __forceinline__ static void merge_pair(float& H, float& L, float h, float l) {
    two_sum(H, L, h);
    L = __fadd_rn(L, l);
    float t = H, e = 0.f;                       // (t, e) = H + L exactly (TwoSum)
    two_sum(t, e, L);
    H = t;
    L = e;
  }
  // level 1 -> level 2 every kGroup elements; level 2 -> FP64 every
  // kGroups groups
  __device__ void merge() {
    if (PASS == 0) {
      merge_pair(SH, SL, sh, sl);
      merge_pair(QH, QL, qh, ql);
      merge_pair(AH, AL, ah, al);
      sh = sl = qh = ql = ah = al = 0.f;
    } else {
      merge_pair(QH, QL, qh, ql);
      qh = ql = 0.f;
    }
    n = 0;
    if (++g == kGroups) flush_groups();
  }
  __device__ void flush_groups() {
    if (PASS == 0) {
      s += (double)SH + (double)SL;
      s2 += (double)QH + (double)QL;
      sa += (double)AH + (double)AL;
      SH = SL = QH = QL = AH = AL = 0.f;
    } else {
      c2 += (double)QH + (double)QL;
      QH = QL = 0.f;
    }
    g = 0;
  }
  // everything into the FP64 totals (before a reduction)
  __device__ void flush() {
    merge();
    flush_groups();
    mx = fmax(mx, (double)fmx);
    mn = fmin(mn, (double)fmn);
    fmx = -INFINITY;
    fmn = INFINITY;
  }
};

template <typename T, int PASS>
__device__ void to_global(double* acc, int64_t i, const Part<T, PASS>& p) {
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

// Block reduction of the FP64 totals into thread 0 (all threads call it).
template <typename T, int PASS>
__device__ void block_reduce(Part<T, PASS>& p) {
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
}

// rows regime: grid (row blocks, column chunks).  P >= 256: thread = virtual
// row q, one column at a time; P < 256: the block covers C = 256 / P columns
// at a time (thread t: row t % P, column offset t / P).
template <typename T, int PASS>
__global__ void __launch_bounds__(kThreads) k_stats_rows(const T* __restrict__ x, int64_t L,
                                                          int64_t P, int64_t Rt, int ncol,
                                                          const double* __restrict__ mean,
                                                          double* __restrict__ acc) {
  const int C = P < kThreads ? (int)(kThreads / P) : 1;
  const int64_t q = P < kThreads ? threadIdx.x % P : (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const int c = P < kThreads ? (int)(threadIdx.x / P) : 0;
  if (q >= P || c >= C) return;
  const int64_t i = q / L;
  const int64_t r0 = Rt * blockIdx.y / ncol, r1 = Rt * (blockIdx.y + 1) / ncol;
  Part<T, PASS> p;
  p.init(PASS ? mean[i] : 0.0);
  const int64_t step = (int64_t)C * P;
  const T* ptr = x + q + P * (r0 + c);
  int64_t r = r0 + c;
  for (; r + 3 * C < r1; r += 4 * C, ptr += 4 * step) {   // four loads in flight
    const T a = __ldg(ptr), b = __ldg(ptr + step), d = __ldg(ptr + 2 * step),
            e = __ldg(ptr + 3 * step);
    p.add(a);
    p.add(b);
    p.add(d);
    p.add(e);
  }
  for (; r < r1; r += C, ptr += step) p.add(__ldg(ptr));
  p.flush();
  if (r1 > r0) to_global(acc, i, p);
}

// runs regime (L >= 4096): units (i, r, chunk) in i-major order, a
// contiguous range of units per CTA, walked without divisions.
template <typename T, int PASS>
__global__ void __launch_bounds__(kThreads) k_stats_runs(const T* __restrict__ x, int64_t L,
                                                          int64_t I, int64_t Rt,
                                                          const double* __restrict__ mean,
                                                          double* __restrict__ acc) {
  const int64_t nch = (L + kChunk - 1) / kChunk;
  const int64_t per_i = Rt * nch, units = I * per_i;
  const int64_t u0 = units * blockIdx.x / gridDim.x, u1 = units * (blockIdx.x + 1) / gridDim.x;
  if (u0 >= u1) return;
  int64_t cur = u0 / per_i, rest0 = u0 % per_i;
  int64_t i = cur, r = rest0 / nch, ch = rest0 % nch;
  Part<T, PASS> p;
  p.init(PASS ? mean[cur] : 0.0);
  for (int64_t u = u0; u < u1; ++u) {
    if (i != cur) {                       // uniform across the block
      p.flush();
      block_reduce(p);
      if (threadIdx.x == 0) to_global(acc, cur, p);
      cur = i;
      p.init(PASS ? mean[cur] : 0.0);
    }
    const int64_t l0 = ch * kChunk, l1 = min(L, l0 + kChunk);
    const T* run = x + L * (i + I * r);
    int64_t l = l0 + threadIdx.x;
    for (; l + 3 * kThreads < l1; l += 4 * kThreads) {
      const T a = __ldg(run + l), b = __ldg(run + l + kThreads),
              d = __ldg(run + l + 2 * kThreads), e = __ldg(run + l + 3 * kThreads);
      p.add(a);
      p.add(b);
      p.add(d);
      p.add(e);
    }
    for (; l < l1; l += kThreads) p.add(__ldg(run + l));
    if (++ch == nch) {
      ch = 0;
      if (++r == Rt) { r = 0; ++i; }
    }
  }
  p.flush();
  block_reduce(p);
  if (threadIdx.x == 0) to_global(acc, cur, p);
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
  if (!isfinite(a[0]) || !isfinite(a[1]) || !isfinite(a[5]) || !isfinite(mx) || !isfinite(mn))
    atomicOr(bad, 1u);
}

// ---- the linear map per hyperslice
// FP64 data: FP64.  FP32 data: shift and scale (or 1 / scale) as FP32 pairs,
// (x - shift) * scale or x * (1 / scale) + shift in pair arithmetic, one
// rounding to FP32 at the end.
template <typename T, bool INV> struct Map;

template <bool INV> struct Map<double, INV> {
  double sh, sc;
  __device__ Map(double shift, double scale) : sh(shift), sc(scale) {}
  __device__ __forceinline__ double operator()(double v) const {
    return INV ? v / sc + sh : (v - sh) * sc;
  }
};

template <bool INV> struct Map<float, INV> {
  float shh, shl, sch, scl;   // shift and scale (INV: 1 / scale) as FP32 pairs
  __device__ Map(double shift, double scale) {
    const double m = INV ? 1.0 / scale : scale;
    shh = (float)shift;
    shl = (float)(shift - (double)shh);
    sch = (float)m;
    scl = (float)(m - (double)sch);
  }
  __device__ __forceinline__ float operator()(float v) const {
    if (INV) {
      // v * m + shift: p + pe = v * sch exactly, then + v * scl, then the shift
      const float p = __fmul_rn(v, sch);
      const float pe = __fmaf_rn(v, sch, -p);
      const float t = __fmaf_rn(v, scl, pe);
      float s = p, e = 0.f;
      two_sum(s, e, shh);
      return __fadd_rn(s, __fadd_rn(e, __fadd_rn(t, shl)));
    }
    // (v - shift) * scale with v - shh = d + e exactly
    float d = v, e = 0.f;
    two_sum(d, e, -shh);
    const float dl = __fsub_rn(e, shl);
    const float p = __fmul_rn(d, sch);
    const float pe = __fmaf_rn(d, sch, -p);
    return __fadd_rn(p, __fmaf_rn(d, scl, __fmaf_rn(dl, sch, pe)));
  }
};

template <typename T, bool INV>
__global__ void __launch_bounds__(kThreads) k_apply_rows(const T* x, int64_t L, int64_t P,
                                                          int64_t Rt, int ncol,
                                                          const double* __restrict__ shift,
                                                          const double* __restrict__ scale, T* y) {
  const int C = P < kThreads ? (int)(kThreads / P) : 1;
  const int64_t q = P < kThreads ? threadIdx.x % P : (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const int c = P < kThreads ? (int)(threadIdx.x / P) : 0;
  if (q >= P || c >= C) return;
  const int64_t i = q / L;
  const Map<T, INV> f(shift[i], scale[i]);
  const int64_t r0 = Rt * blockIdx.y / ncol, r1 = Rt * (blockIdx.y + 1) / ncol;
  const int64_t step = (int64_t)C * P;
  int64_t r = r0 + c;
  int64_t o = q + P * r;
  for (; r + 3 * C < r1; r += 4 * C, o += 4 * step) {
    const T a = x[o], b = x[o + step], d = x[o + 2 * step], e = x[o + 3 * step];
    y[o] = f(a);
    y[o + step] = f(b);
    y[o + 2 * step] = f(d);
    y[o + 3 * step] = f(e);
  }
  for (; r < r1; r += C, o += step) y[o] = f(x[o]);
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
    const Map<T, INV> f(shift[i], scale[i]);
    const int64_t l0 = ch * kChunk, l1 = min(L, l0 + kChunk);
    const int64_t base = L * j;
    if (VEC) {
      for (int64_t l = l0 + (int64_t)threadIdx.x * V; l < l1; l += (int64_t)kThreads * V) {
        if constexpr (sizeof(T) == 4) {
          float4 v = *reinterpret_cast<const float4*>(x + base + l);
          v.x = f(v.x);
          v.y = f(v.y);
          v.z = f(v.z);
          v.w = f(v.w);
          *reinterpret_cast<float4*>(y + base + l) = v;
        } else {
          double2 v = *reinterpret_cast<const double2*>(x + base + l);
          v.x = f(v.x);
          v.y = f(v.y);
          *reinterpret_cast<double2*>(y + base + l) = v;
        }
      }
    } else {
      for (int64_t l = l0 + threadIdx.x; l < l1; l += kThreads) y[base + l] = f(x[base + l]);
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

// rows-regime grid: (row blocks, column chunks) about 8 CTAs per SM
void rows_grid(int64_t P, int64_t Rt, int num_sms, unsigned& gx, int& nc) {
  const int64_t rb = P < kThreads ? 1 : (P + kThreads - 1) / kThreads;
  int64_t c = ((int64_t)num_sms * 8 + rb - 1) / rb;
  if (c > Rt) c = Rt;
  if (c > 65535) c = 65535;
  gx = (unsigned)rb;
  nc = (int)(c < 1 ? 1 : c);
}

template <typename T, int PASS>
void stats_pass(const T* x, int64_t L, int64_t I, int64_t Rt, const double* mean, double* acc,
                int num_sms, cudaStream_t st) {
  if (L < kRowsMaxL) {
    const int64_t P = L * I;
    unsigned gx;
    int nc;
    rows_grid(P, Rt, num_sms, gx, nc);
    k_stats_rows<T, PASS><<<dim3(gx, (unsigned)nc), kThreads, 0, st>>>(x, L, P, Rt, nc, mean,
                                                                        acc);
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
  if (L < kRowsMaxL) {
    const int64_t P = L * I;
    unsigned gx;
    int nc;
    rows_grid(P, Rt, num_sms, gx, nc);
    k_apply_rows<T, INV><<<dim3(gx, (unsigned)nc), kThreads, 0, st>>>(x, L, P, Rt, nc, shift,
                                                                       scale, y);
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
