// C ABI of the library: argument checks, workspace, and the host loop of
// ST-HOSVD (Algorithm 1 of the TuckerMPI paper) and of the multi-TTM
// reconstruction (Section 7).  Every arithmetic step runs in a device kernel.
#include <algorithm>
#include <array>
#include <map>
#include <mutex>
#include <set>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.h"

using namespace tk;

#include <atomic>
static std::atomic<unsigned long long> g_launches{0};
void tk::count_launches(int n) { g_launches.fetch_add((unsigned long long)n); }

cudaError_t tk::allow_max_dyn_smem(const void* f) {
  static std::mutex mu;
  static std::set<std::pair<int, const void*>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  if (done.count({dev, f})) return cudaSuccess;
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, f);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           optin - (int)fa.sharedSizeBytes);
  if (e != cudaSuccess) return e;
  done.insert({dev, f});
  return cudaSuccess;
}

struct tucker_ctx {
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  int timing = 0;
  int max_sweeps = 40;
  double tol_rel = 1e-15;
  double tol_abs = 1e-15;
  int eig_solver = 0;            // 0 auto, 1 Jacobi, 2 tridiagonal
  unsigned long long barrier_polls = 1ull << 24;   // grid-barrier poll limit of the eigensolvers
  double mem_limit = 0.0;        // bytes assumed available to a call (0: ask the device)
  int gram_digits = 0;           // digits of the exact-digit Gram: 0 auto, 2 or 3
  int autotune = 0;              // 1: split-K of the Gram kernels chosen by timing
  double host_chunk = 1073741824.0;   // bytes per piece of tucker_sthosvd_host's copy
  std::string err;
  // small device scratch
  unsigned* d_words = nullptr;   // 256 words
  double* d_small = nullptr;     // 64 doubles
  int* d_info = nullptr;         // 16 ints
  int64_t* d_i64 = nullptr;      // 16 int64
  // side streams for independent work of a batch (fork / join by events)
  static constexpr int kSide = 8;
  cudaStream_t side[kSide] = {};
  cudaEvent_t side_ev[kSide] = {};
  cudaEvent_t fork_ev = nullptr;
};

namespace {

constexpr size_t kWords = 256;

tucker_status set_err(tucker_ctx* c, tucker_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

tucker_status cuda_status(tucker_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return TUCKER_OK;
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return set_err(c, TUCKER_ERR_OOM, m);
  return set_err(c, TUCKER_ERR_CUDA, m);
}

#define TK_CUDA(ctx, expr)                                              \
  do {                                                                  \
    cudaError_t _e = (expr);                                            \
    if (_e != cudaSuccess) return cuda_status((ctx), _e, #expr);        \
  } while (0)

#define TK_TRY(expr)                                                    \
  do {                                                                  \
    tucker_status _s = (expr);                                          \
    if (_s != TUCKER_OK) return _s;                                     \
  } while (0)

// Stream-ordered device buffer, freed on the context stream.
struct DevBuf {
  void* p = nullptr;
  cudaStream_t st = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { reset(); }
  void reset() {
    if (p) cudaFreeAsync(p, st);
    p = nullptr;
  }
  void* release() { void* q = p; p = nullptr; return q; }
  template <typename T> T* as() const { return static_cast<T*>(p); }
};

tucker_status dev_alloc(tucker_ctx* c, DevBuf& b, size_t bytes) {
  b.reset();
  b.st = c->stream;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMallocAsync(&b.p, bytes, c->stream);
  if (e != cudaSuccess) {
    b.p = nullptr;
    cudaGetLastError();
    char m[128];
    snprintf(m, sizeof m, "device allocation of %zu bytes failed", bytes);
    return set_err(c, TUCKER_ERR_OOM, m);
  }
  return TUCKER_OK;
}

bool check_dims(int ndim, const int64_t* dims) {
  if (ndim < 1 || ndim > TUCKER_MAX_MODES || !dims) return false;
  for (int k = 0; k < ndim; ++k)
    if (dims[k] < 1) return false;
  return true;
}

int64_t numel(int ndim, const int64_t* dims) {
  int64_t n = 1;
  for (int k = 0; k < ndim; ++k) n *= dims[k];
  return n;
}

bool check_order(int ndim, const int* order, int* out) {
  bool seen[TUCKER_MAX_MODES] = {false};
  for (int k = 0; k < ndim; ++k) {
    int m = order ? order[k] : k;
    if (m < 0 || m >= ndim || seen[m]) return false;
    seen[m] = true;
    out[k] = m;
  }
  return true;
}

tucker_status sync(tucker_ctx* c) {
  TK_CUDA(c, cudaStreamSynchronize(c->stream));
  return TUCKER_OK;
}

// Side streams start after everything enqueued so far on the context stream
// (fork) and the context stream continues after all of them (join).  Work
// issued while c->stream is switched to a side stream keeps its scratch
// allocations stream-ordered on that side stream.
tucker_status fork_side(tucker_ctx* c) {
  TK_CUDA(c, cudaEventRecord(c->fork_ev, c->stream));
  for (int k = 0; k < tucker_ctx::kSide; ++k)
    TK_CUDA(c, cudaStreamWaitEvent(c->side[k], c->fork_ev, 0));
  return TUCKER_OK;
}
tucker_status join_side(tucker_ctx* c) {
  for (int k = 0; k < tucker_ctx::kSide; ++k) {
    TK_CUDA(c, cudaEventRecord(c->side_ev[k], c->side[k]));
    TK_CUDA(c, cudaStreamWaitEvent(c->stream, c->side_ev[k], 0));
  }
  return TUCKER_OK;
}
struct StreamSwap {
  tucker_ctx* c;
  cudaStream_t main;
  explicit StreamSwap(tucker_ctx* cc) : c(cc), main(cc->stream) {}
  void to(int k) { c->stream = c->side[k % tucker_ctx::kSide]; }
  ~StreamSwap() { c->stream = main; }
};

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  bool on = false;
  void start(tucker_ctx* c) {
    on = c->timing != 0;
    if (!on) return;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, c->stream);
  }
  void stop(tucker_ctx* c) {
    if (on) cudaEventRecord(b, c->stream);
  }
  float ms() {
    if (!on) return 0.f;
    float t = 0.f;
    cudaEventSynchronize(b);
    cudaEventElapsedTime(&t, a, b);
    return t;
  }
  ~Timer() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

// ---------------------------------------------------------------- steps

// rowmax != NULL: y is FP32 with a mode-0 size I0 (n = I0 * ncols) and the
// column-major pass also records the row maxima (for the digit scales of the
// exact tensor-core Gram) into rowmax[I0].
tucker_status do_norm(tucker_ctx* c, const void* y, tucker_dtype dt, int64_t n, double* out,
                      double* maxabs = nullptr, unsigned* rowmax = nullptr, int64_t I0 = 0) {
  // four blocks per SM: 7.73 ms for the 44 GB norm pass with row maxima,
  // against 7.93 ms with eight (each thread keeps eight loads in flight)
  int nb = (int)std::min<int64_t>((n + 255) / 256, (int64_t)c->num_sms * 4);
  if (nb < 1) nb = 1;
  DevBuf part;
  TK_TRY(dev_alloc(c, part, sizeof(double) * 2 * nb));
  TK_CUDA(c, cudaMemsetAsync(c->d_words, 0, sizeof(unsigned), c->stream));
  if (rowmax) {
    TK_CUDA(c, cudaMemsetAsync(rowmax, 0, sizeof(unsigned) * I0, c->stream));
    TK_CUDA(c, launch_sumsq_rowmax((const float*)y, I0, n / I0, part.as<double>(), nb, c->d_words,
                                   rowmax, c->d_small, c->stream));
  } else {
    TK_CUDA(c, launch_sumsq(y, dt, n, part.as<double>(), nb, c->d_words, c->d_small, c->stream));
  }
  double h[2] = {0.0, 0.0};
  unsigned bad = 0;
  TK_CUDA(c, cudaMemcpyAsync(h, c->d_small, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  TK_CUDA(c, cudaMemcpyAsync(&bad, c->d_words, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
  TK_TRY(sync(c));
  *out = h[0];
  if (maxabs) *maxabs = h[1];
  if (bad) return set_err(c, TUCKER_ERR_NONFINITE, "tensor holds NaN or Inf");
  return TUCKER_OK;
}

// Power-of-two scale with max|x| * scale <= 2^14 (FP16 split headroom).
float split_scale(double maxabs) {
  if (!(maxabs > 0.0) || !std::isfinite(maxabs)) return 1.0f;
  int ex = 0;
  std::frexp(maxabs, &ex);          // maxabs < 2^ex
  int e = 14 - ex;
  if (e > 100) e = 100;
  if (e < -100) e = -100;
  return std::ldexp(1.0f, e);
}

// Smallest eps^2 / N at which an eps-driven ST-HOSVD keeps an FP32-product
// Gram (see tucker_sthosvd).
constexpr double kMinFp32GramThreshold = 1e-9;

// Digits of the exact-digit Gram of an I x K view for the eps cut at
// threshold thr: 2 or 3, or 0 when neither is accurate enough (FP64 Gram).
// The Gram's only error is the representation of each value by its digits:
// |r_ik| <= delta_i = 2^(floor(log2 max_k |x_ik|) - 20) with three digits,
// 2^(... - 13) with two, independent of the digits (variance sigma_i^2 <=
// delta_i^2 / 3); the kernel subtracts each row's sum of r^2 from its
// diagonal entry, which leaves the small eigenvalues unbiased (r is x's own
// low part, so the digits' Gram carries + diag(sum r^2) and a relative
// O(sigma^2 / E[x^2]) shrink).  On the discarded subspace (projector P,
// tail <= thr at the cut) the error is then
//   2 sum_k (P x_k).r_k + sum_k sum_{i != j} P_ij r_ik r_jk,
// with variance at most 4 sigma_max^2 tail + 2 K sum_{i != j} P_ij^2
// sigma_i^2 sigma_j^2, and sum_j P_ij^2 = P_ii <= 1 bounds the second term by
// 2 K sigma_max^2 sum_i sigma_i^2.  A digit count is accepted when six
// standard deviations stay below 1 % of thr (the FP64 path's own margins at
// the cut are a few percent of thr on the benchmarked tensors); two digits
// are preferred, four products instead of nine.  With no threshold (ranks
// given) three digits.
double digit_gram_err6(const unsigned* rowmax_bits, int64_t I, int64_t K, double thr, int ndig) {
  double dmax = 0.0, dsum = 0.0;
  for (int64_t i = 0; i < I; ++i) {
    const unsigned b = rowmax_bits[i] & 0x7fffffffu;
    if (b == 0u) continue;
    float m;
    memcpy(&m, &b, sizeof m);
    int e = 0;
    std::frexp((double)m, &e);                      // m in [2^(e-1), 2^e)
    const double d = std::ldexp(1.0, e - (ndig == 3 ? 21 : 14));
    dmax = std::max(dmax, d);
    dsum += d * d;
  }
  const double s2max = dmax * dmax / 3.0, s2sum = dsum / 3.0;
  return 6.0 * std::sqrt(4.0 * s2max * thr + 2.0 * (double)K * s2max * s2sum);
}

int digit_gram_digits(const unsigned* rowmax_bits, int64_t I, int64_t K, double thr) {
  if (!(thr > 0.0)) return 3;
  if (digit_gram_err6(rowmax_bits, I, K, thr, 2) <= 0.01 * thr) return 2;
  if (digit_gram_err6(rowmax_bits, I, K, thr, 3) <= 0.01 * thr) return 3;
  return 0;
}

// Which kernel serves a Gram / TTM step: 0 SIMT FP64, 1 SIMT FP32, 2 tcgen05
// (rounded FP16 split products), 3 small-mode FP64 (I < 64, every
// precision), 4 FP32 with exact (compensated) block sums (row modes with few
// slabs), 5 tcgen05 on exact integer digit products (MIXED, I <= 4096;
// column-mode views from I = 64, row-mode views from 128), three digits;
// 6 the same with two digits.
int gram_kernel_for(tucker_prec prec, tucker_dtype dt, const SlabView& v, int sms) {
  if (plan_gram_small(v.L, v.I, v.Rt, sms, v.L0).nctas > 0) return 3;
  if (prec == TUCKER_PREC_FP64) return 0;
  if (prec == TUCKER_PREC_TENSOR && dt == TUCKER_F32 && plan_gram_tc(v.L, v.I, v.Rt, sms).ok) return 2;
  if (prec == TUCKER_PREC_MIXED && dt == TUCKER_F32 && plan_gram_tcx(v.L, v.I, v.Rt, sms).nctas > 0)
    return 5;
  return 1;
}

// Row maxima of the column-major mode-0 view (as FP32 bits) for the digit
// scales of the exact tensor-core Gram; own scratch, so it may run on a side
// stream.  Also gives the sum of squares, unused here.
tucker_status rowmax_pass(tucker_ctx* c, const float* y, int64_t I0, int64_t ncols,
                          unsigned* rowmax) {
  const int nb = c->num_sms * 4;
  DevBuf scr;
  TK_TRY(dev_alloc(c, scr, sizeof(double) * (2 * (size_t)nb + 2) + sizeof(unsigned)));
  double* part = scr.as<double>();
  double* out = part + 2 * nb;
  unsigned* bad = reinterpret_cast<unsigned*>(out + 2);
  TK_CUDA(c, cudaMemsetAsync(bad, 0, sizeof(unsigned), c->stream));
  TK_CUDA(c, cudaMemsetAsync(rowmax, 0, sizeof(unsigned) * I0, c->stream));
  TK_CUDA(c, launch_sumsq_rowmax(y, I0, ncols, part, nb, bad, rowmax, out, c->stream));
  return TUCKER_OK;
}

// Row maxima of any slab view for the digit Gram's scales: the column-major
// pass for column views, else one warp per (row, run of slabs).
tucker_status view_rowmax(tucker_ctx* c, const float* y, const SlabView& v, unsigned* rowmax) {
  if (v.L == 1 && v.I <= 8192) return rowmax_pass(c, y, v.I, v.Rt, rowmax);
  TK_CUDA(c, launch_rowmax_slab(y, v.L, v.I, v.Rt, c->num_sms, rowmax, c->stream));
  return TUCKER_OK;
}

// maxabs: max|y| if the caller knows it (e.g. from the norm pass), else <= 0.
// check = false: the tensor-core kernel's error word (d_words[8]) is neither
// cleared nor read here; the caller clears it before and reads it after a
// batch of calls.
// ndig: digits of the exact-digit Gram (2 or 3; TUCKER_OPT_GRAM_DIGITS
// overrides it).
// sms: the SM count the split-K planners size their one wave of CTAs for
// (the device's, or the autotuner's choice).
tucker_status gram_once(tucker_ctx* c, const void* y, tucker_dtype dt, const SlabView& v,
                        tucker_prec prec, double* S, int* kernel_used, double maxabs, bool check,
                        const unsigned* rowmax, int ndig, int kern, int sms) {
  if (kernel_used) *kernel_used = (kern == 5 && ndig == 2) ? 6 : kern;
  if (kern == 5) {
    const GramPlan p = plan_gram_tcx(v.L, v.I, v.Rt, sms);
    DevBuf scratch, rm;
    TK_TRY(dev_alloc(c, scratch, p.scratch_bytes));
    if (!rowmax) {
      TK_TRY(dev_alloc(c, rm, sizeof(unsigned) * v.I));
      TK_TRY(view_rowmax(c, (const float*)y, v, rm.as<unsigned>()));
      rowmax = rm.as<unsigned>();
    }
    if (check) TK_CUDA(c, cudaMemsetAsync(c->d_words + 8, 0, sizeof(unsigned), c->stream));
    TK_CUDA(c, launch_gram_tcx((const float*)y, v.L, v.I, v.Rt, p, rowmax, scratch.p,
                               c->d_words + 8, S, c->stream, ndig));
    if (!check) return TUCKER_OK;
    unsigned err = 0;
    TK_CUDA(c, cudaMemcpyAsync(&err, c->d_words + 8, sizeof(unsigned), cudaMemcpyDeviceToHost,
                               c->stream));
    TK_TRY(sync(c));
    if (err) {
      char m[96];
      snprintf(m, sizeof m, "tensor-core Gram reported device error word 0x%x", err);
      return set_err(c, TUCKER_ERR_CUDA, m);
    }
    return TUCKER_OK;
  }
  if (kern == 2) {
    if (!(maxabs > 0.0)) {
      double nrm;
      TK_TRY(do_norm(c, y, dt, v.L * v.I * v.Rt, &nrm, &maxabs));
    }
    TcGramPlan p = plan_gram_tc(v.L, v.I, v.Rt, c->num_sms);
    DevBuf scratch;
    TK_TRY(dev_alloc(c, scratch, p.scratch_bytes));
    if (check) TK_CUDA(c, cudaMemsetAsync(c->d_words + 8, 0, sizeof(unsigned), c->stream));
    TK_CUDA(c, launch_gram_tc((const float*)y, v.L, v.I, v.Rt, p, split_scale(maxabs),
                              scratch.as<double>(), c->d_words + 8, S, c->stream));
    if (!check) return TUCKER_OK;
    unsigned err = 0;
    TK_CUDA(c, cudaMemcpyAsync(&err, c->d_words + 8, sizeof(unsigned), cudaMemcpyDeviceToHost,
                               c->stream));
    TK_TRY(sync(c));
    if (err) {
      char m[96];
      snprintf(m, sizeof m, "tensor-core Gram reported device error word 0x%x", err);
      return set_err(c, TUCKER_ERR_CUDA, m);
    }
    return TUCKER_OK;
  }
  if (kern == 3) {
    const GramPlan ps = plan_gram_small(v.L, v.I, v.Rt, sms, v.L0);
    DevBuf scratch;
    TK_TRY(dev_alloc(c, scratch, ps.scratch_bytes));
    TK_CUDA(c, launch_gram_small(y, dt, v.L, v.I, v.Rt, v.L0, ps, scratch.as<double>(), S,
                                 c->stream));
    return TUCKER_OK;
  }
  if (kern == 1 && dt == TUCKER_F32) {
    const GramPlan pc = plan_gram_f32(v.L, v.I, v.Rt, sms, v.L0);
    if (pc.ntiles > 0) {
      if (kernel_used && gram_f32_compensated(v.L, v.Rt)) *kernel_used = 4;
      DevBuf scratch;
      TK_TRY(dev_alloc(c, scratch, pc.scratch_bytes));
      TK_CUDA(c, launch_gram_f32((const float*)y, v.L, v.I, v.Rt, v.L0, pc, scratch.as<double>(),
                                 S, c->stream));
      return TUCKER_OK;
    }
  }
  GramPlan p = plan_gram_simt(v.L, v.I, v.Rt, sms, v.L0);
  DevBuf scratch;
  TK_TRY(dev_alloc(c, scratch, p.scratch_bytes));
  TK_CUDA(c, launch_gram_simt(y, dt, kern == 0, v.L, v.I, v.Rt, v.L0, p, scratch.as<double>(), S,
                              c->stream));
  return TUCKER_OK;
}

// Per device, the event of the last host-to-device input copy that
// tucker_sthosvd_host issued (the calls chain their copies on it).
std::mutex g_h2d_mu;
std::map<int, cudaEvent_t> g_h2d_last;

// Process-wide cache of the split-K autotuner: for each (device, kernel,
// view shape, dtype, digits) the SM count whose one-wave plan ran fastest.
std::mutex g_tune_mu;
std::map<std::array<int64_t, 7>, int> g_tune;

// maxabs: max|y| if the caller knows it (e.g. from the norm pass), else <= 0.
// check = false: the tensor-core kernel's error word (d_words[8]) is neither
// cleared nor read here; the caller clears it before and reads it after a
// batch of calls.
// ndig: digits of the exact-digit Gram (2 or 3; TUCKER_OPT_GRAM_DIGITS
// overrides it).
// With TUCKER_OPT_AUTOTUNE the split-K planners size their wave for the SM
// count the autotuner chose for this kernel and view: on the first call of
// a (kernel, shape) the candidates 0.5, 1, 1.5 and 2 waves are each run twice
// on the context stream, timed by CUDA events, and the fastest is cached
// for the process (tile shapes are those of the kernels; only the K split
// is tuned).
tucker_status do_gram(tucker_ctx* c, const void* y, tucker_dtype dt, const SlabView& v,
                      tucker_prec prec, double* S, int* kernel_used, double maxabs = -1.0,
                      bool check = true, const unsigned* rowmax = nullptr, int ndig = 3) {
  int kern = gram_kernel_for(prec, dt, v, c->num_sms);
  if (kern == 2 && (((uintptr_t)y) & 15) != 0) kern = 1;
  if (kern == 5 && (((uintptr_t)y) & 3) != 0) kern = 1;
  if (c->gram_digits) ndig = c->gram_digits;
  if (!c->autotune || kern == 2)
    return gram_once(c, y, dt, v, prec, S, kernel_used, maxabs, check, rowmax, ndig, kern,
                     c->num_sms);
  const std::array<int64_t, 7> key{c->device, kern, v.L, v.I, v.Rt, (int64_t)dt,
                                   kern == 5 ? ndig : 0};
  int best = 0;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) best = it->second;
  }
  if (best == 0) {
    // the digit Gram's row maxima once, outside the timed runs
    DevBuf rm;
    if (kern == 5 && !rowmax) {
      TK_TRY(dev_alloc(c, rm, sizeof(unsigned) * v.I));
      TK_TRY(view_rowmax(c, (const float*)y, v, rm.as<unsigned>()));
      rowmax = rm.as<unsigned>();
    }
    cudaEvent_t e0, e1;
    TK_CUDA(c, cudaEventCreate(&e0));
    TK_CUDA(c, cudaEventCreate(&e1));
    float best_ms = 0.f;
    tucker_status st = TUCKER_OK;
    for (double f : {0.5, 1.0, 1.5, 2.0}) {
      const int sms = std::max(1, (int)std::lround(c->num_sms * f));
      for (int rep = 0; rep < 2 && st == TUCKER_OK; ++rep) {
        cudaEventRecord(e0, c->stream);
        st = gram_once(c, y, dt, v, prec, S, nullptr, maxabs, true, rowmax, ndig, kern, sms);
        cudaEventRecord(e1, c->stream);
        float ms = 0.f;
        if (st == TUCKER_OK && cudaEventSynchronize(e1) == cudaSuccess &&
            cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && (best == 0 || ms < best_ms)) {
          best = sms;
          best_ms = ms;
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    if (st != TUCKER_OK) return st;
    if (best == 0) best = c->num_sms;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = best;
  }
  return gram_once(c, y, dt, v, prec, S, kernel_used, maxabs, check, rowmax, ndig, kern, best);
}

// Device bytes of the split-K scratch do_gram allocates for a view.
size_t gram_scratch_bytes(const tucker_ctx* c, tucker_prec prec, tucker_dtype dt,
                          const SlabView& v) {
  const int kern = gram_kernel_for(prec, dt, v, c->num_sms);
  if (kern == 5) return plan_gram_tcx(v.L, v.I, v.Rt, c->num_sms).scratch_bytes + 8 * (size_t)v.I;
  if (kern == 2) return plan_gram_tc(v.L, v.I, v.Rt, c->num_sms).scratch_bytes;
  if (kern == 3) return plan_gram_small(v.L, v.I, v.Rt, c->num_sms, v.L0).scratch_bytes;
  if (kern == 1 && dt == TUCKER_F32) {
    const GramPlan pc = plan_gram_f32(v.L, v.I, v.Rt, c->num_sms, v.L0);
    if (pc.ntiles > 0) return pc.scratch_bytes;
  }
  return plan_gram_simt(v.L, v.I, v.Rt, c->num_sms, v.L0).scratch_bytes;
}

// Bytes a call may still allocate: with TUCKER_OPT_MEM_LIMIT set, that
// figure less what the call already holds; otherwise the device's free
// memory plus what the default memory pool has reserved and not handed out.
double mem_available(tucker_ctx* c, double held) {
  if (c->mem_limit > 0.0) return c->mem_limit - held;
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    return std::numeric_limits<double>::infinity();
  }
  double avail = (double)fr;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, c->device) == cudaSuccess) {
    uint64_t reserved = 0, used = 0;
    if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) ==
            cudaSuccess &&
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) == cudaSuccess &&
        reserved > used)
      avail += (double)(reserved - used);
  }
  cudaGetLastError();
  return avail;
}

tucker_status predict_oom(tucker_ctx* c, double need, double held, const char* what) {
  const double avail = mem_available(c, held);
  if (need <= avail) return TUCKER_OK;
  char m[192];
  snprintf(m, sizeof m, "predicted out of memory before %s: %.0f bytes needed, %.0f available",
           what, need, avail > 0.0 ? avail : 0.0);
  return set_err(c, TUCKER_ERR_OOM, m);
}

tucker_status do_eig(tucker_ctx* c, const double* S, int n, double* w, double* V, int* sweeps) {
  DevBuf work;
  TK_TRY(dev_alloc(c, work, jacobi_work_bytes(n)));
  // ||S||_F^2 for the absolute part of the Jacobi threshold
  int nb = (int)std::min<int64_t>(((int64_t)n * n + 255) / 256, 1024);
  DevBuf part;
  TK_TRY(dev_alloc(c, part, sizeof(double) * 2 * std::max(nb, 1)));
  TK_CUDA(c, launch_sumsq(S, TUCKER_F64, (int64_t)n * n, part.as<double>(), std::max(nb, 1),
                          c->d_words + 16, c->d_small + 8, c->stream));
  int ms = c->max_sweeps;
  if (ms > 200) ms = 200;
  TK_CUDA(c, launch_jacobi(S, n, work.as<double>(), c->d_small + 8, c->d_words + 32, ms,
                           c->tol_rel, c->tol_abs, c->num_sms, w, V, c->d_info, c->stream,
                           c->barrier_polls));
  int info[4] = {0, 0, 0, -1};
  unsigned words[3] = {0, 0, 0};
  TK_CUDA(c, cudaMemcpyAsync(info, c->d_info, sizeof(info), cudaMemcpyDeviceToHost, c->stream));
  TK_CUDA(c, cudaMemcpyAsync(words, c->d_words + 32, sizeof(words), cudaMemcpyDeviceToHost,
                             c->stream));
  TK_TRY(sync(c));
  if (words[2] & DEV_ERR_BARRIER_TIMEOUT)
    return set_err(c, TUCKER_ERR_CUDA, "Jacobi grid barrier gave up waiting");
  if (ms == 0) { info[2] = 0; info[3] = (n & 1) ? n : -1; }
  TK_CUDA(c, launch_eig_finish(n, work.as<double>(), info, c->d_info, w, V, c->stream));
  TK_TRY(sync(c));
  if (sweeps) *sweeps = info[0];
  if (!info[1] && ms > 0)
    return set_err(c, TUCKER_ERR_EIG_NOCONV, "Jacobi reached the sweep cap without converging");
  if (ms == 0) return set_err(c, TUCKER_ERR_EIG_NOCONV, "Jacobi sweep cap is 0");
  return TUCKER_OK;
}

// Whether the truncated eigensolve of an n x n Gram takes the tridiagonal
// solver: every n up to the size whose three work vectors fit in shared
// memory (measured faster than the Jacobi sweeps at every size: 0.23 vs
// 0.29 ms at n = 8, 0.30 vs 0.46 at n = 11, 0.80 vs 3.45 at n = 50).
bool use_tridiag(const tucker_ctx* c, int n) {
  if (c->eig_solver == 1) return false;
  return n >= 1 && n <= 4096;
}

// All eigenvalues (descending, into w) and the leading R eigenvectors of S by
// the tridiagonal solver (tridiag.cu); R from the cut at thr, or fixed_R > 0.
// U is allocated here (I x R, column-major).  *failed: the Cholesky QR
// rejected the inverse-iteration vectors (the caller then takes Jacobi); w,
// R and the discarded sum are valid either way.
tucker_status do_eig_tri(tucker_ctx* c, const double* S, int n, double thr, int fixed_R,
                         double* w, DevBuf& U, int64_t* R_out, double* disc, bool* failed) {
  const int G = tridiag_team_size(n, c->num_sms);
  const size_t nn = (size_t)n * n;
  const size_t nwy = eig_wy_doubles(n);
  const size_t ndbl = nn + 3 * (size_t)n + 4 * (size_t)n + 2 * (size_t)G + (size_t)n + 1 + nwy;
  DevBuf work;
  TK_TRY(dev_alloc(c, work, sizeof(double) * ndbl + sizeof(EigProblem) + 16));
  EigProblem h{};
  h.A = work.as<double>();
  h.d = h.A + nn;
  h.e = h.d + n;
  h.tau = h.e + n;
  h.xch = h.tau + n;
  double* tail = h.xch + 4 * (size_t)n + 2 * (size_t)G;
  h.wyT = tail + n + 1;
  EigProblem* pd = reinterpret_cast<EigProblem*>(h.wyT + nwy);
  int* info = reinterpret_cast<int*>(pd + 1);
  h.w = w;
  h.info = info;
  h.n = n;
  h.team_off = 0;
  h.team_size = G;
  cudaStream_t st = c->stream;
  TK_CUDA(c, cudaMemcpyAsync(h.A, S, sizeof(double) * nn, cudaMemcpyDeviceToDevice, st));
  TK_CUDA(c, cudaMemsetAsync(c->d_words + 32, 0, sizeof(unsigned) * 3, st));
  TK_CUDA(c, cudaMemsetAsync(info, 0, sizeof(int), st));
  TK_CUDA(c, launch_tridiag(pd, &h, 1, c->d_words + 32, c->d_words + 34, st, c->barrier_polls));
  TK_CUDA(c, launch_bisect(pd, 1, n, n, c->num_sms, st));
  TK_CUDA(c, launch_rank_cut(w, n, thr, fixed_R, c->d_i64, c->d_small + 2, tail, st));
  int64_t R = 0;
  unsigned werr = 0;
  TK_CUDA(c, cudaMemcpyAsync(&R, c->d_i64, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  TK_CUDA(c, cudaMemcpyAsync(disc, c->d_small + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
  TK_CUDA(c, cudaMemcpyAsync(&werr, c->d_words + 34, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  TK_TRY(sync(c));
  if (werr & DEV_ERR_BARRIER_TIMEOUT)
    return set_err(c, TUCKER_ERR_CUDA, "tridiagonalization grid barrier gave up waiting");
  if (R < 1 || R > n) return set_err(c, TUCKER_ERR_CUDA, "rank cut returned an invalid rank");
  *R_out = R;
  const int Ri = (int)R;
  TK_TRY(dev_alloc(c, U, sizeof(double) * (size_t)n * Ri));
  DevBuf vec;
  const size_t zb = sizeof(double) * (size_t)n * Ri, gb = sizeof(double) * (size_t)Ri * Ri;
  TK_TRY(dev_alloc(c, vec, zb + gb + eig_lu_bytes(n, Ri)));
  h.z = vec.as<double>();
  h.gram = h.z + (size_t)n * Ri;
  h.lu = h.gram + (size_t)Ri * Ri;
  h.U = U.as<double>();
  h.R = Ri;
  h.zoff = 0;
  h.roff = 0;
  TK_CUDA(c, cudaMemcpyAsync(pd, &h, sizeof(h), cudaMemcpyHostToDevice, st));
  TK_CUDA(c, launch_invit(pd, 1, Ri, st));
  // Cholesky QR, twice (the second pass restores orthogonality to rounding
  // when eigenvalues are clustered and the vectors are far from orthogonal).
  // Z^T Z is the Gram of the column-major view of Z (L = 1, I = R, Rt = n).
  const SlabView zv{1, (int64_t)Ri, (int64_t)n, 1};
  for (int pass = 0; pass < 2; ++pass) {
    TK_TRY(do_gram(c, h.z, TUCKER_F64, zv, TUCKER_PREC_FP64, h.gram, nullptr));
    TK_CUDA(c, launch_chol(pd, 1, st));
    TK_CUDA(c, launch_trsm_rows(pd, 1, n, st));
  }
  TK_CUDA(c, launch_backtransform(pd, 1, Ri, n, st));
  int hinfo = 0;
  TK_CUDA(c, cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, st));
  TK_TRY(sync(c));
  *failed = hinfo != 0;
  return TUCKER_OK;
}

tucker_status do_cut(tucker_ctx* c, const double* w, int n, double thr, int fixed_R, int64_t* R,
                     double* disc) {
  DevBuf tail;
  TK_TRY(dev_alloc(c, tail, sizeof(double) * (n + 1)));
  TK_CUDA(c, launch_rank_cut(w, n, thr, fixed_R, c->d_i64, c->d_small + 2, tail.as<double>(),
                             c->stream));
  TK_CUDA(c, cudaMemcpyAsync(R, c->d_i64, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
  TK_CUDA(c, cudaMemcpyAsync(disc, c->d_small + 2, sizeof(double), cudaMemcpyDeviceToHost,
                             c->stream));
  return sync(c);
}

// ymax: max|y| if the caller knows it (e.g. from the norm pass), else <= 0.
// check = false: as do_gram, for the tensor-core TTM's error word (d_words[9]).
// zt (column-mode views): Z written transposed, slab fastest (the new mode
// becomes the slowest index).
tucker_status do_ttm(tucker_ctx* c, const void* y, tucker_dtype ydt, const SlabView& v,
                     const double* A, int64_t K, int64_t lda, int arow, tucker_prec prec, void* z,
                     tucker_dtype zdt, int* kernel_used, double ymax = -1.0, bool check = true,
                     bool zt = false) {
  // (the split scale needs max|y|: without it and without host syncs, SIMT)
  const bool tc = (prec == TUCKER_PREC_MIXED || prec == TUCKER_PREC_TENSOR) && ydt == TUCKER_F32 &&
                  zdt == TUCKER_F32 && (((uintptr_t)y) & 15) == 0 && (check || ymax >= 0.0) &&
                  (!zt || (((uintptr_t)z) & 15) == 0) && ttm_tc_supported(v.L, v.I, v.Rt, K);
  if (kernel_used) *kernel_used = tc ? 2 : (prec == TUCKER_PREC_FP64 ? 0 : 1);
  if (tc) {
    if (!(ymax >= 0.0)) {
      double nrm;
      TK_TRY(do_norm(c, y, ydt, v.L * v.I * v.Rt, &nrm, &ymax));
    }
    DevBuf scratch;
    TK_TRY(dev_alloc(c, scratch, ttm_tc_scratch_bytes(v.I, K)));
    if (check) TK_CUDA(c, cudaMemsetAsync(c->d_words + 9, 0, sizeof(unsigned), c->stream));
    TK_CUDA(c, launch_ttm_tc((const float*)y, v.L, v.I, v.Rt, A, K, lda, arow, split_scale(ymax),
                             (float*)z, zt, scratch.p, c->d_words + 9, c->num_sms, c->stream));
    if (!check) return TUCKER_OK;
    unsigned err = 0;
    TK_CUDA(c, cudaMemcpyAsync(&err, c->d_words + 9, sizeof(unsigned), cudaMemcpyDeviceToHost,
                               c->stream));
    TK_TRY(sync(c));
    if (err) {
      char m[96];
      snprintf(m, sizeof m, "tensor-core TTM reported device error word 0x%x", err);
      return set_err(c, TUCKER_ERR_CUDA, m);
    }
    return TUCKER_OK;
  }
  // row-mode views with a short contraction (I <= 64: the reconstruction's
  // expansions) on the tensor cores, l as the MMA's M.  Its split scale needs
  // max|y|: a caller that runs without host syncs (check = false, the batched
  // path on side streams) and does not know it keeps the SIMT TTM rather than
  // pay a synchronizing norm pass.
  const bool tc_row = !zt && (check || ymax >= 0.0) &&
                      (prec == TUCKER_PREC_MIXED || prec == TUCKER_PREC_TENSOR) &&
                      ydt == TUCKER_F32 && zdt == TUCKER_F32 && (((uintptr_t)y) & 15) == 0 &&
                      ttm_tc_row_supported(v.L, v.I, v.Rt, K);
  if (tc_row) {
    if (kernel_used) *kernel_used = 2;
    if (!(ymax >= 0.0)) {
      double nrm;
      TK_TRY(do_norm(c, y, ydt, v.L * v.I * v.Rt, &nrm, &ymax));
    }
    DevBuf scratch;
    TK_TRY(dev_alloc(c, scratch, ttm_tc_row_scratch_bytes(K)));
    if (check) TK_CUDA(c, cudaMemsetAsync(c->d_words + 9, 0, sizeof(unsigned), c->stream));
    TK_CUDA(c, launch_ttm_tc_row((const float*)y, v.L, v.I, v.Rt, A, K, lda, arow,
                                 split_scale(ymax), (float*)z, scratch.p, c->d_words + 9,
                                 c->num_sms, c->stream));
    if (!check) return TUCKER_OK;
    unsigned err = 0;
    TK_CUDA(c, cudaMemcpyAsync(&err, c->d_words + 9, sizeof(unsigned), cudaMemcpyDeviceToHost,
                               c->stream));
    TK_TRY(sync(c));
    if (err) {
      char m[96];
      snprintf(m, sizeof m, "tensor-core TTM reported device error word 0x%x", err);
      return set_err(c, TUCKER_ERR_CUDA, m);
    }
    return TUCKER_OK;
  }
  // the FP32 copy of the operator pays off once the TTM spans several waves
  DevBuf a32;
  if (prec != TUCKER_PREC_FP64 && (double)v.L * (double)v.Rt * (double)K >= 16777216.0)
    TK_TRY(dev_alloc(c, a32, sizeof(float) * (size_t)K * v.I));
  TK_CUDA(c, launch_ttm_simt(y, ydt, prec == TUCKER_PREC_FP64, v.L, v.I, v.Rt, A, K, lda, arow,
                             a32.as<float>(), z, zdt, c->stream, zt));
  return TUCKER_OK;
}

void order_search(int N, const int64_t* R, const int64_t* K, int objective, int* out) {
  std::vector<int> perm(N);
  for (int k = 0; k < N; ++k) perm[k] = k;
  bool first = true;
  long double best = 0;
  do {
    int64_t cur[TUCKER_MAX_MODES];
    for (int k = 0; k < N; ++k) cur[k] = R[k];
    long double cost = 0, prev = 1;
    for (int k = 0; k < N; ++k) prev *= (long double)cur[k];
    long double peak = 0;
    for (int s = 0; s < N; ++s) {
      int n = perm[s];
      long double sz = 1;
      for (int k = 0; k < N; ++k) sz *= (long double)cur[k];
      cost += sz * (long double)K[n];
      cur[n] = K[n];
      long double nsz = 1;
      for (int k = 0; k < N; ++k) nsz *= (long double)cur[k];
      peak = std::max(peak, sz + nsz);
    }
    long double obj = objective == 0 ? cost : peak;
    if (first || obj < best) {
      best = obj;
      first = false;
      for (int k = 0; k < N; ++k) out[k] = perm[k];
    }
  } while (std::next_permutation(perm.begin(), perm.end()));
}

}  // namespace

extern "C" {

tucker_status tucker_create(tucker_ctx** out, void* stream) {
  if (!out) return TUCKER_ERR_INVALID;
  *out = nullptr;
  tucker_ctx* c = new tucker_ctx();
  c->stream = (cudaStream_t)stream;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e == cudaSuccess) {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, c->device) == cudaSuccess) {
      uint64_t thr = std::numeric_limits<uint64_t>::max();
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    e = cudaMalloc(&c->d_words, sizeof(unsigned) * kWords);
  }
  if (e == cudaSuccess) e = cudaMalloc(&c->d_small, sizeof(double) * 64);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_info, sizeof(int) * 16);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_i64, sizeof(int64_t) * 16);
  for (int k = 0; k < tucker_ctx::kSide && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&c->side[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->side_ev[k], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaFree(c->d_words); cudaFree(c->d_small); cudaFree(c->d_info); cudaFree(c->d_i64);
    for (int k = 0; k < tucker_ctx::kSide; ++k) {
      if (c->side[k]) cudaStreamDestroy(c->side[k]);
      if (c->side_ev[k]) cudaEventDestroy(c->side_ev[k]);
    }
    if (c->fork_ev) cudaEventDestroy(c->fork_ev);
    delete c;
    return e == cudaErrorMemoryAllocation ? TUCKER_ERR_OOM : TUCKER_ERR_CUDA;
  }
  *out = c;
  return TUCKER_OK;
}

tucker_status tucker_destroy(tucker_ctx* c) {
  if (!c) return TUCKER_ERR_INVALID;
  cudaStreamSynchronize(c->stream);
  cudaFree(c->d_words);
  cudaFree(c->d_small);
  cudaFree(c->d_info);
  cudaFree(c->d_i64);
  for (int k = 0; k < tucker_ctx::kSide; ++k) {
    cudaStreamSynchronize(c->side[k]);
    cudaStreamDestroy(c->side[k]);
    cudaEventDestroy(c->side_ev[k]);
  }
  cudaEventDestroy(c->fork_ev);
  delete c;
  return TUCKER_OK;
}

const char* tucker_last_error(const tucker_ctx* c) { return c ? c->err.c_str() : "null context"; }

uint64_t tucker_kernel_launches(void) { return g_launches.load(); }

int64_t tucker_autotune_entries(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return (int64_t)g_tune.size();
}

tucker_status tucker_set_option(tucker_ctx* c, int key, double value) {
  if (!c) return TUCKER_ERR_INVALID;
  switch (key) {
    case TUCKER_OPT_TIMING: c->timing = value != 0.0; return TUCKER_OK;
    case TUCKER_OPT_MAX_SWEEPS:
      if (value < 0 || value > 200) return set_err(c, TUCKER_ERR_INVALID, "sweep cap out of [0, 200]");
      c->max_sweeps = (int)value;
      return TUCKER_OK;
    case TUCKER_OPT_EIG_SOLVER:
      if (value != 0.0 && value != 1.0 && value != 2.0)
        return set_err(c, TUCKER_ERR_INVALID, "eigensolver must be 0 (auto), 1 or 2");
      c->eig_solver = (int)value;
      return TUCKER_OK;
    case TUCKER_OPT_AUTOTUNE:
      if (value != 0.0 && value != 1.0) return set_err(c, TUCKER_ERR_INVALID, "autotune must be 0 or 1");
      c->autotune = (int)value;
      return TUCKER_OK;
    case TUCKER_OPT_GRAM_DIGITS:
      if (value != 0.0 && value != 2.0 && value != 3.0)
        return set_err(c, TUCKER_ERR_INVALID, "Gram digits must be 0 (auto), 2 or 3");
      c->gram_digits = (int)value;
      return TUCKER_OK;
    case TUCKER_OPT_BARRIER_POLLS:
      if (!(value >= 1.0 && value <= 1099511627776.0))
        return set_err(c, TUCKER_ERR_INVALID, "barrier poll limit out of [1, 2^40]");
      c->barrier_polls = (unsigned long long)value;
      return TUCKER_OK;
    case TUCKER_OPT_MEM_LIMIT:
      if (!(value >= 0.0 && std::isfinite(value)))
        return set_err(c, TUCKER_ERR_INVALID, "memory limit must be >= 0");
      c->mem_limit = value;
      return TUCKER_OK;
    case TUCKER_OPT_HOST_CHUNK:
      if (!(value >= 1.0 && std::isfinite(value)))
        return set_err(c, TUCKER_ERR_INVALID, "host piece size must be >= 1 byte");
      c->host_chunk = value;
      return TUCKER_OK;
    case TUCKER_OPT_JACOBI_TOL:
      if (!(value > 0.0 && value < 1e-3)) return set_err(c, TUCKER_ERR_INVALID, "tolerance out of (0, 1e-3)");
      c->tol_rel = value;
      return TUCKER_OK;
    default: return set_err(c, TUCKER_ERR_INVALID, "unknown option");
  }
}

tucker_status tucker_norm_sq(tucker_ctx* c, const void* y, tucker_dtype dt, int64_t count,
                             double* out) {
  if (!c) return TUCKER_ERR_INVALID;
  if (!y || !out || count < 0 || (dt != TUCKER_F32 && dt != TUCKER_F64))
    return set_err(c, TUCKER_ERR_INVALID, "tucker_norm_sq: bad argument");
  if (count == 0) { *out = 0.0; return TUCKER_OK; }
  return do_norm(c, y, dt, count, out);
}

tucker_status tucker_gram(tucker_ctx* c, const void* y, tucker_dtype dt, int ndim,
                          const int64_t* dims, int mode, tucker_prec prec, double* S) {
  if (!c) return TUCKER_ERR_INVALID;
  if (!y || !S || !check_dims(ndim, dims) || mode < 0 || mode >= ndim ||
      (dt != TUCKER_F32 && dt != TUCKER_F64) || prec < 0 || prec > 3)
    return set_err(c, TUCKER_ERR_INVALID, "tucker_gram: bad argument");
  if ((prec == TUCKER_PREC_MIXED || prec == TUCKER_PREC_TENSOR) && dt != TUCKER_F32)
    return set_err(c, TUCKER_ERR_UNSUPPORTED, "MIXED/TENSOR precision needs FP32 input");
  SlabView v = slab_view(ndim, dims, mode);
  TK_TRY(do_gram(c, y, dt, v, prec, S, nullptr));
  return sync(c);
}

tucker_status tucker_eig(tucker_ctx* c, const double* S, int64_t I, double* w, double* V,
                         int* sweeps) {
  if (!c) return TUCKER_ERR_INVALID;
  if (!S || !w || !V || I < 1 || I > 8192)
    return set_err(c, TUCKER_ERR_INVALID, "tucker_eig: bad argument");
  return do_eig(c, S, (int)I, w, V, sweeps);
}

tucker_status tucker_eig_trunc(tucker_ctx* c, const double* S, int64_t I, double thr,
                               int64_t fixed_R, double* w, double* U, int64_t* R, double* disc) {
  if (!c) return TUCKER_ERR_INVALID;
  if (!S || !w || !U || !R || !disc || I < 1 || I > 8192 || !(thr >= 0.0) || fixed_R < 0 ||
      fixed_R > I)
    return set_err(c, TUCKER_ERR_INVALID, "tucker_eig_trunc: bad argument");
  const int n = (int)I;
  if (use_tridiag(c, n)) {
    DevBuf Ub;
    bool failed = false;
    TK_TRY(do_eig_tri(c, S, n, thr, (int)fixed_R, w, Ub, R, disc, &failed));
    if (!failed) {
      TK_CUDA(c, cudaMemcpyAsync(U, Ub.p, sizeof(double) * n * (*R), cudaMemcpyDeviceToDevice,
                                 c->stream));
      return sync(c);
    }
  }
  DevBuf V;
  TK_TRY(dev_alloc(c, V, sizeof(double) * (size_t)n * n));
  tucker_status es = do_eig(c, S, n, w, V.as<double>(), nullptr);
  if (es != TUCKER_OK && es != TUCKER_ERR_EIG_NOCONV) return es;
  TK_TRY(do_cut(c, w, n, thr, (int)fixed_R, R, disc));
  TK_CUDA(c, cudaMemcpyAsync(U, V.p, sizeof(double) * n * (*R), cudaMemcpyDeviceToDevice,
                             c->stream));
  TK_TRY(sync(c));
  return es;
}

tucker_status tucker_rank_cut(tucker_ctx* c, const double* w, int64_t I, double thr, int64_t* R,
                              double* disc) {
  if (!c) return TUCKER_ERR_INVALID;
  if (!w || !R || !disc || I < 1 || !(thr >= 0.0))
    return set_err(c, TUCKER_ERR_INVALID, "tucker_rank_cut: bad argument");
  return do_cut(c, w, (int)I, thr, 0, R, disc);
}

tucker_status tucker_ttm(tucker_ctx* c, const void* y, tucker_dtype ydt, int ndim,
                         const int64_t* dims, int mode, const double* A, int64_t K, int64_t lda,
                         int arow, tucker_prec prec, void* z, tucker_dtype zdt) {
  if (!c) return TUCKER_ERR_INVALID;
  if (!y || !A || !z || !check_dims(ndim, dims) || mode < 0 || mode >= ndim || K < 1 ||
      (ydt != TUCKER_F32 && ydt != TUCKER_F64) || (zdt != TUCKER_F32 && zdt != TUCKER_F64) ||
      prec < 0 || prec > 3)
    return set_err(c, TUCKER_ERR_INVALID, "tucker_ttm: bad argument");
  if (arow ? lda < dims[mode] : lda < K)
    return set_err(c, TUCKER_ERR_INVALID, "tucker_ttm: leading dimension too small");
  SlabView v = slab_view(ndim, dims, mode);
  TK_TRY(do_ttm(c, y, ydt, v, A, K, lda, arow, prec, z, zdt, nullptr));
  return sync(c);
}

tucker_status tucker_result_destroy(tucker_result* r) {
  if (!r) return TUCKER_ERR_INVALID;
  cudaDeviceSynchronize();
  cudaFree(r->core);
  for (int k = 0; k < TUCKER_MAX_MODES; ++k) {
    cudaFree(r->factors[k]);
    cudaFree(r->eigvals[k]);
  }
  delete r;
  return TUCKER_OK;
}

// Argument checks shared by tucker_sthosvd and tucker_sthosvd_host; fills
// order (the default 0..N-1 when order_in is null).
static tucker_status check_sthosvd_args(tucker_ctx* c, const void* x, tucker_dtype dt, int ndim,
                                 const int64_t* dims, double eps, const int64_t* ranks,
                                 const int* order_in, tucker_prec prec, int* order,
                                 const char* what) {
  if (!x || !check_dims(ndim, dims) || (dt != TUCKER_F32 && dt != TUCKER_F64) || prec < 0 ||
      prec > 3) {
    char m[96];
    snprintf(m, sizeof m, "%s: bad argument", what);
    return set_err(c, TUCKER_ERR_INVALID, m);
  }
  if (!ranks && !(eps >= 0.0 && std::isfinite(eps)))
    return set_err(c, TUCKER_ERR_INVALID, "eps must be finite and >= 0");
  if (ranks)
    for (int k = 0; k < ndim; ++k)
      if (ranks[k] < 1 || ranks[k] > dims[k])
        return set_err(c, TUCKER_ERR_INVALID, "ranks must satisfy 1 <= R_n <= I_n");
  if (!check_order(ndim, order_in, order))
    return set_err(c, TUCKER_ERR_INVALID, "mode order is not a permutation");
  if ((prec == TUCKER_PREC_MIXED || prec == TUCKER_PREC_TENSOR) && dt != TUCKER_F32)
    return set_err(c, TUCKER_ERR_UNSUPPORTED, "MIXED/TENSOR precision needs FP32 input");
  int64_t imax = 0;
  for (int k = 0; k < ndim; ++k) imax = std::max(imax, dims[k]);
  if (imax > 8192) return set_err(c, TUCKER_ERR_INVALID, "mode size above 8192");
  return TUCKER_OK;
}

// What tucker_sthosvd_host computes while the input streams in: the norm
// pass and, when the first mode is mode 0, that mode's Gram.
struct StreamedMode0 {
  double nrm2 = 0.0, xmax = 0.0;
  const unsigned* rowmax = nullptr;   // mode-0 row maxima (FP32 bits, device) or null
  const double* S0 = nullptr;         // Gram of the first mode (device) or null
  int gram_kernel0 = 0;
  float ms_norm = 0.f, ms_gram0 = 0.f;
};

// Algorithm 1 on the device tensor x; pre != null: the norm (and maybe the
// first Gram) come from a streamed input (tucker_sthosvd_host).
static tucker_status sthosvd_impl(tucker_ctx* c, const void* x, tucker_dtype dt, int ndim,
                           const int64_t* dims, double eps, const int64_t* ranks,
                           const int* order, tucker_prec prec, tucker_result** out,
                           const StreamedMode0* pre) {
  int64_t imax = 0;
  for (int k = 0; k < ndim; ++k) imax = std::max(imax, dims[k]);

  const tucker_dtype wdt = (prec == TUCKER_PREC_FP64) ? TUCKER_F64 : dt;
  // workspace the first mode needs at least (nothing is launched or
  // allocated when it does not fit): the Gram and eigenvector matrices,
  // the first Gram's split-K scratch and its TTM output at rank 1
  const double ws_fixed = 16.0 * (double)imax * (double)imax;
  {
    const SlabView v0 = slab_view(ndim, dims, order[0]);
    const double need0 = ws_fixed + (double)gram_scratch_bytes(c, prec, dt, v0) +
                         (double)dtype_size(wdt) * (double)(numel(ndim, dims) / dims[order[0]]);
    TK_TRY(predict_oom(c, need0, 0.0, "the first mode"));
  }

  tucker_result* r = new tucker_result();
  memset(r, 0, sizeof(*r));
  struct Guard {
    tucker_result*& r;
    ~Guard() { if (r) tucker_result_destroy(r); }
  } guard{r};
  r->ndim = ndim;
  r->core_dtype = wdt;
  for (int k = 0; k < ndim; ++k) { r->dims[k] = dims[k]; r->mode_order[k] = order[k]; }
  double held_factors = 0.0;

  Timer t_total, t_norm;
  t_total.start(c);
  t_norm.start(c);
  const int64_t nx = numel(ndim, dims);
  double nrm2 = 0.0, xmax = 0.0;
  // the exact tensor-core Gram of a first mode 0 takes its digit scales from
  // row maxima that the norm pass records on the way
  DevBuf rowmax;
  const unsigned* rowmax0 = nullptr;
  if (pre) {
    nrm2 = pre->nrm2;
    xmax = pre->xmax;
    rowmax0 = pre->rowmax;
  } else {
    const SlabView v0 = slab_view(ndim, dims, 0);
    const bool tcx = order[0] == 0 && gram_kernel_for(prec, dt, v0, c->num_sms) == 5 &&
                     (((uintptr_t)x) & 3) == 0;
    // the norm pass records the row maxima on the way
    const bool in_norm = tcx && v0.I <= 8192;
    if (tcx) TK_TRY(dev_alloc(c, rowmax, sizeof(unsigned) * v0.I));
    TK_TRY(do_norm(c, x, dt, nx, &nrm2, &xmax, in_norm ? rowmax.as<unsigned>() : nullptr,
                   dims[0]));
    if (tcx && !in_norm) TK_TRY(view_rowmax(c, (const float*)x, v0, rowmax.as<unsigned>()));
    rowmax0 = rowmax.as<unsigned>();
  }
  t_norm.stop(c);
  r->norm_x_sq = nrm2;
  const double thr = ranks ? 0.0 : eps * eps * nrm2 / ndim;
  r->threshold = thr;
  // Gram precision.  The rank cut compares a tail sum with eps^2 ||X||^2 / N.
  // An FP32-product Gram (unbiased rounding, split and ordered as in the
  // kernels) leaves up to ~1.5e-10 ||X||^2 on the discarded subspace of the
  // later modes, whose energy sits in a few components; below
  // eps^2 / N = 1e-9 that is no longer far below the threshold, so those
  // Grams are computed in FP64 there (the TTMs keep their precision).  The
  // exact-digit Gram's error is bounded per view from its row maxima
  // (digit_gram_digits): it keeps the tensor cores, with two digits or
  // three, while that bound allows.
  const bool small_eps =
      !ranks && prec != TUCKER_PREC_FP64 && eps * eps / ndim < kMinFp32GramThreshold;

  DevBuf S, V, ycur;
  TK_TRY(dev_alloc(c, S, sizeof(double) * imax * imax));
  TK_TRY(dev_alloc(c, V, sizeof(double) * imax * imax));
  const void* y = x;
  tucker_dtype ydt = dt;
  int64_t cur[TUCKER_MAX_MODES];
  for (int k = 0; k < ndim; ++k) cur[k] = dims[k];
  // Rotated layout (mode order 0, 1, ..., N-1): every TTM contracts the
  // fastest mode and writes its new mode last (transposed output), so mode n
  // is always the fastest index of the working tensor and every Gram and TTM
  // sees a column-mode view; after N modes the core is back in the natural
  // order.  Other orders keep the natural layout (row-mode views).
  bool rotate = true;
  for (int k = 0; k < ndim; ++k) rotate = rotate && order[k] == k;
  bool noconv = false;
  for (int s = 0; s < ndim; ++s) {
    const int n = order[s];
    SlabView v = slab_view(ndim, cur, n);
    if (rotate) v = SlabView{1, v.I, v.L * v.Rt, 1};
    const int I = (int)v.I;
    Timer tmg, tme, tmt;
    tmg.start(c);
    // later modes of the rotated layout: digit scales from a row-maxima pass
    // of the column-mode view, whose largest entry is the TTM's split scale
    DevBuf rowmax_s;
    double ymax = s == 0 ? xmax : -1.0;
    const unsigned* rmx = s == 0 ? rowmax0 : nullptr;
    const bool streamed = s == 0 && pre && pre->S0;   // Gram summed while the input streamed in
    const int gk = streamed ? -1 : gram_kernel_for(prec, ydt, v, c->num_sms);
    tucker_prec gram_prec = prec;
    int ndig = 3;
    if (gk == 5 && rotate && s > 0 && ydt == TUCKER_F32 && (((uintptr_t)y) & 3) == 0) {
      TK_TRY(dev_alloc(c, rowmax_s, sizeof(unsigned) * v.I));
      TK_TRY(view_rowmax(c, (const float*)y, v, rowmax_s.as<unsigned>()));
      rmx = rowmax_s.as<unsigned>();
    }
    if (gk == 5 && rmx) {
      std::vector<unsigned> hb((size_t)v.I);
      TK_CUDA(c, cudaMemcpyAsync(hb.data(), rmx, sizeof(unsigned) * v.I, cudaMemcpyDeviceToHost,
                                 c->stream));
      TK_TRY(sync(c));
      if (s > 0) {
        unsigned mb = 0;
        for (unsigned b : hb) mb = std::max(mb, b & 0x7fffffffu);
        float mf;
        memcpy(&mf, &mb, sizeof mf);
        ymax = (double)mf;
      }
      ndig = digit_gram_digits(hb.data(), v.I, v.L * v.Rt, thr);
      if (ndig == 0) gram_prec = TUCKER_PREC_FP64;
    } else if (small_eps && gk != 3 && !streamed) {
      gram_prec = TUCKER_PREC_FP64;
    }
    const double* Sn = S.as<double>();
    if (streamed) {
      Sn = pre->S0;
      r->gram_kernel[n] = pre->gram_kernel0;
    } else {
      TK_TRY(do_gram(c, y, ydt, v, gram_prec, S.as<double>(), &r->gram_kernel[n], ymax, true, rmx,
                     ndig > 0 ? ndig : 3));
    }
    tmg.stop(c);
    DevBuf w, U;
    TK_TRY(dev_alloc(c, w, sizeof(double) * I));
    tme.start(c);
    int sweeps = 0;
    int64_t R = 0;
    double disc = 0.0;
    tucker_status es = TUCKER_OK;
    bool have = false;
    const int fixed_R = ranks ? (int)ranks[n] : 0;
    if (use_tridiag(c, I)) {
      bool failed = false;
      TK_TRY(do_eig_tri(c, Sn, I, thr, fixed_R, w.as<double>(), U, &R, &disc, &failed));
      have = !failed;
      r->eig_kernel[n] = 1;
    }
    if (!have) {
      es = do_eig(c, Sn, I, w.as<double>(), V.as<double>(), &sweeps);
      if (es != TUCKER_OK && es != TUCKER_ERR_EIG_NOCONV) return es;
      TK_TRY(do_cut(c, w.as<double>(), I, thr, fixed_R, &R, &disc));
      TK_TRY(dev_alloc(c, U, sizeof(double) * I * R));
      TK_CUDA(c, cudaMemcpyAsync(U.p, V.p, sizeof(double) * I * R, cudaMemcpyDeviceToDevice,
                                 c->stream));
      r->eig_kernel[n] = 0;
    }
    tme.stop(c);
    r->jacobi_sweeps[n] = sweeps;
    r->ranks[n] = R;
    r->discarded_sq[n] = disc;
    r->eigvals[n] = w.as<double>();
    w.release();
    r->factors[n] = U.as<double>();
    U.release();
    // Y <- Y x_n U_n^T : A = U^T is U's column-major storage read row-major
    int64_t nd[TUCKER_MAX_MODES];
    for (int k = 0; k < ndim; ++k) nd[k] = cur[k];
    nd[n] = R;
    held_factors += 8.0 * (double)I * (double)(R + 1);
    {
      const double held = ws_fixed + held_factors +
                          (s > 0 ? (double)dtype_size(ydt) * (double)numel(ndim, cur) : 0.0);
      TK_TRY(predict_oom(c, (double)dtype_size(wdt) * (double)numel(ndim, nd), held,
                         "a TTM"));
    }
    DevBuf z;
    TK_TRY(dev_alloc(c, z, dtype_size(wdt) * numel(ndim, nd)));
    tmt.start(c);
    TK_TRY(do_ttm(c, y, ydt, v, r->factors[n], R, I, 1, prec, z.p, wdt, &r->ttm_kernel[n],
                  ymax, true, rotate));
    tmt.stop(c);
    ycur.reset();
    ycur.p = z.release();
    ycur.st = c->stream;
    y = ycur.p;
    ydt = wdt;
    cur[n] = R;
    if (es == TUCKER_ERR_EIG_NOCONV) noconv = true;
    TK_TRY(sync(c));
    if (c->timing) {
      r->ms_gram[n] = streamed ? pre->ms_gram0 : tmg.ms();
      r->ms_eig[n] = tme.ms();
      r->ms_ttm[n] = tmt.ms();
    }
  }
  r->core = ycur.release();
  t_total.stop(c);
  TK_TRY(sync(c));
  if (c->timing) {
    r->ms_norm = pre ? pre->ms_norm : t_norm.ms();
    r->ms_total = t_total.ms();
  }
  *out = r;
  r = nullptr;  // disarm guard
  if (noconv) return set_err(c, TUCKER_ERR_EIG_NOCONV, "Jacobi reached the sweep cap in some mode");
  return TUCKER_OK;
}

tucker_status tucker_sthosvd(tucker_ctx* c, const void* x, tucker_dtype dt, int ndim,
                             const int64_t* dims, double eps, const int64_t* ranks,
                             const int* order_in, tucker_prec prec, tucker_result** out) {
  if (!c) return TUCKER_ERR_INVALID;
  if (!out) return set_err(c, TUCKER_ERR_INVALID, "null result pointer");
  *out = nullptr;
  int order[TUCKER_MAX_MODES];
  TK_TRY(check_sthosvd_args(c, x, dt, ndim, dims, eps, ranks, order_in, prec, order,
                            "tucker_sthosvd"));
  return sthosvd_impl(c, x, dt, ndim, dims, eps, ranks, order, prec, out, nullptr);
}

// ST-HOSVD of a tensor in host memory.  The input is copied to the device in
// pieces of about c->host_chunk bytes on a copy stream, all enqueued first;
// the context stream takes each piece as its copy lands: the norm pass
// (with the mode-0 row maxima) and, when the first mode is mode 0, that
// mode's Gram over the piece's columns, summed in FP64.  So the norm and the
// largest Gram run under the copy, which bounds the call.
//   Pieces of the mode-0 Gram: whole columns of the I0 x K view (a multiple
// of 4, so every piece starts 16-byte aligned).  The exact-digit Gram of a
// piece takes its scales from the piece's own row maxima and runs with three
// digits (the digit count needs the threshold, which needs the whole norm);
// once the norm is complete, the bound of the whole view decides as in
// tucker_sthosvd, and where it asks for an FP64 Gram, that Gram is computed
// again over the resident copy.  Then Algorithm 1 goes on as in
// tucker_sthosvd on the device copy, which is freed before the call returns.
tucker_status tucker_sthosvd_host(tucker_ctx* c, const void* x_host, tucker_dtype dt, int ndim,
                                  const int64_t* dims, double eps, const int64_t* ranks,
                                  const int* order_in, tucker_prec prec, tucker_result** out) {
  if (!c) return TUCKER_ERR_INVALID;
  if (!out) return set_err(c, TUCKER_ERR_INVALID, "null result pointer");
  *out = nullptr;
  int order[TUCKER_MAX_MODES];
  TK_TRY(check_sthosvd_args(c, x_host, dt, ndim, dims, eps, ranks, order_in, prec, order,
                            "tucker_sthosvd_host"));
  const int64_t nx = numel(ndim, dims);
  const size_t esz = dtype_size(dt);
  const int64_t I0 = dims[0];
  int64_t imax = 0;
  for (int k = 0; k < ndim; ++k) imax = std::max(imax, dims[k]);
  // the device copy, then the first mode's workspace (as tucker_sthosvd)
  {
    const tucker_dtype wdt = (prec == TUCKER_PREC_FP64) ? TUCKER_F64 : dt;
    const SlabView v0 = slab_view(ndim, dims, order[0]);
    const double need = (double)esz * (double)nx + 16.0 * (double)imax * (double)imax * 2.0 +
                        (double)gram_scratch_bytes(c, prec, dt, v0) +
                        (double)dtype_size(wdt) * (double)(nx / dims[order[0]]);
    TK_TRY(predict_oom(c, need, 0.0, "the host input's device copy"));
  }
  DevBuf xd;
  TK_TRY(dev_alloc(c, xd, esz * (size_t)nx));

  // pieces: whole mode-0 columns (4 at a time) when mode 0 comes first
  const SlabView v0 = slab_view(ndim, dims, 0);
  const bool gram0 = order[0] == 0;
  const int64_t ncols = nx / I0;
  int64_t unit = gram0 ? 4 * I0 : 1024;                 // elements
  int64_t per = std::max<int64_t>(1, (int64_t)(c->host_chunk / (double)esz) / unit) * unit;
  if (per > nx) per = nx;
  const int64_t npieces = (nx + per - 1) / per;

  // copies first (copy stream, after the allocation), one event per piece
  cudaStream_t cs = nullptr;
  TK_CUDA(c, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  std::vector<cudaEvent_t> ev((size_t)npieces, nullptr);
  struct Cleanup {
    cudaStream_t& cs;
    std::vector<cudaEvent_t>& ev;
    ~Cleanup() {
      if (cs) { cudaStreamSynchronize(cs); cudaStreamDestroy(cs); }
      for (cudaEvent_t e : ev) if (e) cudaEventDestroy(e);
    }
  } cleanup{cs, ev};
  TK_CUDA(c, cudaEventRecord(c->fork_ev, c->stream));
  TK_CUDA(c, cudaStreamWaitEvent(cs, c->fork_ev, 0));
  {
    // The input copies of concurrent calls on one device run one call after
    // the other (each waits for the previous call's last copy): each gets the
    // whole host-to-device link in turn, and one call's compute and copies
    // back overlap the next call's input.  Issued under the lock, so the
    // chain follows the order in which calls reach this point.
    std::lock_guard<std::mutex> lk(g_h2d_mu);
    cudaEvent_t& last = g_h2d_last[c->device];
    if (last) TK_CUDA(c, cudaStreamWaitEvent(cs, last, 0));
    for (int64_t p = 0; p < npieces; ++p) {
      const int64_t e0 = p * per, e1 = std::min(nx, e0 + per);
      TK_CUDA(c, cudaEventCreateWithFlags(&ev[(size_t)p], cudaEventDisableTiming));
      TK_CUDA(c, cudaMemcpyAsync(xd.as<char>() + esz * (size_t)e0,
                                 static_cast<const char*>(x_host) + esz * (size_t)e0,
                                 esz * (size_t)(e1 - e0), cudaMemcpyHostToDevice, cs));
      TK_CUDA(c, cudaEventRecord(ev[(size_t)p], cs));
    }
    if (!last) TK_CUDA(c, cudaEventCreateWithFlags(&last, cudaEventDisableTiming));
    TK_CUDA(c, cudaEventRecord(last, cs));
  }

  // per piece on the context stream: norm (+ row maxima), Gram of mode 0
  const tucker_prec gprec = prec;
  const int gk = gram0 ? gram_kernel_for(gprec, dt, v0, c->num_sms) : -1;
  const bool tcx = gk == 5;
  const bool small_eps =
      !ranks && prec != TUCKER_PREC_FP64 && eps * eps / ndim < kMinFp32GramThreshold;
  const tucker_prec piece_prec = (gram0 && small_eps && gk != 3 && gk != 5) ? TUCKER_PREC_FP64
                                                                             : gprec;
  DevBuf rmx_all, rmx_p, S0, Sp;
  std::vector<unsigned> rmx_h, rmx_acc;
  if (tcx) {
    TK_TRY(dev_alloc(c, rmx_all, sizeof(unsigned) * I0));
    TK_TRY(dev_alloc(c, rmx_p, sizeof(unsigned) * I0));
    rmx_h.resize((size_t)I0);
    rmx_acc.assign((size_t)I0, 0u);
  }
  if (gram0) {
    TK_TRY(dev_alloc(c, S0, sizeof(double) * I0 * I0));
    TK_TRY(dev_alloc(c, Sp, sizeof(double) * I0 * I0));
  }
  StreamedMode0 pre;
  double xmax = 0.0;
  // the per-piece sums of squares are added in piece order (FP64)
  double nrm2 = 0.0;
  float ms_norm = 0.f, ms_gram = 0.f;
  int kern0 = 0;
  for (int64_t p = 0; p < npieces; ++p) {
    const int64_t e0 = p * per, e1 = std::min(nx, e0 + per);
    const void* yp = xd.as<char>() + esz * (size_t)e0;
    TK_CUDA(c, cudaStreamWaitEvent(c->stream, ev[(size_t)p], 0));
    Timer tn, tg;
    tn.start(c);
    double n2 = 0.0, mx = 0.0;
    const bool in_norm = tcx && I0 <= 8192;
    TK_TRY(do_norm(c, yp, dt, e1 - e0, &n2, &mx, in_norm ? rmx_p.as<unsigned>() : nullptr, I0));
    if (tcx && !in_norm)
      TK_TRY(view_rowmax(c, (const float*)yp, SlabView{1, I0, (e1 - e0) / I0, 1},
                         rmx_p.as<unsigned>()));
    tn.stop(c);
    nrm2 += n2;
    xmax = std::max(xmax, mx);
    if (c->timing) ms_norm += tn.ms();
    if (!gram0) continue;
    const SlabView vp{1, I0, (e1 - e0) / I0, 1};
    tg.start(c);
    double* dst = p == 0 ? S0.as<double>() : Sp.as<double>();
    TK_TRY(do_gram(c, yp, dt, vp, piece_prec, dst, &kern0, mx, true,
                   tcx ? rmx_p.as<unsigned>() : nullptr, 3));
    if (p > 0) TK_CUDA(c, launch_add_f64(Sp.as<double>(), S0.as<double>(), I0 * I0, c->num_sms,
                                         c->stream));
    tg.stop(c);
    if (c->timing) ms_gram += tg.ms();
    if (tcx) {
      TK_CUDA(c, cudaMemcpyAsync(rmx_h.data(), rmx_p.p, sizeof(unsigned) * I0,
                                 cudaMemcpyDeviceToHost, c->stream));
      TK_TRY(sync(c));
      for (int64_t i = 0; i < I0; ++i)
        rmx_acc[(size_t)i] = std::max(rmx_acc[(size_t)i], rmx_h[(size_t)i] & 0x7fffffffu);
    }
  }
  if (tcx) {
    TK_CUDA(c, cudaMemcpyAsync(rmx_all.p, rmx_acc.data(), sizeof(unsigned) * I0,
                               cudaMemcpyHostToDevice, c->stream));
    // the whole view's bound decides as in tucker_sthosvd; a view that needs
    // an FP64 Gram gets it over the resident copy
    const double thr = ranks ? 0.0 : eps * eps * nrm2 / ndim;
    const int nd = c->gram_digits ? c->gram_digits : digit_gram_digits(rmx_acc.data(), I0, ncols,
                                                                       thr);
    if (nd == 0) {
      Timer tg;
      tg.start(c);
      TK_TRY(do_gram(c, xd.p, dt, v0, TUCKER_PREC_FP64, S0.as<double>(), &kern0, xmax, true,
                     nullptr, 3));
      tg.stop(c);
      if (c->timing) ms_gram += tg.ms();
    }
  }
  TK_TRY(sync(c));
  pre.nrm2 = nrm2;
  pre.xmax = xmax;
  pre.rowmax = tcx ? rmx_all.as<unsigned>() : nullptr;
  pre.S0 = gram0 ? S0.as<double>() : nullptr;
  pre.gram_kernel0 = kern0;
  pre.ms_norm = ms_norm;
  pre.ms_gram0 = ms_gram;
  return sthosvd_impl(c, xd.p, dt, ndim, dims, eps, ranks, order, prec, out, &pre);
}

// The batched ST-HOSVD runs modes 0, 1, ... in order on every tensor and keeps
// each working tensor rotated (every TTM writes its new mode last), so mode s
// is the fastest index when its turn comes: the column-mode view of slab_view's
// (L, I, Rt).
static SlabView rot_view(const SlabView& v) { return SlabView{1, v.I, v.L * v.Rt, 1}; }

tucker_status tucker_sthosvd_batched(tucker_ctx* c, int count, const void* const* xs,
                                     tucker_dtype dt, const int* ndims,
                                     const int64_t* const* dimss, double eps, tucker_prec prec,
                                     tucker_result** out) {
  if (!c) return TUCKER_ERR_INVALID;
  if (!out || !xs || !ndims || !dimss || count < 1 || (dt != TUCKER_F32 && dt != TUCKER_F64) ||
      prec < 0 || prec > 3 || !(eps >= 0.0 && std::isfinite(eps)))
    return set_err(c, TUCKER_ERR_INVALID, "tucker_sthosvd_batched: bad argument");
  for (int i = 0; i < count; ++i) out[i] = nullptr;
  if ((prec == TUCKER_PREC_MIXED || prec == TUCKER_PREC_TENSOR) && dt != TUCKER_F32)
    return set_err(c, TUCKER_ERR_UNSUPPORTED, "MIXED/TENSOR precision needs FP32 input");
  int maxN = 0;
  for (int i = 0; i < count; ++i) {
    if (!xs[i] || !check_dims(ndims[i], dimss[i]))
      return set_err(c, TUCKER_ERR_INVALID, "tucker_sthosvd_batched: bad tensor");
    for (int k = 0; k < ndims[i]; ++k)
      if (dimss[i][k] > 4096)
        return set_err(c, TUCKER_ERR_INVALID, "tucker_sthosvd_batched: mode size above 4096");
    maxN = std::max(maxN, ndims[i]);
  }
  cudaStream_t st = c->stream;
  const tucker_dtype wdt = (prec == TUCKER_PREC_FP64) ? TUCKER_F64 : dt;
  std::vector<tucker_result*> res(count, nullptr);
  struct Guard {
    std::vector<tucker_result*>& r;
    ~Guard() { for (auto* p : r) if (p) tucker_result_destroy(p); }
  } guard{res};
  for (int i = 0; i < count; ++i) {
    res[i] = new tucker_result();
    memset(res[i], 0, sizeof(tucker_result));
    res[i]->ndim = ndims[i];
    res[i]->core_dtype = wdt;
    for (int k = 0; k < ndims[i]; ++k) { res[i]->dims[k] = dimss[i][k]; res[i]->mode_order[k] = k; }
  }
  Timer t_total;
  t_total.start(c);
  // ---- norms of all tensors, one synchronization
  std::vector<double> nrm2(count), xmax(count);
  {
    std::vector<int> nb(count);
    size_t off = 0;
    for (int i = 0; i < count; ++i) {
      const int64_t ne = numel(ndims[i], dimss[i]);
      nb[i] = (int)std::max<int64_t>(1, std::min<int64_t>((ne + 255) / 256, (int64_t)c->num_sms * 8));
      off += 2 * (size_t)nb[i];
    }
    DevBuf part, outb;
    TK_TRY(dev_alloc(c, part, sizeof(double) * off));
    TK_TRY(dev_alloc(c, outb, sizeof(double) * 2 * count + sizeof(unsigned) * count));
    unsigned* bad_d = reinterpret_cast<unsigned*>(outb.as<double>() + 2 * count);
    TK_CUDA(c, cudaMemsetAsync(bad_d, 0, sizeof(unsigned) * count, st));
    off = 0;
    for (int i = 0; i < count; ++i) {
      TK_CUDA(c, launch_sumsq(xs[i], dt, numel(ndims[i], dimss[i]), part.as<double>() + off, nb[i],
                              bad_d + i, outb.as<double>() + 2 * i, st));
      off += 2 * (size_t)nb[i];
    }
    std::vector<double> h(2 * count);
    std::vector<unsigned> bad(count);
    TK_CUDA(c, cudaMemcpyAsync(h.data(), outb.p, sizeof(double) * 2 * count, cudaMemcpyDeviceToHost, st));
    TK_CUDA(c, cudaMemcpyAsync(bad.data(), bad_d, sizeof(unsigned) * count, cudaMemcpyDeviceToHost, st));
    TK_TRY(sync(c));
    for (int i = 0; i < count; ++i) {
      if (bad[i]) return set_err(c, TUCKER_ERR_NONFINITE, "a tensor of the batch holds NaN or Inf");
      nrm2[i] = h[2 * i];
      xmax[i] = h[2 * i + 1];
      res[i]->norm_x_sq = nrm2[i];
      res[i]->threshold = eps * eps * nrm2[i] / ndims[i];
    }
  }
  // FP64 Grams below eps^2 / N = 1e-9, as in tucker_sthosvd
  std::vector<tucker_prec> gprec(count, prec);
  for (int i = 0; i < count; ++i)
    if (prec != TUCKER_PREC_FP64 && eps * eps / ndims[i] < kMinFp32GramThreshold)
      gprec[i] = TUCKER_PREC_FP64;
  std::vector<std::vector<int64_t>> cur(count);
  std::vector<const void*> y(count);
  std::vector<DevBuf> ycur(count);
  std::vector<tucker_dtype> ydt(count, dt);
  for (int i = 0; i < count; ++i) {
    cur[i].assign(dimss[i], dimss[i] + ndims[i]);
    y[i] = xs[i];
  }
  TK_CUDA(c, cudaMemsetAsync(c->d_words + 8, 0, 2 * sizeof(unsigned), st));
  for (int s = 0; s < maxN; ++s) {
    std::vector<int> act;
    for (int i = 0; i < count; ++i)
      if (ndims[i] > s) act.push_back(i);
    const int m = (int)act.size();
    // ---- per-problem workspace: A (Gram, reduced in place), d, e, tau, xch, wyT
    std::vector<size_t> wo(m);
    std::vector<int> nq(m), team(m);
    size_t wtot = 0;
    int nmax = 0;
    for (int q = 0; q < m; ++q) nq[q] = (int)cur[act[q]][s];
    tridiag_batch_teams(nq.data(), m, c->num_sms, team.data());
    for (int q = 0; q < m; ++q) {
      const int n = nq[q];
      nmax = std::max(nmax, n);
      wo[q] = wtot;
      wtot += (size_t)n * n + 3 * (size_t)n + 4 * (size_t)n + 2 * (size_t)team[q] + eig_wy_doubles(n);
    }
    DevBuf work, meta;
    TK_TRY(dev_alloc(c, work, sizeof(double) * wtot));
    TK_TRY(dev_alloc(c, meta, sizeof(EigProblem) * m + sizeof(double) * m + sizeof(int64_t) * m +
                                  sizeof(double) * m + sizeof(int) * m + sizeof(unsigned) * (m + 1)));
    EigProblem* pd = meta.as<EigProblem>();
    double* thr_d = reinterpret_cast<double*>(pd + m);
    int64_t* R_d = reinterpret_cast<int64_t*>(thr_d + m);
    double* disc_d = reinterpret_cast<double*>(R_d + m);
    int* info_d = reinterpret_cast<int*>(disc_d + m);
    unsigned* bars_d = reinterpret_cast<unsigned*>(info_d + m);   // m team barriers + error word
    std::vector<EigProblem> h(m);
    std::vector<DevBuf> wbuf(m);
    std::vector<double> thr(m);
    for (int q = 0; q < m; ++q) TK_TRY(dev_alloc(c, wbuf[q], sizeof(double) * nq[q]));
    Timer tg, te, tt;
    tg.start(c);
    TK_TRY(fork_side(c));
    for (int q = 0; q < m; ++q) {
      const int i = act[q], n = (int)cur[i][s];
      EigProblem& P = h[q];
      P = EigProblem{};
      P.A = work.as<double>() + wo[q];
      P.d = P.A + (size_t)n * n;
      P.e = P.d + n;
      P.tau = P.e + n;
      P.xch = P.tau + n;
      P.wyT = P.xch + 4 * (size_t)n + 2 * (size_t)team[q];
      P.info = info_d + q;
      P.n = n;
      P.team_size = team[q];
      P.team_off = q == 0 ? 0 : h[q - 1].team_off + h[q - 1].team_size;
      P.w = wbuf[q].as<double>();
      thr[q] = res[i]->threshold;
      const SlabView v = rot_view(slab_view(ndims[i], cur[i].data(), s));
      StreamSwap sw(c);
      sw.to(q);
      TK_TRY(do_gram(c, y[i], ydt[i], v, gprec[i], P.A, &res[i]->gram_kernel[s],
                     s == 0 ? xmax[i] : -1.0, false));
    }
    TK_TRY(join_side(c));
    tg.stop(c);
    te.start(c);
    TK_CUDA(c, cudaMemsetAsync(info_d, 0, sizeof(int) * m + sizeof(unsigned) * (m + 1), st));
    TK_CUDA(c, cudaMemcpyAsync(thr_d, thr.data(), sizeof(double) * m, cudaMemcpyHostToDevice, st));
    TK_CUDA(c, launch_tridiag(pd, h.data(), m, bars_d, bars_d + m, st, c->barrier_polls));
    int neig = 0;
    for (int q = 0; q < m; ++q) neig += h[q].n;
    TK_CUDA(c, launch_bisect(pd, m, nmax, neig, c->num_sms, st));
    TK_CUDA(c, launch_rank_cut_batched(pd, m, thr_d, nullptr, R_d, disc_d, st));
    std::vector<int64_t> R(m);
    std::vector<double> disc(m);
    TK_CUDA(c, cudaMemcpyAsync(R.data(), R_d, sizeof(int64_t) * m, cudaMemcpyDeviceToHost, st));
    TK_CUDA(c, cudaMemcpyAsync(disc.data(), disc_d, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
    TK_TRY(sync(c));
    // ---- leading eigenvectors of all problems
    size_t vtot = 0;
    int zoff = 0, roff = 0;
    std::vector<size_t> vo(m);
    std::vector<DevBuf> ubuf(m);
    for (int q = 0; q < m; ++q) {
      const int n = h[q].n, Rq = (int)R[q];
      if (Rq < 1 || Rq > n) return set_err(c, TUCKER_ERR_CUDA, "rank cut returned an invalid rank");
      vo[q] = vtot;
      vtot += (size_t)n * Rq + (size_t)Rq * Rq + (eig_lu_bytes(n, Rq) + 7) / 8;
      TK_TRY(dev_alloc(c, ubuf[q], sizeof(double) * (size_t)n * Rq));
    }
    DevBuf vec;
    TK_TRY(dev_alloc(c, vec, sizeof(double) * vtot));
    for (int q = 0; q < m; ++q) {
      EigProblem& P = h[q];
      P.R = (int)R[q];
      P.z = vec.as<double>() + vo[q];
      P.gram = P.z + (size_t)P.n * P.R;
      P.lu = P.gram + (size_t)P.R * P.R;
      P.U = ubuf[q].as<double>();
      P.zoff = zoff;
      P.roff = roff;
      zoff += P.R;
      roff += P.n;
    }
    TK_CUDA(c, cudaMemcpyAsync(pd, h.data(), sizeof(EigProblem) * m, cudaMemcpyHostToDevice, st));
    TK_CUDA(c, launch_invit(pd, m, zoff, st));
    for (int pass = 0; pass < 2; ++pass) {
      TK_CUDA(c, launch_zgram_batched(pd, m, st));   // problems with R <= 64
      for (int q = 0; q < m; ++q)
        if (h[q].R > zgram_batched_max_r()) {
          const SlabView zv{1, (int64_t)h[q].R, (int64_t)h[q].n, 1};
          TK_TRY(do_gram(c, h[q].z, TUCKER_F64, zv, TUCKER_PREC_FP64, h[q].gram, nullptr));
        }
      TK_CUDA(c, launch_chol(pd, m, st));
      TK_CUDA(c, launch_trsm_rows(pd, m, roff, st));
    }
    TK_CUDA(c, launch_backtransform(pd, m, zoff, nmax, st));
    std::vector<int> info(m);
    unsigned berr = 0;
    TK_CUDA(c, cudaMemcpyAsync(info.data(), info_d, sizeof(int) * m, cudaMemcpyDeviceToHost, st));
    TK_CUDA(c, cudaMemcpyAsync(&berr, bars_d + m, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    TK_TRY(sync(c));
    if (berr & DEV_ERR_BARRIER_TIMEOUT)
      return set_err(c, TUCKER_ERR_CUDA, "tridiagonalization team barrier gave up waiting");
    // ---- results of the step, Jacobi where the Cholesky QR refused
    for (int q = 0; q < m; ++q) {
      const int i = act[q], n = h[q].n;
      int64_t Rq = R[q];
      double dq = disc[q];
      res[i]->eig_kernel[s] = 1;
      if (info[q]) {
        DevBuf S2, V2, U2;
        TK_TRY(dev_alloc(c, S2, sizeof(double) * (size_t)n * n));
        TK_TRY(dev_alloc(c, V2, sizeof(double) * (size_t)n * n));
        const SlabView v = rot_view(slab_view(ndims[i], cur[i].data(), s));
        TK_TRY(do_gram(c, y[i], ydt[i], v, gprec[i], S2.as<double>(), nullptr, -1.0, false));
        int sweeps = 0;
        tucker_status es = do_eig(c, S2.as<double>(), n, h[q].w, V2.as<double>(), &sweeps);
        if (es != TUCKER_OK && es != TUCKER_ERR_EIG_NOCONV) return es;
        TK_TRY(do_cut(c, h[q].w, n, thr[q], 0, &Rq, &dq));
        TK_TRY(dev_alloc(c, U2, sizeof(double) * (size_t)n * Rq));
        TK_CUDA(c, cudaMemcpyAsync(U2.p, V2.p, sizeof(double) * n * Rq, cudaMemcpyDeviceToDevice, st));
        ubuf[q].reset();
        ubuf[q].p = U2.release();
        ubuf[q].st = st;
        res[i]->eig_kernel[s] = 0;
        res[i]->jacobi_sweeps[s] = sweeps;
      }
      res[i]->ranks[s] = Rq;
      res[i]->discarded_sq[s] = dq;
      res[i]->eigvals[s] = static_cast<double*>(wbuf[q].release());
      res[i]->factors[s] = ubuf[q].as<double>();
      ubuf[q].release();
    }
    te.stop(c);
    tt.start(c);
    // ---- TTMs of all tensors on the side streams; outputs allocated (and the
    // inputs released, after the join) on the context stream
    std::vector<DevBuf> znew(m);
    for (int q = 0; q < m; ++q) {
      const int i = act[q];
      std::vector<int64_t> nd = cur[i];
      nd[s] = res[i]->ranks[s];
      TK_TRY(dev_alloc(c, znew[q], dtype_size(wdt) * numel(ndims[i], nd.data())));
    }
    TK_TRY(fork_side(c));
    for (int q = 0; q < m; ++q) {
      const int i = act[q];
      const SlabView v = rot_view(slab_view(ndims[i], cur[i].data(), s));
      StreamSwap sw(c);
      sw.to(q);
      TK_TRY(do_ttm(c, y[i], ydt[i], v, res[i]->factors[s], res[i]->ranks[s], h[q].n, 1, prec,
                    znew[q].p, wdt, &res[i]->ttm_kernel[s], s == 0 ? xmax[i] : -1.0, false, true));
    }
    TK_TRY(join_side(c));
    for (int q = 0; q < m; ++q) {
      const int i = act[q];
      ycur[i].reset();
      ycur[i].p = znew[q].release();
      ycur[i].st = st;
      y[i] = ycur[i].p;
      ydt[i] = wdt;
      cur[i][s] = res[i]->ranks[s];
    }
    tt.stop(c);
    if (c->timing) {
      // phases are shared by the whole batch: every result gets their times
      const float g = tg.ms(), e = te.ms(), t = tt.ms();
      for (int q = 0; q < m; ++q) {
        res[act[q]]->ms_gram[s] = g;
        res[act[q]]->ms_eig[s] = e;
        res[act[q]]->ms_ttm[s] = t;
      }
    }
  }
  unsigned werr[2] = {0, 0};
  TK_CUDA(c, cudaMemcpyAsync(werr, c->d_words + 8, sizeof(werr), cudaMemcpyDeviceToHost, st));
  t_total.stop(c);
  TK_TRY(sync(c));
  if (werr[0] | werr[1]) {
    char msg[96];
    snprintf(msg, sizeof msg, "tensor-core kernel reported device error words 0x%x 0x%x", werr[0], werr[1]);
    return set_err(c, TUCKER_ERR_CUDA, msg);
  }
  const float ms = c->timing ? t_total.ms() : 0.f;
  for (int i = 0; i < count; ++i) {
    res[i]->core = ycur[i].release();
    res[i]->ms_total = ms;
    out[i] = res[i];
    res[i] = nullptr;
  }
  return TUCKER_OK;
}

tucker_status tucker_ttm_order(int ndim, const int64_t* core_dims, const int64_t* out_dims,
                               int objective, int* order_out) {
  if (!check_dims(ndim, core_dims) || !check_dims(ndim, out_dims) || !order_out ||
      (objective != 0 && objective != 1))
    return TUCKER_ERR_INVALID;
  order_search(ndim, core_dims, out_dims, objective, order_out);
  return TUCKER_OK;
}

tucker_status tucker_multi_ttm(tucker_ctx* c, const void* core, tucker_dtype cdt, int ndim,
                               const int64_t* core_dims, const double* const* mats,
                               const int64_t* lda, const int64_t* out_dims, const int* order_in,
                               tucker_prec prec, void* out, tucker_dtype odt) {
  if (!c) return TUCKER_ERR_INVALID;
  if (!core || !mats || !lda || !out || !check_dims(ndim, core_dims) ||
      !check_dims(ndim, out_dims) || (cdt != TUCKER_F32 && cdt != TUCKER_F64) ||
      (odt != TUCKER_F32 && odt != TUCKER_F64) || prec < 0 || prec > 3)
    return set_err(c, TUCKER_ERR_INVALID, "tucker_multi_ttm: bad argument");
  for (int k = 0; k < ndim; ++k)
    if (!mats[k] || lda[k] < out_dims[k])
      return set_err(c, TUCKER_ERR_INVALID, "tucker_multi_ttm: bad factor or leading dimension");
  int order[TUCKER_MAX_MODES];
  if (order_in) {
    if (!check_order(ndim, order_in, order))
      return set_err(c, TUCKER_ERR_INVALID, "mode order is not a permutation");
  } else {
    order_search(ndim, core_dims, out_dims, 0, order);
  }
  const tucker_dtype wdt = (prec == TUCKER_PREC_FP64) ? TUCKER_F64 : (cdt == TUCKER_F64 ? TUCKER_F64 : TUCKER_F32);
  int64_t cur[TUCKER_MAX_MODES];
  for (int k = 0; k < ndim; ++k) cur[k] = core_dims[k];
  const void* y = core;
  tucker_dtype ydt = cdt;
  DevBuf hold;
  for (int s = 0; s < ndim; ++s) {
    const int n = order[s];
    const SlabView v = slab_view(ndim, cur, n);
    int64_t nd[TUCKER_MAX_MODES];
    for (int k = 0; k < ndim; ++k) nd[k] = cur[k];
    nd[n] = out_dims[n];
    const bool last = (s == ndim - 1);
    DevBuf z;
    void* zp = out;
    tucker_dtype zdt = odt;
    if (!last) {
      TK_TRY(dev_alloc(c, z, dtype_size(wdt) * numel(ndim, nd)));
      zp = z.p;
      zdt = wdt;
    }
    TK_TRY(do_ttm(c, y, ydt, v, mats[n], out_dims[n], lda[n], 0, prec, zp, zdt, nullptr));
    if (!last) {
      hold.reset();
      hold.p = z.release();
      hold.st = c->stream;
      y = hold.p;
      ydt = wdt;
    }
    cur[n] = out_dims[n];
  }
  return sync(c);
}

tucker_status tucker_reconstruct(tucker_ctx* c, const tucker_result* r, const int64_t* begin,
                                 const int64_t* end, const int* order, tucker_prec prec,
                                 void* out, tucker_dtype odt) {
  if (!c) return TUCKER_ERR_INVALID;
  if (!r || !out) return set_err(c, TUCKER_ERR_INVALID, "tucker_reconstruct: bad argument");
  const int N = r->ndim;
  const double* mats[TUCKER_MAX_MODES];
  int64_t lda[TUCKER_MAX_MODES], od[TUCKER_MAX_MODES];
  for (int k = 0; k < N; ++k) {
    int64_t b = begin ? begin[k] : 0, e = end ? end[k] : r->dims[k];
    if (b < 0 || e > r->dims[k] || e <= b)
      return set_err(c, TUCKER_ERR_INVALID, "reconstruction range out of bounds or empty");
    mats[k] = r->factors[k] + b;
    lda[k] = r->dims[k];
    od[k] = e - b;
  }
  return tucker_multi_ttm(c, r->core, r->core_dtype, N, r->ranks, mats, lda, od, order, prec,
                          out, odt);
}

// ---------------------------------------------------------------- HOSVD

namespace {

// Eigendecomposition and cut of one mode (Algorithm 1's steps after the
// Gram): all eigenvalues into w, R by Eq. Un (or fixed_R), the R leading
// eigenvectors into U (I x R column-major), by the tridiagonal solver where
// it applies, else (or when its Cholesky QR rejects the vectors) Jacobi.
tucker_status do_truncate(tucker_ctx* c, const double* S, int I, double thr, int fixed_R,
                          DevBuf& w, DevBuf& U, int64_t* R, double* disc, int* sweeps,
                          int* eig_kernel, bool* noconv) {
  TK_TRY(dev_alloc(c, w, sizeof(double) * I));
  *sweeps = 0;
  if (use_tridiag(c, I)) {
    bool failed = false;
    TK_TRY(do_eig_tri(c, S, I, thr, fixed_R, w.as<double>(), U, R, disc, &failed));
    *eig_kernel = 1;
    if (!failed) return TUCKER_OK;
  }
  DevBuf V;
  TK_TRY(dev_alloc(c, V, sizeof(double) * (size_t)I * I));
  tucker_status es = do_eig(c, S, I, w.as<double>(), V.as<double>(), sweeps);
  if (es != TUCKER_OK && es != TUCKER_ERR_EIG_NOCONV) return es;
  if (es == TUCKER_ERR_EIG_NOCONV) *noconv = true;
  TK_TRY(do_cut(c, w.as<double>(), I, thr, fixed_R, R, disc));
  TK_TRY(dev_alloc(c, U, sizeof(double) * I * (*R)));
  TK_CUDA(c, cudaMemcpyAsync(U.p, V.p, sizeof(double) * I * (*R), cudaMemcpyDeviceToDevice,
                             c->stream));
  *eig_kernel = 0;
  return TUCKER_OK;
}

// Flops of ST-HOSVD in mode order `perm` with ranks R (the cost analysis of
// Section 6, without the eigensolve, which every order pays alike): the
// mode-n Gram of the current tensor costs numel I_n, its TTM 2 numel R_n.
long double sthosvd_order_cost(int N, const int64_t* I, const int64_t* R, const int* perm) {
  long double cur[TUCKER_MAX_MODES], cost = 0;
  for (int k = 0; k < N; ++k) cur[k] = (long double)I[k];
  for (int s = 0; s < N; ++s) {
    const int n = perm[s];
    long double numel = 1;
    for (int k = 0; k < N; ++k) numel *= cur[k];
    cost += numel * (long double)(I[n] + 2 * R[n]);
    cur[n] = (long double)R[n];
  }
  return cost;
}

}  // namespace

tucker_status tucker_selftest_rcp64(const double* x_dev, double* y_dev, int64_t n,
                                   void* stream) {
  if (!x_dev || !y_dev || n < 0) return TUCKER_ERR_INVALID;
  if (launch_rcp64_probe(x_dev, y_dev, n, (cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return TUCKER_ERR_CUDA;
  }
  return cudaStreamSynchronize((cudaStream_t)stream) == cudaSuccess ? TUCKER_OK : TUCKER_ERR_CUDA;
}

tucker_status tucker_sthosvd_order(int ndim, const int64_t* dims, const int64_t* ranks,
                                   int* order_out) {
  if (!check_dims(ndim, dims) || !ranks || !order_out) return TUCKER_ERR_INVALID;
  for (int k = 0; k < ndim; ++k)
    if (ranks[k] < 1 || ranks[k] > dims[k]) return TUCKER_ERR_INVALID;
  std::vector<int> perm(ndim);
  for (int k = 0; k < ndim; ++k) perm[k] = k;
  bool first = true;
  long double best = 0;
  do {
    const long double cost = sthosvd_order_cost(ndim, dims, ranks, perm.data());
    if (first || cost < best) {
      best = cost;
      first = false;
      for (int k = 0; k < ndim; ++k) order_out[k] = perm[k];
    }
  } while (std::next_permutation(perm.begin(), perm.end()));
  return TUCKER_OK;
}

tucker_status tucker_hosvd(tucker_ctx* c, const void* x, tucker_dtype dt, int ndim,
                           const int64_t* dims, double eps, const int64_t* ranks,
                           tucker_prec prec, tucker_result** out) {
  if (!c) return TUCKER_ERR_INVALID;
  if (!out) return set_err(c, TUCKER_ERR_INVALID, "null result pointer");
  *out = nullptr;
  if (!x || !check_dims(ndim, dims) || (dt != TUCKER_F32 && dt != TUCKER_F64) || prec < 0 ||
      prec > 3)
    return set_err(c, TUCKER_ERR_INVALID, "tucker_hosvd: bad argument");
  if (!ranks && !(eps >= 0.0 && std::isfinite(eps)))
    return set_err(c, TUCKER_ERR_INVALID, "eps must be finite and >= 0");
  if (ranks)
    for (int k = 0; k < ndim; ++k)
      if (ranks[k] < 1 || ranks[k] > dims[k])
        return set_err(c, TUCKER_ERR_INVALID, "ranks must satisfy 1 <= R_n <= I_n");
  if ((prec == TUCKER_PREC_MIXED || prec == TUCKER_PREC_TENSOR) && dt != TUCKER_F32)
    return set_err(c, TUCKER_ERR_UNSUPPORTED, "MIXED/TENSOR precision needs FP32 input");
  int64_t imax = 0;
  for (int k = 0; k < ndim; ++k) imax = std::max(imax, dims[k]);
  if (imax > 8192) return set_err(c, TUCKER_ERR_INVALID, "mode size above 8192");

  tucker_result* r = new tucker_result();
  memset(r, 0, sizeof(*r));
  struct Guard {
    tucker_result*& r;
    ~Guard() { if (r) tucker_result_destroy(r); }
  } guard{r};
  r->ndim = ndim;
  const tucker_dtype wdt = (prec == TUCKER_PREC_FP64) ? TUCKER_F64 : dt;
  r->core_dtype = wdt;
  for (int k = 0; k < ndim; ++k) { r->dims[k] = dims[k]; r->mode_order[k] = k; }
  Timer t_total, t_norm;
  t_total.start(c);
  t_norm.start(c);
  double nrm2 = 0.0, xmax = 0.0;
  // Gram precision as in tucker_sthosvd: the mode-0 digit Gram by its
  // bound from the row maxima, FP32-product Grams (and row-mode digit Grams,
  // whose row maxima stay on the device) in FP64 below eps^2 / N = 1e-9
  const bool small_eps = !ranks && prec != TUCKER_PREC_FP64 &&
                         eps * eps / ndim < kMinFp32GramThreshold;
  DevBuf rowmax;
  {
    const SlabView v0 = slab_view(ndim, dims, 0);
    if (gram_kernel_for(prec, dt, v0, c->num_sms) == 5 && (((uintptr_t)x) & 3) == 0)
      TK_TRY(dev_alloc(c, rowmax, sizeof(unsigned) * v0.I));
  }
  {
    const SlabView v0 = slab_view(ndim, dims, 0);
    const bool in_norm = rowmax.p && v0.I <= 8192;
    TK_TRY(do_norm(c, x, dt, numel(ndim, dims), &nrm2, &xmax,
                   in_norm ? rowmax.as<unsigned>() : nullptr, dims[0]));
    if (rowmax.p && !in_norm) TK_TRY(view_rowmax(c, (const float*)x, v0, rowmax.as<unsigned>()));
  }
  t_norm.stop(c);
  r->norm_x_sq = nrm2;
  const double thr = ranks ? 0.0 : eps * eps * nrm2 / ndim;
  r->threshold = thr;
  DevBuf S;
  TK_TRY(dev_alloc(c, S, sizeof(double) * imax * imax));
  bool noconv = false;
  // every factor from the Gram of X itself (Section 3.2)
  for (int n = 0; n < ndim; ++n) {
    const SlabView v = slab_view(ndim, dims, n);
    Timer tmg, tme;
    tmg.start(c);
    const int gk = gram_kernel_for(prec, dt, v, c->num_sms);
    tucker_prec gram_prec = prec;
    int ndig = 3;
    if (gk == 5 && n == 0 && rowmax.p) {
      std::vector<unsigned> hb((size_t)v.I);
      TK_CUDA(c, cudaMemcpyAsync(hb.data(), rowmax.p, sizeof(unsigned) * v.I,
                                 cudaMemcpyDeviceToHost, c->stream));
      TK_TRY(sync(c));
      ndig = digit_gram_digits(hb.data(), v.I, v.L * v.Rt, thr);
      if (ndig == 0) gram_prec = TUCKER_PREC_FP64;
    } else if (small_eps && gk != 3) {
      gram_prec = TUCKER_PREC_FP64;
    }
    TK_TRY(do_gram(c, x, dt, v, gram_prec, S.as<double>(), &r->gram_kernel[n], xmax, true,
                   n == 0 ? rowmax.as<unsigned>() : nullptr, ndig > 0 ? ndig : 3));
    tmg.stop(c);
    tme.start(c);
    DevBuf w, U;
    int64_t R = 0;
    double disc = 0.0;
    TK_TRY(do_truncate(c, S.as<double>(), (int)v.I, thr, ranks ? (int)ranks[n] : 0, w, U, &R,
                       &disc, &r->jacobi_sweeps[n], &r->eig_kernel[n], &noconv));
    tme.stop(c);
    r->ranks[n] = R;
    r->discarded_sq[n] = disc;
    r->eigvals[n] = w.as<double>();
    w.release();
    r->factors[n] = U.as<double>();
    U.release();
    TK_TRY(sync(c));
    if (c->timing) {
      r->ms_gram[n] = tmg.ms();
      r->ms_eig[n] = tme.ms();
    }
  }
  // core G = X x_0 U_0^T ... x_{N-1} U_{N-1}^T, the TTMs in the flop-minimal
  // order of the shrinking chain; A = U_n^T is U_n's storage read row-major
  int order[TUCKER_MAX_MODES];
  order_search(ndim, dims, r->ranks, 0, order);
  int64_t cur[TUCKER_MAX_MODES];
  for (int k = 0; k < ndim; ++k) cur[k] = dims[k];
  const void* y = x;
  tucker_dtype ydt = dt;
  DevBuf hold;
  for (int s = 0; s < ndim; ++s) {
    const int n = order[s];
    const SlabView v = slab_view(ndim, cur, n);
    int64_t nd[TUCKER_MAX_MODES];
    for (int k = 0; k < ndim; ++k) nd[k] = cur[k];
    nd[n] = r->ranks[n];
    DevBuf z;
    TK_TRY(dev_alloc(c, z, dtype_size(wdt) * numel(ndim, nd)));
    Timer tmt;
    tmt.start(c);
    TK_TRY(do_ttm(c, y, ydt, v, r->factors[n], r->ranks[n], v.I, 1, prec, z.p, wdt,
                  &r->ttm_kernel[n], s == 0 ? xmax : -1.0));
    tmt.stop(c);
    hold.reset();
    hold.p = z.release();
    hold.st = c->stream;
    y = hold.p;
    ydt = wdt;
    cur[n] = r->ranks[n];
    TK_TRY(sync(c));
    if (c->timing) r->ms_ttm[n] = tmt.ms();
  }
  r->core = hold.release();
  t_total.stop(c);
  TK_TRY(sync(c));
  if (c->timing) {
    r->ms_norm = t_norm.ms();
    r->ms_total = t_total.ms();
  }
  *out = r;
  r = nullptr;
  if (noconv) return set_err(c, TUCKER_ERR_EIG_NOCONV, "Jacobi reached the sweep cap in some mode");
  return TUCKER_OK;
}

// ------------------------------------------------ pre- and post-processing

tucker_status tucker_slice_stats(tucker_ctx* c, const void* x, tucker_dtype dt, int ndim,
                                 const int64_t* dims, int mode, double* stats) {
  if (!c) return TUCKER_ERR_INVALID;
  if (!x || !stats || !check_dims(ndim, dims) || mode < 0 || mode >= ndim ||
      (dt != TUCKER_F32 && dt != TUCKER_F64))
    return set_err(c, TUCKER_ERR_INVALID, "tucker_slice_stats: bad argument");
  const SlabView v = slab_view(ndim, dims, mode);
  DevBuf work;
  TK_TRY(dev_alloc(c, work, slice_stats_work_bytes(v.I)));
  TK_CUDA(c, cudaMemsetAsync(c->d_words + 40, 0, sizeof(unsigned), c->stream));
  TK_CUDA(c, launch_slice_stats(x, dt, v.L, v.I, v.Rt, work.p, stats, c->d_words + 40,
                                c->num_sms, c->stream));
  unsigned bad = 0;
  TK_CUDA(c, cudaMemcpyAsync(&bad, c->d_words + 40, sizeof(unsigned), cudaMemcpyDeviceToHost,
                             c->stream));
  TK_TRY(sync(c));
  if (bad) return set_err(c, TUCKER_ERR_NONFINITE, "tensor holds NaN or Inf");
  return TUCKER_OK;
}

tucker_status tucker_slice_transform(tucker_ctx* c, const void* x, tucker_dtype dt, int ndim,
                                     const int64_t* dims, int mode, const double* shift,
                                     const double* scale, int inverse, void* y) {
  if (!c) return TUCKER_ERR_INVALID;
  if (!x || !y || !shift || !scale || !check_dims(ndim, dims) || mode < 0 || mode >= ndim ||
      (dt != TUCKER_F32 && dt != TUCKER_F64) || (inverse != 0 && inverse != 1))
    return set_err(c, TUCKER_ERR_INVALID, "tucker_slice_transform: bad argument");
  const SlabView v = slab_view(ndim, dims, mode);
  TK_CUDA(c, launch_slice_apply(x, dt, v.L, v.I, v.Rt, shift, scale, inverse, y, c->num_sms,
                                c->stream));
  return sync(c);
}

tucker_status tucker_preprocess(tucker_ctx* c, const void* x, tucker_dtype dt, int ndim,
                                const int64_t* dims, int mode, int method, double* shift,
                                double* scale, void* y) {
  if (!c) return TUCKER_ERR_INVALID;
  if (!x || !y || !shift || !scale || !check_dims(ndim, dims) || mode < 0 || mode >= ndim ||
      (dt != TUCKER_F32 && dt != TUCKER_F64) || (method != 0 && method != 1))
    return set_err(c, TUCKER_ERR_INVALID, "tucker_preprocess: bad argument");
  const int64_t I = dims[mode];
  DevBuf st;
  TK_TRY(dev_alloc(c, st, sizeof(double) * 6 * I));
  TK_TRY(tucker_slice_stats(c, x, dt, ndim, dims, mode, st.as<double>()));
  TK_CUDA(c, launch_slice_params(st.as<double>(), I, method, shift, scale, c->stream));
  return tucker_slice_transform(c, x, dt, ndim, dims, mode, shift, scale, 0, y);
}

}  // extern "C"
