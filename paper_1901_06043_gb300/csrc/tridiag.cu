// FP64 symmetric eigensolver for the truncation step of ST-HOSVD (Section
// 5.2 computes the eigenpairs of the I_n x I_n Gram matrix with LAPACK's
// syev, whose first stage is a Householder reduction to tridiagonal form).
// Only what Algorithm 1 consumes is computed: all eigenvalues (the rank cut
// of Eq. Un sums their tail) and the leading R eigenvectors (U_n).
//
//   1. Householder tridiagonalization  Q^T S Q = T          (k_tridiag)
//   2. all eigenvalues of T by bisection on Sturm counts    (k_bisect)
//   3. the rank cut (k_rank_cut of jacobi.cu)
//   4. eigenvectors of T for the leading R eigenvalues by
//      inverse iteration                                     (k_invit)
//   5. their Cholesky QR in descending eigenvalue order, two passes:
//      Gram (gram kernels), L = chol (k_chol), Z L^-T        (k_trsm_rows)
//   6. back-transformation U = Q Z                           (k_backtransform)
//
// Every stage is FP64.  Work is ~(4/3) n^3 for stage 1 and O(n^2 R) for the
// rest, against ~4 n^3 per sweep (matrix plus vectors) of a cyclic Jacobi
// method, which needs ~15 sweeps on the graded Gram matrices of a Tucker
// tensor; on this part FP64 runs at 1/64 of the FP32 rate, so the FP64
// operation count decides.
//
// Stage 1 runs on a team of CTAs: the whole grid (one matrix, a
// cooperative launch with ONE bounded grid barrier per Householder step) or
// one CTA (batched matrices, one CTA each).  Rows are owned cyclically
// (row i by team rank i mod G), so each CTA keeps a balanced share of the
// shrinking trailing matrix.  Step k (reflector H_k = I - tau_k v_k v_k^T
// acting on indices k+1..n-1) needs p_k = tau_k A v_k (rows spread over the
// team) and then w_k = p_k - (tau_k/2)(p_k . v_k) v_k for the rank-2 update
// A <- A - v_k w_k^T - w_k v_k^T.  After the barrier that publishes p_k, every
// CTA forms w_k itself, applies step k's update to the next pivot row (which
// its owner published before the barrier) to obtain v_{k+1}, and then, in
// one pass over its own rows, applies step k's update and computes its part
// of p_{k+1}: the update of step k and the product of step k+1 share a
// barrier.
#include <cfloat>

#include "common.cuh"
#include "kernels.h"

namespace tk {
namespace {

constexpr int TNT = 256;            // threads per CTA of k_tridiag / k_chol
constexpr int TNW = TNT / 32;

__device__ __forceinline__ double warp_sum(double v) {
  // xor butterfly: every lane adds the same two operands at every level
  // (addition commutes exactly), so all lanes end with the same value
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// FP64 instructions occupy a sub-partition's FP64 pipe for ~64 cycles per
// warp whatever they compute, so scalar work that every thread needs is done
// by warp 0 and broadcast through shared memory.

// Sum over the CTA, in a fixed order, returned to every thread.  `red` holds
// TNW + 1 doubles; consecutive calls must alternate between two buffers.
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = (threadIdx.x < TNW) ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = TNW / 2; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) red[TNW] = t;
  }
  __syncthreads();
  return red[TNW];
}

// Householder reflector (Golub & Van Loan Alg. 5.1.1, with the sign of beta
// opposite to alpha): for x = vx[k2..n-1] (alpha = x[k2]) find v (v[k2] = 1),
// tau and beta with (I - tau v v^T) x = beta e_1.  Written in place into vx.
// All threads of the CTA call it and return the same tau and beta.  `red`
// holds TNW + 4 doubles.
__device__ void house(double* vx, int k2, int n, double* red, double& tau, double& beta) {
  double s = 0.0;
  for (int j = k2 + 1 + threadIdx.x; j < n; j += TNT) s = fma(vx[j], vx[j], s);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = (threadIdx.x < TNW) ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = TNW / 2; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) {
      const double alpha = vx[k2];
      double ta = 0.0, be = alpha, sc = 0.0;
      if (t != 0.0) {
        const double mu = sqrt(fma(alpha, alpha, t));
        be = (alpha > 0.0) ? -mu : mu;
        ta = (be - alpha) / be;
        sc = 1.0 / (alpha - be);
      }
      red[TNW + 1] = ta;
      red[TNW + 2] = be;
      red[TNW + 3] = sc;
      vx[k2] = 1.0;
    }
  }
  __syncthreads();
  tau = red[TNW + 1];
  beta = red[TNW + 2];
  const double sc = red[TNW + 3];
  for (int j = k2 + 1 + threadIdx.x; j < n; j += TNT) vx[j] *= sc;
  __syncthreads();
}

}  // namespace

// ---------------------------------------------------------------- stage 1
// One team of P.team_size CTAs per problem (teams back to back in the grid);
// a team of one synchronizes with __syncthreads, a larger one with its own
// bounded barrier.  P.srows: the CTA's own rows live in shared memory;
// otherwise they are read and written in place in A (L2-resident).
__global__ void __launch_bounds__(TNT, 1) k_tridiag(const EigProblem* probs, int count,
                                                    unsigned* bar_counts, unsigned* err,
                                                    unsigned long long poll_limit) {
  extern __shared__ __align__(16) double tsm[];
  int pidx = 0;
  while (pidx + 1 < count && probs[pidx + 1].team_off <= (int)blockIdx.x) ++pidx;
  const EigProblem P = probs[pidx];
  const int n = P.n;
  const int G = P.team_size;
  const int c = (int)blockIdx.x - P.team_off;
  if (c < 0 || c >= G) return;
  const bool SROWS = P.srows != 0;
  const GridBarrier bar{bar_counts + pidx, nullptr, err};
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* A = P.A;
  double* const xp = P.xch;               // p_k: 2 x n
  double* const xr = P.xch + 2 * n;       // next pivot row: 2 x n
  double* const xv = P.xch + 4 * n;       // partial p . v per CTA: 2 x G
  double* vk = tsm;                       // v_k by global index
  double* vn = tsm + n;                   // v_{k+1}
  double* const w = tsm + 2 * n;          // w_k
  double* const red0 = tsm + 3 * n;       // TNW + 4 each
  double* const red1 = red0 + TNW + 4;
  double* const srows = red1 + TNW + 4;   // own rows t = 0, 1, ... (row c + G t) when SROWS
  unsigned gen = 0;
  auto row = [&](int i) -> double* {
    return SROWS ? srows + (size_t)((i - c) / G) * n : A + (int64_t)i * n;
  };

  if (n <= 2) {
    if (c == 0 && threadIdx.x == 0) {
      P.d[0] = A[0];
      if (n == 2) { P.e[0] = A[1]; P.d[1] = A[3]; }
    }
    return;
  }
  if (SROWS) {
    for (int i = c; i < n; i += G) {
      const double* src = A + (int64_t)i * n;
      double* dst = row(i);
      for (int j = threadIdx.x; j < n; j += TNT) dst[j] = src[j];
    }
  }
  // ---- phase -1: v_0 from row 0, p_0 over own rows
  for (int j = threadIdx.x; j < n; j += TNT) vn[j] = (j >= 1) ? A[j] : 0.0;
  __syncthreads();
  double tau_k, beta;
  house(vn, 1, n, red0, tau_k, beta);
  if (c == 0 && threadIdx.x == 0) { P.d[0] = A[0]; P.e[0] = beta; P.tau[0] = tau_k; }
  // (row 0 of A receives its reflector only after the team's first barrier:
  // every CTA reads row 0 above, and a CTA that starts late must not see it
  // overwritten)
  {
    double pv = 0.0;
    const int i0 = 1 + ((c - 1) % G + G) % G;   // smallest own row >= 1
    for (int i = i0 + G * warp; i < n; i += G * TNW) {
      const double* Ai = row(i);
      double acc = 0.0;
      for (int j = 1 + lane; j < n; j += 32) {
        const double a = Ai[j];
        if (i == 1) xr[j] = a;                  // pivot row of phase 0 (buffer 0)
        acc = fma(a, vn[j], acc);
      }
      acc = warp_sum(acc) * tau_k;
      if (lane == 0) xp[i] = acc;               // buffer 0
      pv = fma(acc, vn[i], pv);
    }
    // one value per warp (identical in its lanes): sum the warps
    const double s = block_sum(lane == 0 ? pv : 0.0, red1);
    if (threadIdx.x == 0) xv[c] = s;
  }
  { double* t = vk; vk = vn; vn = t; }
  if (G > 1) { if (!grid_sync(bar, gen, poll_limit, (unsigned)G)) return; } else __syncthreads();
  if (c == 0)   // v_0 (now vk) into row 0, read by nobody after the barrier
    for (int j = 2 + threadIdx.x; j < n; j += TNT) A[j] = vk[j];

  // ---- phases 0 .. n-3
  for (int k = 0; k <= n - 3; ++k) {
    const int b = k & 1, nb = b ^ 1;
    const double* pk = xp + b * n;
    const double* rk = xr + b * n;
    double* const red = (k & 1) ? red1 : red0;
    double* const redo = (k & 1) ? red0 : red1;
    // this thread's entries of p_k and of the pivot row (issued first), and
    // p_k . v_k from the CTAs' partials in a fixed order (warp 0)
    constexpr int JPT = 4;                  // j values per thread kept in registers
    double pj[JPT], rj[JPT];
#pragma unroll
    for (int q = 0; q < JPT; ++q) {
      const int j = k + 1 + threadIdx.x + q * TNT;
      pj[q] = (j < n) ? __ldcg(pk + j) : 0.0;
      rj[q] = (j < n) ? __ldcg(rk + j) : 0.0;
    }
    if (warp == 0) {
      double s = 0.0;
      for (int q = lane; q < G; q += 32) s += __ldcg(xv + b * G + q);
      s = warp_sum(s);
      if (lane == 0) {
        const double K = 0.5 * tau_k * s;
        redo[TNW + 1] = K;
        redo[TNW + 2] = __ldcg(pk + k + 1) - K;   // w_k at k+1 (v_k[k+1] = 1)
      }
    }
    __syncthreads();
    const double K = redo[TNW + 1], wk1 = redo[TNW + 2];
    const bool owner = ((k + 1) % G) == c;
    auto wr = [&](int j, double pjq, double rjq) {
      const double wj = fma(-K, vk[j], pjq);
      w[j] = wj;
      // row k+1 of the updated matrix: r_j = a_j - w_j - w_{k+1} v_j
      const double r = fma(-wk1, vk[j], rjq - wj);
      if (j == k + 1) {
        if (owner) P.d[k + 1] = r;
      } else {
        vn[j] = r;
      }
    };
#pragma unroll
    for (int q = 0; q < JPT; ++q) {
      const int j = k + 1 + threadIdx.x + q * TNT;
      if (j < n) wr(j, pj[q], rj[q]);
    }
    for (int j = k + 1 + threadIdx.x + JPT * TNT; j < n; j += TNT) wr(j, __ldcg(pk + j), __ldcg(rk + j));
    __syncthreads();
    const bool more = (k + 1 <= n - 3);
    double tau_n = 0.0;
    if (more) {
      house(vn, k + 2, n, red, tau_n, beta);
      if (owner) {
        if (threadIdx.x == 0) { P.e[k + 1] = beta; P.tau[k + 1] = tau_n; }
        double* Ar = A + (int64_t)(k + 1) * n;
        for (int j = k + 3 + threadIdx.x; j < n; j += TNT) Ar[j] = vn[j];
      }
    } else if (owner && threadIdx.x == 0) {
      P.e[n - 2] = vn[n - 1];
    }
    // own rows i >= k+2: update of step k, then the product of step k+1
    double pv = 0.0;
    {
      const int lo = k + 2;
      const int i0 = lo + ((c - lo) % G + G) % G;
      for (int i = i0 + G * warp; i < n; i += G * TNW) {
        double* Ai = row(i);
        const double vi = vk[i], wi = w[i];
        double acc = 0.0;
#pragma unroll 4
        for (int j = lo + lane; j < n; j += 32) {
          const double a = fma(-wi, vk[j], fma(-vi, w[j], Ai[j]));
          Ai[j] = a;
          if (i == lo) xr[nb * n + j] = a;
          if (more) acc = fma(a, vn[j], acc);
          else if (i == n - 1) P.d[n - 1] = a;
        }
        if (more) {
          acc = warp_sum(acc) * tau_n;
          if (lane == 0) xp[nb * n + i] = acc;
          pv = fma(acc, vn[i], pv);
        }
      }
    }
    if (!more) break;
    const double sp = block_sum(lane == 0 ? pv : 0.0, redo);
    if (threadIdx.x == 0) xv[nb * G + c] = sp;
    { double* t = vk; vk = vn; vn = t; }
    tau_k = tau_n;
    if (G > 1) { if (!grid_sync(bar, gen, poll_limit, (unsigned)G)) return; } else __syncthreads();
  }
}

// ---------------------------------------------------------------- stage 2
// Sturm count: the number of eigenvalues of T below x = the number of sign
// changes in the leading principal minors p_0 = 1, p_1, ..., p_n of T - x I,
// from the three-term recurrence p_i = (d_{i-1} - x) p_{i-1} -
// e_{i-2}^2 p_{i-2} (Wilkinson, The Algebraic Eigenvalue Problem, Ch. 5: the
// computed signs are exact for a matrix within a few ulps of T).  No
// division: three FP64 operations a step (a division costs ~7 FMAs here).
// T arrives scaled by a power of two to entries of magnitude <= 1, so the
// minors grow by at most ~3 per step: both are rescaled by a power of two
// when their exponents leave [-256, 256], tested every 8 steps.  An exact
// zero minor becomes -sign(previous) 2^-600 (integer operations only), the
// counterpart of the -pivmin safeguard of the ratio form; with e_i != 0 the
// count is then the same as with the zero counted either way.
__device__ __forceinline__ int exp_bits(double v) {
  return (int)((__double_as_longlong(v) >> 52) & 0x7ff);
}
__device__ __forceinline__ double nonzero_or_tiny(double pn, double pc) {
  const long long b = __double_as_longlong(pn);
  if ((b << 1) != 0) return pn;
  // -sign(pc) * 2^-600
  const long long t = (~__double_as_longlong(pc) & (long long)0x8000000000000000ull) |
                      ((long long)(1023 - 600) << 52);
  return __longlong_as_double(t);
}
__device__ __forceinline__ int sturm_count(const double* d, const double* e2, int n, double x) {
  double pm = 1.0;          // p_{i-1}
  double pc = nonzero_or_tiny(d[0] - x, 1.0);
  int cnt = (int)((unsigned long long)__double_as_longlong(pc) >> 63);
  int i = 1;
  while (i < n) {
    const int iend = min(n, i + 8);
#pragma unroll 8
    for (; i < iend; ++i) {
      const double pn = nonzero_or_tiny(fma(d[i] - x, pc, -e2[i - 1] * pm), pc);
      cnt += (int)(((unsigned long long)(__double_as_longlong(pn) ^ __double_as_longlong(pc))) >> 63);
      pm = pc;
      pc = pn;
    }
    const int em = max(exp_bits(pc), exp_bits(pm));
    if (em > 1023 + 256 || em < 1023 - 256) {
      const double f = __longlong_as_double((long long)(2046 - em) << 52);   // 2^(1023 - em)
      pc *= f;
      pm *= f;
    }
  }
  return cnt;
}

// Bisection by multisection: L lanes (1 <= L <= 32, a power of two) work on
// one eigenvalue, each round counting at L interior points of [lo, hi] and
// keeping the sub-interval that holds eigenvalue number a (ascending), until
// its width is below 2 eps ||T|| (the accuracy of the counts).  A warp issues
// one FP64 instruction per step whatever its lanes do, so L trades rounds
// (53 / log2(L + 1)) against warps: wide L for a few eigenvalues, narrow L for
// many.  CTA = BNW warps of one problem.
constexpr int BNW = 4;
__global__ void __launch_bounds__(BNW * 32) k_bisect(const EigProblem* probs, int L) {
  extern __shared__ __align__(16) double bsm[];
  const EigProblem P = probs[blockIdx.y];
  const int n = P.n;
  const int per_warp = 32 / L;
  const int per_cta = BNW * per_warp;
  if ((int)blockIdx.x * per_cta >= n) return;
  double* d = bsm;
  double* e2 = bsm + n;
  __shared__ double s_lo[BNW * 32], s_hi[BNW * 32];
  double glo = INFINITY, ghi = -INFINITY;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double di = P.d[i];
    const double el = (i > 0) ? fabs(P.e[i - 1]) : 0.0;
    const double er = (i < n - 1) ? fabs(P.e[i]) : 0.0;
    glo = fmin(glo, di - el - er);
    ghi = fmax(ghi, di + el + er);
  }
  s_lo[threadIdx.x] = glo;
  s_hi[threadIdx.x] = ghi;
  __syncthreads();
  for (int i = 0; i < BNW * 32; ++i) {
    glo = fmin(glo, s_lo[i]);
    ghi = fmax(ghi, s_hi[i]);
  }
  const double tnorm = fmax(fabs(glo), fabs(ghi));
  // scale by 2^-ex (exact) so that ||T|| / 2^ex is in [0.5, 1)
  const int ex = (tnorm > 0.0) ? exp_bits(tnorm) - 1022 : 0;
  const double sc = __longlong_as_double((long long)(1023 - ex) << 52);
  const double isc = __longlong_as_double((long long)(1023 + ex) << 52);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    d[i] = P.d[i] * sc;
    if (i < n - 1) { const double ei = P.e[i] * sc; e2[i] = ei * ei; }
  }
  __syncthreads();
  const double tn = tnorm * sc;
  const double atol = 2.0 * DBL_EPSILON * tn + DBL_MIN;
  glo = glo * sc - (2.0 * DBL_EPSILON * tn * n + DBL_MIN);
  ghi = ghi * sc + (2.0 * DBL_EPSILON * tn * n + DBL_MIN);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane / L, l = lane % L;                         // group, lane in group
  const int j = blockIdx.x * per_cta + warp * per_warp + g;     // descending index
  const bool valid = j < n;
  const int a = n - 1 - (valid ? j : n - 1);                    // ascending index
  const unsigned gmask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << (g * L));
  double lo = glo, hi = ghi;
  for (int round = 0; round < 64; ++round) {
    const bool active = valid && (hi - lo > atol);
    if (!__any_sync(0xffffffffu, active)) break;
    const double x = lo + (hi - lo) * ((double)(l + 1) / (double)(L + 1));
    const int cnt = active ? sturm_count(d, e2, n, x) : 0;
    const unsigned above = __ballot_sync(0xffffffffu, active && cnt > a) & gmask;
    const int m = above ? (__ffs(above) - 1 - g * L) : L;      // first point above, in group
    const double xm = __shfl_sync(0xffffffffu, x, g * L + (m < L ? m : L - 1));
    const double xl = __shfl_sync(0xffffffffu, x, g * L + (m > 0 ? m - 1 : 0));
    if (active) {
      if (m < L) hi = xm;
      if (m > 0) lo = xl;
    }
  }
  if (valid && l == 0) P.w[j] = 0.5 * (lo + hi) * isc;
}

// ---------------------------------------------------------------- stage 4
// Inverse iteration, one thread per wanted eigenvector: Gaussian elimination
// with partial pivoting of T - lambda I (a tridiagonal; U gets a second
// superdiagonal from the row swaps), then two solves, the first from a
// pseudo-random right-hand side, each followed by normalization.  Pivots
// below eps ||T|| are raised to that size (the shift is an eigenvalue, so
// one pivot is ~0); a running power-of-two rescale (|z| <= 2^400, so the
// sum of squares stays finite) keeps the back substitution finite.  Output
// column j of Z (n x R, row-major: Z[i*R + j]).
//
// The factorization runs fused with the first forward elimination, and the
// pivots are stored as reciprocals, so the only reciprocal on the dependent
// chain is the factorization's; it is an FP32 seed refined by two
// Newton-Raphson steps r <- r (2 - x r) in FP64 (quadratic convergence:
// 2^-23 -> 2^-46 -> below FP64 rounding), ~5 dependent FP64 operations
// against ~7 for a full division.
__device__ __forceinline__ uint32_t hash_u32(uint32_t i, uint32_t j) {
  uint32_t h = i * 0x9E3779B1u ^ (j + 0x7F4A7C15u) * 0x85EBCA77u;
  h ^= h >> 15; h *= 0x2C1B3C6Du; h ^= h >> 12; h *= 0x297A2D39u; h ^= h >> 15;
  return h;
}
__device__ __forceinline__ double hash_unit(uint32_t i, uint32_t j) {
  return (double)hash_u32(i, j) * (2.0 / 4294967296.0) - 1.0;
}

// 1/x for a normal x with |x| in [2^-1000, 2^1000]: the FP32 reciprocal of
// x's mantissa (moved into FP32 by integer operations), rescaled by the
// exponent, then two Newton-Raphson steps.
__device__ __forceinline__ double rcp64(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7ff);
  if (ex < 24 || ex > 2022) return 1.0 / x;
  const float mf = __uint_as_float(0x3f800000u | (unsigned)((b >> 29) & 0x7fffff));   // [1, 2)
  float rf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(mf));                              // (0.5, 1]
  const unsigned rb = __float_as_uint(rf);
  const int re = (int)((rb >> 23) & 0xff) - 127 + 1023 - (ex - 1023);
  double r = __longlong_as_double((long long)((b >> 63) << 63 | (unsigned long long)re << 52 |
                                              (unsigned long long)(rb & 0x7fffff) << 29));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

__global__ void k_rcp64_probe(const double* x, double* y, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = rcp64(x[i]);
}

__global__ void k_invit(const EigProblem* probs, int nprob) {
  // flattened (problem, vector): probs[p].zoff is the first thread of p
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  int p = 0;
  while (p + 1 < nprob && probs[p + 1].zoff <= t) ++p;
  const EigProblem P = probs[p];
  const int j = t - P.zoff;
  if (j < 0 || j >= P.R) return;
  const int n = P.n, R = P.R;
  const double lam = P.w[j];
  const double* __restrict__ d = P.d;
  const double* __restrict__ e = P.e;
  double* __restrict__ RI = P.lu;                        // 1 / pivot
  double* __restrict__ U1 = RI + (int64_t)n * R;
  double* __restrict__ U2 = U1 + (int64_t)n * R;
  double* __restrict__ M = U2 + (int64_t)n * R;
  unsigned char* __restrict__ flag = reinterpret_cast<unsigned char*>(M + (int64_t)n * R);
  unsigned char* __restrict__ scnt = flag + (int64_t)n * R;
  double* __restrict__ Z = P.z;
  auto at = [&](int k) { return (int64_t)k * R + j; };
  // ||T||_1 bound for the pivot floor
  double tn = 0.0;
  for (int i = 0; i < n; ++i) {
    const double r = fabs(d[i]) + (i > 0 ? fabs(e[i - 1]) : 0.0) + (i < n - 1 ? fabs(e[i]) : 0.0);
    tn = fmax(tn, r);
  }
  const double ptol = fmax(DBL_EPSILON * tn, 0x1p-990);
  const unsigned long long ptol_bits = (unsigned long long)__double_as_longlong(ptol);
  auto absb = [](double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
  };
  // factorization fused with the forward elimination of b (random); y -> Z
  double p0 = d[0] - lam, p1 = (n > 1) ? e[0] : 0.0;
  double pb = hash_unit(0, j);
  for (int k = 0; k + 1 < n; ++k) {
    const double ek = e[k];
    const double a1 = d[k + 1] - lam;
    const double e1 = (k + 2 < n) ? e[k + 1] : 0.0;
    const double bk1 = hash_unit(k + 1, j);
    const bool swap = absb(ek) > absb(p0);
    if (!swap && absb(p0) < ptol_bits) p0 = (p0 < 0.0) ? -ptol : ptol;
    const double piv = swap ? ek : p0;
    const double r = rcp64(piv);
    const double m = (swap ? p0 : ek) * r;
    RI[at(k)] = r;
    U1[at(k)] = swap ? a1 : p1;
    U2[at(k)] = swap ? e1 : 0.0;
    M[at(k)] = m;
    flag[at(k)] = swap ? 1 : 0;
    double yk;
    if (swap) {
      yk = bk1;
      pb = fma(-m, bk1, pb);
      p0 = fma(-m, a1, p1);
      p1 = -m * e1;
    } else {
      yk = pb;
      pb = fma(-m, pb, bk1);
      p0 = fma(-m, p1, a1);
      p1 = e1;
    }
    Z[at(k)] = yk;
  }
  if (absb(p0) < ptol_bits) p0 = (p0 < 0.0) ? -ptol : ptol;
  RI[at(n - 1)] = rcp64(p0);
  U1[at(n - 1)] = 0.0;
  U2[at(n - 1)] = 0.0;
  Z[at(n - 1)] = pb;
  const double SMALL = 0x1p-400;
  double bscale = 1.0;
  // the passes below prefetch the operands of the next PF steps into
  // registers before working through the current ones, which keeps the L2
  // latency off the dependent chain (each step stores into Z, so the
  // compiler cannot move the next loads ahead by itself)
  constexpr int PF = 8;
  for (int it = 0; it < 2; ++it) {
    if (it == 1) {
      // forward elimination of the previous solution (times bscale)
      double pv = Z[at(0)] * bscale;
      double nb_[PF], nm_[PF];
      unsigned char nf_[PF];
      auto load_f = [&](int k0) {
#pragma unroll
        for (int q = 0; q < PF; ++q) {
          const int k = k0 + q;
          const bool ok = k + 1 < n;
          nb_[q] = ok ? Z[at(k + 1)] : 0.0;
          nm_[q] = ok ? M[at(k)] : 0.0;
          nf_[q] = ok ? flag[at(k)] : 0;
        }
      };
      load_f(0);
      for (int k0 = 0; k0 + 1 < n; k0 += PF) {
        double cb[PF], cm[PF];
        unsigned char cf[PF];
#pragma unroll
        for (int q = 0; q < PF; ++q) { cb[q] = nb_[q]; cm[q] = nm_[q]; cf[q] = nf_[q]; }
        if (k0 + PF + 1 < n) load_f(k0 + PF);
#pragma unroll
        for (int q = 0; q < PF; ++q) {
          const int k = k0 + q;
          if (k + 1 < n) {
            const double bk1 = cb[q] * bscale;
            double yk;
            if (cf[q] == 0) { yk = pv; pv = fma(-cm[q], pv, bk1); }
            else { yk = bk1; pv = fma(-cm[q], bk1, pv); }
            Z[at(k)] = yk;
          }
        }
      }
      Z[at(n - 1)] = pv;
    }
    // back substitution with rescaling; scnt[i] = rescales before z_i was
    // stored; the sum of squares is kept at the running scale
    int nres = 0;
    double sc = 1.0;             // 2^(-400 nres): the scale of z1, z2 and zk
    double z1 = 0.0, z2 = 0.0;   // z_{k+1}, z_{k+2} at the current scale
    double ss = 0.0;
    double ny[PF], n1[PF], n2[PF], nr[PF];
    auto load_b = [&](int k0) {   // steps k0, k0 - 1, ..., k0 - PF + 1
#pragma unroll
      for (int q = 0; q < PF; ++q) {
        const int k = k0 - q;
        const bool ok = k >= 0;
        ny[q] = ok ? Z[at(k)] : 0.0;
        n1[q] = ok ? U1[at(k)] : 0.0;
        n2[q] = ok ? U2[at(k)] : 0.0;
        nr[q] = ok ? RI[at(k)] : 0.0;
      }
    };
    load_b(n - 1);
    for (int k0 = n - 1; k0 >= 0; k0 -= PF) {
      double cy[PF], c1[PF], c2[PF], cr[PF];
#pragma unroll
      for (int q = 0; q < PF; ++q) { cy[q] = ny[q]; c1[q] = n1[q]; c2[q] = n2[q]; cr[q] = nr[q]; }
      if (k0 - PF >= 0) load_b(k0 - PF);
#pragma unroll
      for (int q = 0; q < PF; ++q) {
        const int k = k0 - q;
        if (k >= 0) {
          double rr = cy[q] * sc;
          rr = fma(-c2[q], z2, rr);     // U2 and U1 are 0 past the end
          rr = fma(-c1[q], z1, rr);
          double zk = rr * cr[q];
          if (absb(zk) > 0x58F0000000000000ull) {   // |zk| > 2^400: rescale by 2^-400
            zk *= SMALL; z1 *= SMALL; z2 *= SMALL; sc *= SMALL; ss *= 0x1p-800;
            ++nres;
          }
          Z[at(k)] = zk;
          scnt[at(k)] = (unsigned char)(nres > 255 ? 255 : nres);
          ss = fma(zk, zk, ss);
          z2 = z1;
          z1 = zk;
        }
      }
    }
    if (nres > 0) {
      for (int k = 0; k < n; ++k) {
        double zk = Z[at(k)];
        for (int q = scnt[at(k)]; q < nres; ++q) zk *= SMALL;
        Z[at(k)] = zk;
      }
    }
    bscale = (ss > 0.0) ? rcp64(sqrt(ss)) : 1.0;
  }
  for (int k = 0; k < n; ++k) Z[at(k)] *= bscale;
}

// ---------------------------------------------------------------- stage 5
// Cholesky factor of the R x R Gram G = Z^T Z (lower, in place), one CTA per
// problem, column by column.  A pivot <= 0 (info = 1) or a condition number
// of Z above 1e6 (info = 2: inverse iteration returned nearly dependent
// vectors, and the QR would lose orthogonality) marks the problem as failed;
// the host then takes another solver for it.
__global__ void __launch_bounds__(TNT) k_chol(const EigProblem* probs) {
  const EigProblem P = probs[blockIdx.x];
  const int R = P.R;
  double* Gm = P.gram;
  double lmin = INFINITY, lmax = 0.0;
  for (int col = 0; col < R; ++col) {
    const double piv = Gm[(int64_t)col * R + col];
    if (!(piv > 0.0)) {
      if (threadIdx.x == 0) *P.info = 1;
      return;
    }
    const double l = sqrt(piv);
    const double il = 1.0 / l;
    lmin = fmin(lmin, l);
    lmax = fmax(lmax, l);
    __syncthreads();   // every thread has read the pivot
    // scale the column below the pivot, then update the trailing lower part
    for (int r = col + threadIdx.x; r < R; r += TNT)
      Gm[(int64_t)r * R + col] = (r == col) ? l : Gm[(int64_t)r * R + col] * il;
    __syncthreads();
    const int m = R - col - 1;
    for (int q = threadIdx.x; q < m * m; q += TNT) {
      const int r = col + 1 + q / m, s = col + 1 + q % m;
      if (s <= r)
        Gm[(int64_t)r * R + s] = fma(-Gm[(int64_t)r * R + col], Gm[(int64_t)s * R + col],
                                     Gm[(int64_t)r * R + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && lmin < 1e-6 * lmax) *P.info = 2;
}

// Q = Z L^-T, one thread per row of Z (forward substitution with L).
__global__ void k_trsm_rows(const EigProblem* probs, int nprob) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  int p = 0;
  while (p + 1 < nprob && probs[p + 1].roff <= t) ++p;
  const EigProblem P = probs[p];
  const int i = t - P.roff;
  if (i < 0 || i >= P.n || *P.info) return;
  const int R = P.R;
  double* z = P.z + (int64_t)i * R;
  const double* L = P.gram;
  for (int c = 0; c < R; ++c) {
    double s = z[c];
    for (int q = 0; q < c; ++q) s = fma(-L[(int64_t)c * R + q], z[q], s);
    z[c] = s / L[(int64_t)c * R + c];
  }
}

// ---------------------------------------------------------------- stage 6
// U = Q_H Z with Q_H = H_0 H_1 ... H_{n-3}, in blocks of WYB reflectors: a
// block H_k0 ... H_{k0+m-1} equals I - V T V^T with V = [v_k0 ... v_{k0+m-1}]
// and T upper triangular (the compact WY form, Schreiber & Van Loan 1989:
// T_jj = tau_j, T[0:j, j] = -tau_j T[0:j, 0:j] (V[:, 0:j]^T v_j)).  The blocks
// are applied from the last to the first: z <- z - V (T (V^T z)).  U is
// I x R column-major.
constexpr int WYB = 32;
__host__ __device__ __forceinline__ int wy_blocks(int n) { return n > 2 ? (n - 2 + WYB - 1) / WYB : 0; }

// One CTA per block of reflectors: the T factor into wyT (WYB x WYB, row-major).
__global__ void __launch_bounds__(256) k_wy_t(const EigProblem* probs) {
  const EigProblem P = probs[blockIdx.y];
  const int n = P.n, b = blockIdx.x;
  if (b >= wy_blocks(n)) return;
  const int k0 = b * WYB, m = min(WYB, n - 2 - k0);
  __shared__ double W[WYB][WYB + 1];
  __shared__ double T[WYB][WYB + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // W[i][j] = v_{k0+i} . v_{k0+j} for i < j; v_{k0+j} is 1 at k0+j+1 and
  // A[k0+j][c] beyond, and v_{k0+i} is A[k0+i][c] there
  for (int q = warp; q < m * m; q += 8) {
    const int i = q / m, jj = q % m;
    if (i >= jj) continue;
    const double* vi = P.A + (int64_t)(k0 + i) * n;
    const double* vj = P.A + (int64_t)(k0 + jj) * n;
    const int s0 = k0 + jj + 1;
    double acc = 0.0;
    for (int c = s0 + 1 + lane; c < n; c += 32) acc = fma(vi[c], vj[c], acc);
    acc = warp_sum(acc);
    if (lane == 0) W[i][jj] = acc + vi[s0];
  }
  __syncthreads();
  if (warp == 0) {
    for (int jj = 0; jj < m; ++jj) {
      const double tj = P.tau[k0 + jj];
      if (lane < jj) {
        double s = 0.0;
        for (int l = lane; l < jj; ++l) s = fma(T[lane][l], W[l][jj], s);
        T[lane][jj] = -tj * s;
      } else if (lane == jj) {
        T[lane][jj] = tj;
      }
      __syncwarp();
    }
  }
  __syncthreads();
  double* To = P.wyT + (size_t)b * WYB * WYB;
  for (int q = threadIdx.x; q < WYB * WYB; q += 256) {
    const int i = q / WYB, jj = q % WYB;
    To[q] = (i < m && jj < m && i <= jj) ? T[i][jj] : 0.0;
  }
}

// One CTA per eigenvector (flattened over problems), the vector in shared memory.
__global__ void __launch_bounds__(256) k_backtransform(const EigProblem* probs, int nprob) {
  extern __shared__ __align__(16) double zs[];
  __shared__ double y[WYB], y2[WYB];
  const int t = blockIdx.x;
  int p = 0;
  while (p + 1 < nprob && probs[p + 1].zoff <= t) ++p;
  const EigProblem P = probs[p];
  const int j = t - P.zoff;
  if (j < 0 || j >= P.R || *P.info) return;
  const int n = P.n, R = P.R;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double* A = P.A;
  for (int i = threadIdx.x; i < n; i += blockDim.x) zs[i] = P.z[(int64_t)i * R + j];
  __syncthreads();
  for (int b = wy_blocks(n) - 1; b >= 0; --b) {
    const int k0 = b * WYB, m = min(WYB, n - 2 - k0);
    // y = V^T z
    for (int q = warp; q < m; q += 8) {
      const double* v = A + (int64_t)(k0 + q) * n;
      const int s0 = k0 + q + 1;
      double acc = 0.0;
      for (int c = s0 + 1 + lane; c < n; c += 32) acc = fma(v[c], zs[c], acc);
      acc = warp_sum(acc);
      if (lane == 0) y[q] = acc + zs[s0];
    }
    __syncthreads();
    // y2 = T y
    if (warp == 0 && lane < m) {
      const double* Tb = P.wyT + (size_t)b * WYB * WYB + (size_t)lane * WYB;
      double s = 0.0;
      for (int l = lane; l < m; ++l) s = fma(Tb[l], y[l], s);
      y2[lane] = s;
    }
    __syncthreads();
    // z <- z - V y2 (entry i gets the reflectors q with k0 + q + 1 <= i)
    for (int i = k0 + 1 + threadIdx.x; i < n; i += blockDim.x) {
      const int qmax = min(m, i - k0);
      double s = 0.0;
      for (int q = 0; q < qmax; ++q) {
        const double coef = (i == k0 + q + 1) ? 1.0 : A[(int64_t)(k0 + q) * n + i];
        s = fma(coef, y2[q], s);
      }
      zs[i] -= s;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) P.U[(int64_t)j * n + i] = zs[i];
}

// ---------------------------------------------------------------- batched helpers
// Rank cut of Eq. Un for each problem (one thread each): R = min{R in 1..n :
// tail(R) <= thr}, tail accumulated from the smallest eigenvalue up (the same
// order as k_rank_cut), or R = fixed when fixed > 0; disc = tail(R).
__global__ void k_rank_cut_batched(const EigProblem* probs, int count, const double* thr,
                                   const int* fixed, int64_t* R_out, double* disc_out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  const EigProblem P = probs[p];
  const int n = P.n;
  const int fr = fixed ? fixed[p] : 0;
  double tail = 0.0, best_tail = 0.0;
  int best = n;
  for (int R = n - 1; R >= 1; --R) {
    tail += P.w[R];
    if (fr > 0 ? (R == fr) : (tail <= thr[p])) { best = R; best_tail = tail; }
  }
  if (fr > 0 && fr == n) { best = n; best_tail = 0.0; }
  R_out[p] = best;
  disc_out[p] = best_tail;
}

// G = Z^T Z (R x R, full) for each problem with R <= 64, one CTA each: rows of
// Z staged 16 at a time in shared memory, one thread per lower-triangle entry
// (several when R(R+1)/2 > 256), FP64 sums in row order.
constexpr int ZG_MAXR = 64, ZG_ROWS = 16, ZG_PPT = (ZG_MAXR * (ZG_MAXR + 1) / 2 + TNT - 1) / TNT;
__global__ void __launch_bounds__(TNT) k_zgram_batched(const EigProblem* probs) {
  const EigProblem P = probs[blockIdx.x];
  const int n = P.n, R = P.R;
  if (R > ZG_MAXR || *P.info) return;
  __shared__ double zs[ZG_ROWS][ZG_MAXR + 1];
  const int npair = R * (R + 1) / 2;
  int pa[ZG_PPT], pb[ZG_PPT];
  double acc[ZG_PPT];
#pragma unroll
  for (int q = 0; q < ZG_PPT; ++q) {
    const int t = threadIdx.x + TNT * q;
    int a = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
    while ((a + 1) * (a + 2) / 2 <= t) ++a;
    while (a * (a + 1) / 2 > t) --a;
    pa[q] = (t < npair) ? a : 0;
    pb[q] = (t < npair) ? t - a * (a + 1) / 2 : 0;
    acc[q] = 0.0;
  }
  for (int i0 = 0; i0 < n; i0 += ZG_ROWS) {
    __syncthreads();
    for (int c = threadIdx.x; c < ZG_ROWS * R; c += TNT) {
      const int r = c / R, a = c - r * R;
      zs[r][a] = (i0 + r < n) ? P.z[(int64_t)(i0 + r) * R + a] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < ZG_PPT; ++q) {
      if (threadIdx.x + TNT * q >= npair) break;
      double s = acc[q];
#pragma unroll
      for (int r = 0; r < ZG_ROWS; ++r) s = fma(zs[r][pa[q]], zs[r][pb[q]], s);
      acc[q] = s;
    }
  }
#pragma unroll
  for (int q = 0; q < ZG_PPT; ++q) {
    if (threadIdx.x + TNT * q >= npair) break;
    P.gram[(int64_t)pa[q] * R + pb[q]] = acc[q];
    P.gram[(int64_t)pb[q] * R + pa[q]] = acc[q];
  }
}

// ---------------------------------------------------------------- launchers
cudaError_t launch_rank_cut_batched(const EigProblem* probs_dev, int count, const double* thr,
                                    const int* fixed, int64_t* R_out, double* disc_out,
                                    cudaStream_t st) {
  k_rank_cut_batched<<<(count + 127) / 128, 128, 0, st>>>(probs_dev, count, thr, fixed, R_out,
                                                           disc_out);
  count_launches(1);
  return cudaGetLastError();
}

int zgram_batched_max_r() { return ZG_MAXR; }

cudaError_t launch_zgram_batched(const EigProblem* probs_dev, int count, cudaStream_t st) {
  k_zgram_batched<<<count, TNT, 0, st>>>(probs_dev);
  count_launches(1);
  return cudaGetLastError();
}

namespace {
int tridiag_rows_per_cta(int n, int G) { return (n + G - 1) / G; }
size_t tridiag_base_smem(int n) { return sizeof(double) * (3 * (size_t)n + 2 * (TNW + 4)); }
constexpr size_t kTridiagSmemRowsCap = 120 * 1024;
}  // namespace

// ~6 rows per CTA at the first step (the step time is latency-bound: 2 to 8
// rows per CTA measured within 8% of each other at n = 500), at most one CTA
// per SM
int tridiag_team_size(int n, int num_sms) {
  int G = (n + 5) / 6;
  return G > num_sms ? num_sms : (G < 1 ? 1 : G);
}

void tridiag_batch_teams(const int* n, int count, int num_sms, int* team) {
  for (int p = 0; p < count; ++p) team[p] = 1;
  if (count >= num_sms) return;
  double tot = 0.0;
  for (int p = 0; p < count; ++p) tot += (double)n[p] * n[p] * n[p];
  const int extra = num_sms - count;
  for (int p = 0; p < count; ++p) {
    int g = 1 + (int)(extra * ((double)n[p] * n[p] * n[p]) / (tot > 0.0 ? tot : 1.0));
    const int cap = tridiag_team_size(n[p], num_sms);
    team[p] = g < cap ? g : cap;
  }
}

cudaError_t launch_tridiag(const EigProblem* probs_dev, EigProblem* probs_host, int count,
                           unsigned* bar_counts, unsigned* err, cudaStream_t st,
                           unsigned long long poll_limit) {
  int nmax = 0, grid = 0, multi = 0;
  size_t rows_max = 0;
  for (int p = 0; p < count; ++p) {
    EigProblem& P = probs_host[p];
    nmax = P.n > nmax ? P.n : nmax;
    const size_t rb = sizeof(double) * (size_t)tridiag_rows_per_cta(P.n, P.team_size) * P.n;
    P.srows = rb <= kTridiagSmemRowsCap;
    if (P.srows && rb > rows_max) rows_max = rb;
    grid += P.team_size;
    multi |= P.team_size > 1;
  }
  const size_t smem = tridiag_base_smem(nmax) + rows_max;
  cudaError_t e = allow_max_dyn_smem((const void*)k_tridiag);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(const_cast<EigProblem*>(probs_dev), probs_host, sizeof(EigProblem) * count,
                      cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  count_launches(1);
  if (multi) {
    // teams of several CTAs spin on each other: all CTAs must be resident
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tridiag, TNT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorLaunchOutOfResources;
    void* args[] = {(void*)&probs_dev, (void*)&count, (void*)&bar_counts, (void*)&err,
                    (void*)&poll_limit};
    return cudaLaunchCooperativeKernel((void*)k_tridiag, dim3(grid), dim3(TNT), args, smem, st);
  }
  k_tridiag<<<grid, TNT, smem, st>>>(probs_dev, count, bar_counts, err, poll_limit);
  return cudaGetLastError();
}

cudaError_t launch_bisect(const EigProblem* probs_dev, int count, int nmax, int total_eigs,
                          int num_sms, cudaStream_t st) {
  // lanes per eigenvalue: about one warp per SM sub-partition in total
  int L = 32;
  while (L > 1 && (int64_t)total_eigs * L > (int64_t)num_sms * 4 * 32) L >>= 1;
  const size_t smem = sizeof(double) * 2 * (size_t)nmax;
  cudaError_t e = allow_max_dyn_smem((const void*)k_bisect);
  if (e != cudaSuccess) return e;
  const int per_cta = BNW * (32 / L);
  k_bisect<<<dim3((nmax + per_cta - 1) / per_cta, count), BNW * 32, smem, st>>>(probs_dev, L);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_invit(const EigProblem* probs_dev, int count, int total_vectors, cudaStream_t st) {
  if (total_vectors < 1) return cudaSuccess;
  k_invit<<<(total_vectors + 63) / 64, 64, 0, st>>>(probs_dev, count);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_chol(const EigProblem* probs_dev, int count, cudaStream_t st) {
  k_chol<<<count, TNT, 0, st>>>(probs_dev);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_trsm_rows(const EigProblem* probs_dev, int count, int total_rows, cudaStream_t st) {
  if (total_rows < 1) return cudaSuccess;
  k_trsm_rows<<<(total_rows + 127) / 128, 128, 0, st>>>(probs_dev, count);
  count_launches(1);
  return cudaGetLastError();
}

size_t eig_wy_doubles(int n) { return (size_t)wy_blocks(n) * WYB * WYB; }

cudaError_t launch_backtransform(const EigProblem* probs_dev, int count, int total_vectors,
                                 int nmax, cudaStream_t st) {
  if (total_vectors < 1) return cudaSuccess;
  const int nb = wy_blocks(nmax);
  if (nb > 0) {
    k_wy_t<<<dim3(nb, count), 256, 0, st>>>(probs_dev);
    count_launches(1);
  }
  const size_t smem = sizeof(double) * (size_t)nmax;
  cudaError_t e = allow_max_dyn_smem((const void*)k_backtransform);
  if (e != cudaSuccess) return e;
  k_backtransform<<<total_vectors, 256, smem, st>>>(probs_dev, count);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_rcp64_probe(const double* x, double* y, int64_t n, cudaStream_t st) {
  if (n > 0) k_rcp64_probe<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, y, n);
  count_launches(n > 0 ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace tk
