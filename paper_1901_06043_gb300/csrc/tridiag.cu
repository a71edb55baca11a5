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

// Sum over the CTA, returned to every thread, in a fixed order.  `red` holds
// TNW doubles; consecutive calls must alternate between two buffers.
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = red[0];
#pragma unroll
  for (int i = 1; i < TNW; ++i) s += red[i];
  return s;
}

// Householder reflector (Golub & Van Loan Alg. 5.1.1, with the sign of beta
// opposite to alpha): for x = vx[k2..n-1] (alpha = x[k2]) find v (v[k2] = 1),
// tau and beta with (I - tau v v^T) x = beta e_1.  Written in place into vx.
// All threads of the CTA call it and return the same tau and beta.
__device__ void house(double* vx, int k2, int n, double* red, double& tau, double& beta) {
  const double alpha = vx[k2];
  double s = 0.0;
  for (int j = k2 + 1 + threadIdx.x; j < n; j += TNT) s = fma(vx[j], vx[j], s);
  const double sigma2 = block_sum(s, red);
  if (sigma2 == 0.0) {
    tau = 0.0;
    beta = alpha;
    __syncthreads();
    if (threadIdx.x == 0) vx[k2] = 1.0;
    for (int j = k2 + 1 + threadIdx.x; j < n; j += TNT) vx[j] = 0.0;
  } else {
    const double mu = sqrt(fma(alpha, alpha, sigma2));
    beta = (alpha > 0.0) ? -mu : mu;
    tau = (beta - alpha) / beta;
    const double sc = 1.0 / (alpha - beta);
    __syncthreads();
    if (threadIdx.x == 0) vx[k2] = 1.0;
    for (int j = k2 + 1 + threadIdx.x; j < n; j += TNT) vx[j] *= sc;
  }
  __syncthreads();
}

}  // namespace

// ---------------------------------------------------------------- stage 1
template <bool GRID>
__global__ void __launch_bounds__(TNT) k_tridiag(const EigProblem* probs, GridBarrier bar) {
  extern __shared__ __align__(16) double tsm[];
  const EigProblem P = probs[GRID ? 0 : blockIdx.x];
  const int n = P.n;
  const int G = GRID ? (int)gridDim.x : 1;
  const int c = GRID ? (int)blockIdx.x : 0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* A = P.A;
  double* const xp = P.xch;               // p_k: 2 x n
  double* const xr = P.xch + 2 * n;       // next pivot row: 2 x n
  double* const xv = P.xch + 4 * n;       // partial p . v per CTA: 2 x G
  double* vk = tsm;                       // v_k by global index
  double* vn = tsm + n;                   // v_{k+1}
  double* const w = tsm + 2 * n;          // w_k
  double* const red0 = tsm + 3 * n;
  double* const red1 = red0 + TNW;
  unsigned gen = 0;

  if (n <= 2) {
    if (c == 0 && threadIdx.x == 0) {
      P.d[0] = A[0];
      if (n == 2) { P.e[0] = A[1]; P.d[1] = A[3]; }
    }
    return;
  }
  // ---- phase -1: v_0 from row 0, p_0 over own rows
  for (int j = threadIdx.x; j < n; j += TNT) vn[j] = (j >= 1) ? A[j] : 0.0;
  __syncthreads();
  double tau_k, beta;
  house(vn, 1, n, red0, tau_k, beta);
  if (c == 0) {
    if (threadIdx.x == 0) { P.d[0] = A[0]; P.e[0] = beta; P.tau[0] = tau_k; }
    for (int j = 2 + threadIdx.x; j < n; j += TNT) A[j] = vn[j];
  }
  {
    double pv = 0.0;
    const int i0 = 1 + ((c - 1) % G + G) % G;   // smallest own row >= 1
    for (int i = i0 + G * warp; i < n; i += G * TNW) {
      const double* Ai = A + (int64_t)i * n;
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
  if (GRID) { if (!grid_sync(bar, gen)) return; } else __syncthreads();

  // ---- phases 0 .. n-3
  for (int k = 0; k <= n - 3; ++k) {
    const int b = k & 1, nb = b ^ 1;
    const double* pk = xp + b * n;
    const double* rk = xr + b * n;
    // p_k . v_k from the CTAs' partials, fixed order (every warp alike)
    double s = 0.0;
    for (int q = lane; q < G; q += 32) s += __ldcg(xv + b * G + q);
    s = warp_sum(s);
    const double K = 0.5 * tau_k * s;
    const double wk1 = __ldcg(pk + k + 1) - K;          // w_k at k+1 (v_k[k+1] = 1)
    const bool owner = ((k + 1) % G) == c;
    for (int j = k + 1 + threadIdx.x; j < n; j += TNT) {
      const double wj = fma(-K, vk[j], __ldcg(pk + j));
      w[j] = wj;
      // row k+1 of the updated matrix: r_j = a_j - w_j - w_{k+1} v_j
      const double r = fma(-wk1, vk[j], __ldcg(rk + j) - wj);
      if (j == k + 1) {
        if (owner) P.d[k + 1] = r;
      } else {
        vn[j] = r;
      }
    }
    __syncthreads();
    const bool more = (k + 1 <= n - 3);
    double tau_n = 0.0;
    if (more) {
      house(vn, k + 2, n, (k & 1) ? red1 : red0, tau_n, beta);
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
        double* Ai = A + (int64_t)i * n;
        const double vi = vk[i], wi = w[i];
        double acc = 0.0;
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
    const double sp = block_sum(lane == 0 ? pv : 0.0, (k & 1) ? red0 : red1);
    if (threadIdx.x == 0) xv[nb * G + c] = sp;
    { double* t = vk; vk = vn; vn = t; }
    tau_k = tau_n;
    if (GRID) { if (!grid_sync(bar, gen)) return; } else __syncthreads();
  }
}

// ---------------------------------------------------------------- stage 2
// Sturm count: the number of eigenvalues of T below x, from the signs of the
// pivots of the LDL^T factorization of T - x I (q_0 = d_0 - x,
// q_i = d_i - x - e_{i-1}^2 / q_{i-1}); a pivot smaller than pivmin in
// magnitude is replaced by -pivmin (Kahan's safeguard).
__device__ __forceinline__ int sturm_count(const double* d, const double* e2, int n, double x,
                                           double pivmin) {
  int cnt = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  cnt += (q < 0.0);
  for (int i = 1; i < n; ++i) {
    q = (d[i] - x) - e2[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    cnt += (q < 0.0);
  }
  return cnt;
}

// One warp per eigenvalue.  Multisection: each round the 32 lanes count at
// 32 interior points of [lo, hi] and the interval shrinks to the sub-interval
// that holds eigenvalue number a (ascending), ~5 bits a round, until its width
// is below 2 eps ||T|| (the accuracy of the counts).
constexpr int BNW = 8;   // warps (eigenvalues) per CTA
__global__ void __launch_bounds__(BNW * 32) k_bisect(const EigProblem* probs) {
  extern __shared__ __align__(16) double bsm[];
  const EigProblem P = probs[blockIdx.y];
  const int n = P.n;
  if ((int)blockIdx.x * BNW >= n) return;
  double* d = bsm;
  double* e2 = bsm + n;
  __shared__ double s_lo[BNW * 32], s_hi[BNW * 32], s_piv[BNW * 32];
  double glo = INFINITY, ghi = -INFINITY, emax = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double di = P.d[i];
    const double el = (i > 0) ? fabs(P.e[i - 1]) : 0.0;
    const double er = (i < n - 1) ? fabs(P.e[i]) : 0.0;
    d[i] = di;
    if (i < n - 1) e2[i] = er * er;
    glo = fmin(glo, di - el - er);
    ghi = fmax(ghi, di + el + er);
    emax = fmax(emax, er * er);
  }
  s_lo[threadIdx.x] = glo;
  s_hi[threadIdx.x] = ghi;
  s_piv[threadIdx.x] = emax;
  __syncthreads();
  for (int i = 0; i < BNW * 32; ++i) {
    glo = fmin(glo, s_lo[i]);
    ghi = fmax(ghi, s_hi[i]);
    emax = fmax(emax, s_piv[i]);
  }
  const double tnorm = fmax(fabs(glo), fabs(ghi));
  const double pivmin = DBL_MIN * fmax(1.0, emax);
  const double atol = 2.0 * DBL_EPSILON * tnorm;
  glo -= 2.0 * DBL_EPSILON * tnorm * n + pivmin;
  ghi += 2.0 * DBL_EPSILON * tnorm * n + pivmin;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * BNW + warp;          // descending index
  if (j >= n) return;
  const int a = n - 1 - j;                        // ascending index
  double lo = glo, hi = ghi;
  for (int round = 0; round < 16 && hi - lo > atol; ++round) {
    const double x = lo + (hi - lo) * ((double)(lane + 1) / 33.0);
    const int cnt = sturm_count(d, e2, n, x, pivmin);
    const unsigned above = __ballot_sync(0xffffffffu, cnt > a);
    const int m = above ? (__ffs(above) - 1) : 32;
    const double xm = __shfl_sync(0xffffffffu, x, m < 32 ? m : 31);
    const double xl = __shfl_sync(0xffffffffu, x, m > 0 ? m - 1 : 0);
    if (m < 32) hi = xm;
    if (m > 0) lo = xl;
  }
  if (lane == 0) P.w[j] = 0.5 * (lo + hi);
}

// ---------------------------------------------------------------- stage 4
// Inverse iteration, one thread per wanted eigenvector: Gaussian elimination
// with partial pivoting of T - lambda I (a tridiagonal; U gets a second
// superdiagonal from the row swaps), then two solves, the first from a
// pseudo-random right-hand side, each followed by normalization.  Pivots
// below eps ||T|| are raised to that size (the shift is an eigenvalue, so
// one pivot is ~0); a running power-of-two rescale keeps the back
// substitution finite.  Output column j of Z (n x R, row-major: Z[i*R + j]).
__device__ __forceinline__ double hash_unit(uint32_t i, uint32_t j) {
  uint32_t h = i * 0x9E3779B1u ^ (j + 0x7F4A7C15u) * 0x85EBCA77u;
  h ^= h >> 15; h *= 0x2C1B3C6Du; h ^= h >> 12; h *= 0x297A2D39u; h ^= h >> 15;
  return (double)h * (2.0 / 4294967296.0) - 1.0;
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
  double* U0 = P.lu;
  double* U1 = U0 + (int64_t)n * R;
  double* U2 = U1 + (int64_t)n * R;
  double* M = U2 + (int64_t)n * R;
  unsigned char* flag = reinterpret_cast<unsigned char*>(M + (int64_t)n * R);
  unsigned char* scnt = flag + (int64_t)n * R;
  double* Z = P.z;
  auto at = [&](int k) { return (int64_t)k * R + j; };
  // ||T||_1 bound for the pivot floor
  double tn = 0.0;
  for (int i = 0; i < n; ++i) {
    const double r = fabs(P.d[i]) + (i > 0 ? fabs(P.e[i - 1]) : 0.0) + (i < n - 1 ? fabs(P.e[i]) : 0.0);
    tn = fmax(tn, r);
  }
  const double ptol = fmax(DBL_EPSILON * tn, DBL_MIN);
  // factor
  double p0 = P.d[0] - lam, p1 = (n > 1) ? P.e[0] : 0.0;
  for (int k = 0; k + 1 < n; ++k) {
    const double ek = P.e[k];
    const double a1 = P.d[k + 1] - lam;
    const double e1 = (k + 2 < n) ? P.e[k + 1] : 0.0;
    if (fabs(p0) >= fabs(ek)) {
      if (fabs(p0) < ptol) p0 = (p0 < 0.0) ? -ptol : ptol;
      const double m = ek / p0;
      U0[at(k)] = p0; U1[at(k)] = p1; U2[at(k)] = 0.0; M[at(k)] = m; flag[at(k)] = 0;
      p0 = fma(-m, p1, a1);
      p1 = e1;
    } else {
      const double m = p0 / ek;
      U0[at(k)] = ek; U1[at(k)] = a1; U2[at(k)] = e1; M[at(k)] = m; flag[at(k)] = 1;
      p0 = fma(-m, a1, p1);
      p1 = -m * e1;
    }
  }
  if (fabs(p0) < ptol) p0 = (p0 < 0.0) ? -ptol : ptol;
  U0[at(n - 1)] = p0;
  const double BIG = 0x1p+600, SMALL = 0x1p-600;
  double bscale = 1.0;
  for (int it = 0; it < 2; ++it) {
    // forward elimination of the right-hand side b (random, then the
    // previous solution times bscale), y into Z
    double pb = (it == 0) ? hash_unit(0, j) : Z[at(0)] * bscale;
    for (int k = 0; k + 1 < n; ++k) {
      const double bk1 = (it == 0) ? hash_unit(k + 1, j) : Z[at(k + 1)] * bscale;
      const double m = M[at(k)];
      double yk;
      if (flag[at(k)] == 0) { yk = pb; pb = fma(-m, pb, bk1); }
      else { yk = bk1; pb = fma(-m, bk1, pb); }
      Z[at(k)] = yk;
    }
    Z[at(n - 1)] = pb;
    // back substitution with rescaling; scnt[i] = rescales before z_i was stored
    int nres = 0;
    double sc = 1.0;             // 2^(-600 nres): the scale of z1, z2 and zk
    double z1 = 0.0, z2 = 0.0;   // z_{k+1}, z_{k+2} at the current scale
    for (int k = n - 1; k >= 0; --k) {
      double r = Z[at(k)] * sc;
      if (k + 1 < n) r = fma(-U1[at(k)], z1, r);
      if (k + 2 < n) r = fma(-U2[at(k)], z2, r);
      double zk = r / U0[at(k)];
      if (fabs(zk) > BIG) {   // scale everything from here on down by 2^-600
        zk *= SMALL; z1 *= SMALL; z2 *= SMALL; sc *= SMALL;
        ++nres;
      }
      Z[at(k)] = zk;
      scnt[at(k)] = (unsigned char)(nres > 255 ? 255 : nres);
      z2 = z1;
      z1 = zk;
    }
    // bring all entries to the final scale and normalize
    double ss = 0.0;
    for (int k = 0; k < n; ++k) {
      double zk = Z[at(k)];
      for (int q = scnt[at(k)]; q < nres; ++q) zk *= SMALL;
      Z[at(k)] = zk;
      ss = fma(zk, zk, ss);
    }
    bscale = (ss > 0.0) ? 1.0 / sqrt(ss) : 1.0;
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
// U = Q_H Z with Q_H = H_0 H_1 ... H_{n-3}: the reflectors applied from the
// last to the first; one warp per vector, the vector in shared memory.
// U is I x R column-major.
__global__ void k_backtransform(const EigProblem* probs, int nprob, int warps_per_cta,
                                int zstride) {
  extern __shared__ __align__(16) double zsm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x * warps_per_cta + warp;   // flattened (problem, vector)
  int p = 0;
  while (p + 1 < nprob && probs[p + 1].zoff <= t) ++p;
  const EigProblem P = probs[p];
  const int j = t - P.zoff;
  if (j < 0 || j >= P.R || *P.info) return;
  const int n = P.n, R = P.R;
  double* z = zsm + (size_t)warp * zstride;
  for (int i = lane; i < n; i += 32) z[i] = P.z[(int64_t)i * R + j];
  __syncwarp();
  for (int k = n - 3; k >= 0; --k) {
    const double tau = P.tau[k];
    if (tau == 0.0) continue;
    const double* vrow = P.A + (int64_t)k * n;   // v_k[k+1] = 1, v_k[i] = A[k][i] for i >= k+2
    double s = 0.0;
    for (int i = k + 2 + lane; i < n; i += 32) s = fma(vrow[i], z[i], s);
    s = warp_sum(s);
    const double f = tau * (z[k + 1] + s);
    __syncwarp();
    if (lane == 0) z[k + 1] -= f;
    for (int i = k + 2 + lane; i < n; i += 32) z[i] = fma(-f, vrow[i], z[i]);
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) P.U[(int64_t)j * n + i] = z[i];
}

// ---------------------------------------------------------------- launchers
size_t tridiag_smem_bytes(int n) { return sizeof(double) * (3 * (size_t)n + 2 * TNW); }

cudaError_t launch_tridiag(const EigProblem* probs_dev, int count, int nmax, bool grid,
                           int num_sms, GridBarrier bar, cudaStream_t st) {
  const size_t smem = tridiag_smem_bytes(nmax);
  cudaError_t e;
  if (grid) {
    e = cudaFuncSetAttribute(k_tridiag<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tridiag<true>, TNT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorLaunchOutOfResources;
    // ~4 rows per CTA at the first step, at most one CTA per SM
    int G = (nmax + 3) / 4;
    if (G > num_sms) G = num_sms;
    if (G < 1) G = 1;
    void* args[] = {(void*)&probs_dev, (void*)&bar};
    e = cudaLaunchCooperativeKernel((void*)k_tridiag<true>, dim3(G), dim3(TNT), args, smem, st);
    count_launches(1);
    return e;
  }
  e = cudaFuncSetAttribute(k_tridiag<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_tridiag<false><<<count, TNT, smem, st>>>(probs_dev, bar);
  count_launches(1);
  return cudaGetLastError();
}

int tridiag_team_size(int n, int num_sms) {
  int G = (n + 3) / 4;
  return G > num_sms ? num_sms : (G < 1 ? 1 : G);
}

cudaError_t launch_bisect(const EigProblem* probs_dev, int count, int nmax, cudaStream_t st) {
  const size_t smem = sizeof(double) * 2 * (size_t)nmax;
  cudaError_t e = cudaFuncSetAttribute(k_bisect, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_bisect<<<dim3((nmax + BNW - 1) / BNW, count), BNW * 32, smem, st>>>(probs_dev);
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

cudaError_t launch_backtransform(const EigProblem* probs_dev, int count, int total_vectors,
                                 int nmax, cudaStream_t st) {
  if (total_vectors < 1) return cudaSuccess;
  int wpc = (int)((96 * 1024) / (sizeof(double) * (size_t)nmax));
  if (wpc > 8) wpc = 8;
  if (wpc < 1) wpc = 1;
  const size_t smem = sizeof(double) * (size_t)nmax * wpc;
  cudaError_t e = cudaFuncSetAttribute(k_backtransform, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_backtransform<<<(total_vectors + wpc - 1) / wpc, wpc * 32, smem, st>>>(probs_dev, count, wpc,
                                                                          nmax);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace tk
