// FP64 symmetric eigensolver (Section 5.2 of the TuckerMPI paper computes all
// eigenpairs of the I_n x I_n Gram matrix; this is a parallel cyclic Jacobi
// method instead of LAPACK's syev) plus the descending sort and the eps rank
// cut of Eq. Un.
//
// Parallel ordering: the round-robin ("circle") tournament.  Storage is kept
// permuted so that the pairs of the current step always sit at positions
// (2j, 2j+1); every step writes the rotated matrix into the other buffer at
// the positions of the next step's pairing, so all pairs of a step are
// disjoint 2x2 blocks and every 2x2 block of A updates independently.
// A and V are permuted together, so column p of V always belongs to the
// diagonal entry p of A.  One persistent cooperative kernel runs every
// sweep; a bounded grid barrier separates the rotation and update phases.
#include "common.cuh"
#include "kernels.h"

namespace tk {

__device__ __forceinline__ int slot_of_pos(int pos, int np) {
  int k = pos >> 1;
  return (pos & 1) ? (np - 1 - k) : k;
}
__device__ __forceinline__ int pos_of_slot(int s, int np) {
  return (s < (np >> 1)) ? (2 * s) : (2 * (np - 1 - s) + 1);
}
// Storage position at the next step of the element now at `pos`.
__device__ __forceinline__ int next_pos(int pos, int np) {
  int s = slot_of_pos(pos, np);
  int ns = (s == 0) ? 0 : (s % (np - 1)) + 1;
  return pos_of_slot(ns, np);
}

struct JacobiArgs {
  double* A[2];       // np x np row-major, ping-pong
  double* V[2];       // n x np row-major (rows: coordinates, cols: storage positions)
  double* rot;        // 3 * P: c, s, t
  unsigned* counts;   // non-skipped rotations per sweep (max_sweeps entries, zeroed)
  int* info;          // [0] sweeps, [1] converged, [2] final buffer, [3] dummy position
  const double* fro2; // ||S||_F^2
  GridBarrier bar;
  int n, np, max_sweeps;
  double tol_rel, tol_abs;
};

__global__ void __launch_bounds__(256) k_jacobi(JacobiArgs a) {
  const int n = a.n, np = a.np, P = np >> 1;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gsz = (int64_t)gridDim.x * blockDim.x;
  const double floor_abs = a.tol_abs * sqrt(*a.fro2);
  const int64_t nblk = (int64_t)P * (P + 1) / 2;
  const int64_t nvit = (int64_t)n * P;
  unsigned gen = 0;
  int cur = 0;
  int dpos = (n & 1) ? n : -1;   // dummy index (odd n) sits at position n initially
  int sweeps = 0, converged = 0;
  for (int sweep = 0; sweep < a.max_sweeps; ++sweep) {
    for (int t = 0; t < np - 1; ++t) {
      const double* A = a.A[cur];
      double* An = a.A[cur ^ 1];
      const double* V = a.V[cur];
      double* Vn = a.V[cur ^ 1];
      // phase 1: one rotation per pair (sym.schur2 of Golub & Van Loan)
      for (int64_t j = gtid; j < P; j += gsz) {
        const int p = 2 * (int)j, q = p + 1;
        const double app = A[(int64_t)p * np + p], aqq = A[(int64_t)q * np + q];
        const double apq = A[(int64_t)p * np + q];
        double c = 1.0, s = 0.0, tt = 0.0;
        const double thr = fmax(a.tol_rel * sqrt(fabs(app)) * sqrt(fabs(aqq)), floor_abs);
        if (fabs(apq) > thr) {
          const double tau = (aqq - app) / (2.0 * apq);
          tt = (tau >= 0.0) ? 1.0 / (tau + sqrt(1.0 + tau * tau))
                            : -1.0 / (-tau + sqrt(1.0 + tau * tau));
          c = 1.0 / sqrt(1.0 + tt * tt);
          s = tt * c;
          atomicAdd(&a.counts[sweep], 1u);
        }
        a.rot[3 * j] = c;
        a.rot[3 * j + 1] = s;
        a.rot[3 * j + 2] = tt;
      }
      if (!grid_sync(a.bar, gen)) return;
      // phase 2a: 2x2 blocks (ja <= jb) of A' = J^T A J, written permuted
      for (int64_t it = gtid; it < nblk; it += gsz) {
        int jb = (int)((sqrtf(8.f * (float)it + 1.f) - 1.f) * 0.5f);
        while ((int64_t)(jb + 1) * (jb + 2) / 2 <= it) ++jb;
        while ((int64_t)jb * (jb + 1) / 2 > it) --jb;
        const int ja = (int)(it - (int64_t)jb * (jb + 1) / 2);
        const int pa = 2 * ja, pb = 2 * jb;
        const int na0 = next_pos(pa, np), na1 = next_pos(pa + 1, np);
        const int nb0 = next_pos(pb, np), nb1 = next_pos(pb + 1, np);
        const double a00 = A[(int64_t)pa * np + pb], a01 = A[(int64_t)pa * np + pb + 1];
        const double a10 = A[(int64_t)(pa + 1) * np + pb], a11 = A[(int64_t)(pa + 1) * np + pb + 1];
        if (ja == jb) {
          const double s = a.rot[3 * ja + 1], tt = a.rot[3 * ja + 2];
          double d0 = a00, d1 = a11, off = a01;
          if (s != 0.0) { d0 = a00 - tt * a01; d1 = a11 + tt * a01; off = 0.0; }
          An[(int64_t)na0 * np + na0] = d0;
          An[(int64_t)na1 * np + na1] = d1;
          An[(int64_t)na0 * np + na1] = off;
          An[(int64_t)na1 * np + na0] = off;
        } else {
          const double ca = a.rot[3 * ja], sa = a.rot[3 * ja + 1];
          const double cb = a.rot[3 * jb], sb = a.rot[3 * jb + 1];
          const double r00 = ca * a00 - sa * a10, r01 = ca * a01 - sa * a11;
          const double r10 = sa * a00 + ca * a10, r11 = sa * a01 + ca * a11;
          const double n00 = r00 * cb - r01 * sb, n01 = r00 * sb + r01 * cb;
          const double n10 = r10 * cb - r11 * sb, n11 = r10 * sb + r11 * cb;
          An[(int64_t)na0 * np + nb0] = n00; An[(int64_t)nb0 * np + na0] = n00;
          An[(int64_t)na0 * np + nb1] = n01; An[(int64_t)nb1 * np + na0] = n01;
          An[(int64_t)na1 * np + nb0] = n10; An[(int64_t)nb0 * np + na1] = n10;
          An[(int64_t)na1 * np + nb1] = n11; An[(int64_t)nb1 * np + na1] = n11;
        }
      }
      // phase 2b: V' = V J, columns written permuted
      for (int64_t it = gtid; it < nvit; it += gsz) {
        const int64_t i = it / P;
        const int j = (int)(it - i * P);
        const double c = a.rot[3 * j], s = a.rot[3 * j + 1];
        const double v0 = V[i * np + 2 * j], v1 = V[i * np + 2 * j + 1];
        Vn[i * np + next_pos(2 * j, np)] = c * v0 - s * v1;
        Vn[i * np + next_pos(2 * j + 1, np)] = s * v0 + c * v1;
      }
      if (dpos >= 0) dpos = next_pos(dpos, np);
      cur ^= 1;
      if (!grid_sync(a.bar, gen)) return;
    }
    sweeps = sweep + 1;
    if (ld_acquire_u32(&a.counts[sweep]) == 0u) { converged = 1; break; }
  }
  if (gtid == 0) {
    a.info[0] = sweeps;
    a.info[1] = converged;
    a.info[2] = cur;
    a.info[3] = dpos;
  }
}

// Padded copy S (n x n) -> A (np x np) and V = [I | 0] (n x np).
__global__ void k_jacobi_init(const double* __restrict__ S, int n, int np, double* __restrict__ A,
                              double* __restrict__ V) {
  int64_t tot = (int64_t)np * np;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / np, j = e % np;
    A[e] = (i < n && j < n) ? S[i * n + j] : 0.0;
    if (i < n) V[i * np + j] = (i == j) ? 1.0 : 0.0;
  }
}

// Ranks eigenvalues (descending; ties by position) and writes them out.
__global__ void __launch_bounds__(1024) k_eig_rank(const double* __restrict__ A, int n, int np,
                                                   const int* __restrict__ info,
                                                   int* __restrict__ rank, double* __restrict__ w) {
  const int dpos = info[3];
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    if (p == dpos) { rank[p] = -1; continue; }
    const double lp = A[(int64_t)p * np + p];
    int r = 0;
    for (int q = 0; q < np; ++q) {
      if (q == dpos || q == p) continue;
      const double lq = A[(int64_t)q * np + q];
      r += (lq > lp) || (lq == lp && q < p);
    }
    rank[p] = r;
    w[r] = lp;
  }
}

// V_out (n x n column-major) column rank[p] = V column p.
__global__ void k_eig_gather(const double* __restrict__ V, int n, int np, const int* __restrict__ rank,
                             double* __restrict__ Vout) {
  int64_t tot = (int64_t)n * np;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / np;
    int p = (int)(e % np);
    int r = rank[p];
    if (r >= 0) Vout[i + (int64_t)n * r] = V[e];
  }
}

// Eq. Un: R = min{R in 1..n : sum_{i>=R} max(w_i, 0) <= thr}; the tail is
// accumulated from the smallest eigenvalue up.  out_R[0] = R, out_d[0] = tail(R).
// With fixed_R > 0 the rank is given (rank-specified variant) and only the
// discarded tail is computed.
__global__ void k_rank_cut(const double* __restrict__ w, int n, double thr, int fixed_R,
                           int64_t* out_R, double* out_d, double* tail) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  tail[n] = 0.0;
  for (int i = n - 1; i >= 0; --i) tail[i] = tail[i + 1] + w[i];
  int R = n;
  if (fixed_R > 0) {
    R = fixed_R;
  } else {
    for (int r = 1; r <= n; ++r)
      if (tail[r] <= thr) { R = r; break; }
  }
  out_R[0] = R;
  out_d[0] = tail[R];
}

cudaError_t launch_jacobi(const double* S, int n, double* work, const double* fro2, unsigned* words,
                          int max_sweeps, double tol_rel, double tol_abs, int num_sms,
                          double* w_out, double* V_out, int* info_dev, cudaStream_t st) {
  const int np = n + (n & 1), P = np / 2;
  double* A0 = work;
  double* A1 = A0 + (size_t)np * np;
  double* V0 = A1 + (size_t)np * np;
  double* V1 = V0 + (size_t)n * np;
  double* rot = V1 + (size_t)n * np;
  // words: [0] barrier count, [1] barrier gen, [2] err, [3..] per-sweep counts
  cudaError_t e = cudaMemsetAsync(words, 0, sizeof(unsigned) * (3 + max_sweeps + 1), st);
  if (e != cudaSuccess) return e;
  k_jacobi_init<<<256, 256, 0, st>>>(S, n, np, A0, V0);
  count_launches(max_sweeps > 0 ? 2 : 1);
  JacobiArgs a;
  a.A[0] = A0; a.A[1] = A1; a.V[0] = V0; a.V[1] = V1;
  a.rot = rot;
  a.counts = words + 3;
  a.info = info_dev;
  a.fro2 = fro2;
  a.bar = GridBarrier{words, words + 1, words + 2};
  a.n = n; a.np = np; a.max_sweeps = max_sweeps;
  a.tol_rel = tol_rel; a.tol_abs = tol_abs;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi, 256, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 2) per_sm = 2;
  int64_t items = (int64_t)P * (P + 1) / 2 + (int64_t)n * P;
  int64_t want = (items + 255) / 256;
  int64_t cap = (int64_t)num_sms * per_sm;
  int grid = (int)(want < 1 ? 1 : (want > cap ? cap : want));
  if (max_sweeps > 0) {
    void* args[] = {&a};
    e = cudaLaunchCooperativeKernel((void*)k_jacobi, dim3(grid), dim3(256), args, 0, st);
    if (e != cudaSuccess) return e;
  } else {
    int h[4] = {0, 0, 0, (n & 1) ? n : -1};
    e = cudaMemcpyAsync(info_dev, h, sizeof(h), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
  }
  // the final buffer is chosen on the device: rank from both, gather from the right one
  return cudaGetLastError();
}

cudaError_t launch_eig_finish(int n, double* work, const int* info_host, int* info_dev,
                              double* w_out, double* V_out, cudaStream_t st) {
  const int np = n + (n & 1), P = np / 2;
  double* A0 = work;
  double* A1 = A0 + (size_t)np * np;
  double* V0 = A1 + (size_t)np * np;
  double* V1 = V0 + (size_t)n * np;
  double* rot = V1 + (size_t)n * np;
  int* rank = (int*)(rot + 3 * (size_t)P + 1);
  const int cur = info_host[2];
  const double* A = cur ? A1 : A0;
  const double* V = cur ? V1 : V0;
  k_eig_rank<<<1, 1024, 0, st>>>(A, n, np, info_dev, rank, w_out);
  count_launches(2);
  int64_t tot = (int64_t)n * np;
  int blocks = (int)((tot + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  k_eig_gather<<<blocks, 256, 0, st>>>(V, n, np, rank, V_out);
  return cudaGetLastError();
}

size_t jacobi_work_bytes(int n) {
  const size_t np = n + (n & 1), P = np / 2;
  return sizeof(double) * (2 * np * np + 2 * (size_t)n * np + 3 * P + 1) + sizeof(int) * (np + 4);
}

cudaError_t launch_rank_cut(const double* w, int n, double thr, int fixed_R, int64_t* out_R,
                            double* out_d, double* tail, cudaStream_t st) {
  k_rank_cut<<<1, 32, 0, st>>>(w, n, thr, fixed_R, out_R, out_d, tail);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace tk
