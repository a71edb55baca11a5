// Launchers of the device kernels (internal to the library).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "tucker_gb300.h"
#include "common.cuh"

namespace tk {

// ---- FP64 sum of squares: partial per block, then a fixed-order reduction
cudaError_t launch_sumsq(const void* y, tucker_dtype dt, int64_t n, double* partial, int nblocks,
                         unsigned* nonfinite, double* out, cudaStream_t st);

// The same over the column-major I0 x ncols mode-0 view, also recording each
// row's max |x| as FP32 bits (atomicMax into the zeroed rowmax_bits[I0]);
// I0 <= 8192, 4-byte aligned y (16-byte loads when I0 % 4 == 0 and y is
// 16-byte aligned)
cudaError_t launch_sumsq_rowmax(const float* y, int64_t I0, int64_t ncols, double* partial,
                                int nblocks, unsigned* nonfinite, unsigned* rowmax_bits, double* out,
                                cudaStream_t st);

// ---- b[i] += a[i] over n FP64 values (sums of Grams computed in pieces)
cudaError_t launch_add_f64(const double* a, double* b, int64_t n, int num_sms, cudaStream_t st);

// ---- SIMT Gram (FP64 or FP32 products), split-K partial tiles + reduction
struct GramPlan {
  int ntiles = 0, ksplit = 0;
  int ksplit_diag = 0;   // plan_gram_f32: K splits of a diagonal tile (ksplit: off-diagonal)
  int nctas = 0;         // plan_gram_f32: CTAs (= partial tiles)
  size_t scratch_bytes = 0;
};
// ---- tensor-core Gram of a slab view on exact digit products
// (gram_tcx.cu): plan.nctas == 0 when it does not apply (I <= 4096;
// column mode 64 <= I, row mode 128 <= I;
// column mode L == 1 (16-byte loads when I % 4 == 0 and y is 16-byte aligned,
// else 4-byte loads); row mode L > 1 with l-blocks of 16 at
// most 25 % zero fill); rowmax_bits: FP32 bits of the row maxima, from
// launch_sumsq_rowmax (column mode) or launch_rowmax_slab (row mode)
GramPlan plan_gram_tcx(int64_t L, int64_t I, int64_t Rt, int num_sms);
// ndig: 3 (three 7-bit digits, all nine products) or 2 (two digits, four
// products; representation error 2^-13 instead of 2^-20 of the row maximum)
cudaError_t launch_gram_tcx(const float* y, int64_t L, int64_t I, int64_t Rt, const GramPlan& p,
                            const unsigned* rowmax_bits, void* scratch, unsigned* err, double* S,
                            cudaStream_t st, int ndig);
cudaError_t launch_rowmax_slab(const float* y, int64_t L, int64_t I, int64_t Rt, int num_sms,
                               unsigned* rowmax_bits, cudaStream_t st);

// L0: the fastest sub-index of l (the first dim of the tensor for a mode
// n > 0); row-mode K-blocks never cross a multiple of it
GramPlan plan_gram_simt(int64_t L, int64_t I, int64_t Rt, int num_sms, int64_t L0);
GramPlan plan_gram_simt_capped(int64_t L, int64_t I, int64_t Rt, int num_sms, size_t max_bytes,
                               int* ok, int64_t L0);
cudaError_t launch_gram_simt(const void* y, tucker_dtype dt, bool fp64, int64_t L, int64_t I,
                             int64_t Rt, int64_t L0, const GramPlan& p, double* scratch, double* S,
                             cudaStream_t st);

// ---- FP32-product Gram of FP32 input, I >= 64: 128 x 128 tiles, cp.async
// pipeline; plan.ntiles == 0 when it does not apply
GramPlan plan_gram_f32(int64_t L, int64_t I, int64_t Rt, int num_sms, int64_t L0);
// Whether launch_gram_f32 runs its compensated (exact block sums) variant:
// row-mode views with fewer than 4096 slabs
int gram_f32_compensated(int64_t L, int64_t Rt);
cudaError_t launch_gram_f32(const float* y, int64_t L, int64_t I, int64_t Rt, int64_t L0,
                            const GramPlan& p, double* scratch, double* S, cudaStream_t st);

// ---- Gram of a small mode (I < 64) in FP64 (products of FP32 inputs are
// exact), for every precision; plan.nctas == 0 when it does not apply
GramPlan plan_gram_small(int64_t L, int64_t I, int64_t Rt, int num_sms, int64_t L0);
cudaError_t launch_gram_small(const void* y, tucker_dtype dt, int64_t L, int64_t I, int64_t Rt,
                              int64_t L0, const GramPlan& p, double* scratch, double* S,
                              cudaStream_t st);

// ---- SIMT TTM
// a32_scratch: K * I floats for the FP32 copy of A (FP32 arithmetic), or NULL
// zt (column mode only): Z written transposed, z[slab + Rt k] (the new mode last)
cudaError_t launch_ttm_simt(const void* y, tucker_dtype ydt, bool fp64, int64_t L, int64_t I,
                            int64_t Rt, const double* A, int64_t K, int64_t lda, int a_rowmajor,
                            float* a32_scratch, void* z, tucker_dtype zdt, cudaStream_t st,
                            bool zt = false);

// ---- tensor-core (tcgen05) Gram and TTM on the FP16 hi/lo split
struct TcGramPlan {
  int ok = 0;
  int64_t ntiles = 0, nsplit = 0;
  size_t scratch_bytes = 0;
};
TcGramPlan plan_gram_tc(int64_t L, int64_t I, int64_t Rt, int num_sms);
cudaError_t launch_gram_tc(const float* y, int64_t L, int64_t I, int64_t Rt, const TcGramPlan& p,
                           float scale, double* scratch, unsigned* err, double* S, cudaStream_t st);
// TTM of the column-major mode-0 view (L == 1, I % 4 == 0, K <= 128); sy =
// power-of-two scale of y with max|y sy| <= 2^14
int ttm_tc_supported(int64_t L, int64_t I, int64_t Rt, int64_t K);
cudaError_t launch_ttm_tc(const float* y, int64_t L, int64_t I, int64_t Rt, const double* A,
                          int64_t K, int64_t lda, int a_rowmajor, float sy, float* z, bool zt,
                          void* scratch, unsigned* err, int num_sms, cudaStream_t st);
size_t ttm_tc_scratch_bytes(int64_t I, int64_t K);
// row-mode views (L > 1, L % 4 == 0, I <= 64, K <= 1024): Z(l, k, r) =
// sum_i A(k, i) Y(l, i, r), z[l + L (k + K r)] (ttm_tc.cu)
int ttm_tc_row_supported(int64_t L, int64_t I, int64_t Rt, int64_t K);
size_t ttm_tc_row_scratch_bytes(int64_t K);
cudaError_t launch_ttm_tc_row(const float* y, int64_t L, int64_t I, int64_t Rt, const double* A,
                              int64_t K, int64_t lda, int a_rowmajor, float sy, float* z,
                              void* scratch, unsigned* err, int num_sms, cudaStream_t st);

// ---- Jacobi eigensolver, sort and rank cut
size_t jacobi_work_bytes(int n);
cudaError_t launch_jacobi(const double* S, int n, double* work, const double* fro2, unsigned* words,
                          int max_sweeps, double tol_rel, double tol_abs, int num_sms,
                          double* w_out, double* V_out, int* info_dev, cudaStream_t st,
                          unsigned long long poll_limit);
cudaError_t launch_eig_finish(int n, double* work, const int* info_host, int* info_dev,
                              double* w_out, double* V_out, cudaStream_t st);
cudaError_t launch_rank_cut(const double* w, int n, double thr, int fixed_R, int64_t* out_R,
                            double* out_d, double* tail, cudaStream_t st);

// ---- tridiagonal eigensolver (tridiag.cu): all eigenvalues, the leading R
// eigenvectors.  One descriptor per matrix (device array of descriptors).
struct EigProblem {
  double* A;      // n x n row-major symmetric input copy; overwritten with the reflectors
  double* d;      // n: diagonal of T
  double* e;      // n: off-diagonal of T (e[k] = T[k+1][k])
  double* tau;    // n: reflector scalars
  double* xch;    // 4 n + 2 G: exchange buffers of the team reduction (G CTAs)
  double* w;      // n: eigenvalues, descending
  double* z;      // n x R row-major: eigenvectors of T, then their QR factor
  double* lu;     // inverse-iteration factors: 4 n R doubles + 2 n R bytes
  double* gram;   // R x R
  double* U;      // n x R column-major output
  double* wyT;    // eig_wy_doubles(n): T factors of the blocked back-transformation
  int* info;      // 0 ok; 1 / 2 the Cholesky QR failed (see k_chol)
  int n, R;
  int zoff;       // first flattened vector index of this problem
  int roff;       // first flattened row index of this problem
  int team_off;   // k_tridiag: first CTA of this problem's team
  int team_size;  // k_tridiag: CTAs of the team (xch holds 4 n + 2 team_size)
  int srows;      // k_tridiag: the team's rows live in shared memory
};
int tridiag_team_size(int n, int num_sms);
// Team sizes for a batch: 1 CTA each plus the remaining SMs shared in
// proportion to n^3; all 1 when count >= num_sms.
void tridiag_batch_teams(const int* n, int count, int num_sms, int* team);
inline size_t eig_lu_bytes(int n, int R) { return (size_t)n * R * (4 * sizeof(double) + 2); }
size_t eig_wy_doubles(int n);
// Problems with their team_off / team_size set (teams back to back) and
// team_size * n / ... as planned; probs_host is the host copy of the
// descriptors (it sets the launch shape and each team's shared-memory rows).
// bar_counts: `count` zeroed words (one barrier per team), err: error word.
// poll_limit: polls before a team's grid barrier gives up (sets *err)
cudaError_t launch_tridiag(const EigProblem* probs_dev, EigProblem* probs_host, int count,
                           unsigned* bar_counts, unsigned* err, cudaStream_t st,
                           unsigned long long poll_limit);
// y[i] = the tridiagonal solver's FP64 reciprocal of x[i] (diagnostics)
cudaError_t launch_rcp64_probe(const double* x, double* y, int64_t n, cudaStream_t st);
// total_eigs: the sum of n over the problems (sets the lanes per eigenvalue)
cudaError_t launch_bisect(const EigProblem* probs_dev, int count, int nmax, int total_eigs,
                          int num_sms, cudaStream_t st);
cudaError_t launch_invit(const EigProblem* probs_dev, int count, int total_vectors, cudaStream_t st);
cudaError_t launch_chol(const EigProblem* probs_dev, int count, cudaStream_t st);
cudaError_t launch_trsm_rows(const EigProblem* probs_dev, int count, int total_rows, cudaStream_t st);
cudaError_t launch_backtransform(const EigProblem* probs_dev, int count, int total_vectors,
                                 int nmax, cudaStream_t st);
// batched rank cut (thr[p], fixed[p] > 0 or NULL) and Z^T Z for problems with R <= 64
cudaError_t launch_rank_cut_batched(const EigProblem* probs_dev, int count, const double* thr,
                                    const int* fixed, int64_t* R_out, double* disc_out,
                                    cudaStream_t st);
int zgram_batched_max_r();
cudaError_t launch_zgram_batched(const EigProblem* probs_dev, int count, cudaStream_t st);

// ---- pre- and post-processing of Section 3.5 (prepost.cu)
// Statistics of every hyperslice of the slab view (Rt, I, L): stats[6 i + k]
// = mean, population standard deviation, max, min, 1-norm, 2-norm (FP64);
// work: slice_stats_work_bytes(I); *bad |= 1 when a statistic is not finite
size_t slice_stats_work_bytes(int64_t I);
cudaError_t launch_slice_stats(const void* x, tucker_dtype dt, int64_t L, int64_t I, int64_t Rt,
                               void* work, double* stats, unsigned* bad, int num_sms,
                               cudaStream_t st);
// shift/scale of a method (0 standardization, 1 max rescaling) from stats
cudaError_t launch_slice_params(const double* stats, int64_t I, int method, double* shift,
                                double* scale, cudaStream_t st);
// y = (x - shift_i) * scale_i, or (inverse) x / scale_i + shift_i; y may be x
cudaError_t launch_slice_apply(const void* x, tucker_dtype dt, int64_t L, int64_t I, int64_t Rt,
                               const double* shift, const double* scale, int inverse, void* y,
                               int num_sms, cudaStream_t st);

}  // namespace tk
