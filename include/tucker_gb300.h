/*
 * tucker_gb300.h -- C ABI of the GB300 (sm_103a) ST-HOSVD Tucker library.
 *
 * The library computes the hot path of sequentially truncated HOSVD
 * (Ballard, Klinvex, Kolda, "TuckerMPI", arXiv 1901.06043, Algorithm 1):
 * per mode n the Gram matrix of the mode-n unfolding (Algorithm 2), its
 * eigendecomposition (Section 5.2), the eps rank cut (Eq. Un) and the TTM
 * that shrinks the working tensor (Algorithm 3); plus the multi-TTM that
 * reconstructs a tensor or a subtensor from the core and factors (Section 7).
 *
 * Conventions used by every entry point
 * -------------------------------------
 * - Tensors are dense and stored in natural-descending order (Section 4.1,
 *   Eq. idxtolin): element (j_0, ..., j_{N-1}) of a J_0 x ... x J_{N-1}
 *   tensor sits at sum_n j_n * (J_0 * ... * J_{n-1}); the first index is
 *   fastest.  1 <= N <= TUCKER_MAX_MODES, every J_n >= 1.
 * - "_dev" pointers are CUDA device pointers of the current device; "_host"
 *   pointers are host memory.  The library never frees memory it did not
 *   allocate, and never writes through a const pointer.
 * - Every call is enqueued on the context's stream.  Calls that return a
 *   value to the host (a rank, a norm, a status that depends on device
 *   data) synchronise that stream before returning.
 * - Every entry point returns a tucker_status.  On failure nothing is
 *   freed that the caller owns, results are left undefined, and
 *   tucker_last_error() describes the failure.  No failure is reported by
 *   trapping or hanging the device: device-side checks write an error word
 *   that the host reads.
 * - Matrices of FP64 values: U_n (I_n x R_n) and eigenvector matrices are
 *   column-major; Gram matrices are symmetric I x I (either order).
 */
#ifndef TUCKER_GB300_H
#define TUCKER_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TUCKER_MAX_MODES 8

typedef enum {
  TUCKER_OK = 0,
  TUCKER_ERR_INVALID = 1,    /* bad argument: ndim, dims, eps, ranks, ranges, order, null */
  TUCKER_ERR_OOM = 2,        /* device allocation failed or predicted to fail */
  TUCKER_ERR_NONFINITE = 3,  /* NaN or Inf in the input tensor */
  TUCKER_ERR_EIG_NOCONV = 4, /* Jacobi sweep cap reached (results still written) */
  TUCKER_ERR_CUDA = 5,       /* a CUDA runtime error, or a device-side wait that gave up */
  TUCKER_ERR_UNSUPPORTED = 6 /* valid request this build cannot serve (e.g. dtype/precision pair) */
} tucker_status;

typedef enum { TUCKER_F32 = 0, TUCKER_F64 = 1 } tucker_dtype;

/* Arithmetic of the Gram and TTM steps.  The eigensolve and the rank cut
 * are FP64 in every mode, and the Gram is always reduced across slabs in
 * FP64.  In every precision a mode with I_n < 64 gets an FP64 Gram (the
 * energy of the later, small modes sits in a few components, where FP32
 * block sums do not average out), and an eps-driven tucker_sthosvd with
 * eps^2 / N < 1e-9 computes all its Grams in FP64: FP32-product Grams leave
 * up to ~1.5e-10 ||X||^2 on the discarded subspace, too close to the
 * threshold eps^2 ||X||^2 / N below that.  The result reports the kernel of
 * every step.
 *   FP64   : products and sums in FP64 (any input dtype); core in FP64.
 *   FP32   : FP32 products, round-to-nearest FP32 sums over short chunks
 *            combined exactly (TwoSum) and in FP64; working tensor and core
 *            in the input dtype.
 *   MIXED  : Grams of column-mode views with 64 <= I_n <= 4096 (row-mode
 *            views: 128 <= I_n <= 4096) on the tensor cores with exact
 *            integer digit products: each value is split under a per-row
 *            power-of-two scale into two or three 7-bit digits (exact in
 *            FP16), all digit products accumulate exactly in FP32 over
 *            windows of 2048 or 1024 columns, and the windows are summed in
 *            exact FP32 pairs; the only error is the last digit's rounding,
 *            2^-13 (two digits) or 2^-20 (three) of the row maximum,
 *            unbiased (its squared mean is removed from the diagonal).  An
 *            eps-driven tucker_sthosvd bounds that error on the discarded
 *            subspace from the row maxima, the view's size and the
 *            threshold, and takes two digits where six standard deviations
 *            stay below 1 % of eps^2 ||X||^2 / N, else three, else an FP64
 *            Gram; a single tucker_gram uses three.  Other Grams as FP32.
 *            TTMs on the tensor cores
 *            (tcgen05) with a two-term FP16 split of both operands where the
 *            shape allows (column-mode views with K <= 128; row-mode views
 *            with L % 4 == 0 and I_n <= 64, the reconstruction's expansions).
 *            In the natural mode order the working tensor is kept rotated
 *            (every TTM writes its new mode last), so every mode's Gram and
 *            TTM see a column-mode view.  FP32 input only.  The rank cut at
 *            small eps is decided by a tail sum that is ~1e-9 of the trace;
 *            the Gram needs unbiased rounding for that, while TTM rounding
 *            errors act as perturbations of the data and do not bias the
 *            next cut.
 *   TENSOR : MIXED plus the Gram of the column-major mode-0 view on tcgen05
 *            (two-term FP16 split, all four products).  The tensor-core FP32
 *            accumulator truncates toward zero, a relative bias of ~1e-7
 *            per accumulation step; safe for the rank cut when
 *            eps^2 / N >> 1e-8 (e.g. eps = 1e-2), not at eps = 1e-4. */
typedef enum {
  TUCKER_PREC_FP64 = 0,
  TUCKER_PREC_FP32 = 1,
  TUCKER_PREC_MIXED = 2,
  TUCKER_PREC_TENSOR = 3
} tucker_prec;

typedef struct tucker_ctx tucker_ctx;

/* Result of tucker_sthosvd.  All pointers are device memory owned by the
 * result and released by tucker_result_destroy. */
typedef struct tucker_result {
  int ndim;
  tucker_dtype core_dtype;
  int64_t dims[TUCKER_MAX_MODES];    /* I_n of the input                               */
  int64_t ranks[TUCKER_MAX_MODES];   /* R_n chosen (eps) or given (ranks)              */
  int mode_order[TUCKER_MAX_MODES];  /* order in which the modes were processed        */
  void* core;                        /* R_0 x ... x R_{N-1}, natural-descending        */
  double* factors[TUCKER_MAX_MODES]; /* U_n: I_n x R_n column-major, orthonormal cols  */
  double* eigvals[TUCKER_MAX_MODES]; /* all I_n eigenvalues of the mode-n Gram, desc.  */
  double norm_x_sq;                  /* ||X||^2 (FP64 sum of squares)                  */
  double threshold;                  /* eps^2 ||X||^2 / N (0 when ranks were given)    */
  double discarded_sq[TUCKER_MAX_MODES]; /* sum of discarded eigenvalues per mode      */
  int jacobi_sweeps[TUCKER_MAX_MODES];
  int gram_kernel[TUCKER_MAX_MODES]; /* kernel that ran: 0 SIMT FP64, 1 SIMT FP32, 2 tcgen05
                                        (rounded split), 3 small-mode FP64, 4 FP32 with
                                        exact block sums, 5 / 6 tcgen05 on exact three- /
                                        two-digit products */
  int ttm_kernel[TUCKER_MAX_MODES];
  int eig_kernel[TUCKER_MAX_MODES];  /* 0 Jacobi, 1 tridiagonal + inverse iteration          */
  float ms_norm;                     /* device time per step (CUDA events), ms         */
  float ms_gram[TUCKER_MAX_MODES];
  float ms_eig[TUCKER_MAX_MODES];
  float ms_ttm[TUCKER_MAX_MODES];
  float ms_total;
} tucker_result;

/* Context: a stream, a device workspace and the last error string.
 * `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  The context must be used from one host thread at a time. */
tucker_status tucker_create(tucker_ctx** ctx, void* stream);
tucker_status tucker_destroy(tucker_ctx* ctx);
const char* tucker_last_error(const tucker_ctx* ctx);

/* Options (key, value):
 *   TUCKER_OPT_TIMING      1 = record per-step CUDA-event times into results
 *   TUCKER_OPT_MAX_SWEEPS  Jacobi sweep cap (default 40; 0 = no sweep)
 *   TUCKER_OPT_JACOBI_TOL  relative off-diagonal tolerance (default 1e-15)
 *   TUCKER_OPT_EIG_SOLVER  eigensolver of the truncation step (tucker_sthosvd,
 *                          tucker_eig_trunc): 0 auto and 2: tridiagonal for
 *                          I <= 4096 (Jacobi above, and where the Cholesky
 *                          QR of the inverse-iteration vectors fails),
 *                          1 Jacobi
 *   TUCKER_OPT_BARRIER_POLLS  polls a CTA of the eigensolvers' grid barriers
 *                          (Jacobi sweeps, Householder reduction) makes
 *                          before it gives up (default 2^24, about a second
 *                          with its back-off; 1 .. 2^40).  A barrier that
 *                          gives up makes every CTA return, and the call
 *                          returns TUCKER_ERR_CUDA ("grid barrier gave up
 *                          waiting"); the context stays usable.
 *   TUCKER_OPT_MEM_LIMIT   device bytes tucker_sthosvd may hold at once
 *                          (0, the default: the device's free memory plus
 *                          what the default memory pool holds unused).
 *                          tucker_sthosvd predicts its workspace from the
 *                          mode sizes before it starts (the Gram and
 *                          eigenvector matrices, the first Gram's split-K
 *                          scratch, the first TTM output at rank 1) and, once
 *                          each rank is cut, the TTM output; a prediction
 *                          above the figure returns TUCKER_ERR_OOM before
 *                          that step launches or allocates anything.
 *   TUCKER_OPT_GRAM_DIGITS digits per value of the exact-digit Gram (MIXED):
 *                          0 (default) chooses per view (see MIXED), 2 or 3
 *                          forces that count wherever the digit Gram runs.
 *   TUCKER_OPT_AUTOTUNE    1: the K split of every Gram kernel (the number of
 *                          CTAs the split-K planners give one wave) is chosen
 *                          by timing: the first call of each (kernel, view
 *                          shape, dtype, digit count) runs the plans for 0.5,
 *                          1, 1.5 and 2 waves twice each on the context stream
 *                          (CUDA events, synchronising) and the fastest is
 *                          kept for the rest of the process, for every
 *                          context.  Results differ from the untuned ones only
 *                          by the order of the FP64 split sums.  0 (default):
 *                          one wave.
 *   TUCKER_OPT_HOST_CHUNK  bytes per piece in which tucker_sthosvd_host copies
 *                          its input (rounded to whole mode-0 columns, four at
 *                          a time); default 2^30, at least 1. */
#define TUCKER_OPT_TIMING 1
#define TUCKER_OPT_MAX_SWEEPS 2
#define TUCKER_OPT_JACOBI_TOL 3
#define TUCKER_OPT_EIG_SOLVER 4
#define TUCKER_OPT_BARRIER_POLLS 5
#define TUCKER_OPT_MEM_LIMIT 6
#define TUCKER_OPT_GRAM_DIGITS 7
#define TUCKER_OPT_AUTOTUNE 8
#define TUCKER_OPT_HOST_CHUNK 9
tucker_status tucker_set_option(tucker_ctx* ctx, int key, double value);

/* Diagnostics: number of device kernels this library has launched in the
 * process so far (all contexts).  Host only; never fails. */
uint64_t tucker_kernel_launches(void);

/* Diagnostics: number of (kernel, shape) entries the split-K autotuner has
 * cached in this process (TUCKER_OPT_AUTOTUNE).  Host only; never fails. */
int64_t tucker_autotune_entries(void);

/* Diagnostics: y_dev[i] = the FP64 reciprocal the tridiagonal eigensolver
 * uses (an FP32 seed refined by two Newton-Raphson steps, within one ulp of
 * 1/x for normal x) of x_dev[i], i < n, on `stream` (a cudaStream_t, NULL =
 * legacy default stream); synchronises it.  Errors: INVALID, CUDA. */
tucker_status tucker_selftest_rcp64(const double* x_dev, double* y_dev, int64_t n,
                                    void* stream);

/* ST-HOSVD, Algorithm 1 (Section 3.3).
 *   x_dev      input tensor (dtype, dims), read only.
 *   eps        relative accuracy; R_n = min{R in 1..I_n : sum_{i>=R} lambda_i
 *              <= eps^2 ||X||^2 / N} (Eq. Un, 0-based, inclusive; the
 *              computed eigenvalues are summed with their signs, as
 *              Algorithm 1 does).  Ignored when ranks_or_null != NULL.
 *   ranks      the core size of the rank-specified variant (Section 8.4),
 *              1 <= R_n <= I_n.
 *   mode_order permutation of 0..N-1 (NULL = 0..N-1).
 * On success *out receives a result to release with tucker_result_destroy.
 * Errors: INVALID, OOM (predicted before the first mode or before a TTM, see
 * TUCKER_OPT_MEM_LIMIT, or a failed allocation), NONFINITE (input has
 * NaN/Inf), EIG_NOCONV (a result is still returned), UNSUPPORTED (MIXED with
 * FP64 input), CUDA. */
tucker_status tucker_sthosvd(tucker_ctx* ctx, const void* x_dev, tucker_dtype dtype,
                             int ndim, const int64_t* dims, double eps,
                             const int64_t* ranks_or_null, const int* mode_order_or_null,
                             tucker_prec prec, tucker_result** out);

/* ST-HOSVD, Algorithm 1 (Section 3.3), of a tensor in HOST memory.
 *   x_host     input tensor (dtype, dims) in host memory, read only; page-
 *              locked memory (cudaHostAlloc, cudaHostRegister) lets the copy
 *              overlap the computation, pageable memory works but is staged
 *              by the driver.
 *   other arguments, the result and its ownership as tucker_sthosvd.
 * The library copies the tensor into a device buffer of its own, in pieces
 * (TUCKER_OPT_HOST_CHUNK), and runs the norm pass and, when the first mode is
 * mode 0, that mode's Gram on each piece as it lands (Gram of the piece's
 * columns, summed in FP64; the exact-digit Gram of a piece uses its own row
 * maxima and three digits, and an FP64 Gram replaces the sum when the whole
 * view's bound asks for one, as in tucker_sthosvd).  The rest is
 * tucker_sthosvd on the device copy, which is freed before the call returns.
 * Results equal tucker_sthosvd's up to the order of the FP64 sums and the
 * digit count of the first Gram.  Synchronises the context stream.
 * Calls on several contexts of one device may run at once (one host thread
 * each): their input copies then run one call after the other, in the order
 * the calls issue them, so each has the whole host-to-device link and one
 * call's computation overlaps the next one's copy.
 * Errors: those of tucker_sthosvd; OOM also when the device copy does not
 * fit (predicted before anything is allocated). */
tucker_status tucker_sthosvd_host(tucker_ctx* ctx, const void* x_host, tucker_dtype dtype,
                                  int ndim, const int64_t* dims, double eps,
                                  const int64_t* ranks_or_null, const int* mode_order_or_null,
                                  tucker_prec prec, tucker_result** out);
tucker_status tucker_result_destroy(tucker_result* res);

/* Batched ST-HOSVD: Algorithm 1, eps-driven, mode order 0..N_i-1, for each of
 * `count` independent tensors of any orders and shapes (x_dev[i], ndims[i],
 * dims[i][0..ndims[i]-1], all of one dtype; every mode size <= 4096).  Each
 * result is exactly what tucker_sthosvd would compute with the tridiagonal
 * eigensolver.  The tensors advance through their modes together: step s
 * takes mode s of every tensor with more than s modes, issues their Gram
 * kernels, then one reduction, eigenvalue, rank-cut, eigenvector and
 * back-transformation launch for all of them (one CTA per matrix where the
 * eigensolver is sequential), then their TTMs; the host synchronises twice
 * per step (to size the factors from the ranks, and to check the Cholesky QR
 * of the eigenvectors, which falls back to Jacobi for a matrix it rejects).
 * out[0..count-1] receive results to release with tucker_result_destroy
 * (all NULL on failure).  Errors as tucker_sthosvd. */
tucker_status tucker_sthosvd_batched(tucker_ctx* ctx, int count, const void* const* x_dev,
                                     tucker_dtype dtype, const int* ndims,
                                     const int64_t* const* dims, double eps, tucker_prec prec,
                                     tucker_result** out);

/* (Partial) reconstruction, Section 7: Z = G x_n A_n over the modes in
 * `mode_order_or_null` (NULL = the flop-minimal order by exhaustive
 * search), with A_n = rows begin_n..end_n-1 of U_n.  NULL begin/end = the
 * whole range.  out_dev (caller-owned) holds prod(end_n - begin_n)
 * elements of out_dtype.  Errors: INVALID (ranges, order), OOM, CUDA. */
tucker_status tucker_reconstruct(tucker_ctx* ctx, const tucker_result* res,
                                 const int64_t* begin_or_null, const int64_t* end_or_null,
                                 const int* mode_order_or_null, tucker_prec prec,
                                 void* out_dev, tucker_dtype out_dtype);

/* General multi-TTM, Section 7: Z = G x_{p(0)} A_{p(0)} ... x_{p(N-1)} A_{p(N-1)}.
 *   core_dev   R_0 x ... x R_{N-1} tensor (core_dtype).
 *   mats_dev   N device pointers; A_n is out_dims[n] x core_dims[n], FP64,
 *              column-major with leading dimension lda[n] >= out_dims[n]
 *              (so a row range of U_n is U_n + begin with lda = I_n).
 *   order      permutation (NULL = flop-minimal order, exhaustive search).
 * out_dev holds prod(out_dims) elements.  The last TTM writes straight
 * into out_dev; intermediates live in the context workspace. */
tucker_status tucker_multi_ttm(tucker_ctx* ctx, const void* core_dev, tucker_dtype core_dtype,
                               int ndim, const int64_t* core_dims,
                               const double* const* mats_dev, const int64_t* lda,
                               const int64_t* out_dims, const int* mode_order_or_null,
                               tucker_prec prec, void* out_dev, tucker_dtype out_dtype);

/* Mode order of a multi-TTM chain from core_dims to out_dims (host only).
 * objective 0 = fewest multiply-adds sum_steps J^* K_n (Section 5.3 cost),
 * 1 = smallest peak input+output of one step; exhaustive over N! orders,
 * ties to the lexicographically first.  order_out receives N modes. */
tucker_status tucker_ttm_order(int ndim, const int64_t* core_dims, const int64_t* out_dims,
                               int objective, int* order_out);

/* HOSVD, Section 3.2: every factor from the Gram of X's own mode-n
 * unfolding (Eq. Xeigprob), R_n by Eq. Un with the threshold
 * eps^2 ||X||^2 / N (or the given ranks), U_n its leading R_n eigenvectors;
 * then the core G = X x_0 U_0^T ... x_{N-1} U_{N-1}^T (TTMs in the
 * flop-minimal order of that chain).  Theorem 1 bounds the error:
 * ||X - Xhat||^2 <= sum_n discarded_sq[n].  Arguments, precision, result and
 * errors as tucker_sthosvd (mode_order records 0..N-1, the order of the
 * Grams, which all read X). */
tucker_status tucker_hosvd(tucker_ctx* ctx, const void* x_dev, tucker_dtype dtype, int ndim,
                           const int64_t* dims, double eps, const int64_t* ranks_or_null,
                           tucker_prec prec, tucker_result** out);

/* ST-HOSVD mode order for given (or estimated) ranks, host only: the
 * permutation of 0..N-1 with the fewest flops under the cost analysis of
 * Section 6 (mode-n Gram L I_n^2 Rt, TTM 2 L R_n I_n Rt on the current
 * tensor; the eigensolves cost the same in every order), by exhaustive
 * search over the N! orders, ties to the lexicographically first.  Pass it
 * as tucker_sthosvd's mode order; for an eps-driven run the ranks are an
 * estimate (e.g. those of a similar tensor), since they are not known before
 * the run (Section 8.4).  1 <= ranks[n] <= dims[n].  Errors: INVALID. */
tucker_status tucker_sthosvd_order(int ndim, const int64_t* dims, const int64_t* ranks,
                                   int* order_out);

/* ---- pre- and post-processing, Section 3.5 ---- */

/* Statistics of every mode-`mode` hyperslice X(:, .., i, .., :) (its
 * J^* / I_n entries), FP64: stats_dev[6 i + k] with k = TUCKER_STAT_*.
 * The standard deviation is the population one (sum (x - mean)^2 / count),
 * computed in a second pass over the data.  FP32 data is summed in exact
 * FP32 pairs moved into FP64 (within a few units of 2^-48 of the FP64 sums),
 * FP64 data in FP64.  stats_dev (6 I_n doubles) is
 * caller-owned.  Synchronises.  Errors: INVALID, NONFINITE (a statistic is
 * NaN or Inf: the tensor holds NaN or Inf), OOM, CUDA. */
#define TUCKER_STAT_MEAN 0
#define TUCKER_STAT_STD 1
#define TUCKER_STAT_MAX 2
#define TUCKER_STAT_MIN 3
#define TUCKER_STAT_NORM1 4
#define TUCKER_STAT_NORM2 5
tucker_status tucker_slice_stats(tucker_ctx* ctx, const void* x_dev, tucker_dtype dtype, int ndim,
                                 const int64_t* dims, int mode, double* stats_dev);

/* One linear function per mode-`mode` hyperslice i:
 *   inverse = 0 (pre-processing):  y = (x - shift_i) * scale_i
 *   inverse = 1 (post-processing): y = x / scale_i + shift_i
 * FP64 data in FP64; FP32 data in FP32-pair arithmetic (about 48 bits, the
 * inverse as x * (1 / scale_i)), rounded once to FP32: within one ulp of the
 * exact value.  shift_dev, scale_dev: I_n
 * FP64 values each (for a reconstructed subtensor whose mode-`mode` range
 * starts at b, pass shift + b and scale + b); scale_i must be nonzero for
 * the inverse.  y_dev (same dims and dtype) may equal x_dev (in place).
 * Synchronises.  Errors: INVALID, CUDA. */
tucker_status tucker_slice_transform(tucker_ctx* ctx, const void* x_dev, tucker_dtype dtype,
                                     int ndim, const int64_t* dims, int mode,
                                     const double* shift_dev, const double* scale_dev,
                                     int inverse, void* y_dev);

/* Pre-processing in one call (Section 3.5): the hyperslice statistics, the
 * parameters of `method` into shift_dev and scale_dev (I_n FP64 each,
 * caller-owned, kept for the post-processing inverse), then the transform
 * into y_dev (may equal x_dev).
 *   TUCKER_PRE_STANDARDIZE: shift = mean, scale = 1 / std (mean 0, variance 1)
 *   TUCKER_PRE_MAX_RESCALE: shift = 0, scale = 1 / max |x| (range -1..1)
 * A slice with std 0 (standardization) or all zeros (max rescaling) keeps
 * scale 1.  Synchronises.  Errors as tucker_slice_stats. */
#define TUCKER_PRE_STANDARDIZE 0
#define TUCKER_PRE_MAX_RESCALE 1
tucker_status tucker_preprocess(tucker_ctx* ctx, const void* x_dev, tucker_dtype dtype, int ndim,
                                const int64_t* dims, int mode, int method, double* shift_dev,
                                double* scale_dev, void* y_dev);

/* ---- single steps of the hot path (each one row of Algorithm 1) ---- */

/* ||Y||^2 as an FP64 sum of squares (Section 2.2.2).  Synchronises.
 * Returns NONFINITE (with *out_host set to the sum) if Y holds NaN/Inf. */
tucker_status tucker_norm_sq(tucker_ctx* ctx, const void* y_dev, tucker_dtype dtype,
                             int64_t count, double* out_host);

/* Gram S = Y_(n) Y_(n)^T of the mode-n unfolding (Algorithm 2) over the
 * strided slab view (Rt, I, L) of Y, with no unfolding materialised.
 * S_dev: caller-owned I x I FP64 (full symmetric matrix written). */
tucker_status tucker_gram(tucker_ctx* ctx, const void* y_dev, tucker_dtype dtype, int ndim,
                          const int64_t* dims, int mode, tucker_prec prec, double* S_dev);

/* All eigenpairs of the symmetric I x I FP64 matrix S (Section 5.2) by
 * parallel cyclic Jacobi in FP64 on the whole GPU.  eigvals_dev (I) gets
 * them in descending order, V_dev (I x I, column-major) the matching
 * orthonormal eigenvectors.  *sweeps_host (may be NULL) the sweeps used.
 * 1 <= I <= 8192 (also the largest mode size tucker_sthosvd accepts).
 * Synchronises.  EIG_NOCONV if the sweep cap was reached. */
tucker_status tucker_eig(tucker_ctx* ctx, const double* S_dev, int64_t I,
                         double* eigvals_dev, double* V_dev, int* sweeps_host);

/* Truncated eigensolve, the eigenvalue step of Algorithm 1 (Section 5.2;
 * rank cut of Eq. Un): all eigenvalues of the symmetric I x I FP64 matrix S
 * into eigvals_dev (I, descending), then R = the cut at thr (as in
 * tucker_rank_cut) or R = fixed_R when fixed_R > 0, and the R leading
 * orthonormal eigenvectors into U_dev (caller-owned, capacity I x I doubles;
 * the first I x R hold them, column-major).  Solver per
 * TUCKER_OPT_EIG_SOLVER: the tridiagonal one is Householder reduction,
 * bisection, inverse iteration and a Cholesky QR, with Jacobi taken instead
 * if that QR finds the vectors nearly dependent.  1 <= I <= 8192,
 * 0 <= fixed_R <= I, thr >= 0.  Synchronises; *R_host and *discarded_host =
 * tail(R).  EIG_NOCONV as tucker_eig when Jacobi ran and hit its cap. */
tucker_status tucker_eig_trunc(tucker_ctx* ctx, const double* S_dev, int64_t I, double thr,
                               int64_t fixed_R, double* eigvals_dev, double* U_dev,
                               int64_t* R_host, double* discarded_host);

/* Rank cut of Eq. Un on descending eigenvalues: R = min{R in 1..I :
 * sum_{i>=R} lambda_i <= thr}, the signed computed eigenvalues accumulated
 * in FP64 from the smallest up.  Synchronises; *R_host and
 * *discarded_host = tail(R). */
tucker_status tucker_rank_cut(tucker_ctx* ctx, const double* eigvals_dev, int64_t I, double thr,
                              int64_t* R_host, double* discarded_host);

/* TTM Z = Y x_n A (Algorithm 3) for A of size K x J_n, FP64, column-major
 * with leading dimension lda >= K, or row-major (a_rowmajor = 1, leading
 * dimension lda >= J_n).  A = U_n^T is U_n's column-major storage read
 * row-major.  z_dev (caller-owned) holds Y's dims with J_n -> K. */
tucker_status tucker_ttm(tucker_ctx* ctx, const void* y_dev, tucker_dtype y_dtype, int ndim,
                         const int64_t* dims, int mode, const double* A_dev, int64_t K,
                         int64_t lda, int a_rowmajor, tucker_prec prec,
                         void* z_dev, tucker_dtype z_dtype);

/* ---- Gram without allocation ----
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc -- code whose device memory is all owned by its own
 * allocator (a framework's caching pool that reserved the device), or code
 * on a path where an allocation may not happen or may not stall (a
 * fixed-budget service loop).  It computes exactly what tucker_gram
 * computes, with the SIMT kernel (prec FP64 or FP32; MIXED is UNSUPPORTED),
 * and needs no context.
 *   - Its split-K scratch is a static 16 MiB device array inside the
 *     library, so every GPU that loads the library holds those 16 MiB until
 *     the process exits.  The partial tiles of one call must fit in it:
 *     I_n <= 1984 (larger I_n returns TUCKER_ERR_INVALID, nothing launched).
 *   - The first call on a device looks up that array's device address
 *     (cudaGetSymbolAddress) with the device current; make that first call
 *     before any stream capture.
 *   - All calls share the one array: calls that overlap on the GPU (other
 *     streams, other host threads) race and corrupt each other's results.
 *     Every call overwrites the partial tiles it reads, so nothing carries
 *     over from the previous call.
 *   - The call is asynchronous on `stream` (a cudaStream_t, NULL = legacy
 *     default stream); S_dev (I_n x I_n FP64, caller-owned) is complete when
 *     the stream reaches this point.  It calls no cudaMalloc, cudaFree or
 *     allocating library routine.
 * Errors: INVALID (arguments, size limit), UNSUPPORTED (MIXED), CUDA. */
tucker_status tucker_gram_noalloc(const void* y_dev, tucker_dtype dtype, int ndim,
                                  const int64_t* dims, int mode, tucker_prec prec,
                                  double* S_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* TUCKER_GB300_H */
