/* ihsbin.h -- C ABI of a GB300 (sm_103a) implementation of IHS-BIN, the iterative
 * Hessian sketch with binomial decomposition of Wang & Pilanci, "Sketching the
 * Krylov Subspace: Faster Computation of the Entire Ridge Regularization Path".
 *
 * Problem (Section 1, eq. 1):  x*(lam) = argmin 1/2||A x - b||^2 + lam/2 ||x||^2
 *                                       = (A^T A + lam I)^-1 A^T b,
 * for every lam of a grid Lambda in [lambda_min, lambda_max]; matrix-valued
 * right-hand sides B (n x K) per Section 5.3; under-determined A (n < d)
 * through the dual of Section 5.2 (x = A^T z).
 *
 * Call order on a problem:  ihsbin_sketch -> ihsbin_build_basis -> ihsbin_eval_path
 * (eval may be repeated with any lambdas inside the range).  Any other order
 * returns IHSBIN_ERR_STATE.
 *
 * Conventions for every call:
 *  - returns an ihsbin_status; no C++ exception crosses the ABI and no device
 *    kernel traps: faults detected on the device (non-positive pivot, NaN)
 *    come back through a device status word read at the call's synchronisation
 *    point;
 *  - `stream` is a cudaStream_t passed as void* (NULL = the calling thread's
 *    default stream; the library is built with per-thread default streams, so
 *    calls from different host threads never serialise on a shared stream);
 *    every call is stream-ordered and returns after its own work on that
 *    stream has completed (the status word is read there);
 *  - device memory comes from a stream-ordered pool owned by the context
 *    (freed blocks are kept for reuse), so no call synchronises the device;
 *  - on error, outputs are unspecified; a failed ihsbin_sketch leaves the problem unsketched
 *    and a failed ihsbin_build_basis leaves it sketched without a basis (their previous result
 *    is discarded when they start); every other call leaves the problem as it was;
 *  - ihsbin_last_error() returns a thread-local description of the last error.
 */
#ifndef IHSBIN_H
#define IHSBIN_H

#include <stdint.h>

#if defined(__GNUC__)
#define IHSBIN_API __attribute__((visibility("default")))
#else
#define IHSBIN_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  IHSBIN_OK = 0,
  IHSBIN_ERR_INVALID_ARG = 1,
  IHSBIN_ERR_OUT_OF_MEMORY = 2,
  IHSBIN_ERR_CUDA = 3,
  IHSBIN_ERR_NOT_SPD = 4,      /* a factor of (SA)^T SA + lam0 I had a non-positive pivot  */
  IHSBIN_ERR_LAMBDA_RANGE = 5, /* a requested lambda lies outside [lambda_min, lambda_max] */
  IHSBIN_ERR_STATE = 6,        /* call out of order                                      */
  IHSBIN_ERR_TIMEOUT = 7,      /* a bounded wait expired                                 */
  IHSBIN_ERR_ADMISSION = 8,    /* request larger than the device-memory budget           */
  IHSBIN_ERR_UNSUPPORTED = 9,
  IHSBIN_ERR_NAN = 11          /* a non-finite value was produced on the device          */
} ihsbin_status;

/* Element type of caller-provided arrays.  IHSBIN_TF32 (the data matrix only): FP32 storage whose
 * values enter the method rounded to TF32 (10 fraction bits, to nearest, ties away from zero);
 * the library rounds a copy of A at problem creation and solves the problem of the rounded data. */
typedef enum { IHSBIN_F64 = 0, IHSBIN_F32 = 1, IHSBIN_BF16 = 2, IHSBIN_TF32 = 3 } ihsbin_dtype;

/* Arithmetic of the accuracy-critical contractions (Gram, preconditioner,
 * basis loop, right-hand side, path evaluation):
 *  IHSBIN_COMPUTE_F64  IEEE double throughout;
 *  IHSBIN_COMPUTE_F32X2 float-float pairs (about 44 significant bits) built from
 *                      error-free transformations on the FP32 pipe; the
 *                      sketch itself is applied in FP64 (Gaussian), in exact
 *                      int64 fixed point (the SRHT's Hadamard transform) or
 *                      with FP64 accumulation (CountSketch). */
typedef enum { IHSBIN_COMPUTE_F64 = 0, IHSBIN_COMPUTE_F32X2 = 1 } ihsbin_compute;

typedef enum { IHSBIN_DENSE_ROWMAJOR = 0, IHSBIN_CSR = 1 } ihsbin_layout;

/* Section 3: Gaussian N(0, 1/m); CountSketch (s = 1) / SJLT (s > 1 stacked
 * CountSketches of m/s rows, entries +-1/sqrt(s)); SRHT (1/sqrt(m)) R H D on
 * the rows zero-padded to a power of two. */
typedef enum { IHSBIN_SK_GAUSSIAN = 0, IHSBIN_SK_SRHT = 1, IHSBIN_SK_COUNTSKETCH = 2 } ihsbin_sketch_kind;

/* How A^T (A V) is formed inside the basis loop (Algorithm 2):
 *  IHSBIN_PRODUCT_AUTO   = GRAM;
 *  IHSBIN_PRODUCT_GRAM   form G = A^T A once (dense: a split-K contraction;
 *                        CSR: the nonzero pairs of every row), then every
 *                        product of the loop is G V;
 *  IHSBIN_PRODUCT_ASPACE stream A twice per step: W = A V, Y = A^T W (dense only). */
typedef enum { IHSBIN_PRODUCT_AUTO = 0, IHSBIN_PRODUCT_GRAM = 1, IHSBIN_PRODUCT_ASPACE = 2 } ihsbin_product;

/* The data matrix A (n x d).  Borrowed: when on_device = 1 the arrays must stay
 * valid until the problem is destroyed; when on_device = 0 they are copied
 * during ihsbin_problem_create.
 *  dense: `values` row-major with row stride `ld` (>= d) elements of `dtype`;
 *  CSR:   row_ptr[n+1] (int64), col_idx[nnz] (int32, sorted within each row,
 *         no duplicates), values[nnz] of `dtype`. */
typedef struct {
  int64_t n, d;
  ihsbin_layout layout;
  ihsbin_dtype dtype;
  const void* values;
  int64_t ld;
  const int64_t* row_ptr;
  const int32_t* col_idx;
  int64_t nnz;
  int on_device;
} ihsbin_matrix;

/* How the Gaussian sketch S A_hat is contracted (Section 3, Gaussian sketch):
 *  AUTO   : TENSOR for BF16 entries of dense BF16 data, FMA otherwise;
 *  TENSOR : BF16 entries and dense BF16 data only (else IHSBIN_ERR_UNSUPPORTED).  S is drawn
 *           once per call into the tensor cores' shared-memory image (every BF16 entry equal to
 *           the FP64 value rounded FP64 -> FP32 -> BF16), and S A_hat runs as a BF16 tcgen05
 *           contraction: products exact, accumulated in FP32 over at most a k-split of the rows
 *           (a few thousand products per entry), the k-splits added in FP64;
 *  FMA    : CUDA-core contraction, FP64 accumulation (FP64 entries) or float-float (BF16 entries
 *           of FP32/BF16 data). */
typedef enum { IHSBIN_APPLY_AUTO = 0, IHSBIN_APPLY_TENSOR = 1, IHSBIN_APPLY_FMA = 2 } ihsbin_sketch_apply;

typedef struct {
  ihsbin_sketch_kind kind;
  int64_t m;     /* sketch rows (m % s == 0 for CountSketch/SJLT)           */
  int32_t s;     /* SJLT sparsity; 1 = CountSketch; ignored for other kinds */
  uint64_t seed; /* Philox4x32-10 key                                       */
  ihsbin_dtype entries; /* Gaussian only: IHSBIN_F64 (default) keeps the FP64 entries z/sqrt(m);
                         * IHSBIN_BF16 rounds them (FP64 -> FP32 -> BF16, to nearest even), and with
                         * FP32/BF16 data every product of the sketch is then exact in FP32 */
  ihsbin_sketch_apply apply; /* Gaussian only: the contraction (see ihsbin_sketch_apply) */
} ihsbin_sketch_desc;

/* Interval plan and iteration parameters (Section 4.2, Theorem 4).
 *  L        number of intervals; 0 selects floor(2 ln(lambda_max/lambda_min)) (at least 1).
 *           Interval l covers [lambda_min beta^(l/L), lambda_min beta^((l+1)/L)),
 *           the last one closed; lam0_l is the geometric mean of its ends.
 *  k        per-interval term counts k_l (array of L), or NULL to use k_default.
 *  rho1/rho2 per-interval eigenvalue bounds of the sketched Hessian (arrays of L),
 *           or NULL to use rho: rho1 = (1+sqrt rho)^2, rho2 = (1-sqrt rho)^2
 *           (Gaussian-sketch theorem with ||D||_2 = 1); rho <= 0 selects
 *           min(D/m, 0.81) with D the dimension of the (dual) unknown.
 *  tau_l = 2 lam0_l / (lo_l/rho1_l + hi_l/rho2_l)   (Theorem 4, from its proof).
 *  jmax     0 keeps every basis term utilde_0..utilde_{k-1} (Algorithm 2); a
 *           positive value keeps only the terms j < jmax.  The recursion for
 *           j < jmax is unchanged, so the result differs from the full basis
 *           only by the omitted high-order terms of the expansion in
 *           theta = tau (lam - lam0) / lam0.
 *  auto_rho nonzero (with rho1/rho2 NULL): rho_l = min(d_e(lam0_l)/m, 0.95) with the
 *           effective dimension of Section 4.2 estimated from the sketch,
 *           d_e = tr(G_S (G_S + lam0 I)^-1) = D - lam0 tr(P_l) (taking ||D||_2 = 1).
 *  eps      with k == NULL and k_default <= 0, k_l is Theorem 4's iteration
 *           count for relative error eps: ceil(ln eps / ln((kt-1)/(kt+1))) with
 *           kt = rho1 hi_l / (rho2 lo_l) (eps <= 0 selects 1e-7). */
/* Kernel for the Gram A_hat^T A_hat of the Gram product mode.
 *  AUTO   : SLICES for dense FP32/BF16 data, FMA otherwise.
 *  SLICES : dense FP32/BF16 data only.  Every column is scaled by a power of two
 *           and cut into 6 integer slices exact in BF16; the slice products run
 *           on the tensor cores (tcgen05, FP32 accumulation of integer products,
 *           exact in chunks of 512 rows, drained into int32), and the pairs are
 *           combined in FP64.  The result matches the exact Gram to about FP64
 *           rounding (entries within 2^-17 of their column's largest magnitude
 *           are represented exactly; smaller ones to 2^-41 of that maximum).
 *  FMA    : CUDA-core contraction in FP64 (F64 compute) or float-float (F32X2). */
typedef enum { IHSBIN_GRAM_AUTO = 0, IHSBIN_GRAM_SLICES = 1, IHSBIN_GRAM_FMA = 2 } ihsbin_gram;

/* Kernel for the two products of every step of the basis recursion
 * (A_hat^T A_hat U in the Gram product mode, and P_l R).
 *  AUTO   : SLICES in the F32X2 compute mode, FMA otherwise.
 *  SLICES : F32X2 compute only.  The Gram and every P_l are cut by rows, and the
 *           step's columns by columns, into 6 integer slices exact in BF16 (each
 *           entry held to 2^-47 of its row's / column's largest magnitude); the 26
 *           slice pairs with s + t <= 6 run on the tensor cores (tcgen05), exact in
 *           chunks and drained into int32, and are combined in FP64 into the
 *           float-float state: the accuracy class of the float-float contraction.
 *  FMA    : CUDA-core contraction in the compute mode's arithmetic. */
typedef enum { IHSBIN_LOOP_AUTO = 0, IHSBIN_LOOP_SLICES = 1, IHSBIN_LOOP_FMA = 2 } ihsbin_loop;

/* Kernel for the explicit inverse P_l = W_l^T W_l (W_l = L_l^-1) of every interval.
 *  AUTO   : SLICES in the F32X2 compute mode, FMA otherwise.
 *  SLICES : F32X2 compute only.  The columns of W_l are cut into exact BF16 slices and the
 *           product runs on the tensor cores as the recursion's products do, skipping the
 *           zero blocks of the triangular W_l and the mirrored half of the symmetric result.
 *  FMA    : CUDA-core contraction in the compute mode's arithmetic. */
typedef enum { IHSBIN_FACTOR_AUTO = 0, IHSBIN_FACTOR_SLICES = 1, IHSBIN_FACTOR_FMA = 2 } ihsbin_factor;

/* Form in which the SLICES recursion carries the basis (the FMA kernels always run INCREMENT).
 *  AUTO      : RESIDUAL where available (Gram product mode, D <= 20480) and the automatic
 *              precond_weight below is at most 4, else INCREMENT.
 *  INCREMENT : Algorithm 2 as printed: the per-step terms u_{i,j} are carried and added into
 *              utilde_j; every product keeps slice_weight's pairs; the longest intervals switch to
 *              the two-product steps with M_l = P_l (G + lam0_l I) once at most six are running.
 *  RESIDUAL  : the same polynomial carried as its partial sums v_{i,j} = sum_{i' <= i} u_{i',j},
 *              which are utilde_j after the last step.  Summing the recursion of Proposition 1 over
 *              the steps gives v_j <- v_j + P_l r_j with the residual
 *              r_j = [j = 0] c - tau (G + lam0 I) v_j - lam0 v_{j-1}  (re-centred, re-scaled form),
 *              equal to the INCREMENT result in exact arithmetic.  An error made in applying P_l
 *              reappears in the next residual and is removed by the following steps (the residual
 *              correction of IHS), so only G v needs the float-float class: P_l r keeps the pairs
 *              s + t <= precond_weight. */
typedef enum { IHSBIN_FORM_AUTO = 0, IHSBIN_FORM_RESIDUAL = 1, IHSBIN_FORM_INCREMENT = 2 } ihsbin_form;

typedef struct {
  double lambda_min, lambda_max;
  int32_t L;
  const int32_t* k;
  int32_t k_default;
  const double* rho1;
  const double* rho2;
  double rho;
  int32_t jmax;
  ihsbin_compute compute;
  ihsbin_product product;
  double eps;
  int32_t auto_rho;
  ihsbin_gram gram;
  ihsbin_loop loop;
  ihsbin_factor factor;
  double sigma_d2;  /* >= 0: a known lower bound on the smallest eigenvalue of A_hat^T A_hat (the remark
                     * after Theorem 4); > 0 centres interval [lo, hi] at
                     * lam0 = sqrt((hi + s)(lo + s)) - s, takes tau = 2 (lam0 + s) / ((lo + s)/rho1 + (hi + s)/rho2)
                     * and, for auto k, Theorem 4's rate with kt = rho1 (hi + s) / (rho2 (lo + s)); 0 is the
                     * default rule (lam0 = sqrt(lo hi)) */
  const double* tau; /* NULL: tau_l from Theorem 4's rule above; else an array of L explicit steps (each finite
                      * and > 0; needs L > 0), for callers who tuned them (Theorem 4's rho are not computable
                      * from data in practice); rho1/rho2 still set k_l when k is NULL and k_default <= 0 */
  int32_t slice_weight; /* SLICES loop / factor kernels only: the slice pairs (s, t) with s + t <= slice_weight
                         * are kept (0 selects 6, the float-float accuracy class; 4 or 5 drop the pairs
                         * weighing below 2^-40 / 2^-48 of an entry's leading product, 1.8x / 1.3x fewer
                         * tensor-core products; the Gram of A keeps every pair it needs regardless) */
  int32_t form;          /* ihsbin_form (0 = AUTO) */
  int32_t precond_weight; /* RESIDUAL form: the slice pairs kept by the P_l r products (1..6; each step
                           * of 1 divides the weight of the dropped pairs by 2^8; up to 3 the
                           * products run on 64-column tiles).  0 = the smallest w in 2..5 with
                           * (1) 2^(-8(w+1)) sqrt(D) kappa <= 2^-5, kappa = 1 + tr(G_S) / min_l lam0_l
                           * (the iteration map keeps its contraction), and
                           * (2) 2^(-8(w+1)) max_l k_l rate_l^(k_l - 1) <= max_l k_l 2^-47, rate_l
                           * Theorem 4's contraction bound of interval l (the error the steps carry
                           * to the end is no larger than the increment form's); 6 when none is.
                           * A nonzero value selects the RESIDUAL form under AUTO. */
} ihsbin_path_desc;

typedef struct ihsbin_ctx ihsbin_ctx;
typedef struct ihsbin_problem ihsbin_problem;

/* Library context bound to CUDA device `device`.  hbm_budget_bytes caps the
 * device memory all problems of this context may hold (0 = no cap); a problem
 * that would exceed it fails with IHSBIN_ERR_ADMISSION.  Owned by the caller;
 * release with ihsbin_ctx_destroy after every problem of it is destroyed. */
IHSBIN_API ihsbin_status ihsbin_ctx_create(int device, uint64_t hbm_budget_bytes, ihsbin_ctx** out);
IHSBIN_API ihsbin_status ihsbin_ctx_destroy(ihsbin_ctx* ctx);
/* Test hook for the error paths: after `after` more device allocations of this context succeed,
 * every further one fails (the call returns IHSBIN_ERR_OUT_OF_MEMORY) until the hook is reset with
 * after < 0.  The failure is made on the host, before any device memory is requested. */
IHSBIN_API ihsbin_status ihsbin_ctx_fail_allocations(ihsbin_ctx* ctx, int64_t after);
/* Bytes of device memory currently held by the context's problems. */
IHSBIN_API ihsbin_status ihsbin_ctx_memory(const ihsbin_ctx* ctx, uint64_t* bytes_in_use);
IHSBIN_API const char* ihsbin_last_error(void);

/* Create a problem for A and right-hand side(s) B (n x K, row stride ldb >= K,
 * element type b_dtype, host or device per b_on_device; copied).  If n < d the
 * problem is solved through the dual (Section 5.2).  Allocates the problem's
 * device state (counted against the context budget).  CSR structure is checked on the device
 * before any kernel indexes with it: row_ptr must run from 0 to nnz without decreasing and each
 * row's column indices must lie in [0, d) and increase strictly; otherwise the call fails with
 * IHSBIN_ERR_INVALID_ARG and creates nothing.  Release with ihsbin_problem_destroy. */
IHSBIN_API ihsbin_status ihsbin_problem_create(ihsbin_ctx* ctx, const ihsbin_matrix* A, const void* B,
                                    int64_t K, int64_t ldb, ihsbin_dtype b_dtype, int b_on_device,
                                    ihsbin_problem** out);
IHSBIN_API ihsbin_status ihsbin_problem_destroy(ihsbin_problem* p);

/* Step a1 of the hot path: S A_hat (m x D) for the sketch of Section 3 and
 * its Gram (S A_hat)^T (S A_hat), where A_hat = A (over-determined) or A^T
 * (under-determined).  S A_hat is returned in FP64.  The SRHT converts each column of
 * D A_hat once to int64 fixed point at 2^-(62 - log2 N_pad) of the column's largest
 * magnitude and then adds exactly; the other sketches accumulate in FP64.  Its Gram is
 * formed on the tensor cores from seven exact BF16 slices of S A_hat and combined in FP64
 * (FP64-class accuracy).  Re-sketching an already sketched problem discards the basis.
 * Limits: the SRHT needs dense A, m <= N_pad and N_pad <= 2^24 rows (beyond that its
 * launches exceed the grid limits and the call fails with IHSBIN_ERR_CUDA); CountSketch and
 * Gaussian sketches take any row count.
 * For dense FP32/BF16/TF32 data with K >= 32 (not the dual), and unless per-launch timing is on,
 * the call also starts the Gram of A_hat and A_hat^T B on the problem's low-priority internal
 * stream; it returns when the sketch is done, with that Gram still running.  The next
 * ihsbin_build_basis takes it when it runs the float-float mode with the sliced Gram (the
 * defaults); any other call that needs the problem's memory waits for it first.  An error of
 * that background work is reported by the build. */
IHSBIN_API ihsbin_status ihsbin_sketch(ihsbin_problem* p, const ihsbin_sketch_desc* sk, void* stream);

/* Bit-exact export of the sketch's integer draws, for tests.
 *  SRHT:        idx[0..m) = kept rows of H (ascending), sign[0..N_pad) = diagonal of D;
 *  CountSketch: idx[i*s+t] = row of S hit by input row i in block t, sign[i*s+t];
 *  Gaussian:    nothing (count = 0).
 * `cap` bounds both arrays; *count receives the number of idx entries. */
IHSBIN_API ihsbin_status ihsbin_sketch_export(ihsbin_problem* p, int64_t* idx, int8_t* sign, int64_t cap,
                                   int64_t* count);

/* Copy S A_hat (m x D, row-major FP64) and/or its Gram (D x D) to host arrays
 * (either may be NULL), for tests. */
IHSBIN_API ihsbin_status ihsbin_sketch_matrix_export(ihsbin_problem* p, double* SA, double* GS);

/* BF16 bits of the entries S[i][j], row0 <= i < row0 + nrows, col0 <= j < col0 + ncols, of a
 * problem sketched with the Gaussian sketch with BF16 entries (Section 3), drawn by the same
 * device code the tensor-core contraction uses; written row-major to the host array `out`
 * (nrows * ncols values), for tests.  IHSBIN_ERR_STATE when the problem is not sketched that
 * way, IHSBIN_ERR_INVALID_ARG for a window outside the m x N sketch. */
IHSBIN_API ihsbin_status ihsbin_sketch_entries_export(ihsbin_problem* p, int64_t row0, int64_t nrows, int64_t col0,
                                                      int64_t ncols, uint16_t* out);

/* Steps a2-a4: per interval, the factor of (S A_hat)^T S A_hat + lam0_l I and
 * its explicit inverse P_l; the right-hand side c = A^T B (dual: c = B); then
 * Algorithm 2 / 5 (Proposition 1's recursion, re-centred at lam0_l):
 *   u_00 = P c;  for i = 1..k_l-1:  u_i = -lam0 P u_{i-1},
 *   u_j <- u_j - P(tau (A^T A u_j + lam0 u_j) + lam0 u_{j-1})  (j = i-1..1),
 *   u_0 <- u_0 - P tau (A^T A u_0 + lam0 u_0),  utilde_j += u_j.
 * The bases stay resident on the device until the problem is destroyed.
 * Ordered after earlier work on `stream` and synchronous: it returns when the basis
 * is complete.  Internally the call forks two streams of the problem (created on its
 * first build, destroyed with the problem) from `stream` -- the Gram and right-hand
 * side on one, the factorization on the other -- and joins both back into `stream`
 * before the recursion; nothing is left running on them when the call returns. */
IHSBIN_API ihsbin_status ihsbin_build_basis(ihsbin_problem* p, const ihsbin_path_desc* desc, void* stream);

/* Copy the Gram G = A_hat^T A_hat (D x D, row-major) built by the last
 * ihsbin_build_basis in the Gram product mode to a host FP64 array, for tests.
 * Fails with IHSBIN_ERR_STATE when there is no basis or the product mode was
 * A-space (no Gram is formed). */
IHSBIN_API ihsbin_status ihsbin_gram_export(ihsbin_problem* p, double* G);

/* The form and the preconditioner pair weight the last ihsbin_build_basis ran with (ihsbin_form
 * RESIDUAL or INCREMENT; in the INCREMENT form the weight is slice_weight's).  Either pointer may be NULL.
 * Fails with STATE before the first build. */
IHSBIN_API ihsbin_status ihsbin_recursion_form(const ihsbin_problem* p, int32_t* form, int32_t* precond_weight);
/* The plan the library derived from the descriptor: arrays of L (edges: L+1),
 * any may be NULL; *L_out receives L.  Fails with INVALID_ARG if cap_L < L. */
IHSBIN_API ihsbin_status ihsbin_plan_export(ihsbin_problem* p, double* edges, double* lam0, double* tau,
                                 int32_t* k, int32_t* jcount, int32_t cap_L, int32_t* L_out);

/* Copy interval l's basis utilde_j (j < jcount_l) to host as FP64, layout
 * [j][r][i] (D x K per term); *need receives the element count. */
IHSBIN_API ihsbin_status ihsbin_basis_export(ihsbin_problem* p, int32_t l, double* buf, int64_t cap,
                                  int64_t* need);

/* Steps a5-a6: X(:, :, t) = tau_l sum_j theta_t^j utilde_j with
 * theta_t = tau_l (lambdas[t] - lam0_l) / lam0_l for the interval l holding
 * lambdas[t] (Algorithm 3 / 6 composition); for an under-determined problem
 * the primal x = A^T z is returned.  lambdas: host array of T doubles.  X:
 * T x d x K row-major per lambda (element [t][i][r]), caller-owned, on the
 * device or host per x_on_device, element type F64 or F32.  Any lambda outside
 * [lambda_min, lambda_max] fails with IHSBIN_ERR_LAMBDA_RANGE before anything
 * is written. */
IHSBIN_API ihsbin_status ihsbin_eval_path(ihsbin_problem* p, const double* lambdas, int64_t T, void* X,
                               ihsbin_dtype x_dtype, int x_on_device, void* stream);

/* Section 6.1's losses along the path without forming X: for each lambdas[t]
 *   train_loss[t] = 1/2 ||A x(lambda_t) - B||_F^2 + lambda_t/2 ||x(lambda_t)||_F^2,
 *   test_loss[t]  = 1/2 ||A_test x(lambda_t) - B_test||_F^2,
 * with x(lambda) the primal solution ihsbin_eval_path returns (the dual's x = A^T z).
 * The basis's images A utilde_j and A_test utilde_j are formed once (a contraction over d
 * per basis column) and the residual of each lambda is a combination of them with the
 * evaluation's coefficients, in the compute mode's arithmetic; the squares are summed in
 * FP64 in a fixed order.  lambdas: host array of T doubles, each in [lambda_min, lambda_max]
 * (else IHSBIN_ERR_LAMBDA_RANGE).  A_test: dense row-major n_test x d (any data dtype,
 * host or device per its on_device; CSR fails with IHSBIN_ERR_UNSUPPORTED); B_test:
 * n_test x K, row stride ldb_test >= K, F64 or F32, host or device per b_test_on_device.
 * train_loss / test_loss: host arrays of T doubles, either may be NULL (test_loss NULL
 * leaves A_test / B_test unread).  Synchronous on `stream`. */
IHSBIN_API ihsbin_status ihsbin_path_losses(ihsbin_problem* p, const double* lambdas, int64_t T,
                                 const ihsbin_matrix* A_test, const void* B_test, int64_t ldb_test,
                                 ihsbin_dtype b_test_dtype, int b_test_on_device, double* train_loss,
                                 double* test_loss, void* stream);

/* Adaptive sketch dimension (Section 5.1, Algorithm 4).  Newton-sketch steps with an
 * Armijo line search on the ridge problem at lambda:
 *   f(x) = 1/2 x^T (A_hat^T A_hat + lambda I) x - c^T x   (c = A_hat^T B; the dual of
 *   Section 5.2, A_hat = A^T and c = B, when n < d), summed over the K columns,
 *   d_k = P_S grad f(x_k), P_S = ((S A_hat)^T S A_hat + lambda I)^-1,
 *   delta_k = <d_k, grad f(x_k)>,  tau_k = gamma1^j with the smallest j >= 0 such that
 *   f(x_k - tau d_k) <= f(x_k) - gamma2 tau delta_k,  x_{k+1} = x_k - tau_k d_k;
 * when delta_{k+1} >= gamma3 delta_k the sketch dimension doubles (while 2m <= m_max) and a
 * new sketch is drawn with seed + (number of doublings), d_{k+1} and delta_{k+1} recomputed
 * with it.  Stops when delta_k <= eps delta_0 or after max_iter steps. */
typedef struct {
  ihsbin_sketch_desc sketch; /* kind, initial m, s, seed, entries                              */
  double lambda;             /* > 0: the shift (normally lambda_min of the path)               */
  double eps;                /* relative stop on the decrement; <= 0 selects 1e-10             */
  double gamma1, gamma2;     /* Armijo backtracking factor and constant in (0,1); <= 0: 0.5, 0.25 */
  double gamma3;             /* doubling threshold on delta_{k+1} / delta_k; <= 0: 0.5         */
  int32_t max_iter;          /* <= 0 selects 100                                               */
  int64_t m_max;             /* <= 0: the row count of A_hat (its power-of-two padding for SRHT) */
  ihsbin_compute compute;    /* arithmetic of the iteration (the factor, P_S and the products)  */
} ihsbin_adaptive_desc;

typedef struct {
  int64_t m;                 /* the final sketch dimension                                     */
  int32_t iterations, doublings;
  double delta0, delta;      /* first and last decrement                                       */
} ihsbin_adaptive_result;

/* Runs Algorithm 4 on the problem and leaves it sketched with the final S (as after
 * ihsbin_sketch with the final m and seed), ready for ihsbin_build_basis; any basis is
 * discarded.  Optional host outputs (NULL to skip): delta_trace / m_trace / step_trace of
 * trace_cap entries (delta_k and the m in force for k = 0..iterations, tau_k for k <
 * iterations; entries past trace_cap are dropped), x_out the final iterate (D x K row-major
 * FP64, the dual variable for n < d).  Synchronous on `stream`.  Errors: INVALID_ARG for bad
 * parameters, the sketch's own errors, NOT_SPD from a factor. */
IHSBIN_API ihsbin_status ihsbin_adaptive_sketch(ihsbin_problem* p, const ihsbin_adaptive_desc* desc,
                                     ihsbin_adaptive_result* res, double* delta_trace, int64_t* m_trace,
                                     double* step_trace, int32_t trace_cap, double* x_out, void* stream);

/* Device time (ms) of the phases of the last sketch / build_basis / eval_path
 * calls: [0] sketch, [1] factor+inverse, [2] Gram+rhs, [3] basis loop, [4] eval. */
IHSBIN_API ihsbin_status ihsbin_phase_times(ihsbin_problem* p, float* ms5);

/* Per-kernel accounting, for measurement.  Every launch is counted with the
 * method's algorithmic work: flops = 2 per multiply-add of the contraction the
 * paper's step performs (FP64 class), bytes = one pass over the step's operands
 * at 8 bytes per FP64-class entry (the Gram G once per recursion step, each live
 * P_l once, the data at its storage width).  When timing is enabled each launch
 * is also bracketed by CUDA events on the stream it runs on and its device time
 * is added at the call's synchronisation point.  Categories 0 ..
 * IHSBIN_KCAT_COUNT-1 (names returned in *name, static storage; categories not
 * in use report no launches and the name "unused"). */
#define IHSBIN_KCAT_COUNT 40
IHSBIN_API ihsbin_status ihsbin_set_timing(ihsbin_problem* p, int enable);
IHSBIN_API ihsbin_status ihsbin_reset_stats(ihsbin_problem* p);
IHSBIN_API ihsbin_status ihsbin_kernel_stats(ihsbin_problem* p, int32_t cat, int64_t* launches, double* ms,
                                             double* flops, double* bytes, const char** name);
/* The work the same launches execute: for the exact-slice tensor-core products the
 * BF16 flops of every kept slice pair and the bytes of the slice images they stream
 * (12 bytes per FP64-class entry), for every other kernel the algorithmic figures. */
IHSBIN_API ihsbin_status ihsbin_kernel_exec(ihsbin_problem* p, int32_t cat, double* xflops, double* xbytes);

/* Launch geometry chosen by measurement (the library's own autotuner; the paper has none).
 * Launch sites whose candidate geometries compute identical values (cluster size of the
 * recursion's per-column kernels; the SMs the Gram of A leaves to the factorization beside
 * it) try each candidate on their first launches of a shape class, timed with CUDA events,
 * and settle on the fastest once every candidate has two samples.  The table is process-wide.
 * ihsbin_tuning_report writes one text line per tuned site and shape class (the chosen value and
 * every candidate's best time) into buf (cap bytes, NUL-terminated; *need receives the size
 * needed); ihsbin_tuning_reset forgets every choice. */
IHSBIN_API ihsbin_status ihsbin_tuning_report(char* buf, int64_t cap, int64_t* need);
IHSBIN_API ihsbin_status ihsbin_tuning_reset(void);

/* ---- Serving: a continuous-batching request loop (the library's runtime; the
 * paper solves one problem at a time).  `slots` worker threads each own a CUDA
 * stream; a worker admits the first queued request whose estimated device
 * footprint (ihsbin_request_footprint) fits the budget left, runs its whole
 * path (create, sketch, basis, evaluation, destroy) on its stream, and frees
 * the footprint when done, so requests arriving while others run enter as
 * slots and memory free up and their kernels overlap on the device.  Each
 * request is an independent problem: its result does not depend on what else
 * runs (up to the order of FP64 atomic additions in CSR Gram and CountSketch
 * accumulation). */
typedef struct ihsbin_server ihsbin_server;
typedef struct {
  int32_t slots;             /* concurrent requests; 0 selects 4                                  */
  uint64_t hbm_budget_bytes; /* admission budget; 0 selects the context's budget (0 = unlimited)  */
} ihsbin_serve_config;
typedef struct {
  ihsbin_matrix A;           /* borrowed until the request completes                               */
  const void* B;             /* n x K, row stride ldb, borrowed until completion                   */
  int64_t K, ldb;
  ihsbin_dtype b_dtype;
  int b_on_device;
  ihsbin_sketch_desc sketch;
  ihsbin_path_desc path;     /* its arrays (k, rho1, rho2) borrowed until completion               */
  const double* lambdas;     /* T values, copied at submission                                     */
  int64_t T;
  void* X;                   /* T x d x K output (ihsbin_eval_path layout), written on completion   */
  ihsbin_dtype x_dtype;
  int x_on_device;
} ihsbin_request;

/* Upper estimate of the device memory the request holds at its peak. */
IHSBIN_API ihsbin_status ihsbin_request_footprint(const ihsbin_request* q, uint64_t* bytes);
/* Start the workers.  Release with ihsbin_serve_destroy. */
IHSBIN_API ihsbin_status ihsbin_serve_create(ihsbin_ctx* ctx, const ihsbin_serve_config* cfg, ihsbin_server** out);
/* Queue a request (non-blocking).  IHSBIN_ERR_ADMISSION if its footprint can never fit the budget. */
IHSBIN_API ihsbin_status ihsbin_serve_submit(ihsbin_server* s, const ihsbin_request* q, uint64_t* ticket);
/* Wait up to timeout_us (0 = poll) for a request: IHSBIN_ERR_TIMEOUT if it is not done (the ticket
 * stays valid); otherwise *result is the request's status and the ticket is released.  times4 (may
 * be NULL) receives seconds of queueing, service, submission-to-completion, and device time. */
IHSBIN_API ihsbin_status ihsbin_serve_wait(ihsbin_server* s, uint64_t ticket, int64_t timeout_us,
                                           ihsbin_status* result, double* times4);
/* Finish every queued and running request, then stop the workers. */
IHSBIN_API ihsbin_status ihsbin_serve_destroy(ihsbin_server* s);
/* Blocking driver: submits reqs[i] at arrival_s[i] seconds after the call (NULL = all at once),
 * waits for all, and reports each status and its latency from scheduled arrival to completion. */
IHSBIN_API ihsbin_status ihsbin_serve(ihsbin_ctx* ctx, const ihsbin_serve_config* cfg, const ihsbin_request* reqs,
                                      int64_t n, const double* arrival_s, ihsbin_status* results,
                                      double* latency_s);

/* Allocation-free variant of the sketched Gram matrix (the paper has no
 * counterpart; this exists for callers that cannot allocate device memory).
 *
 * GS (D x D, row-major FP64, device) = SA^T SA for SA (m x D, row-major FP64,
 * device) -- the same matrix ihsbin_sketch forms from its sketch.  Callers
 * that cannot call cudaMalloc where they need it (latency-bound callers that
 * cannot absorb the device-wide synchronisation an allocation or free may
 * cause; hosts that hand all device memory to their own pool or fixed arena and
 * forbid allocations by libraries) use this entry point: it
 * calls no cudaMalloc, cudaFree or allocating library routine.  Its split-K
 * partial sums live in one file-scope device array of
 * IHSBIN_NOALLOC_SCRATCH_BYTES (16 MiB), which every GPU that loads the
 * library holds until the process exits; D*D must fit in it (D <= 1448),
 * otherwise IHSBIN_ERR_INVALID_ARG is returned before anything is launched.
 * All calls share that array: calls that overlap on the GPU race, so
 * serialise them.  The first call on a device (with that device current) looks
 * up the array's device address and caches it; make that first call before any
 * stream capture.  Stream-ordered on `stream` (a cudaStream_t, NULL = the
 * calling thread's default stream); returns after enqueueing, without
 * synchronising.  Inputs and
 * outputs are caller-owned. */
#define IHSBIN_NOALLOC_SCRATCH_BYTES (16u << 20)
IHSBIN_API ihsbin_status ihsbin_sketch_gram_noalloc(const double* SA, int64_t m, int64_t D, double* GS,
                                                    void* stream);

#ifdef __cplusplus
}
#endif
#endif /* IHSBIN_H */
