// Internal interfaces between the ABI layer (api.cu) and the kernel launchers (kernels.cu).
#pragma once
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/ihsbin.h"
#include "common.cuh"

struct ihsbin_ctx {
  int device = 0;
  uint64_t budget = 0;
  uint64_t in_use = 0;
  std::mutex mu;
  cudaMemPool_t pool = nullptr;  // stream-ordered pool that keeps freed memory for reuse
  int64_t fail_after = -1;        // test hook: allocations left before every one fails (-1: off)
};

namespace ihsbin {

// Tall view A_hat (N x D, N >= D) of the data: A itself, or A^T for the dual.
struct Tall {
  int64_t N = 0, D = 0;
  int layout = IHSBIN_DENSE_ROWMAJOR;
  int elem = ELEM_F64;
  // dense row-major (N x D) with row stride ld
  const void* A = nullptr;
  int64_t ld = 0;
  // CSR of A_hat (N rows) and of A_hat^T (D rows)
  const int64_t* rp = nullptr;
  const int32_t* ci = nullptr;
  const void* val = nullptr;
  const int64_t* rpT = nullptr;
  const int32_t* ciT = nullptr;
  const void* valT = nullptr;
  int64_t nnz = 0;
};

struct Plan {
  int L = 0;
  std::vector<double> edges, lam0, tau;
  std::vector<int32_t> k, jcount;
  int32_t jmax = 0;   // 0 = full basis
  int jc = 0;         // max jcount (buffer stride)
  int kmax = 0;
  int compute = IHSBIN_COMPUTE_F64;
  int product = IHSBIN_PRODUCT_GRAM;
  int gram = IHSBIN_GRAM_FMA;   // resolved Gram kernel (never AUTO)
  int loop = IHSBIN_LOOP_FMA;   // resolved product kernel of the basis recursion (never AUTO)
  int factor = IHSBIN_FACTOR_FMA;  // resolved kernel of the explicit inverse (never AUTO)
  int slice_w = 6;                 // slice pairs kept by the recursion's and the inverse's products
  int form = IHSBIN_FORM_AUTO;     // requested; resolved by the build into form_run
  int precond_req = 0;             // requested pair weight of the residual form's P_l r (0: from the bound)
  int form_run = 0, precond_w = 6; // what the last build ran (0: no build yet)
  // parameters completed after the factor phase (rho from the sketch, k from Theorem 4)
  bool auto_rho = false, auto_k = false;
  double eps = 1e-7;
  double sigma_d2 = 0.0;  // known smallest eigenvalue bound (0: the default centring)
  std::vector<double> rho1, rho2;
  std::vector<double> tau_user;  // explicit per-interval steps (empty: Theorem 4's rule)
};

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// Kernel categories for the opt-in per-launch timing (ihsbin_kernel_stats).
enum KCat : int {
  K_SKETCH_DRAW = 0, K_SKETCH_APPLY, K_SKETCH_GRAM, K_FACTOR_SHIFT, K_FACTOR_POTRF, K_FACTOR_TRSM,
  K_FACTOR_SYRK, K_TRTRI, K_INVERSE, K_GRAM, K_RHS, K_LOOP_Y, K_LOOP_P, K_DUAL_MAP, K_EVAL_COEF, K_EVAL,
  K_SPARSE, K_GRAM_SLICE, K_GRAM_TC, K_GRAM_COMBINE, K_LOOP_SLICE, K_LOOP_Y_TC, K_LOOP_P_TC, K_INVERSE_SLICE,
  K_INVERSE_TC, K_TRTRI_TC, K_SYRK_TC, K_LOSS_SLICE, K_LOSS_TC, K_LOSS_IMAGE, K_LOSS_RESID, K_ADAPTIVE,
  K_SKETCH_IMAGE, K_SKETCH_TC, K_SKETCH_REDUCE, K_NCAT
};
struct KStat {
  int64_t launches = 0;
  double ms = 0, flops = 0, bytes = 0;  // the method's (algorithmic) work
  double xflops = 0, xbytes = 0;        // the work the implementation executes (slice products, slice images)
};

}  // namespace ihsbin

namespace ihsbin {
struct TuneLaunch;
}

struct ihsbin_problem {
  ihsbin_ctx* ctx = nullptr;
  cudaStream_t side = nullptr;  // build_basis: the Gram's stream, overlapping ...
  cudaStream_t fac = nullptr;   // ... the factorization's stream
  int64_t n = 0, d = 0, K = 0;
  bool dual = false;
  ihsbin::Tall A;
  bool tf32 = false;                     // A's values were rounded to TF32 (held as FP32)
  std::vector<ihsbin::DevBuf> owned;     // every device allocation of this problem
  double* B = nullptr;                   // n x K (FP64, device)
  int* status = nullptr;                 // device status word
  // sketch
  bool sketched = false;
  ihsbin_sketch_desc sk{};
  double* SA = nullptr;                  // m x D FP64
  double* GS = nullptr;                  // D x D FP64
  double trGS = 0.0;                     // its trace (host copy, for the residual form's pair weight)
  int64_t* sk_idx = nullptr;             // device
  int8_t* sk_sign = nullptr;             // device
  int64_t sk_idx_count = 0, sk_sign_count = 0;
  // basis
  bool built = false;
  ihsbin::Plan plan;
  ihsbin::CBuf G;                        // D x D (gram product mode)
  ihsbin::CBuf Pinv;                     // L x D x D
  ihsbin::CBuf Ut;                       // L x jc x K x D
  ihsbin::CBuf W;                        // dual: L x jc x K x N (primal basis)
  std::vector<ihsbin::DevBuf> basis_bufs;
  // The Gram of A and A^T b that ihsbin_sketch starts on the side stream for the next build
  // (float-float, sliced Gram, dense data; they do not depend on the sketch): taken by that build
  // when its mode matches, else waited for and freed.
  bool gram_pre = false;
  ihsbin::CBuf G_pre, c_pre;
  std::vector<ihsbin::DevBuf> pre_bufs;
  cudaEvent_t pre_ev[2] = {nullptr, nullptr};  // start / end of the background Gram (side stream)
  bool pre_taken = false;                      // the running build uses them
  ihsbin::TuneLaunch* pre_tune = nullptr;      // the SMs it leaves free: tuned from its start to the build's join
  int last_compute = -1, last_gram = -1;       // mode of the last successful build (-1: none)
  bool pre_off = false;                        // set while Algorithm 4 re-sketches (no build follows)
  float phase_ms[5] = {0, 0, 0, 0, 0};
  // per-launch accounting: counts and algorithmic work always; event timing when enabled
  bool timing = false;
  ihsbin::KStat kstat[ihsbin::K_NCAT];
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<std::pair<int, size_t>> ev_pending;  // (category, index of start event)
};

namespace ihsbin {

// Text returned by ihsbin_last_error() on this thread (api.cu).
void set_last_error(const char* msg);

// Stream that the current ABI call allocates and frees on (stream-ordered pool allocations).
extern thread_local cudaStream_t g_call_stream;
struct CallStream {
  cudaStream_t saved;
  explicit CallStream(cudaStream_t s) : saved(g_call_stream) { g_call_stream = s ? s : cudaStreamPerThread; }
  ~CallStream() { g_call_stream = saved; }
};

// ----- allocation helpers (api.cu) --------------------------------------------
// Lifetime of a device allocation: the problem, the current basis, or the current call.
enum Scope : int { SCOPE_PERSIST = 0, SCOPE_BASIS = 1, SCOPE_SCRATCH = 2, SCOPE_PRE = 3 };
cudaError_t prob_alloc(ihsbin_problem* p, size_t bytes, void** out, int scope);
void prob_free_basis(ihsbin_problem* p);
void pre_gram_discard(ihsbin_problem* p);  // waits for a background Gram (if any) and frees it
CBuf alloc_cbuf(ihsbin_problem* p, int compute, size_t elems, int scope, cudaError_t* err);

// Records one launch of category `cat` with its algorithmic flops / bytes, and
// brackets it with events on `st` when timing is enabled (resolved by
// resolve_timing after the call's synchronisation point).
struct KTimer {
  ihsbin_problem* p;
  int cat;
  cudaStream_t st;
  size_t idx = 0;
  // flops / bytes: the method's algorithmic work; xflops / xbytes (< 0: the same) what the launch executes
  KTimer(ihsbin_problem* pp, int c, cudaStream_t s, double flops, double bytes, double xflops = -1,
         double xbytes = -1);
  ~KTimer();
};
void resolve_timing(ihsbin_problem* p);

// ----- online autotuner of launch geometry (tune.cu) ---------------------------
struct TuneLaunch {
  uint64_t key = 0;
  int cand = 0, value = 0;
  bool timed = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
};
enum TuneSite : int { TUNE_COL_R = 1, TUNE_COL_UPDATE = 2, TUNE_COL_MW = 3, TUNE_GRAM_RESERVE = 4, TUNE_PRE_RESERVE = 5 };
uint64_t tune_key(int site, int64_t a, int64_t b, int64_t c);
int shape_class(int64_t n);  // ceil(log2 n)
// The geometry value to launch with (values[cand]); while the key is being tuned the launch is
// bracketed by events: call tune_end after it on the same stream.
TuneLaunch tune_begin(uint64_t key, const char* site, const int* values, int ncand, cudaStream_t st);
void tune_end(TuneLaunch& t, cudaStream_t st);
void tune_resolve();  // after this host thread's tuned launches have completed
void tune_discard();
std::string tune_report();
void tune_reset();

// ----- kernel launchers (kernels.cu); all return the first CUDA error --------
cudaError_t launch_transpose_dense(const void* src, int elem, int64_t rows, int64_t cols, int64_t ld,
                                   void* dst, cudaStream_t st);
cudaError_t launch_csr_check(const int64_t* rp, const int32_t* ci, int64_t rows, int64_t cols, int64_t nnz,
                             int* status, cudaStream_t st);
cudaError_t launch_csr_transpose(ihsbin_problem* p, const int64_t* rp, const int32_t* ci, const void* val,
                                 int elem, int64_t rows, int64_t cols, int64_t nnz, int64_t** rpT,
                                 int32_t** ciT, void** valT, cudaStream_t st);
cudaError_t launch_convert_to_f64(const void* src, int elem, int64_t rows, int64_t cols, int64_t ld,
                                  double* dst, cudaStream_t st);

cudaError_t sketch_gaussian(ihsbin_problem* p, cudaStream_t st);
// Gaussian sketch with BF16 entries of dense BF16 data on the tensor cores (tc_sketch.cu)
bool sketch_gaussian_tc_ok(const ihsbin_problem* p);
cudaError_t sketch_gaussian_tc(ihsbin_problem* p, cudaStream_t st);
// BF16 bits of the entries [i0, i0 + rows) x [j0, j0 + cols) of the problem's Gaussian sketch (row-major)
cudaError_t gaussian_entries_bf16(ihsbin_problem* p, int64_t i0, int64_t rows, int64_t j0, int64_t cols,
                                  uint16_t* out_dev, cudaStream_t st);
cudaError_t sketch_countsketch(ihsbin_problem* p, cudaStream_t st);
cudaError_t sketch_srht(ihsbin_problem* p, cudaStream_t st);
cudaError_t sketch_gram(ihsbin_problem* p, cudaStream_t st);

cudaError_t build_basis_device(ihsbin_problem* p, cudaStream_t st, cudaEvent_t* ev);
// Completes tau, k, jcount, jc, kmax of p->plan; trP[l] = tr(P_l) when rho comes from the sketch (api.cu).
void finalize_plan(ihsbin_problem* p, const double* trP);

// CSR data (sparse.cu)
cudaError_t csr_gram(ihsbin_problem* p, int compute, cudaStream_t st);

// Dense FP32/BF16 Gram on the tensor cores from exact integer slices (tc_gram.cu)
constexpr int kGramSlices = 6;     // BF16 slices per FP32 entry
constexpr int kGramSlicesBf16 = 4; // BF16 slices per BF16 entry (every entry within 2^-23 of its column maximum exact)
constexpr int kGramMaxWeight = 6;  // slice pairs (s, t) kept: s + t <= kGramMaxWeight
constexpr int kRhsSlices = 6;      // BF16 slices per FP64 entry of B in the right-hand side A_hat^T B
inline int gram_slices_for(int elem, bool tf32) { return elem == ELEM_BF16 || tf32 ? kGramSlicesBf16 : kGramSlices; }
// FP32 values rounded to TF32 (to nearest, ties away from zero): rows x cols with row stride ld -> dst (stride cols)
cudaError_t launch_round_tf32(const float* src, int64_t ld, int64_t rows, int64_t cols, float* dst, cudaStream_t st);
// reserve_sms > 0: the tensor-core launches leave that many SMs free (for work on other streams);
// rhs != nullptr: also c = A_hat^T B (column-major D x K) from the same slices of A_hat
cudaError_t gram_dense_slices(ihsbin_problem* p, int compute, cudaStream_t st, int reserve_sms = 0,
                              CBuf* rhs = nullptr);
// The problem's two internal streams (created once): the side stream at the lowest priority (the
// Gram), the factorization's at the highest.
cudaError_t ensure_streams(ihsbin_problem* p);
cudaError_t gs_trace_launch(ihsbin_problem* p, double* out, cudaStream_t st);  // tr(G_S) into out (device)
// Whether ihsbin_sketch starts the Gram of A and A^T b in the background, and the launch itself
// (on p->side, into SCOPE_PRE buffers; the caller owns the scratch scope on that stream).
bool pre_gram_eligible(const ihsbin_problem* p);
cudaError_t pre_gram_launch(ihsbin_problem* p);
// G_S = (S A_hat)^T (S A_hat) from the FP64 sketch on the tensor cores (7 slices, FP64-class)
cudaError_t sketch_gram_slices(ihsbin_problem* p, cudaStream_t st);
uint64_t gram_slices_scratch_bytes(int64_t N, int64_t D);

// Exact-slice tensor-core products of the basis recursion (tc_loop.cu).  A operands
// (D x D, rows sliced, once per build) and B operands (column panels, every step).
int oz_tile_n(int64_t ncolg, int wmax = 6);  // 64-column tiles for products keeping s + t <= 3
size_t oz_rows_elems(int64_t D);
size_t oz_rows_exps(int64_t D);
size_t oz_cols_elems(int64_t D, int64_t ncolg, int NT);
size_t oz_cols_exps(int64_t ncolg, int NT);
// (float-float operands)
cudaError_t oz_slice_rows(CBuf X, int64_t D, int groups, int64_t gs, __nv_bfloat16* out, int* ea, cudaStream_t st);
cudaError_t oz_slice_cols(CBuf X, int64_t D, int ngroups, int64_t ncolg, int NT, int64_t cpg, int64_t gs,
                          const int* perm, __nv_bfloat16* out, int* eb, cudaStream_t st);
int oz_pick_split(int64_t D, int64_t ncolg, int groups, int NT, int cap);
// writes the exact int64 partials ohi / olo (see oz_join in common.cuh), entry ((s * groups + g) * ncolg + j) * D + i
cudaError_t oz_product(const __nv_bfloat16* As, const int* ea, const int* a_perm, bool a_shared,
                       const __nv_bfloat16* Bs, const int* eb, int64_t D, int64_t ncolg, int groups, int NT,
                       int ksplit, long long* ohi, long long* olo, int* status, cudaStream_t st, int wmax = 6);
double oz_pair_flops(int64_t M, int64_t N, int64_t K, int wmax = 6);

// General form: C_g = X_g Y_g^T (M x N, contraction K) for every group g, X sliced into 128-row
// tiles (A operand), Y into NT-row tiles (NT = 16 or 32, B operand).  Triangular operands: zero
// k-blocks skipped per output tile; sym: only the tiles that touch i <= j are computed.
enum OzTri : int { OZ_TRI_GE_ROW = 1, OZ_TRI_GE_COL = 2, OZ_TRI_LE_ROW = 4 };
struct OzGemm {
  const __nv_bfloat16* As = nullptr;
  const int* ea = nullptr;
  const int* a_perm = nullptr;
  bool a_shared = false;
  const __nv_bfloat16* Bs = nullptr;
  const int* eb = nullptr;
  bool b_shared = false;  // one B for every group
  // pair mode: group 2q multiplies A group q of As (a_perm) and group 2q + 1 A group q of As2
  // (a_perm2), both by B group q
  int pair = 0;
  const __nv_bfloat16* As2 = nullptr;
  const int* a_perm2 = nullptr;
  int64_t M = 0, N = 0, K = 0;
  int groups = 1, NT = 32, ksplit = 1, tri = 0, sym = 0;
  long long* ohi = nullptr;  // exact partials, entry ((s * groups + g) * N + j) * M + i
  long long* olo = nullptr;
  int* status = nullptr;
  int wmax = 6;              // slice pairs kept: s + t <= wmax (4 .. 6)
  // float-float epilogue instead of the partials (ksplit = 1 only): C_ij joined with the row and
  // column exponents and written into out (group g at g * out_gs, row stride out_ld):
  //   OZ_EPI_STORE_NEG : out[(r0 + i) ld + c0 + j]  = -C_ij
  //   OZ_EPI_STORE_SYM : out[j ld + i] = out[i ld + j] = C_ij for i <= j
  int epi = 0;
  CBuf out{};
  int64_t out_ld = 0, out_gs = 0, out_r0 = 0, out_c0 = 0;
};
enum OzEpi : int { OZ_EPI_PARTIALS = 0, OZ_EPI_STORE_NEG = 2, OZ_EPI_STORE_SYM = 3 };
cudaError_t oz_gemm(const OzGemm& q, cudaStream_t st);
// the recursion's update in the two-product form (partials of M_q U and P_l U from a pair-mode product)
cudaError_t oz_update_mw_slice(const long long* Phi, const long long* Plo, int S, const int* em, const int* ep,
                               int live, int64_t ncol, int64_t D, int64_t K, CBuf Uin, CBuf Uout, CBuf Ut,
                               const int* perm, const double* tau, const double* lam0, int64_t gs, const int* eu_in,
                               int live_next, __nv_bfloat16* Us, int* eu, cudaStream_t st);
// M_q = P_l (G + lam0_l I) from the exact partials of G P_l
cudaError_t oz_make_M(const long long* hi, const long long* lo, int S, int64_t D, int T, const int* eg, const int* epc,
                      int64_t epc_gs, const int* perm, const double* lam0, CBuf P, CBuf M, cudaStream_t st);
size_t oz_vec_elems(int64_t nvec, int64_t K, int TH);  // slices of nvec vectors of length K, tile height TH
size_t oz_vec_exps(int64_t nvec, int TH);
// vectors = the columns of row-major float-float matrices (K rows, row stride ld, group stride gs)
cudaError_t oz_slice_matcols(CBuf X, int64_t ld, int64_t K, int64_t nvec, int groups, int64_t gs, int TH,
                             __nv_bfloat16* out, int* e, cudaStream_t st);
// vectors with contiguous entries: vector v of group g at g * gs + off + v * vstride, K entries
cudaError_t oz_slice_vecs(CBuf X, int64_t gs, int64_t off, int64_t vstride, int64_t K, int64_t nvec, int groups,
                          int TH, __nv_bfloat16* out, int* e, cudaStream_t st);
int oz_pick_split_mnk(int64_t M, int64_t N, int64_t K, int groups, int NT, int cap);
// rows of a row-major data matrix (element type elem, row stride ld, K entries), tile height TH
cudaError_t oz_slice_data_rows(const void* X, int elem, int64_t ld, int64_t K, int64_t nvec, int TH,
                               __nv_bfloat16* out, int* e, cudaStream_t st);
// The recursion's elementwise steps with the slicing of their output fused (one CTA per column,
// the column in D x 8 bytes of shared memory; oz_fused_ok(D) says whether it fits).
bool oz_fused_ok(int64_t D);
cudaError_t oz_make_R_slice(const long long* Yhi, const long long* Ylo, int ny, int64_t ny_stride, const int* eg,
                            const int* eu, CBuf U, int live, int64_t nold, int64_t nnew, int64_t D, int64_t K, int inew,
                            const int* perm, const double* tau, const double* lam0, int64_t gs, int NT,
                            __nv_bfloat16* Rs, int* er, CBuf c, cudaStream_t st);
cudaError_t oz_update_slice(const long long* Zhi, const long long* Zlo, int S, const int* ep, int64_t ep_gs,
                            const int* er, int64_t er_gs, int live, int64_t ncol, int64_t D, int64_t K, int i, CBuf Uin,
                            CBuf Uout, CBuf Ut, const int* perm, int64_t gs, int live_next, int NTn, __nv_bfloat16* Us,
                            int* eu, int resid, cudaStream_t st);
// device bytes of the recursion's slices (G, every P_l, one step's B operand)
uint64_t loop_slices_bytes(int64_t D, int L, int64_t ncol_max);
cudaError_t csr_rhs(ihsbin_problem* p, int compute, CBuf c, cudaStream_t st);
cudaError_t csr_dual_map(ihsbin_problem* p, int compute, int64_t ncol, cudaStream_t st);
cudaError_t basis_transpose(ihsbin_problem* p, int compute, CBuf W, int64_t d, int64_t nc, CBuf WT, cudaStream_t st);
cudaError_t csr_basis_image(ihsbin_problem* p, int compute, const int64_t* rp, const int32_t* ci, const void* val,
                            int64_t n_rows, CBuf WT, int64_t nc, CBuf V, cudaStream_t st);
// Algorithm 4's device state (D x K column-major vectors in the compute mode's format)
struct AdaptiveBufs {
  CBuf G, c, P, x, g, d, hd;
  double* lam_dev = nullptr;  // the shift lambda (one double)
  double* part = nullptr;     // inner-product partial sums
  double* dots = nullptr;     // [0] = <d, g>, [1] = <d, (G + lam I) d>
};
cudaError_t adaptive_setup(ihsbin_problem* p, AdaptiveBufs& b, cudaStream_t st);      // G, c; x = 0, g = -c
cudaError_t adaptive_precond(ihsbin_problem* p, AdaptiveBufs& b, cudaStream_t st);    // P = (G_S + lam I)^-1
cudaError_t adaptive_direction(ihsbin_problem* p, AdaptiveBufs& b, cudaStream_t st);  // d = P g, dots[0]
cudaError_t adaptive_curvature(ihsbin_problem* p, AdaptiveBufs& b, double lam, cudaStream_t st);  // hd, dots[1]
cudaError_t adaptive_step(ihsbin_problem* p, AdaptiveBufs& b, double t, cudaStream_t st);  // x -= t d, g -= t hd
cudaError_t adaptive_export_x(ihsbin_problem* p, AdaptiveBufs& b, double* out_dev, cudaStream_t st);
// training / test losses along the path (device outputs of T doubles, either may be null)
cudaError_t losses_device(ihsbin_problem* p, const double* lam_host, const double* lam_dev, int64_t T, const void* At,
                          int at_elem, int64_t at_ld, int64_t n_test, const double* Bt, double* train_out,
                          double* test_out, cudaStream_t st);
cudaError_t eval_device(ihsbin_problem* p, const double* lambdas_host, const double* lambdas_dev, int64_t T, void* X_dev, int x_elem,
                        cudaStream_t st);

}  // namespace ihsbin
