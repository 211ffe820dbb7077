// extern "C" entry points of libihsbin (declared in include/ihsbin.h).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.h"
#include <nvtx3/nvToolsExt.h>

using namespace ihsbin;

namespace {

thread_local std::string g_err;

ihsbin_status fail(ihsbin_status s, const std::string& msg) {
  g_err = msg;
  return s;
}
ihsbin_status cuda_fail(cudaError_t e, const char* where) {
  if (e == cudaErrorMemoryAllocation) return fail(IHSBIN_ERR_OUT_OF_MEMORY, std::string(where) + ": out of device memory");
  if (e == cudaErrorNotSupported) return fail(IHSBIN_ERR_UNSUPPORTED, std::string(where) + ": combination not supported");
  if (e == cudaErrorInvalidValue && g_err.rfind("admission", 0) == 0) return IHSBIN_ERR_ADMISSION;
  return fail(IHSBIN_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

thread_local std::vector<DevBuf>* g_scratch = nullptr;

size_t elem_size(int dt) { return dt == IHSBIN_F64 ? 8 : (dt == IHSBIN_F32 || dt == IHSBIN_TF32) ? 4 : 2; }

void free_list(ihsbin_problem* p, std::vector<DevBuf>& v) {
  std::lock_guard<std::mutex> g(p->ctx->mu);
  for (auto& b : v) {
    cudaFreeAsync(b.p, ihsbin::g_call_stream);
    p->ctx->in_use -= b.bytes;
  }
  v.clear();
}

struct ScratchScope {  // frees the call's scratch allocations when the call returns (nests)
  ihsbin_problem* p;
  std::vector<DevBuf> bufs;
  std::vector<DevBuf>* saved;
  explicit ScratchScope(ihsbin_problem* pp) : p(pp), saved(g_scratch) { g_scratch = &bufs; }
  ~ScratchScope() {
    g_scratch = saved;
    free_list(p, bufs);
  }
};

// Status word check after a synchronisation point.
ihsbin_status check_status(ihsbin_problem* p, cudaStream_t st, const char* where) {
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, where);
  resolve_timing(p);
  tune_resolve();
  int s = 0;
  e = cudaMemcpy(&s, p->status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, where);
  if (s != 0) {
    cudaMemset(p->status, 0, sizeof(int));
    if (s == DEV_NOT_SPD) return fail(IHSBIN_ERR_NOT_SPD, std::string(where) + ": non-positive pivot in a factor of (SA)^T SA + lam0 I");
    if (s == DEV_NAN) return fail(IHSBIN_ERR_NAN, std::string(where) + ": non-finite value on the device");
    if (s == DEV_TIMEOUT)
      return fail(IHSBIN_ERR_TIMEOUT, std::string(where) + ": a tensor-core pipeline wait expired (the kernel gave up)");
    return fail(IHSBIN_ERR_CUDA, std::string(where) + ": device status " + std::to_string(s));
  }
  return IHSBIN_OK;
}

}  // namespace

namespace ihsbin {

thread_local cudaStream_t g_call_stream = cudaStreamPerThread;

// tau from Theorem 4's proof; rho from the sketch when asked; k from Theorem 4's rate when asked.
void finalize_plan(ihsbin_problem* p, const double* trP) {
  Plan& pl = p->plan;
  const double D = (double)p->A.D, m = (double)p->sk.m;
  for (int l = 0; l < pl.L; ++l) {
    const double lo = pl.edges[l], hi = pl.edges[l + 1];
    if (pl.auto_rho && trP) {
      const double de = std::max(1.0, D - pl.lam0[l] * trP[l]);
      const double r = std::min(de / m, 0.95);
      pl.rho1[l] = (1.0 + std::sqrt(r)) * (1.0 + std::sqrt(r));
      pl.rho2[l] = (1.0 - std::sqrt(r)) * (1.0 - std::sqrt(r));
    }
    const double s2 = pl.sigma_d2;
    pl.tau[l] = pl.tau_user.empty() ? 2.0 * (pl.lam0[l] + s2) / ((lo + s2) / pl.rho1[l] + (hi + s2) / pl.rho2[l])
                                    : pl.tau_user[l];
    if (pl.auto_k) {
      const double kt = pl.rho1[l] * (hi + s2) / (pl.rho2[l] * (lo + s2));
      const double rate = (kt - 1.0) / (kt + 1.0);
      double k = rate > 0 ? std::ceil(std::log(pl.eps) / std::log(rate)) : 1.0;
      pl.k[l] = (int32_t)std::min(std::max(k, 1.0), 20000.0);
    }
    pl.jcount[l] = pl.jmax > 0 ? std::min(pl.k[l], pl.jmax) : pl.k[l];
  }
  pl.jc = *std::max_element(pl.jcount.begin(), pl.jcount.end());
  pl.kmax = *std::max_element(pl.k.begin(), pl.k.end());
}

void set_last_error(const char* msg) { g_err = msg; }

cudaError_t prob_alloc(ihsbin_problem* p, size_t bytes, void** out, int scope) {
  *out = nullptr;
  if (bytes == 0) bytes = 16;
  {
    std::lock_guard<std::mutex> g(p->ctx->mu);
    if (p->ctx->fail_after == 0) {
      g_err = "allocation failed (the context's allocation-failure hook)";
      return cudaErrorMemoryAllocation;
    }
    if (p->ctx->fail_after > 0) --p->ctx->fail_after;
    if (p->ctx->budget && p->ctx->in_use + bytes > p->ctx->budget) {
      g_err = "admission: request exceeds the context's device-memory budget";
      return cudaErrorInvalidValue;
    }
    p->ctx->in_use += bytes;
  }
  cudaError_t e = cudaMallocFromPoolAsync(out, bytes, p->ctx->pool, g_call_stream);
  if (e != cudaSuccess) {
    std::lock_guard<std::mutex> g(p->ctx->mu);
    p->ctx->in_use -= bytes;
    *out = nullptr;
    return e;
  }
  DevBuf b{*out, bytes};
  if (scope == SCOPE_SCRATCH && g_scratch) g_scratch->push_back(b);
  else if (scope == SCOPE_PERSIST) p->owned.push_back(b);
  else if (scope == SCOPE_PRE) p->pre_bufs.push_back(b);
  else p->basis_bufs.push_back(b);
  return cudaSuccess;
}

// Waits for a background Gram of an earlier sketch and frees its buffers (on the side stream).
void pre_gram_discard(ihsbin_problem* p) {
  if (p->side) cudaStreamSynchronize(p->side);
  {
    CallStream cs(p->side);
    free_list(p, p->pre_bufs);
  }
  if (p->pre_tune) {  // a tuning sample that no build completed
    if (p->pre_tune->timed) {
      cudaEventDestroy(p->pre_tune->e0);
      cudaEventDestroy(p->pre_tune->e1);
    }
    delete p->pre_tune;
    p->pre_tune = nullptr;
  }
  p->gram_pre = p->pre_taken = false;
  p->G_pre = p->c_pre = CBuf{};
}

CBuf alloc_cbuf(ihsbin_problem* p, int compute, size_t elems, int scope, cudaError_t* err) {
  CBuf b;
  if (*err != cudaSuccess) return b;
  cudaError_t e;
  if (compute == IHSBIN_COMPUTE_F64) {
    e = prob_alloc(p, elems * 8, &b.p0, scope);
  } else {
    e = prob_alloc(p, elems * 4, &b.p0, scope);
    if (e == cudaSuccess) e = prob_alloc(p, elems * 4, &b.p1, scope);
  }
  if (e != cudaSuccess) *err = e;
  return b;
}

const char* const kcat_names[K_NCAT] = {
    "sketch_draw", "sketch_apply", "sketch_gram", "factor_shift", "factor_potrf", "factor_trsm", "factor_syrk",
    "trtri", "inverse_syrk", "gram", "rhs", "loop_gram_product", "loop_precond_update", "dual_map",
    "eval_coef", "eval", "sparse", "gram_slice", "gram_tc_mma", "gram_combine", "loop_slice", "loop_gram_tc",
    "loop_precond_tc", "factor_slice", "inverse_tc", "trtri_tc", "factor_syrk_tc", "loss_slice", "loss_image_tc",
    "loss_image", "loss_resid", "adaptive_step", "sketch_image", "sketch_tc", "sketch_reduce"};

// Every KTimer scope is also an NVTX range named by its category, so that a profiler can select
// a category's launches (no cost when no tool is attached).
KTimer::KTimer(ihsbin_problem* pp, int c, cudaStream_t s, double flops, double bytes, double xflops, double xbytes)
    : p(pp), cat(c), st(s) {
  nvtxRangePushA(kcat_names[c]);
  KStat& k = p->kstat[c];
  k.launches += 1;
  k.flops += flops;
  k.bytes += bytes;
  k.xflops += xflops >= 0 ? xflops : flops;
  k.xbytes += xbytes >= 0 ? xbytes : bytes;
  if (!p->timing) return;
  while (p->ev_pool.size() < p->ev_used + 2) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    p->ev_pool.push_back(e);
  }
  idx = p->ev_used;
  p->ev_used += 2;
  cudaEventRecord(p->ev_pool[idx], st);
  p->ev_pending.push_back({c, idx});
}
KTimer::~KTimer() {
  if (p->timing) cudaEventRecord(p->ev_pool[idx + 1], st);
  nvtxRangePop();
}
void resolve_timing(ihsbin_problem* p) {
  for (auto& pr : p->ev_pending) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, p->ev_pool[pr.second], p->ev_pool[pr.second + 1]) == cudaSuccess)
      p->kstat[pr.first].ms += ms;
  }
  p->ev_pending.clear();
  p->ev_used = 0;
}

void prob_free_basis(ihsbin_problem* p) {
  free_list(p, p->basis_bufs);
  p->G = CBuf{};
  p->Pinv = CBuf{};
  p->Ut = CBuf{};
  p->W = CBuf{};
  p->built = false;
}

}  // namespace ihsbin


namespace {
// A named range on the profiler's timeline for each hot-path call (NVTX, header-only; no cost
// when no tool is attached).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};
}  // namespace

extern "C" {

const char* ihsbin_last_error(void) { return g_err.c_str(); }

ihsbin_status ihsbin_ctx_create(int device, uint64_t budget, ihsbin_ctx** out) {
  if (!out) return fail(IHSBIN_ERR_INVALID_ARG, "ctx_create: out is NULL");
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) return fail(IHSBIN_ERR_CUDA, "ctx_create: no CUDA device available");
  if (device < 0 || device >= n) return fail(IHSBIN_ERR_INVALID_ARG, "ctx_create: device index out of range");
  if ((e = cudaSetDevice(device)) != cudaSuccess) return cuda_fail(e, "ctx_create");
  if ((e = cudaFree(nullptr)) != cudaSuccess) return cuda_fail(e, "ctx_create");
  ihsbin_ctx* c = new (std::nothrow) ihsbin_ctx();
  if (!c) return fail(IHSBIN_ERR_OUT_OF_MEMORY, "ctx_create: host allocation failed");
  c->device = device;
  c->budget = budget;
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = device;
  if ((e = cudaMemPoolCreate(&c->pool, &props)) != cudaSuccess) {
    delete c;
    return cuda_fail(e, "ctx_create: memory pool");
  }
  uint64_t keep = UINT64_MAX;  // freed blocks stay in the pool for the next request
  cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  // No reuse that would make an allocation wait for another stream's pending free: the problem's
  // streams run concurrently (the sketch beside the background Gram, the factorization beside the
  // Gram), and such a wait would serialise them; the pool grows instead.
  int no_deps = 0;
  cudaMemPoolSetAttribute(c->pool, cudaMemPoolReuseAllowInternalDependencies, &no_deps);
  *out = c;
  return IHSBIN_OK;
}

ihsbin_status ihsbin_tuning_report(char* buf, int64_t cap, int64_t* need) {
  const std::string r = tune_report();
  if (need) *need = (int64_t)r.size() + 1;
  if (buf && cap > 0) {
    const size_t n = std::min<size_t>(r.size(), (size_t)cap - 1);
    std::copy(r.begin(), r.begin() + n, buf);
    buf[n] = 0;
  }
  return IHSBIN_OK;
}

ihsbin_status ihsbin_tuning_reset(void) {
  tune_reset();
  return IHSBIN_OK;
}

ihsbin_status ihsbin_ctx_fail_allocations(ihsbin_ctx* ctx, int64_t after) {
  if (!ctx) return fail(IHSBIN_ERR_INVALID_ARG, "ctx_fail_allocations: NULL");
  std::lock_guard<std::mutex> g(ctx->mu);
  ctx->fail_after = after < 0 ? -1 : after;
  return IHSBIN_OK;
}

ihsbin_status ihsbin_ctx_destroy(ihsbin_ctx* c) {
  if (!c) return fail(IHSBIN_ERR_INVALID_ARG, "ctx_destroy: NULL");
  if (c->in_use) return fail(IHSBIN_ERR_STATE, "ctx_destroy: problems still hold device memory");
  cudaSetDevice(c->device);
  cudaStreamSynchronize(cudaStreamPerThread);
  if (c->pool) cudaMemPoolDestroy(c->pool);
  delete c;
  return IHSBIN_OK;
}

ihsbin_status ihsbin_ctx_memory(const ihsbin_ctx* c, uint64_t* bytes) {
  if (!c || !bytes) return fail(IHSBIN_ERR_INVALID_ARG, "ctx_memory: NULL argument");
  *bytes = c->in_use;
  return IHSBIN_OK;
}

ihsbin_status ihsbin_problem_create(ihsbin_ctx* ctx, const ihsbin_matrix* A, const void* B, int64_t K, int64_t ldb,
                                    ihsbin_dtype b_dtype, int b_on_device, ihsbin_problem** out) {
  Range range_("ihsbin_problem_create");
  if (!ctx || !A || !B || !out) return fail(IHSBIN_ERR_INVALID_ARG, "problem_create: NULL argument");
  *out = nullptr;
  if (A->n <= 0 || A->d <= 0 || K <= 0 || ldb < K) return fail(IHSBIN_ERR_INVALID_ARG, "problem_create: bad sizes");
  if (A->dtype < IHSBIN_F64 || A->dtype > IHSBIN_TF32) return fail(IHSBIN_ERR_INVALID_ARG, "problem_create: bad dtype");
  if (b_dtype != IHSBIN_F64 && b_dtype != IHSBIN_F32) return fail(IHSBIN_ERR_INVALID_ARG, "problem_create: B must be F64 or F32");
  if (A->layout == IHSBIN_DENSE_ROWMAJOR) {
    if (!A->values || A->ld < A->d) return fail(IHSBIN_ERR_INVALID_ARG, "problem_create: dense values NULL or ld < d");
  } else if (A->layout == IHSBIN_CSR) {
    if (!A->values || !A->row_ptr || !A->col_idx || A->nnz < 0)
      return fail(IHSBIN_ERR_INVALID_ARG, "problem_create: CSR arrays NULL or nnz < 0");
  } else {
    return fail(IHSBIN_ERR_INVALID_ARG, "problem_create: bad layout");
  }
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(e, "problem_create");
  CallStream cs(nullptr);
  ihsbin_problem* p = new (std::nothrow) ihsbin_problem();
  if (!p) return fail(IHSBIN_ERR_OUT_OF_MEMORY, "problem_create: host allocation failed");
  p->ctx = ctx;
  p->n = A->n;
  p->d = A->d;
  p->K = K;
  p->dual = A->n < A->d;
  auto bail = [&](cudaError_t err, const char* where) {
    ihsbin_status s = cuda_fail(err, where);
    ihsbin_problem_destroy(p);
    return s;
  };
  const size_t es = elem_size(A->dtype);
  Tall& T = p->A;
  T.layout = A->layout;
  T.elem = A->dtype == IHSBIN_F64 ? ELEM_F64 : (A->dtype == IHSBIN_F32 || A->dtype == IHSBIN_TF32) ? ELEM_F32 : ELEM_BF16;
  p->tf32 = A->dtype == IHSBIN_TF32;
  if ((e = prob_alloc(p, sizeof(int), (void**)&p->status, SCOPE_PERSIST)) != cudaSuccess) return bail(e, "problem_create");
  cudaMemset(p->status, 0, sizeof(int));
  if (A->layout == IHSBIN_DENSE_ROWMAJOR) {
    const void* src = A->values;
    int64_t ld = A->ld;
    if (!A->on_device) {  // copy, packing rows to ld = d
      void* dptr = nullptr;
      if ((e = prob_alloc(p, (size_t)A->n * A->d * es, &dptr, SCOPE_PERSIST)) != cudaSuccess) return bail(e, "problem_create");
      e = cudaMemcpy2D(dptr, A->d * es, A->values, A->ld * es, A->d * es, A->n, cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return bail(e, "problem_create");
      src = dptr;
      ld = A->d;
    }
    if (p->tf32) {  // the values the method takes: a rounded copy (in place when the copy is ours)
      float* rptr = (float*)(A->on_device ? nullptr : src);
      if (!rptr && (e = prob_alloc(p, (size_t)A->n * A->d * 4, (void**)&rptr, SCOPE_PERSIST)) != cudaSuccess)
        return bail(e, "problem_create");
      if ((e = launch_round_tf32((const float*)src, ld, A->n, A->d, rptr, 0)) != cudaSuccess)
        return bail(e, "problem_create");
      src = rptr;
      ld = A->d;
    }
    if (!p->dual) {
      T.N = A->n;
      T.D = A->d;
      T.A = src;
      T.ld = ld;
    } else {  // A_hat = A^T, materialised row-major (d x n)
      void* tptr = nullptr;
      if ((e = prob_alloc(p, (size_t)A->n * A->d * es, &tptr, SCOPE_PERSIST)) != cudaSuccess) return bail(e, "problem_create");
      if ((e = launch_transpose_dense(src, T.elem, A->n, A->d, ld, tptr, 0)) != cudaSuccess) return bail(e, "problem_create");
      T.N = A->d;
      T.D = A->n;
      T.A = tptr;
      T.ld = A->n;
    }
  } else {
    // CSR: device copies if needed, then the transpose, so that both CSR(A_hat) and CSR(A_hat^T) exist
    const int64_t* rp = A->row_ptr;
    const int32_t* ci = A->col_idx;
    const void* val = A->values;
    if (!A->on_device) {
      void *drp = nullptr, *dci = nullptr, *dval = nullptr;
      if ((e = prob_alloc(p, (size_t)(A->n + 1) * 8, &drp, SCOPE_PERSIST)) != cudaSuccess) return bail(e, "problem_create");
      if ((e = prob_alloc(p, (size_t)std::max<int64_t>(1, A->nnz) * 4, &dci, SCOPE_PERSIST)) != cudaSuccess)
        return bail(e, "problem_create");
      if ((e = prob_alloc(p, (size_t)std::max<int64_t>(1, A->nnz) * es, &dval, SCOPE_PERSIST)) != cudaSuccess)
        return bail(e, "problem_create");
      if ((e = cudaMemcpy(drp, A->row_ptr, (A->n + 1) * 8, cudaMemcpyHostToDevice)) != cudaSuccess ||
          (e = cudaMemcpy(dci, A->col_idx, A->nnz * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
          (e = cudaMemcpy(dval, A->values, A->nnz * es, cudaMemcpyHostToDevice)) != cudaSuccess)
        return bail(e, "problem_create");
      rp = (const int64_t*)drp;
      ci = (const int32_t*)dci;
      val = dval;
    }
    {  // the structure every later kernel indexes with (violations become INVALID_ARG, not faults)
      if ((e = launch_csr_check(rp, ci, A->n, A->d, A->nnz, p->status, 0)) != cudaSuccess) return bail(e, "problem_create");
      int st_word = 0;
      if ((e = cudaMemcpy(&st_word, p->status, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return bail(e, "problem_create");
      if (st_word != 0) {
        ihsbin_problem_destroy(p);
        return fail(IHSBIN_ERR_INVALID_ARG,
                    "problem_create: CSR structure invalid (row_ptr must run from 0 to nnz without decreasing, "
                    "and each row's column indices must lie in [0, d) and increase)");
      }
    }
    if (p->tf32) {  // rounded values (in place when the copy is ours)
      float* rval = (float*)(A->on_device ? nullptr : val);
      if (!rval && (e = prob_alloc(p, (size_t)std::max<int64_t>(1, A->nnz) * 4, (void**)&rval, SCOPE_PERSIST)) != cudaSuccess)
        return bail(e, "problem_create");
      if ((e = launch_round_tf32((const float*)val, A->nnz, 1, A->nnz, rval, 0)) != cudaSuccess)
        return bail(e, "problem_create");
      val = rval;
    }
    int64_t* trp = nullptr;
    int32_t* tci = nullptr;
    void* tval = nullptr;
    T.nnz = A->nnz;
    ScratchScope scratch(p);
    if ((e = launch_csr_transpose(p, rp, ci, val, T.elem, A->n, A->d, A->nnz, &trp, &tci, &tval, 0)) != cudaSuccess)
      return bail(e, "problem_create (CSR transpose)");
    if (!p->dual) {  // A_hat = A
      T.N = A->n;
      T.D = A->d;
      T.rp = rp; T.ci = ci; T.val = val;
      T.rpT = trp; T.ciT = tci; T.valT = tval;
    } else {         // A_hat = A^T: its CSR is the transpose just built; CSR(A_hat^T) = A
      T.N = A->d;
      T.D = A->n;
      T.rp = trp; T.ci = tci; T.val = tval;
      T.rpT = rp; T.ciT = ci; T.valT = val;
    }
    if ((e = cudaStreamSynchronize(cudaStreamPerThread)) != cudaSuccess) return bail(e, "problem_create (CSR transpose)");
  }
  // B -> device FP64, packed n x K
  if ((e = prob_alloc(p, (size_t)A->n * K * 8, (void**)&p->B, SCOPE_PERSIST)) != cudaSuccess) return bail(e, "problem_create");
  const size_t bes = elem_size(b_dtype);
  if (!b_on_device && b_dtype == IHSBIN_F64 && ldb == K) {
    // packed FP64 rows: one copy straight from the caller's buffer (DMA when it is pinned)
    e = cudaMemcpy(p->B, B, (size_t)A->n * K * 8, cudaMemcpyHostToDevice);
  } else if (!b_on_device) {
    std::vector<double> hb((size_t)A->n * K);
    for (int64_t i = 0; i < A->n; ++i)
      for (int64_t r = 0; r < K; ++r)
        hb[i * K + r] = b_dtype == IHSBIN_F64 ? ((const double*)B)[i * ldb + r] : (double)((const float*)B)[i * ldb + r];
    e = cudaMemcpy(p->B, hb.data(), hb.size() * 8, cudaMemcpyHostToDevice);
  } else if (b_dtype == IHSBIN_F64 && ldb == K) {
    e = cudaMemcpy(p->B, B, (size_t)A->n * K * 8, cudaMemcpyDeviceToDevice);
  } else {
    e = launch_convert_to_f64(B, b_dtype == IHSBIN_F64 ? ELEM_F64 : ELEM_F32, A->n, K, ldb, p->B, 0);
    (void)bes;
  }
  if (e != cudaSuccess) return bail(e, "problem_create");
  if ((e = cudaStreamSynchronize(cudaStreamPerThread)) != cudaSuccess) return bail(e, "problem_create");
  *out = p;
  return IHSBIN_OK;
}

ihsbin_status ihsbin_problem_destroy(ihsbin_problem* p) {
  if (!p) return fail(IHSBIN_ERR_INVALID_ARG, "problem_destroy: NULL");
  cudaSetDevice(p->ctx->device);
  CallStream cs(nullptr);
  for (auto e : p->ev_pool) cudaEventDestroy(e);
  p->ev_pool.clear();
  pre_gram_discard(p);
  for (auto& e : p->pre_ev)
    if (e) cudaEventDestroy(e);
  for (cudaStream_t* sp : {&p->side, &p->fac})
    if (*sp) {
      cudaStreamSynchronize(*sp);
      cudaStreamDestroy(*sp);
      *sp = nullptr;
    }
  prob_free_basis(p);
  free_list(p, p->owned);
  delete p;
  return IHSBIN_OK;
}

ihsbin_status ihsbin_sketch(ihsbin_problem* p, const ihsbin_sketch_desc* sk, void* stream) {
  Range range_("ihsbin_sketch");
  if (!p || !sk) return fail(IHSBIN_ERR_INVALID_ARG, "sketch: NULL argument");
  cudaStream_t st = stream ? (cudaStream_t)stream : cudaStreamPerThread;
  const int64_t N = p->A.N, D = p->A.D;
  if (sk->m <= 0) return fail(IHSBIN_ERR_INVALID_ARG, "sketch: m must be positive");
  if (sk->entries != IHSBIN_F64 && sk->entries != IHSBIN_BF16)
    return fail(IHSBIN_ERR_INVALID_ARG, "sketch: entries must be IHSBIN_F64 or IHSBIN_BF16");
  if (sk->apply != IHSBIN_APPLY_AUTO && sk->apply != IHSBIN_APPLY_TENSOR && sk->apply != IHSBIN_APPLY_FMA)
    return fail(IHSBIN_ERR_INVALID_ARG, "sketch: unknown apply selector");
  int64_t Np = 1;
  while (Np < N) Np <<= 1;
  if (sk->kind == IHSBIN_SK_COUNTSKETCH) {
    if (sk->s <= 0 || sk->m % sk->s) return fail(IHSBIN_ERR_INVALID_ARG, "sketch: need s >= 1 and m % s == 0");
  } else if (sk->kind == IHSBIN_SK_SRHT) {
    if (sk->m > Np) return fail(IHSBIN_ERR_INVALID_ARG, "sketch: SRHT needs m <= padded row count");
    if (p->A.layout != IHSBIN_DENSE_ROWMAJOR) return fail(IHSBIN_ERR_UNSUPPORTED, "sketch: SRHT needs dense A (use CountSketch for CSR)");
  } else if (sk->kind == IHSBIN_SK_GAUSSIAN) {
    if (p->A.layout != IHSBIN_DENSE_ROWMAJOR) return fail(IHSBIN_ERR_UNSUPPORTED, "sketch: Gaussian needs dense A");
    if (sk->apply == IHSBIN_APPLY_TENSOR && !(p->A.elem == ELEM_BF16 && sk->entries == IHSBIN_BF16))
      return fail(IHSBIN_ERR_UNSUPPORTED, "sketch: the tensor-core Gaussian sketch needs BF16 entries and BF16 data");
  } else {
    return fail(IHSBIN_ERR_INVALID_ARG, "sketch: unknown kind");
  }
  cudaError_t e = cudaSetDevice(p->ctx->device);
  if (e != cudaSuccess) return cuda_fail(e, "sketch");
  pre_gram_discard(p);
  CallStream cs(st);
  // discard any previous sketch and basis
  prob_free_basis(p);
  p->sketched = false;
  p->sk = *sk;
  {
    std::vector<DevBuf> keep;
    for (auto& b : p->owned) {
      if (b.p == p->SA || b.p == p->GS || b.p == p->sk_idx || b.p == p->sk_sign) {
        std::lock_guard<std::mutex> g(p->ctx->mu);
        cudaFree(b.p);
        p->ctx->in_use -= b.bytes;
      } else {
        keep.push_back(b);
      }
    }
    p->owned.swap(keep);
    p->SA = p->GS = nullptr;
    p->sk_idx = nullptr;
    p->sk_sign = nullptr;
  }
  ScratchScope scratch(p);
  if ((e = prob_alloc(p, (size_t)sk->m * D * 8, (void**)&p->SA, SCOPE_PERSIST)) != cudaSuccess) return cuda_fail(e, "sketch");
  if ((e = prob_alloc(p, (size_t)D * D * 8, (void**)&p->GS, SCOPE_PERSIST)) != cudaSuccess) return cuda_fail(e, "sketch");
  p->sk_idx_count = p->sk_sign_count = 0;
  if (sk->kind == IHSBIN_SK_SRHT) {
    p->sk_idx_count = sk->m;
    p->sk_sign_count = Np;
  } else if (sk->kind == IHSBIN_SK_COUNTSKETCH) {
    p->sk_idx_count = p->sk_sign_count = N * sk->s;
  }
  if ((e = prob_alloc(p, std::max<int64_t>(1, p->sk_idx_count) * 8, (void**)&p->sk_idx, SCOPE_PERSIST)) != cudaSuccess)
    return cuda_fail(e, "sketch");
  if ((e = prob_alloc(p, std::max<int64_t>(1, p->sk_sign_count), (void**)&p->sk_sign, SCOPE_PERSIST)) != cudaSuccess)
    return cuda_fail(e, "sketch");
  if (pre_gram_eligible(p) && ensure_streams(p) == cudaSuccess) {
    // the Gram of A and A^T b for the next build, on the side stream beside the sketch (its
    // scratch is freed in that stream's order); a failure here only means the build forms them
    CallStream side(p->side);
    ScratchScope pre_scratch(p);
    if (pre_gram_launch(p) != cudaSuccess) {
      cudaGetLastError();
      pre_gram_discard(p);
    }
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // With a background Gram running, the sketch's kernels go to the problem's high-priority stream
  // (forked from and joined back to the caller's), so that the Gram only takes what they leave.
  cudaStream_t ks = p->gram_pre ? p->fac : st;
  double* tr_dev = nullptr;
  if (ks != st) {
    cudaEventRecord(e0, st);
    cudaStreamWaitEvent(ks, e0, 0);
  }
  {
    CallStream kcs(ks);
    cudaEventRecord(e0, ks);
    if (sk->kind == IHSBIN_SK_GAUSSIAN) e = sketch_gaussian(p, ks);
    else if (sk->kind == IHSBIN_SK_SRHT) e = sketch_srht(p, ks);
    else e = sketch_countsketch(p, ks);
    if (e == cudaSuccess) e = sketch_gram(p, ks);
    // tr(G_S) for the next build, read after this call's synchronisation
    if (e == cudaSuccess) e = prob_alloc(p, sizeof(double), (void**)&tr_dev, SCOPE_SCRATCH);
    if (e == cudaSuccess) e = gs_trace_launch(p, tr_dev, ks);
    cudaEventRecord(e1, ks);
  }
  if (ks != st) cudaStreamWaitEvent(st, e1, 0);
  if (e != cudaSuccess) {
    cudaStreamSynchronize(ks);
    cudaStreamSynchronize(st);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaMemset(p->status, 0, sizeof(int));  // nothing of the failed sketch is reported later
    return cuda_fail(e, "sketch");
  }
  ihsbin_status s = check_status(p, st, "sketch");
  if (s == IHSBIN_OK && cudaMemcpy(&p->trGS, tr_dev, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    s = fail(IHSBIN_ERR_CUDA, "sketch: trace copy failed");
  cudaEventElapsedTime(&p->phase_ms[0], e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != IHSBIN_OK) return s;
  p->sketched = true;
  return IHSBIN_OK;
}

ihsbin_status ihsbin_sketch_export(ihsbin_problem* p, int64_t* idx, int8_t* sign, int64_t cap, int64_t* count) {
  if (!p || !count) return fail(IHSBIN_ERR_INVALID_ARG, "sketch_export: NULL argument");
  if (!p->sketched) return fail(IHSBIN_ERR_STATE, "sketch_export: not sketched");
  *count = p->sk_idx_count;
  if (idx && p->sk_idx_count) {
    if (cap < p->sk_idx_count) return fail(IHSBIN_ERR_INVALID_ARG, "sketch_export: cap too small");
    if (cudaMemcpy(idx, p->sk_idx, p->sk_idx_count * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(IHSBIN_ERR_CUDA, "sketch_export: copy failed");
  }
  if (sign && p->sk_sign_count) {
    if (cap < p->sk_sign_count) return fail(IHSBIN_ERR_INVALID_ARG, "sketch_export: cap too small");
    if (cudaMemcpy(sign, p->sk_sign, p->sk_sign_count, cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(IHSBIN_ERR_CUDA, "sketch_export: copy failed");
  }
  return IHSBIN_OK;
}

ihsbin_status ihsbin_sketch_matrix_export(ihsbin_problem* p, double* SA, double* GS) {
  if (!p) return fail(IHSBIN_ERR_INVALID_ARG, "sketch_matrix_export: NULL");
  if (!p->sketched) return fail(IHSBIN_ERR_STATE, "sketch_matrix_export: not sketched");
  const int64_t D = p->A.D;
  if (SA && cudaMemcpy(SA, p->SA, (size_t)p->sk.m * D * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(IHSBIN_ERR_CUDA, "sketch_matrix_export: copy failed");
  if (GS && cudaMemcpy(GS, p->GS, (size_t)D * D * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(IHSBIN_ERR_CUDA, "sketch_matrix_export: copy failed");
  return IHSBIN_OK;
}

ihsbin_status ihsbin_sketch_entries_export(ihsbin_problem* p, int64_t row0, int64_t nrows, int64_t col0,
                                           int64_t ncols, uint16_t* out) {
  if (!p || !out) return fail(IHSBIN_ERR_INVALID_ARG, "sketch_entries_export: NULL argument");
  if (!p->sketched || p->sk.kind != IHSBIN_SK_GAUSSIAN || p->sk.entries != IHSBIN_BF16)
    return fail(IHSBIN_ERR_STATE, "sketch_entries_export: not sketched with BF16 Gaussian entries");
  if (row0 < 0 || col0 < 0 || nrows <= 0 || ncols <= 0 || row0 + nrows > p->sk.m || col0 + ncols > p->A.N)
    return fail(IHSBIN_ERR_INVALID_ARG, "sketch_entries_export: window outside the sketch");
  cudaError_t e = cudaSetDevice(p->ctx->device);
  if (e != cudaSuccess) return cuda_fail(e, "sketch_entries_export");
  cudaStream_t st = cudaStreamPerThread;
  CallStream cs(st);
  ScratchScope scratch(p);
  uint16_t* dev = nullptr;
  if ((e = prob_alloc(p, (size_t)nrows * ncols * 2, (void**)&dev, SCOPE_SCRATCH)) != cudaSuccess)
    return cuda_fail(e, "sketch_entries_export");
  if ((e = gaussian_entries_bf16(p, row0, nrows, col0, ncols, dev, st)) != cudaSuccess)
    return cuda_fail(e, "sketch_entries_export");
  if ((e = cudaMemcpyAsync(out, dev, (size_t)nrows * ncols * 2, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_fail(e, "sketch_entries_export");
  return check_status(p, st, "sketch_entries_export");
}

ihsbin_status ihsbin_build_basis(ihsbin_problem* p, const ihsbin_path_desc* d, void* stream) {
  Range range_("ihsbin_build_basis");
  if (!p || !d) return fail(IHSBIN_ERR_INVALID_ARG, "build_basis: NULL argument");
  if (!p->sketched) return fail(IHSBIN_ERR_STATE, "build_basis: call ihsbin_sketch first");
  if (!(d->lambda_min > 0) || !(d->lambda_max >= d->lambda_min) || !std::isfinite(d->lambda_max))
    return fail(IHSBIN_ERR_INVALID_ARG, "build_basis: need 0 < lambda_min <= lambda_max < inf");
  if (d->L < 0 || d->jmax < 0) return fail(IHSBIN_ERR_INVALID_ARG, "build_basis: negative L or jmax");
  if (!(d->sigma_d2 >= 0) || !std::isfinite(d->sigma_d2))
    return fail(IHSBIN_ERR_INVALID_ARG, "build_basis: sigma_d2 must be finite and >= 0");
  if (d->tau && !(d->L > 0)) return fail(IHSBIN_ERR_INVALID_ARG, "build_basis: an explicit tau array needs L > 0");
  if (d->slice_weight != 0 && (d->slice_weight < 4 || d->slice_weight > 6))
    return fail(IHSBIN_ERR_INVALID_ARG, "build_basis: slice_weight must be 0 or 4..6");
  if (d->compute != IHSBIN_COMPUTE_F64 && d->compute != IHSBIN_COMPUTE_F32X2)
    return fail(IHSBIN_ERR_INVALID_ARG, "build_basis: unknown compute mode");
  if (d->form != IHSBIN_FORM_AUTO && d->form != IHSBIN_FORM_RESIDUAL && d->form != IHSBIN_FORM_INCREMENT)
    return fail(IHSBIN_ERR_INVALID_ARG, "build_basis: unknown recursion form");
  if (d->precond_weight < 0 || d->precond_weight > 6)
    return fail(IHSBIN_ERR_INVALID_ARG, "build_basis: precond_weight must be 0..6");
  Plan pl;
  const double beta = d->lambda_max / d->lambda_min;
  pl.L = d->L > 0 ? d->L : std::max(1, (int)std::floor(2.0 * std::log(beta)));
  const int L = pl.L;
  pl.edges.resize(L + 1);
  for (int l = 0; l <= L; ++l) pl.edges[l] = d->lambda_min * std::pow(beta, (double)l / L);
  pl.edges[0] = d->lambda_min;
  pl.edges[L] = d->lambda_max;
  pl.lam0.resize(L);
  pl.tau.resize(L);
  pl.k.resize(L);
  pl.jcount.resize(L);
  double rho = d->rho;
  if (!(rho > 0)) rho = std::min((double)p->A.D / (double)p->sk.m, 0.81);
  pl.auto_rho = d->auto_rho != 0 && !(d->rho1 && d->rho2);
  pl.auto_k = !d->k && d->k_default <= 0;
  pl.eps = d->eps > 0 ? d->eps : 1e-7;
  pl.rho1.resize(L);
  pl.rho2.resize(L);
  pl.sigma_d2 = d->sigma_d2;
  pl.slice_w = d->slice_weight > 0 ? d->slice_weight : 6;
  pl.form = d->form;
  pl.precond_req = d->precond_weight;
  if (d->tau) {
    pl.tau_user.assign(d->tau, d->tau + L);
    for (double t : pl.tau_user)
      if (!(t > 0) || !std::isfinite(t)) return fail(IHSBIN_ERR_INVALID_ARG, "build_basis: every tau must be finite and > 0");
  }
  for (int l = 0; l < L; ++l) {
    const double lo = pl.edges[l], hi = pl.edges[l + 1];
    pl.lam0[l] = pl.sigma_d2 > 0 ? std::sqrt((hi + pl.sigma_d2) * (lo + pl.sigma_d2)) - pl.sigma_d2 : std::sqrt(lo * hi);
    double r1, r2;
    if (d->rho1 && d->rho2) {
      r1 = d->rho1[l];
      r2 = d->rho2[l];
    } else {
      r1 = (1.0 + std::sqrt(rho)) * (1.0 + std::sqrt(rho));
      r2 = (1.0 - std::sqrt(rho)) * (1.0 - std::sqrt(rho));
    }
    if (!(r1 > 0) || !(r2 > 0)) return fail(IHSBIN_ERR_INVALID_ARG, "build_basis: rho1 and rho2 must be positive");
    pl.rho1[l] = r1;
    pl.rho2[l] = r2;
    const int kl = d->k ? d->k[l] : d->k_default;
    if (!pl.auto_k && kl <= 0) return fail(IHSBIN_ERR_INVALID_ARG, "build_basis: every k_l must be >= 1");
    pl.k[l] = pl.auto_k ? 1 : kl;
  }
  pl.jmax = d->jmax;
  pl.compute = d->compute;
  pl.product = d->product == IHSBIN_PRODUCT_AUTO ? IHSBIN_PRODUCT_GRAM : d->product;
  if (p->A.layout == IHSBIN_CSR && pl.product != IHSBIN_PRODUCT_GRAM)
    return fail(IHSBIN_ERR_UNSUPPORTED, "build_basis: CSR data uses the Gram product");
  if (d->gram != IHSBIN_GRAM_AUTO && d->gram != IHSBIN_GRAM_SLICES && d->gram != IHSBIN_GRAM_FMA)
    return fail(IHSBIN_ERR_INVALID_ARG, "build_basis: unknown Gram kernel");
  {
    const bool sliceable = p->A.layout == IHSBIN_DENSE_ROWMAJOR && p->A.elem != ELEM_F64;
    if (d->gram == IHSBIN_GRAM_SLICES && !sliceable)
      return fail(IHSBIN_ERR_UNSUPPORTED, "build_basis: the sliced tensor-core Gram takes dense FP32/BF16 data");
    pl.gram = d->gram == IHSBIN_GRAM_FMA ? IHSBIN_GRAM_FMA
              : d->gram == IHSBIN_GRAM_SLICES ? IHSBIN_GRAM_SLICES
              : (sliceable ? IHSBIN_GRAM_SLICES : IHSBIN_GRAM_FMA);
  }
  if (d->loop != IHSBIN_LOOP_AUTO && d->loop != IHSBIN_LOOP_SLICES && d->loop != IHSBIN_LOOP_FMA)
    return fail(IHSBIN_ERR_INVALID_ARG, "build_basis: unknown loop kernel");
  if (d->loop == IHSBIN_LOOP_SLICES && d->compute != IHSBIN_COMPUTE_F32X2)
    return fail(IHSBIN_ERR_UNSUPPORTED, "build_basis: the sliced tensor-core loop products take the F32X2 compute mode");
  pl.loop = d->loop == IHSBIN_LOOP_FMA ? IHSBIN_LOOP_FMA
            : d->compute == IHSBIN_COMPUTE_F32X2 ? IHSBIN_LOOP_SLICES : IHSBIN_LOOP_FMA;
  if (d->factor != IHSBIN_FACTOR_AUTO && d->factor != IHSBIN_FACTOR_SLICES && d->factor != IHSBIN_FACTOR_FMA)
    return fail(IHSBIN_ERR_INVALID_ARG, "build_basis: unknown factor kernel");
  if (d->factor == IHSBIN_FACTOR_SLICES && d->compute != IHSBIN_COMPUTE_F32X2)
    return fail(IHSBIN_ERR_UNSUPPORTED, "build_basis: the sliced tensor-core inverse takes the F32X2 compute mode");
  pl.factor = d->factor == IHSBIN_FACTOR_FMA ? IHSBIN_FACTOR_FMA
              : d->compute == IHSBIN_COMPUTE_F32X2 ? IHSBIN_FACTOR_SLICES : IHSBIN_FACTOR_FMA;
  cudaError_t e = cudaSetDevice(p->ctx->device);
  if (e != cudaSuccess) return cuda_fail(e, "build_basis");
  cudaStream_t st = stream ? (cudaStream_t)stream : cudaStreamPerThread;
  CallStream cs(st);
  const bool take_pre = p->gram_pre && pl.compute == IHSBIN_COMPUTE_F32X2 && pl.gram == IHSBIN_GRAM_SLICES &&
                        pl.product == IHSBIN_PRODUCT_GRAM;
  if (p->gram_pre && !take_pre) pre_gram_discard(p);
  prob_free_basis(p);
  p->plan = pl;
  if (take_pre) {
    // the background Gram joins the basis; its right-hand side stays a pre buffer until the end
    std::vector<DevBuf> keep;
    for (auto& b : p->pre_bufs)
      (b.p == p->G_pre.p0 || b.p == p->G_pre.p1 ? p->basis_bufs : keep).push_back(b);
    p->pre_bufs.swap(keep);
    p->G = p->G_pre;
    p->pre_taken = true;
  }
  if (!pl.auto_rho) finalize_plan(p, nullptr);
  // phases: factor ev[0] -> ev[1] (factor stream); Gram + rhs ev[5] -> ev[2] (side stream,
  // overlapping the factor); recursion ev[6] -> ev[3] (caller's stream, after both joins)
  cudaEvent_t ev[7];
  for (auto& x : ev) cudaEventCreate(&x);
  ihsbin_status s;
  {
    ScratchScope scratch(p);
    // persistent members (Pinv, G, Ut, W) are taken out of the scratch scope by the device code
    e = build_basis_device(p, st, ev);
    if (e != cudaSuccess) {
      cudaStreamSynchronize(st);
      if (p->side) cudaStreamSynchronize(p->side);
      if (p->fac) cudaStreamSynchronize(p->fac);
      for (auto& x : ev) cudaEventDestroy(x);
      prob_free_basis(p);
      pre_gram_discard(p);
      cudaMemset(p->status, 0, sizeof(int));  // nothing of the failed build is reported later
      tune_discard();
      return cuda_fail(e, "build_basis");
    }
    s = check_status(p, st, "build_basis");
  }
  float t01 = 0, t12 = 0, t23 = 0;
  cudaEventElapsedTime(&t01, ev[0], ev[1]);
  if (p->pre_taken) cudaEventElapsedTime(&t12, p->pre_ev[0], p->pre_ev[1]);
  else cudaEventElapsedTime(&t12, ev[5], ev[2]);
  cudaEventElapsedTime(&t23, ev[6], ev[3]);
  pre_gram_discard(p);  // the right-hand side of a background Gram (the stream is idle here)
  p->phase_ms[1] = t01;
  p->phase_ms[2] = t12;
  p->phase_ms[3] = t23;
  for (auto& x : ev) cudaEventDestroy(x);
  if (s != IHSBIN_OK) {
    prob_free_basis(p);
    return s;
  }
  p->built = true;
  p->last_compute = pl.compute;
  p->last_gram = pl.gram;
  return IHSBIN_OK;
}

ihsbin_status ihsbin_recursion_form(const ihsbin_problem* p, int32_t* form, int32_t* precond_weight) {
  if (!p) return fail(IHSBIN_ERR_INVALID_ARG, "recursion_form: NULL");
  if (!p->built || p->plan.form_run == 0) return fail(IHSBIN_ERR_STATE, "recursion_form: no basis built");
  if (form) *form = p->plan.form_run;
  if (precond_weight) *precond_weight = p->plan.precond_w;
  return IHSBIN_OK;
}

ihsbin_status ihsbin_plan_export(ihsbin_problem* p, double* edges, double* lam0, double* tau, int32_t* k,
                                 int32_t* jcount, int32_t cap_L, int32_t* L_out) {
  if (!p) return fail(IHSBIN_ERR_INVALID_ARG, "plan_export: NULL");
  if (!p->built) return fail(IHSBIN_ERR_STATE, "plan_export: no basis");
  const Plan& pl = p->plan;
  if (L_out) *L_out = pl.L;
  if ((edges || lam0 || tau || k || jcount) && cap_L < pl.L) return fail(IHSBIN_ERR_INVALID_ARG, "plan_export: cap_L < L");
  for (int l = 0; l < pl.L; ++l) {
    if (lam0) lam0[l] = pl.lam0[l];
    if (tau) tau[l] = pl.tau[l];
    if (k) k[l] = pl.k[l];
    if (jcount) jcount[l] = pl.jcount[l];
  }
  if (edges) {
    if (cap_L < pl.L + 1) return fail(IHSBIN_ERR_INVALID_ARG, "plan_export: edges need L+1 entries");
    for (int l = 0; l <= pl.L; ++l) edges[l] = pl.edges[l];
  }
  return IHSBIN_OK;
}

ihsbin_status ihsbin_basis_export(ihsbin_problem* p, int32_t l, double* buf, int64_t cap, int64_t* need) {
  if (!p || !need) return fail(IHSBIN_ERR_INVALID_ARG, "basis_export: NULL argument");
  if (!p->built) return fail(IHSBIN_ERR_STATE, "basis_export: no basis");
  const Plan& pl = p->plan;
  if (l < 0 || l >= pl.L) return fail(IHSBIN_ERR_INVALID_ARG, "basis_export: interval out of range");
  const int64_t D = p->A.D, K = p->K;
  const int64_t cnt = (int64_t)pl.jcount[l] * K * D;
  *need = cnt;
  if (!buf) return IHSBIN_OK;
  if (cap < cnt) return fail(IHSBIN_ERR_INVALID_ARG, "basis_export: cap too small");
  const int64_t off = (int64_t)l * pl.jc * K * D;
  if (pl.compute == IHSBIN_COMPUTE_F64) {
    if (cudaMemcpy(buf, (double*)p->Ut.p0 + off, cnt * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(IHSBIN_ERR_CUDA, "basis_export: copy failed");
  } else {
    std::vector<float> hi(cnt), lo(cnt);
    if (cudaMemcpy(hi.data(), (float*)p->Ut.p0 + off, cnt * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(lo.data(), (float*)p->Ut.p1 + off, cnt * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(IHSBIN_ERR_CUDA, "basis_export: copy failed");
    for (int64_t i = 0; i < cnt; ++i) buf[i] = (double)hi[i] + (double)lo[i];
  }
  return IHSBIN_OK;
}

ihsbin_status ihsbin_gram_export(ihsbin_problem* p, double* G) {
  if (!p || !G) return fail(IHSBIN_ERR_INVALID_ARG, "gram_export: NULL argument");
  if (!p->built) return fail(IHSBIN_ERR_STATE, "gram_export: no basis");
  if (p->plan.product != IHSBIN_PRODUCT_GRAM || !p->G.p0) return fail(IHSBIN_ERR_STATE, "gram_export: no Gram (A-space product)");
  const int64_t cnt = p->A.D * p->A.D;
  if (p->plan.compute == IHSBIN_COMPUTE_F64) {
    if (cudaMemcpy(G, p->G.p0, cnt * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(IHSBIN_ERR_CUDA, "gram_export: copy failed");
  } else {
    std::vector<float> hi(cnt), lo(cnt);
    if (cudaMemcpy(hi.data(), p->G.p0, cnt * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(lo.data(), p->G.p1, cnt * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(IHSBIN_ERR_CUDA, "gram_export: copy failed");
    for (int64_t i = 0; i < cnt; ++i) G[i] = (double)hi[i] + (double)lo[i];
  }
  return IHSBIN_OK;
}

ihsbin_status ihsbin_eval_path(ihsbin_problem* p, const double* lambdas, int64_t T, void* X, ihsbin_dtype x_dtype,
                               int x_on_device, void* stream) {
  Range range_("ihsbin_eval_path");
  if (!p || !lambdas || !X) return fail(IHSBIN_ERR_INVALID_ARG, "eval_path: NULL argument");
  if (!p->built) return fail(IHSBIN_ERR_STATE, "eval_path: call ihsbin_build_basis first");
  if (T <= 0) return fail(IHSBIN_ERR_INVALID_ARG, "eval_path: T must be positive");
  if (x_dtype != IHSBIN_F64 && x_dtype != IHSBIN_F32) return fail(IHSBIN_ERR_INVALID_ARG, "eval_path: X must be F64 or F32");
  const Plan& pl = p->plan;
  for (int64_t t = 0; t < T; ++t)
    if (!(lambdas[t] >= pl.edges[0] && lambdas[t] <= pl.edges[pl.L]))
      return fail(IHSBIN_ERR_LAMBDA_RANGE, "eval_path: lambda outside [lambda_min, lambda_max]");
  cudaError_t e = cudaSetDevice(p->ctx->device);
  if (e != cudaSuccess) return cuda_fail(e, "eval_path");
  cudaStream_t st = stream ? (cudaStream_t)stream : cudaStreamPerThread;
  CallStream cs(st);
  ScratchScope scratch(p);
  double* lam_dev = nullptr;
  if ((e = prob_alloc(p, T * 8, (void**)&lam_dev, SCOPE_SCRATCH)) != cudaSuccess) return cuda_fail(e, "eval_path");
  if ((e = cudaMemcpyAsync(lam_dev, lambdas, T * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return cuda_fail(e, "eval_path");
  const int64_t outN = (int64_t)T * p->d * p->K;
  const size_t oes = x_dtype == IHSBIN_F64 ? 8 : 4;
  void* Xd = X;
  if (!x_on_device) {
    if ((e = prob_alloc(p, outN * oes, &Xd, SCOPE_SCRATCH)) != cudaSuccess) return cuda_fail(e, "eval_path");
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
  e = eval_device(p, lambdas, lam_dev, T, Xd, x_dtype == IHSBIN_F64 ? ELEM_F64 : ELEM_F32, st);
  cudaEventRecord(e1, st);
  if (e == cudaSuccess && !x_on_device) e = cudaMemcpyAsync(X, Xd, outN * oes, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return cuda_fail(e, "eval_path");
  }
  ihsbin_status s = check_status(p, st, "eval_path");
  cudaEventElapsedTime(&p->phase_ms[4], e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return s;
}

ihsbin_status ihsbin_path_losses(ihsbin_problem* p, const double* lambdas, int64_t T, const ihsbin_matrix* A_test,
                                 const void* B_test, int64_t ldb_test, ihsbin_dtype b_test_dtype, int b_test_on_device,
                                 double* train_loss, double* test_loss, void* stream) {
  Range range_("ihsbin_path_losses");
  if (!p || !lambdas) return fail(IHSBIN_ERR_INVALID_ARG, "path_losses: NULL argument");
  if (!p->built) return fail(IHSBIN_ERR_STATE, "path_losses: call ihsbin_build_basis first");
  if (T <= 0) return fail(IHSBIN_ERR_INVALID_ARG, "path_losses: T must be positive");
  if (test_loss) {
    if (!A_test || !B_test) return fail(IHSBIN_ERR_INVALID_ARG, "path_losses: test loss without A_test / B_test");
    if (A_test->layout != IHSBIN_DENSE_ROWMAJOR) return fail(IHSBIN_ERR_UNSUPPORTED, "path_losses: A_test must be dense");
    if (A_test->d != p->d || A_test->n <= 0 || A_test->ld < A_test->d || !A_test->values)
      return fail(IHSBIN_ERR_INVALID_ARG, "path_losses: A_test must be n_test x d with ld >= d");
    if (A_test->dtype < IHSBIN_F64 || A_test->dtype > IHSBIN_BF16)  // (TF32 test rows are not taken)
      return fail(IHSBIN_ERR_INVALID_ARG, "path_losses: bad A_test dtype");
    if (b_test_dtype != IHSBIN_F64 && b_test_dtype != IHSBIN_F32)
      return fail(IHSBIN_ERR_INVALID_ARG, "path_losses: B_test must be F64 or F32");
    if (ldb_test < p->K) return fail(IHSBIN_ERR_INVALID_ARG, "path_losses: ldb_test < K");
  }
  const Plan& pl = p->plan;
  for (int64_t t = 0; t < T; ++t)
    if (!(lambdas[t] >= pl.edges[0] && lambdas[t] <= pl.edges[pl.L]))
      return fail(IHSBIN_ERR_LAMBDA_RANGE, "path_losses: lambda outside [lambda_min, lambda_max]");
  if (!train_loss && !test_loss) return IHSBIN_OK;
  cudaError_t e = cudaSetDevice(p->ctx->device);
  if (e != cudaSuccess) return cuda_fail(e, "path_losses");
  cudaStream_t st = stream ? (cudaStream_t)stream : cudaStreamPerThread;
  CallStream cs(st);
  ScratchScope scratch(p);
  double *lam_dev = nullptr, *out = nullptr;
  if ((e = prob_alloc(p, T * 8, (void**)&lam_dev, SCOPE_SCRATCH)) != cudaSuccess ||
      (e = prob_alloc(p, 2 * T * 8, (void**)&out, SCOPE_SCRATCH)) != cudaSuccess)
    return cuda_fail(e, "path_losses");
  if ((e = cudaMemcpyAsync(lam_dev, lambdas, T * 8, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return cuda_fail(e, "path_losses");
  const void* At = nullptr;
  int at_elem = ELEM_F64;
  int64_t at_ld = 0, nt = 0;
  double* Bt = nullptr;
  if (test_loss) {
    nt = A_test->n;
    const size_t es = elem_size(A_test->dtype);
    at_elem = A_test->dtype == IHSBIN_F64 ? ELEM_F64 : A_test->dtype == IHSBIN_F32 ? ELEM_F32 : ELEM_BF16;
    At = A_test->values;
    at_ld = A_test->ld;
    if (!A_test->on_device) {  // packed device copy
      void* dptr = nullptr;
      if ((e = prob_alloc(p, (size_t)nt * p->d * es, &dptr, SCOPE_SCRATCH)) != cudaSuccess ||
          (e = cudaMemcpy2DAsync(dptr, p->d * es, A_test->values, A_test->ld * es, p->d * es, nt,
                                 cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(e, "path_losses");
      At = dptr;
      at_ld = p->d;
    }
    if ((e = prob_alloc(p, (size_t)nt * p->K * 8, (void**)&Bt, SCOPE_SCRATCH)) != cudaSuccess)
      return cuda_fail(e, "path_losses");
    const void* bsrc = B_test;
    if (!b_test_on_device) {  // rows as given, converted on the device
      void* dptr = nullptr;
      const size_t bes = elem_size(b_test_dtype);
      if ((e = prob_alloc(p, (size_t)nt * ldb_test * bes, &dptr, SCOPE_SCRATCH)) != cudaSuccess ||
          (e = cudaMemcpyAsync(dptr, B_test, (size_t)((nt - 1) * ldb_test + p->K) * bes, cudaMemcpyHostToDevice,
                               st)) != cudaSuccess)
        return cuda_fail(e, "path_losses");
      bsrc = dptr;
    }
    if ((e = launch_convert_to_f64(bsrc, b_test_dtype == IHSBIN_F64 ? ELEM_F64 : ELEM_F32, nt, p->K, ldb_test, Bt,
                                   st)) != cudaSuccess)
      return cuda_fail(e, "path_losses");
  }
  e = losses_device(p, lambdas, lam_dev, T, At, at_elem, at_ld, nt, Bt, train_loss ? out : nullptr,
                    test_loss ? out + T : nullptr, st);
  if (e == cudaSuccess && train_loss) e = cudaMemcpyAsync(train_loss, out, T * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && test_loss) e = cudaMemcpyAsync(test_loss, out + T, T * 8, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail(e, "path_losses");
  return check_status(p, st, "path_losses");
}

ihsbin_status ihsbin_adaptive_sketch(ihsbin_problem* p, const ihsbin_adaptive_desc* desc, ihsbin_adaptive_result* res,
                                     double* delta_trace, int64_t* m_trace, double* step_trace, int32_t trace_cap,
                                     double* x_out, void* stream) {
  Range range_("ihsbin_adaptive_sketch");
  if (!p || !desc || !res) return fail(IHSBIN_ERR_INVALID_ARG, "adaptive_sketch: NULL argument");
  const double lam = desc->lambda;
  if (!(lam > 0) || !std::isfinite(lam)) return fail(IHSBIN_ERR_INVALID_ARG, "adaptive_sketch: lambda must be positive");
  const double eps = desc->eps > 0 ? desc->eps : 1e-10;
  const double g1 = desc->gamma1 > 0 ? desc->gamma1 : 0.5, g2 = desc->gamma2 > 0 ? desc->gamma2 : 0.25;
  const double g3 = desc->gamma3 > 0 ? desc->gamma3 : 0.5;
  if (!(g1 < 1) || !(g2 < 1)) return fail(IHSBIN_ERR_INVALID_ARG, "adaptive_sketch: gamma1 and gamma2 must lie in (0,1)");
  if (desc->compute != IHSBIN_COMPUTE_F64 && desc->compute != IHSBIN_COMPUTE_F32X2)
    return fail(IHSBIN_ERR_INVALID_ARG, "adaptive_sketch: unknown compute mode");
  if (trace_cap < 0) return fail(IHSBIN_ERR_INVALID_ARG, "adaptive_sketch: negative trace_cap");
  const int max_iter = desc->max_iter > 0 ? desc->max_iter : 100;
  int64_t Np = 1;
  while (Np < p->A.N) Np <<= 1;
  const int64_t m_max = desc->m_max > 0 ? desc->m_max : (desc->sketch.kind == IHSBIN_SK_SRHT ? Np : p->A.N);
  cudaStream_t st = stream ? (cudaStream_t)stream : cudaStreamPerThread;
  ihsbin_sketch_desc sk = desc->sketch;
  const uint64_t seed0 = sk.seed;
  // the re-sketches of Algorithm 4 start no background Gram (no build follows them here)
  struct PreOff {
    ihsbin_problem* p;
    explicit PreOff(ihsbin_problem* q) : p(q) { p->pre_off = true; }
    ~PreOff() { p->pre_off = false; }
  } pre_off_(p);
  ihsbin_status s = ihsbin_sketch(p, &sk, stream);
  if (s != IHSBIN_OK) return s;
  cudaError_t e = cudaSetDevice(p->ctx->device);
  if (e != cudaSuccess) return cuda_fail(e, "adaptive_sketch");
  CallStream cs(st);
  ScratchScope scratch(p);
  // a one-interval plan at lambda for the factor and the Gram kernels
  Plan pl;
  pl.L = 1;
  pl.edges = {lam, lam};
  pl.lam0 = {lam};
  pl.tau = {1.0};
  pl.k = {1};
  pl.jcount = {1};
  pl.compute = desc->compute;
  pl.product = IHSBIN_PRODUCT_GRAM;
  pl.gram = (p->A.layout == IHSBIN_DENSE_ROWMAJOR && p->A.elem != ELEM_F64) ? IHSBIN_GRAM_SLICES : IHSBIN_GRAM_FMA;
  pl.loop = desc->compute == IHSBIN_COMPUTE_F32X2 ? IHSBIN_LOOP_SLICES : IHSBIN_LOOP_FMA;
  pl.factor = desc->compute == IHSBIN_COMPUTE_F32X2 ? IHSBIN_FACTOR_SLICES : IHSBIN_FACTOR_FMA;
  p->plan = pl;
  const int64_t D = p->A.D, K = p->K;
  AdaptiveBufs b;
  auto cb = [&](size_t n) { return alloc_cbuf(p, desc->compute, n, SCOPE_SCRATCH, &e); };
  b.G = cb((size_t)D * D);
  b.P = cb((size_t)D * D);
  b.c = cb((size_t)D * K);
  b.x = cb((size_t)D * K);
  b.g = cb((size_t)D * K);
  b.d = cb((size_t)D * K);
  b.hd = cb((size_t)D * K);
  if (e == cudaSuccess) e = prob_alloc(p, 8, (void**)&b.lam_dev, SCOPE_SCRATCH);
  if (e == cudaSuccess) e = prob_alloc(p, 8 * 256, (void**)&b.part, SCOPE_SCRATCH);
  if (e == cudaSuccess) e = prob_alloc(p, 16, (void**)&b.dots, SCOPE_SCRATCH);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b.lam_dev, &lam, 8, cudaMemcpyHostToDevice, st);
  auto finish = [&](ihsbin_status r) {
    p->plan = Plan{};
    p->G = p->Pinv = CBuf{};
    p->built = false;
    return r;
  };
  if (e == cudaSuccess) e = adaptive_setup(p, b, st);
  if (e == cudaSuccess) e = adaptive_precond(p, b, st);
  if (e == cudaSuccess) e = adaptive_direction(p, b, st);
  double dots[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(dots, b.dots, 16, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return finish(cuda_fail(e, "adaptive_sketch"));
  if ((s = check_status(p, st, "adaptive_sketch")) != IHSBIN_OK) return finish(s);
  double delta = dots[0];
  const double delta0 = delta;
  int64_t m = sk.m;
  int k = 0, r = 0;
  auto record = [&](int idx, double dl, int64_t mm) {
    if (idx < trace_cap) {
      if (delta_trace) delta_trace[idx] = dl;
      if (m_trace) m_trace[idx] = mm;
    }
  };
  record(0, delta, m);
  while (delta > eps * delta0 && k < max_iter) {
    // f(x - t d) - f(x) = -t delta + t^2/2 <d, (G + lam I) d>: the Armijo test reduces to
    // t <d, (G + lam I) d> <= 2 (1 - gamma2) delta
    if ((e = adaptive_curvature(p, b, lam, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(dots, b.dots, 16, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return finish(cuda_fail(e, "adaptive_sketch"));
    const double q = dots[1];
    int j = 0;
    while (std::pow(g1, j) * q > 2.0 * (1.0 - g2) * delta) {
      if (++j > 200) return finish(fail(IHSBIN_ERR_NOT_SPD, "adaptive_sketch: Armijo search found no step"));
    }
    const double t = std::pow(g1, j);
    if (k < trace_cap && step_trace) step_trace[k] = t;
    if ((e = adaptive_step(p, b, t, st)) != cudaSuccess || (e = adaptive_direction(p, b, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(dots, b.dots, 16, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return finish(cuda_fail(e, "adaptive_sketch"));
    double dnew = dots[0];
    if (dnew >= g3 * delta && 2 * m <= m_max) {
      m *= 2;
      ++r;
      sk.m = m;
      sk.seed = seed0 + (uint64_t)r;
      if ((s = ihsbin_sketch(p, &sk, stream)) != IHSBIN_OK) return finish(s);
      p->plan = pl;
      if ((e = adaptive_precond(p, b, st)) != cudaSuccess || (e = adaptive_direction(p, b, st)) != cudaSuccess ||
          (e = cudaMemcpyAsync(dots, b.dots, 16, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return finish(cuda_fail(e, "adaptive_sketch"));
      if ((s = check_status(p, st, "adaptive_sketch")) != IHSBIN_OK) return finish(s);
      dnew = dots[0];
    }
    delta = dnew;
    ++k;
    record(k, delta, m);
  }
  if (x_out) {
    double* xd = nullptr;
    if ((e = prob_alloc(p, (size_t)D * K * 8, (void**)&xd, SCOPE_SCRATCH)) != cudaSuccess ||
        (e = adaptive_export_x(p, b, xd, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(x_out, xd, (size_t)D * K * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      return finish(cuda_fail(e, "adaptive_sketch"));
  }
  if ((s = check_status(p, st, "adaptive_sketch")) != IHSBIN_OK) return finish(s);
  res->m = m;
  res->iterations = k;
  res->doublings = r;
  res->delta0 = delta0;
  res->delta = delta;
  return finish(IHSBIN_OK);
}



ihsbin_status ihsbin_set_timing(ihsbin_problem* p, int enable) {
  if (!p) return fail(IHSBIN_ERR_INVALID_ARG, "set_timing: NULL");
  p->timing = enable != 0;
  return IHSBIN_OK;
}

ihsbin_status ihsbin_reset_stats(ihsbin_problem* p) {
  if (!p) return fail(IHSBIN_ERR_INVALID_ARG, "reset_stats: NULL");
  for (auto& k : p->kstat) k = KStat{};
  return IHSBIN_OK;
}

ihsbin_status ihsbin_kernel_stats(ihsbin_problem* p, int32_t cat, int64_t* launches, double* ms, double* flops,
                                  double* bytes, const char** name) {
  if (!p) return fail(IHSBIN_ERR_INVALID_ARG, "kernel_stats: NULL");
  if (cat < 0 || cat >= IHSBIN_KCAT_COUNT) return fail(IHSBIN_ERR_INVALID_ARG, "kernel_stats: category out of range");
  static const KStat unused{};
  const KStat& k = cat < K_NCAT ? p->kstat[cat] : unused;  // categories not in use report no launches
  if (launches) *launches = k.launches;
  if (ms) *ms = k.ms;
  if (flops) *flops = k.flops;
  if (bytes) *bytes = k.bytes;
  if (name) *name = cat < K_NCAT ? kcat_names[cat] : "unused";
  return IHSBIN_OK;
}

ihsbin_status ihsbin_kernel_exec(ihsbin_problem* p, int32_t cat, double* xflops, double* xbytes) {
  if (!p) return fail(IHSBIN_ERR_INVALID_ARG, "kernel_exec: NULL");
  if (cat < 0 || cat >= IHSBIN_KCAT_COUNT) return fail(IHSBIN_ERR_INVALID_ARG, "kernel_exec: category out of range");
  static const KStat unused{};
  const KStat& k = cat < K_NCAT ? p->kstat[cat] : unused;
  if (xflops) *xflops = k.xflops;
  if (xbytes) *xbytes = k.xbytes;
  return IHSBIN_OK;
}

ihsbin_status ihsbin_phase_times(ihsbin_problem* p, float* ms5) {
  if (!p || !ms5) return fail(IHSBIN_ERR_INVALID_ARG, "phase_times: NULL argument");
  for (int i = 0; i < 5; ++i) ms5[i] = p->phase_ms[i];
  return IHSBIN_OK;
}

}  // extern "C"
