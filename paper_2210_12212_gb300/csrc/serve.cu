// Continuous-batching request loop for ridge-path solves (ihsbin_serve_*).
//
// `slots` worker threads each own a non-blocking CUDA stream.  A worker takes
// the first queued request whose estimated device-memory footprint fits what
// the server budget has left (first fit, so a large request at the head does
// not block smaller ones behind it), runs its whole path (problem creation,
// sketch, basis, evaluation) on its own stream, and releases the footprint
// when it finishes.  Requests that arrive while others are on the GPU are thus
// admitted as slots and memory free up, and their kernels overlap on the
// device.  Every request is an independent problem: its arithmetic and
// reduction order do not depend on what else is running.
//
// All waits on the host are bounded (ihsbin_serve_wait takes a timeout); no
// device code waits on anything.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <memory>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace {

using clk = std::chrono::steady_clock;

struct Req {
  uint64_t ticket = 0;
  ihsbin_request r{};
  std::vector<double> lambdas;
  uint64_t footprint = 0;
  ihsbin_status status = IHSBIN_OK;
  std::string err;
  bool done = false;
  clk::time_point t_submit, t_admit, t_done;
  float device_ms = 0;
};

double secs(clk::time_point a, clk::time_point b) { return std::chrono::duration<double>(b - a).count(); }

size_t esize(int dt) { return dt == IHSBIN_F64 ? 8 : dt == IHSBIN_F32 ? 4 : 2; }

}  // namespace

struct ihsbin_server {
  ihsbin_ctx* ctx = nullptr;
  int slots = 4;
  uint64_t budget = 0;
  uint64_t in_flight = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Req>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<Req>> reqs;
  std::vector<std::thread> workers;
  bool stop = false;
  uint64_t next_ticket = 1;
};

namespace ihsbin {

// Upper estimate of the device memory one request holds at its peak (bytes).
uint64_t request_footprint(const ihsbin_request* q) {
  const ihsbin_matrix& A = q->A;
  const double n = (double)A.n, d = (double)A.d;
  const double N = std::max(n, d), D = std::min(n, d);
  const double K = (double)q->K, m = (double)q->sketch.m, T = (double)q->T;
  const double es = (double)esize(A.dtype);
  double bytes = 0;
  // data and its transposed copy / CSR transpose
  const double data = A.layout == IHSBIN_CSR ? A.nnz * (es + 4) + 8.0 * (A.n + 1) : n * d * es;
  if (!A.on_device) bytes += data;
  if (A.layout == IHSBIN_CSR || A.n < A.d) bytes += data + 8.0 * (N + 1);
  bytes += n * K * 8;                                           // B
  // sketch: SA, G_S, draws, Hadamard intermediates
  double np2 = 1;
  while (np2 < N) np2 *= 2;
  bytes += m * D * 8 + D * D * 8 + np2 * 17;
  if (q->sketch.kind == IHSBIN_SK_SRHT) bytes += 2 * np2 * D * 8;
  if (q->sketch.kind == IHSBIN_SK_GAUSSIAN) bytes += 256.0 * (1 << 20);
  // factor and inverse of every interval, Gram matrix and its split partials
  const ihsbin_path_desc& pd = q->path;
  double L = pd.L > 0 ? pd.L : std::max(1.0, std::floor(2.0 * std::log(pd.lambda_max / pd.lambda_min)));
  double kmax = pd.k_default > 0 ? pd.k_default : 256;
  if (pd.k) for (int l = 0; l < (int)L; ++l) kmax = std::max(kmax, (double)pd.k[l]);
  const double jc = pd.jmax > 0 ? std::min((double)pd.jmax, kmax) : kmax;
  bytes += 3 * L * D * D * 8 + D * D * 8 * 9;
  // slices of the tensor-core products of the recursion (float-float compute)
  if (pd.compute == IHSBIN_COMPUTE_F32X2 && pd.loop != IHSBIN_LOOP_FMA)
    bytes += (double)loop_slices_bytes((int64_t)D, (int)L, (int64_t)(jc * K));
  // slices and exact partials of the tensor-core inverse W^T W
  if (pd.compute == IHSBIN_COMPUTE_F32X2 && pd.factor != IHSBIN_FACTOR_FMA)
    bytes += L * (2.0 * (oz_vec_elems((int64_t)D, (int64_t)D, 128) + oz_vec_elems((int64_t)D, (int64_t)D, 32)) +
                  16.0 * D * D);
  // integer slices and tiles of the tensor-core Gram (dense FP32/BF16 data)
  if (A.layout == IHSBIN_DENSE_ROWMAJOR && A.dtype != IHSBIN_F64 && pd.gram != IHSBIN_GRAM_FMA &&
      pd.product != IHSBIN_PRODUCT_ASPACE)
    bytes += (double)gram_slices_scratch_bytes((int64_t)N, (int64_t)D);
  // recursion buffers: U (2), utilde, R, and the split partials of Y and Z (16 each)
  bytes += (4 + 32) * L * jc * K * D * 8;
  if (A.n < A.d) bytes += L * jc * K * N * 8;                   // dual map
  // evaluation: coefficients and the output staged on the device
  bytes += T * jc * 8 + (q->x_on_device ? 0 : T * d * K * esize(q->x_dtype));
  return (uint64_t)(1.25 * bytes) + (64u << 20);
}

}  // namespace ihsbin

namespace {

void run_request(ihsbin_server* s, Req& r, cudaStream_t st) {
  ihsbin_problem* p = nullptr;
  const ihsbin_request& q = r.r;
  ihsbin_status status = ihsbin_problem_create(s->ctx, &q.A, q.B, q.K, q.ldb, q.b_dtype, q.b_on_device, &p);
  if (status == IHSBIN_OK) status = ihsbin_sketch(p, &q.sketch, st);
  if (status == IHSBIN_OK) status = ihsbin_build_basis(p, &q.path, st);
  if (status == IHSBIN_OK)
    status = ihsbin_eval_path(p, r.lambdas.data(), (int64_t)r.lambdas.size(), q.X, q.x_dtype, q.x_on_device, st);
  if (status != IHSBIN_OK) r.err = ihsbin_last_error();
  if (p) {
    float ms[5];
    if (ihsbin_phase_times(p, ms) == IHSBIN_OK) r.device_ms = ms[0] + ms[1] + ms[2] + ms[3] + ms[4];
    ihsbin_problem_destroy(p);
  }
  r.status = status;
}

void worker_main(ihsbin_server* s) {
  cudaSetDevice(s->ctx->device);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  for (;;) {
    std::shared_ptr<Req> r;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      for (;;) {
        if (s->stop && s->queue.empty()) break;
        auto it = std::find_if(s->queue.begin(), s->queue.end(), [&](const std::shared_ptr<Req>& x) {
          return !s->budget || s->in_flight + x->footprint <= s->budget;
        });
        if (it != s->queue.end()) {
          r = *it;
          s->queue.erase(it);
          s->in_flight += r->footprint;
          r->t_admit = clk::now();
          break;
        }
        s->cv_work.wait_for(lk, std::chrono::milliseconds(50));
      }
    }
    if (!r) break;
    run_request(s, *r, st);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->in_flight -= r->footprint;
      r->t_done = clk::now();
      r->done = true;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
  cudaStreamDestroy(st);
}

}  // namespace

extern "C" {

ihsbin_status ihsbin_request_footprint(const ihsbin_request* q, uint64_t* bytes) {
  if (!q || !bytes) {
    ihsbin::set_last_error("request_footprint: NULL argument");
    return IHSBIN_ERR_INVALID_ARG;
  }
  *bytes = ihsbin::request_footprint(q);
  return IHSBIN_OK;
}

ihsbin_status ihsbin_serve_create(ihsbin_ctx* ctx, const ihsbin_serve_config* cfg, ihsbin_server** out) {
  if (!ctx || !out) {
    ihsbin::set_last_error("serve_create: NULL argument");
    return IHSBIN_ERR_INVALID_ARG;
  }
  *out = nullptr;
  ihsbin_server* s = new (std::nothrow) ihsbin_server();
  if (!s) {
    ihsbin::set_last_error("serve_create: host allocation failed");
    return IHSBIN_ERR_OUT_OF_MEMORY;
  }
  s->ctx = ctx;
  s->slots = (cfg && cfg->slots > 0) ? cfg->slots : 4;
  s->budget = (cfg && cfg->hbm_budget_bytes) ? cfg->hbm_budget_bytes : ctx->budget;
  for (int i = 0; i < s->slots; ++i) s->workers.emplace_back(worker_main, s);
  *out = s;
  return IHSBIN_OK;
}

ihsbin_status ihsbin_serve_submit(ihsbin_server* s, const ihsbin_request* q, uint64_t* ticket) {
  if (!s || !q || !ticket || !q->lambdas || q->T <= 0 || !q->X) {
    ihsbin::set_last_error("serve_submit: NULL argument or T <= 0");
    return IHSBIN_ERR_INVALID_ARG;
  }
  auto r = std::make_shared<Req>();
  r->r = *q;
  r->lambdas.assign(q->lambdas, q->lambdas + q->T);
  r->footprint = ihsbin::request_footprint(q);
  if (s->budget && r->footprint > s->budget) {
    ihsbin::set_last_error("serve_submit: request footprint exceeds the server's device-memory budget");
    return IHSBIN_ERR_ADMISSION;
  }
  r->t_submit = clk::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      ihsbin::set_last_error("serve_submit: server is shutting down");
      return IHSBIN_ERR_STATE;
    }
    r->ticket = s->next_ticket++;
    s->reqs[r->ticket] = r;
    s->queue.push_back(r);
  }
  s->cv_work.notify_one();
  *ticket = r->ticket;
  return IHSBIN_OK;
}

ihsbin_status ihsbin_serve_wait(ihsbin_server* s, uint64_t ticket, int64_t timeout_us, ihsbin_status* result,
                                double* times4) {
  if (!s || !result) {
    ihsbin::set_last_error("serve_wait: NULL argument");
    return IHSBIN_ERR_INVALID_ARG;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) {
    ihsbin::set_last_error("serve_wait: unknown ticket");
    return IHSBIN_ERR_INVALID_ARG;
  }
  std::shared_ptr<Req> r = it->second;
  const auto deadline = clk::now() + std::chrono::microseconds(timeout_us < 0 ? 0 : timeout_us);
  while (!r->done) {
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !r->done) {
      ihsbin::set_last_error("serve_wait: timed out");
      return IHSBIN_ERR_TIMEOUT;
    }
  }
  *result = r->status;
  if (times4) {
    times4[0] = secs(r->t_submit, r->t_admit);  // queueing
    times4[1] = secs(r->t_admit, r->t_done);    // service
    times4[2] = secs(r->t_submit, r->t_done);   // total
    times4[3] = r->device_ms * 1e-3;            // device time of the path's phases
  }
  if (r->status != IHSBIN_OK) ihsbin::set_last_error(r->err.c_str());
  s->reqs.erase(it);
  return IHSBIN_OK;
}

ihsbin_status ihsbin_serve_destroy(ihsbin_server* s) {
  if (!s) {
    ihsbin::set_last_error("serve_destroy: NULL");
    return IHSBIN_ERR_INVALID_ARG;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  delete s;
  return IHSBIN_OK;
}

ihsbin_status ihsbin_serve(ihsbin_ctx* ctx, const ihsbin_serve_config* cfg, const ihsbin_request* reqs, int64_t n,
                           const double* arrival_s, ihsbin_status* results, double* latency_s) {
  if (!ctx || (!reqs && n) || n < 0) {
    ihsbin::set_last_error("serve: bad arguments");
    return IHSBIN_ERR_INVALID_ARG;
  }
  ihsbin_server* s = nullptr;
  ihsbin_status st = ihsbin_serve_create(ctx, cfg, &s);
  if (st != IHSBIN_OK) return st;
  std::vector<uint64_t> tickets(n, 0);
  std::vector<double> lag(n, 0.0);
  const auto t0 = clk::now();
  for (int64_t i = 0; i < n; ++i) {
    const auto sched = t0 + std::chrono::duration_cast<clk::duration>(
                                std::chrono::duration<double>(arrival_s ? arrival_s[i] : 0.0));
    std::this_thread::sleep_until(sched);
    lag[i] = secs(sched, clk::now());  // submission later than the scheduled arrival counts as latency
    ihsbin_status si = ihsbin_serve_submit(s, &reqs[i], &tickets[i]);
    if (si != IHSBIN_OK) {
      if (results) results[i] = si;
      tickets[i] = 0;
    }
  }
  ihsbin_status overall = IHSBIN_OK;
  for (int64_t i = 0; i < n; ++i) {
    if (!tickets[i]) {
      if (latency_s) latency_s[i] = 0;
      continue;
    }
    ihsbin_status res = IHSBIN_ERR_TIMEOUT;
    double t4[4] = {0, 0, 0, 0};
    for (int tries = 0; tries < 3600; ++tries)  // bounded: at most an hour per request
      if (ihsbin_serve_wait(s, tickets[i], 1000000, &res, t4) != IHSBIN_ERR_TIMEOUT) break;
    if (results) results[i] = res;
    if (res == IHSBIN_ERR_TIMEOUT) overall = IHSBIN_ERR_TIMEOUT;
    if (latency_s) latency_s[i] = lag[i] + t4[2];  // scheduled arrival -> completion
  }
  ihsbin_status d = ihsbin_serve_destroy(s);
  return overall != IHSBIN_OK ? overall : d;
}

}  // extern "C"
