// Serving: a persistent request loop over one GPU with continuous batching.
//
// A server owns max_slots worker threads, each bound to its own non-blocking
// CUDA stream.  Submitted requests wait in arrival order; an idle worker admits
// the first waiting request whose footprint estimate fits in what is left of
// the device-memory budget (the oldest request cannot be passed over more than
// a bounded number of times), builds the request's structures on its stream
// and runs its likelihood/gradient or prediction call.  While a request runs,
// its CSR pattern, Sigma_m Cholesky, operator and CG block stay resident on the
// device in its own handle; requests that arrive meanwhile are admitted as
// soon as a slot and memory free up, and the work of all resident requests
// overlaps on the GPU through the slot streams.  Every device allocation is
// stream-ordered on the slot's stream, so one request's frees never wait for
// another request's kernels.
//
// The arithmetic of a request is exactly that of the one-request entry points
// (same kernels, same launch shapes, fixed-order reductions): a result is
// bit-for-bit the same alone and in the mix.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <thread>
#include <vector>

#include "fsa_internal.cuh"
#include "fsa.h"

namespace fsa {
void free_handle(fsa_handle* h, bool trim);
void set_error(const std::string& msg);

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kMaxSlots = 64;
constexpr int kMaxPasses = 8;   // admissions of later requests ahead of the oldest one

struct Job {
  uint64_t ticket = 0;
  fsa_request req;
  std::vector<double> locs, inducing, y, pred;
  int64_t footprint = 0;
  int passes = 0;
  double t_submit = 0, t_start = 0;
};

// expected nonzeros of a taper pattern for points spread over their bounding box
double expected_pairs(const std::vector<double>& a, int64_t na, const std::vector<double>* b, int64_t nb,
                      double gamma) {
  double x0 = INFINITY, x1 = -INFINITY, y0 = INFINITY, y1 = -INFINITY;
  for (int64_t i = 0; i < na; ++i) {
    x0 = std::min(x0, a[2 * i]); x1 = std::max(x1, a[2 * i]);
    y0 = std::min(y0, a[2 * i + 1]); y1 = std::max(y1, a[2 * i + 1]);
  }
  const double area = std::max(x1 - x0, gamma) * std::max(y1 - y0, gamma);
  const double frac = std::min(1.0, M_PI * gamma * gamma / area);
  if (b) return (double)nb * (1.0 + (double)na * frac);
  return (double)na * (1.0 + (double)(na - 1) * frac);
}

}  // namespace

// Device bytes a prediction request holds at its peak (FP64 form): structure,
// operator, the block of CG vectors for [Sigma_mn^T, S^T Z] (m + s columns),
// W1, and the prediction-side matrices.
int64_t predict_footprint(int64_t n, int32_t m, int64_t nnz, int64_t n_p, int32_t s, int64_t nnz_cross) {
  const int64_t cb = (int64_t)m + s, ldb = (cb + 7) / 8 * 8;
  int64_t b = 64 * n + 16 * nnz + 128 * (int64_t)m * m + ((int64_t)64 << 20);
  b += 16 * n * (int64_t)m;                  // A and W1
  b += 16 * n * ldb + 56 * n * ldb;          // [Sigma_mn^T, S^T Z] and its solution; CG vectors
  b += 40 * n_p * (int64_t)m;                // Sigma_{m,np}, G and products
  b += 24 * n_p * (int64_t)s + 128 * n_p;    // prediction probes and outputs
  b += 24 * nnz_cross + 32 * n;              // cross pattern, values and its transpose
  return b + b / 4;
}

}  // namespace fsa

using namespace fsa;

struct fsa_server {
  fsa_server_cfg cfg;
  int64_t budget = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::unique_ptr<Job>> pending;
  std::set<uint64_t> running;
  std::map<uint64_t, fsa_result> done;
  int64_t in_use = 0, peak_in_use = 0;
  int n_running = 0, peak_running = 0;
  int64_t submitted = 0, completed = 0, failed = 0;
  std::vector<double> latencies;
  double first_submit = -1, last_end = 0;
  bool stop = false;
  uint64_t next_ticket = 1;
  std::vector<cudaStream_t> streams;
  std::vector<std::thread> workers;
  Clock::time_point t0 = Clock::now();

  double now_ms() const { return std::chrono::duration<double, std::milli>(Clock::now() - t0).count(); }

  // first waiting request that fits; the oldest one blocks the rest once it
  // has been passed over kMaxPasses times
  std::deque<std::unique_ptr<Job>>::iterator pick() {
    for (auto it = pending.begin(); it != pending.end(); ++it) {
      if (in_use + (*it)->footprint <= budget) {
        if (it != pending.begin()) pending.front()->passes++;
        return it;
      }
      if (it == pending.begin() && (*it)->passes >= kMaxPasses) break;
    }
    return pending.end();
  }

  void run(Job& j, cudaStream_t s, int slot) {
    fsa_result r;
    std::memset(&r, 0, sizeof(r));
    r.kind = j.req.kind;
    r.slot = slot;
    r.footprint_bytes = j.footprint;
    TraceRange trace(j.req.kind == FSA_REQ_LOGLIK_GRAD ? "serve_loglik_grad" : "serve_predict");
    fsa_handle* h = nullptr;
    fsa_status st = fsa_build(j.locs.data(), j.req.n, j.inducing.data(), j.req.m, j.req.taper_range, j.req.cov, s, &h);
    if (st == FSA_OK) {
      if (j.req.kind == FSA_REQ_LOGLIK_GRAD) {
        st = fsa_loglik_grad(h, j.y.data(), &j.req.theta, &j.req.opts, &r.loglik, r.grad, &r.info);
      } else {
        st = fsa_predict(h, j.y.data(), &j.req.theta, &j.req.opts, j.pred.data(), j.req.n_p, j.req.num_var_samples,
                         j.req.mean, j.req.var, &r.info);
      }
    }
    if (st != FSA_OK) std::snprintf(r.message, sizeof(r.message), "%s", fsa_last_error());
    if (h) free_handle(h, false);
    r.status = st;
    const double t_end = now_ms();
    r.queue_ms = j.t_start - j.t_submit;
    r.run_ms = t_end - j.t_start;
    r.latency_ms = t_end - j.t_submit;
    std::lock_guard<std::mutex> lk(mu);
    in_use -= j.footprint;
    n_running--;
    running.erase(j.ticket);
    done[j.ticket] = r;
    completed++;
    if (st != FSA_OK && st != FSA_ERR_NO_CONVERGENCE) failed++;
    latencies.push_back(r.latency_ms);
    last_end = std::max(last_end, t_end);
    cv_done.notify_all();
    cv_work.notify_all();
  }

  void worker(int slot) {
    cudaSetDevice(cfg.device);
    cudaStream_t s = streams[slot];
    for (;;) {
      std::unique_ptr<Job> job;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] { return (stop && pending.empty()) || pick_ready(); });
        if (pending.empty()) return;   // stop requested and nothing left
        auto it = pick();
        if (it == pending.end()) continue;
        job = std::move(*it);
        pending.erase(it);
        in_use += job->footprint;
        peak_in_use = std::max(peak_in_use, in_use);
        n_running++;
        peak_running = std::max(peak_running, n_running);
        running.insert(job->ticket);
        job->t_start = now_ms();
      }
      run(*job, s, slot);
    }
  }

  // predicate form of pick() that does not count passes
  bool pick_ready() const {
    for (auto it = pending.begin(); it != pending.end(); ++it) {
      if (in_use + (*it)->footprint <= budget) return true;
      if (it == pending.begin() && (*it)->passes >= kMaxPasses) return false;
    }
    return false;
  }
};

// the part of fsa_serve_submit that copies the request (host allocations)
static fsa_status submit_job(fsa_server* S, const fsa_request* q, uint64_t* ticket) {
  auto j = std::make_unique<Job>();
  j->req = *q;
  j->locs.assign(q->locs, q->locs + 2 * q->n);
  j->inducing.assign(q->inducing, q->inducing + 2 * (int64_t)q->m);
  j->y.assign(q->y, q->y + q->n);
  const double nnz = 1.25 * expected_pairs(j->locs, q->n, nullptr, 0, q->taper_range);
  if (q->kind == FSA_REQ_LOGLIK_GRAD) {
    j->footprint = fsa_footprint_bytes(q->n, q->m, (int64_t)nnz, q->opts.num_probes, q->opts.precision);
  } else {
    j->pred.assign(q->pred_locs, q->pred_locs + 2 * q->n_p);
    const double cross = 1.25 * expected_pairs(j->locs, q->n, &j->pred, q->n_p, q->taper_range);
    j->footprint = predict_footprint(q->n, q->m, (int64_t)nnz, q->n_p, q->var ? q->num_var_samples : 0,
                                     (int64_t)cross);
  }
  std::lock_guard<std::mutex> lk(S->mu);
  if (j->footprint > S->budget) {
    set_error("request footprint " + std::to_string(j->footprint) + " bytes exceeds the server budget " +
              std::to_string(S->budget));
    return FSA_ERR_OOM;
  }
  if (S->stop) { set_error("server is shutting down"); return FSA_ERR_ARG; }
  j->ticket = S->next_ticket++;
  j->t_submit = S->now_ms();
  if (S->first_submit < 0) S->first_submit = j->t_submit;
  *ticket = j->ticket;
  S->pending.push_back(std::move(j));
  S->submitted++;
  S->cv_work.notify_one();
  return FSA_OK;
}

extern "C" {

void fsa_default_server_cfg(fsa_server_cfg* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->device = 0;
  c->max_slots = 4;
  c->hbm_budget_bytes = 0;
}

fsa_status fsa_server_create(const fsa_server_cfg* cfg, fsa_server** out) {
  if (!out) { set_error("out is NULL"); return FSA_ERR_ARG; }
  *out = nullptr;
  fsa_server_cfg c;
  fsa_default_server_cfg(&c);
  if (cfg) c = *cfg;
  if (c.max_slots < 1 || c.max_slots > kMaxSlots) { set_error("max_slots must be in [1, 64]"); return FSA_ERR_ARG; }
  if (cudaSetDevice(c.device) != cudaSuccess) {
    cudaGetLastError();
    set_error("cannot select the CUDA device");
    return FSA_ERR_CUDA;
  }
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMemGetInfo failed");
    return FSA_ERR_CUDA;
  }
  auto* S = new fsa_server();
  S->cfg = c;
  S->budget = c.hbm_budget_bytes > 0 ? std::min<int64_t>(c.hbm_budget_bytes, (int64_t)free_b)
                                     : (int64_t)(0.85 * (double)free_b);
  S->streams.resize(c.max_slots);
  for (int k = 0; k < c.max_slots; ++k) {
    if (cudaStreamCreateWithFlags(&S->streams[k], cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      for (int j = 0; j < k; ++j) cudaStreamDestroy(S->streams[j]);
      delete S;
      set_error("cudaStreamCreate failed");
      return FSA_ERR_CUDA;
    }
  }
  try {
    for (int k = 0; k < c.max_slots; ++k) S->workers.emplace_back([S, k] { S->worker(k); });
  } catch (const std::exception& e) {
    fsa_server_destroy(S);   // joins the workers that did start, destroys the streams
    return fail_host_exception("fsa_server_create", e);
  }
  *out = S;
  return FSA_OK;
}

fsa_status fsa_serve_submit(fsa_server* S, const fsa_request* q, uint64_t* ticket) {
  if (!S || !q || !ticket) { set_error("NULL argument"); return FSA_ERR_ARG; }
  if (q->kind != FSA_REQ_LOGLIK_GRAD && q->kind != FSA_REQ_PREDICT) { set_error("unknown request kind"); return FSA_ERR_ARG; }
  if (!q->locs || !q->inducing || !q->y || q->n < 2 || q->m < 1 || q->m > q->n || !(q->taper_range > 0)) {
    set_error("bad sizes or NULL inputs");
    return FSA_ERR_ARG;
  }
  if (q->opts.y_on_device) { set_error("serving takes host responses (y_on_device = 0)"); return FSA_ERR_ARG; }
  if (q->kind == FSA_REQ_PREDICT && (!q->pred_locs || q->n_p < 1 || !q->mean)) {
    set_error("prediction needs pred_locs, n_p >= 1 and mean");
    return FSA_ERR_ARG;
  }
  try {
    return submit_job(S, q, ticket);
  } catch (const std::exception& e) {
    return fail_host_exception("fsa_serve_submit", e);
  }
}

static fsa_status take_result(fsa_server* S, uint64_t ticket, fsa_result* out) {
  auto it = S->done.find(ticket);
  if (it == S->done.end()) return FSA_ERR_BUSY;
  if (out) *out = it->second;
  S->done.erase(it);
  return FSA_OK;
}

static bool known(fsa_server* S, uint64_t ticket) {
  if (S->done.count(ticket) || S->running.count(ticket)) return true;
  for (auto& j : S->pending)
    if (j->ticket == ticket) return true;
  return false;
}

fsa_status fsa_serve_poll(fsa_server* S, uint64_t ticket, fsa_result* out) {
  if (!S) { set_error("NULL server"); return FSA_ERR_ARG; }
  std::lock_guard<std::mutex> lk(S->mu);
  if (!known(S, ticket)) { set_error("unknown or already retrieved ticket"); return FSA_ERR_ARG; }
  return take_result(S, ticket, out);
}

fsa_status fsa_serve_wait(fsa_server* S, uint64_t ticket, double timeout_s, fsa_result* out) {
  if (!S) { set_error("NULL server"); return FSA_ERR_ARG; }
  std::unique_lock<std::mutex> lk(S->mu);
  if (!known(S, ticket)) { set_error("unknown or already retrieved ticket"); return FSA_ERR_ARG; }
  auto ready = [&] { return S->done.count(ticket) > 0; };
  if (timeout_s < 0) {
    S->cv_done.wait(lk, ready);
  } else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
    set_error("timed out waiting for the request");
    return FSA_ERR_TIMEOUT;
  }
  return take_result(S, ticket, out);
}

fsa_status fsa_server_get_stats(fsa_server* S, fsa_server_stats* st) {
  if (!S || !st) { set_error("NULL argument"); return FSA_ERR_ARG; }
  std::lock_guard<std::mutex> lk(S->mu);
  std::memset(st, 0, sizeof(*st));
  st->submitted = S->submitted;
  st->completed = S->completed;
  st->failed = S->failed;
  st->pending = (int64_t)S->pending.size();
  st->running = S->n_running;
  st->peak_running = S->peak_running;
  st->budget_bytes = S->budget;
  st->in_use_bytes = S->in_use;
  st->peak_in_use_bytes = S->peak_in_use;
  if (!S->latencies.empty()) {
    std::vector<double> l = S->latencies;
    std::sort(l.begin(), l.end());
    auto rank = [&](double p) {   // nearest-rank percentile
      size_t k = (size_t)std::ceil(p * (double)l.size());
      return l[std::min(l.size(), std::max<size_t>(k, 1)) - 1];
    };
    st->p50_ms = rank(0.50);
    st->p99_ms = rank(0.99);
    double sum = 0;
    for (double v : l) sum += v;
    st->mean_ms = sum / (double)l.size();
    const double span = S->last_end - S->first_submit;
    st->completed_per_s = span > 0 ? 1e3 * (double)S->completed / span : 0.0;
  }
  return FSA_OK;
}

void fsa_server_destroy(fsa_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  cudaSetDevice(S->cfg.device);
  for (auto s : S->streams) cudaStreamDestroy(s);
  release_pool_memory();
  delete S;
}

}  // extern "C"
