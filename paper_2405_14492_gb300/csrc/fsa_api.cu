// C ABI of the FSA library (declared in include/fsa.h).  Every entry point
// catches library errors and returns a status; nothing throws across the ABI.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "fsa_solver.cuh"
#include "fsa_profile.h"

namespace fsa {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

fsa_status fail_host_exception(const char* where, const std::exception& e) {
  const bool oom = dynamic_cast<const std::bad_alloc*>(&e) != nullptr;
  try {
    set_error(std::string(where) + (oom ? ": host memory could not be allocated: " : ": ") + e.what());
  } catch (...) {
  }
  return oom ? FSA_ERR_OOM : FSA_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// stream-ordered allocation: per-thread stream, pool configured once per device
// ---------------------------------------------------------------------------
static thread_local cudaStream_t g_alloc_stream = nullptr;

static void configure_pool() {
  static std::mutex mu;
  static bool done[256] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return;
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    // keep freed blocks in the pool between calls instead of unmapping them at every synchronisation
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  done[dev] = true;
}

cudaStream_t current_alloc_stream() { return g_alloc_stream; }
AllocStreamScope::AllocStreamScope(cudaStream_t s) : prev(g_alloc_stream) {
  configure_pool();
  g_alloc_stream = s;
}
AllocStreamScope::~AllocStreamScope() { g_alloc_stream = prev; }

void release_pool_memory() {
  int dev = 0;
  cudaMemPool_t pool;
  if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess)
    cudaMemPoolTrimTo(pool, 0);
}

// small pinned host buffers (CG polling), recycled: freeing pinned memory
// would synchronise the device
static std::mutex g_pin_mu;
static std::vector<double*> g_pin_free;
static double* pinned_acquire() {
  {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    if (!g_pin_free.empty()) {
      double* p = g_pin_free.back();
      g_pin_free.pop_back();
      return p;
    }
  }
  double* p = nullptr;
  FSA_CUDA(cudaMallocHost(&p, 64 * sizeof(double)));
  return p;
}
static void pinned_release(double* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_pin_mu);
  g_pin_free.push_back(p);
}

static __global__ void k_to_internal(int64_t n, int k, const int64_t* __restrict__ perm,
                                     const double* __restrict__ src, double* __restrict__ dst) {
  int64_t total = n * k;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = t / k;
    int c = (int)(t - i * k);
    dst[t] = src[perm[i] * k + c];
  }
}

static __global__ void k_to_original(int64_t n, int k, const int64_t* __restrict__ perm,
                                     const double* __restrict__ src, double* __restrict__ dst) {
  int64_t total = n * k;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = t / k;
    int c = (int)(t - i * k);
    dst[perm[i] * k + c] = src[t];
  }
}

void to_internal(Handle& H, int k, const double* src, double* dst) {
  k_to_internal<<<grid_for(H.n * k, 256), 256, 0, H.stream>>>(H.n, k, H.perm.p, src, dst);
  FSA_CHECK_LAUNCH();
}
void to_original(Handle& H, int k, const double* src, double* dst) {
  k_to_original<<<grid_for(H.n * k, 256), 256, 0, H.stream>>>(H.n, k, H.perm.p, src, dst);
  FSA_CHECK_LAUNCH();
}

static fsa_status fail(const Error& e) {
  set_error(e.msg);
  return e.code;
}

static bool theta_ok(const fsa_theta* t) {
  return t && std::isfinite(t->sigma1_sq) && std::isfinite(t->rho) && std::isfinite(t->nugget) &&
         t->sigma1_sq > 0 && t->rho > 0 && t->nugget > 0;
}

static fsa_opts resolve_opts(const fsa_opts* o) {
  fsa_opts r;
  fsa_default_opts(&r);
  if (o) r = *o;
  if (r.cg_max_iter <= 0) r.cg_max_iter = 1000;
  return r;
}

}  // namespace fsa

using namespace fsa;


namespace fsa {
// Releases a handle: its buffers are freed in the order of its stream, the
// stream is drained, and (trim) unused pool memory goes back to the driver.
void free_handle(fsa_handle* h, bool trim) {
  Handle& H = h->h;
  cudaStream_t s = H.stream;
  pinned_release(H.host_pinned);
  H.host_pinned = nullptr;
  if (H.ev0) cudaEventDestroy(H.ev0);
  if (H.ev1) cudaEventDestroy(H.ev1);
  if (H.side) cudaStreamSynchronize(H.side);
  if (H.ev_fork) cudaEventDestroy(H.ev_fork);
  if (H.ev_join) cudaEventDestroy(H.ev_join);
  cudaStream_t side = H.side;
  delete h;
  if (side) cudaStreamDestroy(side);
  cudaStreamSynchronize(s);
  if (trim) release_pool_memory();
}
}  // namespace fsa

extern "C" {

void fsa_default_opts(fsa_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->num_probes = 50;
  o->cg_tol = 1e-3;
  o->cg_max_iter = 1000;
  o->fixed_iters = 0;
  o->precision = FSA_FP64;
  o->probe = FSA_PROBE_RADEMACHER;
  o->seed = 14492;
  o->slq_exact_weight = 0;
  o->want_grad = 1;
  o->y_on_device = 0;
}

const char* fsa_status_string(fsa_status s) {
  switch (s) {
    case FSA_OK: return "FSA_OK";
    case FSA_ERR_ARG: return "FSA_ERR_ARG";
    case FSA_ERR_OOM: return "FSA_ERR_OOM";
    case FSA_ERR_NOT_PD: return "FSA_ERR_NOT_PD";
    case FSA_ERR_NO_CONVERGENCE: return "FSA_ERR_NO_CONVERGENCE";
    case FSA_ERR_NAN: return "FSA_ERR_NAN";
    case FSA_ERR_TIMEOUT: return "FSA_ERR_TIMEOUT";
    case FSA_ERR_BUSY: return "FSA_ERR_BUSY";
    case FSA_ERR_CUDA: return "FSA_ERR_CUDA";
    case FSA_ERR_UNSUPPORTED: return "FSA_ERR_UNSUPPORTED";
    case FSA_ERR_BOUNDS: return "FSA_ERR_BOUNDS";
  }
  return "FSA_ERR_UNKNOWN";
}

const char* fsa_last_error(void) { return g_last_error.c_str(); }

int64_t fsa_pool_used_high(int reset) {
  int dev = 0;
  cudaMemPool_t pool;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  uint64_t v = 0;
  if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &v) != cudaSuccess) return -1;
  if (reset) {
    uint64_t zero = 0;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero);
  }
  return (int64_t)v;
}

fsa_status fsa_build(const double* locs, int64_t n, const double* inducing, int32_t m, double taper_range,
                     int32_t cov, void* cuda_stream, fsa_handle** out) {
  if (!out) return fail(Error{FSA_ERR_ARG, "out is NULL"});
  *out = nullptr;
  if (!locs || !inducing || n < 2 || m < 1 || m > n || n > ((int64_t)1 << 31) - 1)
    return fail(Error{FSA_ERR_ARG, "bad sizes or NULL coordinates (need n >= 2, 1 <= m <= n < 2^31)"});
  if (!(taper_range > 0) || !std::isfinite(taper_range)) return fail(Error{FSA_ERR_ARG, "taper_range must be > 0"});
  if (cov != FSA_EXPONENTIAL && cov != FSA_MATERN_1_5) return fail(Error{FSA_ERR_ARG, "unknown covariance"});
  for (int32_t k = 0; k < 2 * m; ++k)
    if (!std::isfinite(inducing[k])) return fail(Error{FSA_ERR_NAN, "non-finite inducing point"});
  fsa_handle* hh = nullptr;
  TraceRange trace("fsa_build");
  try {
    hh = new fsa_handle();
    Handle& H = hh->h;
    H.n = n;
    H.m = m;
    H.gamma = taper_range;
    H.cov = cov;
    H.stream = (cudaStream_t)cuda_stream;
    AllocStreamScope scope(H.stream);
    H.err_buf.alloc(1);
    H.err = H.err_buf.p;
    FSA_CUDA(cudaMemsetAsync(H.err, 0, sizeof(unsigned), H.stream));
    H.host_pinned = pinned_acquire();
    FSA_CUDA(cudaEventCreate(&H.ev0));
    FSA_CUDA(cudaEventCreate(&H.ev1));
    std::vector<double> ix(m), iy(m);
    for (int32_t k = 0; k < m; ++k) { ix[k] = inducing[2 * k]; iy[k] = inducing[2 * k + 1]; }
    H.ind_x.alloc(m);
    H.ind_y.alloc(m);
    FSA_CUDA(cudaMemcpyAsync(H.ind_x.p, ix.data(), sizeof(double) * m, cudaMemcpyHostToDevice, H.stream));
    FSA_CUDA(cudaMemcpyAsync(H.ind_y.p, iy.data(), sizeof(double) * m, cudaMemcpyHostToDevice, H.stream));
    build_structure(H, locs);
    *out = hh;
    return FSA_OK;
  } catch (const Error& e) {
    fsa_free(hh);
    return fail(e);
  } catch (const std::exception& e) {
    fsa_free(hh);
    return fail_host_exception("fsa_build", e);
  }
}

int64_t fsa_nnz(const fsa_handle* h) { return h ? h->h.nnz : -1; }

fsa_status fsa_grad_terms(fsa_handle* h, double* a, double* b, int32_t num_probes) {
  if (!h || !a || !b) return fail(Error{FSA_ERR_ARG, "NULL argument"});
  Handle& H = h->h;
  if (H.gterms_l <= 0 || !H.gterms.p) return fail(Error{FSA_ERR_ARG, "no gradient has been computed on this handle"});
  if (num_probes != H.gterms_l)
    return fail(Error{FSA_ERR_ARG, "num_probes differs from the last call's (" + std::to_string(H.gterms_l) + ")"});
  try {
    const size_t k = (size_t)3 * num_probes;
    FSA_CUDA(cudaMemcpyAsync(a, H.gterms.p, sizeof(double) * k, cudaMemcpyDeviceToHost, H.stream));
    FSA_CUDA(cudaMemcpyAsync(b, H.gterms.p + k, sizeof(double) * k, cudaMemcpyDeviceToHost, H.stream));
    FSA_CUDA(cudaStreamSynchronize(H.stream));
    return FSA_OK;
  } catch (const Error& e) {
    return fail(e);
  }
}

fsa_status fsa_get_csr(fsa_handle* h, int64_t* rowptr, int32_t* col) {
  if (!h || !rowptr || !col) return fail(Error{FSA_ERR_ARG, "NULL argument"});
  try {
    AllocStreamScope scope(h->h.stream);
    export_csr(h->h, rowptr, col);
    return FSA_OK;
  } catch (const Error& e) {
    return fail(e);
  } catch (const std::exception& e) {
    return fail_host_exception("fsa_get_csr", e);
  }
}

fsa_status fsa_loglik_grad(fsa_handle* h, const double* y, const fsa_theta* theta, const fsa_opts* opts,
                           double* loglik, double* grad, fsa_info* info) {
  if (!h || !y || !loglik) return fail(Error{FSA_ERR_ARG, "NULL argument"});
  if (!theta_ok(theta)) return fail(Error{FSA_ERR_ARG, "theta must be finite and > 0"});
  fsa_opts o = resolve_opts(opts);
  if (o.num_probes < 1 || o.num_probes > 1000) return fail(Error{FSA_ERR_ARG, "num_probes must be in [1, 1000]"});
  if (o.want_grad && !grad) return fail(Error{FSA_ERR_ARG, "grad is NULL"});
  if (o.cg_max_iter > 8000 || o.fixed_iters > 8000 || o.fixed_iters < 0)
    return fail(Error{FSA_ERR_ARG, "cg_max_iter / fixed_iters must be <= 8000"});
  if (!(o.cg_tol >= 0.0)) return fail(Error{FSA_ERR_ARG, "cg_tol must be >= 0"});
  if (o.precision < FSA_FP64 || o.precision > FSA_MIXED_BF16X2) return fail(Error{FSA_ERR_ARG, "bad precision"});
  if (o.probe != FSA_PROBE_RADEMACHER && o.probe != FSA_PROBE_GAUSSIAN) return fail(Error{FSA_ERR_ARG, "bad probe"});
  if (o.vec_pieces != 0 && o.vec_pieces != 2 && o.vec_pieces != 3)
    return fail(Error{FSA_ERR_ARG, "vec_pieces must be 0, 2 or 3"});
  if (o.grad_control_variate < 0 || o.grad_control_variate > 3)
    return fail(Error{FSA_ERR_ARG, "grad_control_variate must be 0, 1, 2 or 3"});
  if (o.grad_control_variate != 0 && o.num_probes < 2)
    return fail(Error{FSA_ERR_ARG, "the gradient's control variate needs at least 2 probes"});
  Handle& H = h->h;
  AllocStreamScope scope(H.stream);
  TraceRange trace("fsa_loglik_grad");
  try {
    FSA_CUDA(cudaEventRecord(H.ev0, H.stream));
    H.y.ensure(H.n);
    {
      const double* ydev = y;
      DevPtr<double> tmp;
      if (!o.y_on_device) {
        tmp.alloc(H.n);
        FSA_CUDA(cudaMemcpyAsync(tmp.p, y, sizeof(double) * H.n, cudaMemcpyHostToDevice, H.stream));
        ydev = tmp.p;
      }
      k_gather_y<<<grid_for(H.n, 256), 256, 0, H.stream>>>(H.n, H.perm.p, ydev, H.y.p, H.err);
      FSA_CHECK_LAUNCH();
      check_err(H);
    }
    H.vec_pieces = o.vec_pieces == 3 ? 3 : 2;
    LoglikResult r = run_loglik_grad(H, *theta, o);
    FSA_CUDA(cudaEventRecord(H.ev1, H.stream));
    FSA_CUDA(cudaEventSynchronize(H.ev1));
    float ms = 0;
    cudaEventElapsedTime(&ms, H.ev0, H.ev1);
    *loglik = r.loglik;
    if (o.want_grad)
      for (int q = 0; q < 3; ++q) grad[q] = r.grad[q];
    if (info) {
      info->iters_max = r.iters_max;
      info->iters_y = r.iters_y;
      info->resid_y = r.resid_y;
      info->logdet = r.logdet;
      info->logdet_precond = r.logdetP;
      info->quad_form = r.yu;
      info->logdet_se = r.se;
      info->converged = r.converged ? 1 : 0;
      info->num_probes = o.num_probes;
      info->nnz = H.nnz;
      info->time_ms = ms;
      for (int q = 0; q < 3; ++q) {
        info->grad_trace[q] = o.want_grad ? r.trace[q] : 0.0;
        info->grad_quad[q] = o.want_grad ? r.quad[q] : 0.0;
        info->trace_precond[q] = o.want_grad ? r.traceP[q] : 0.0;
        info->cv_coef[q] = o.want_grad ? r.cv_c[q] : 0.0;
      }
      info->core_scale = H.op.core_scale;
      info->core_fp64 = H.op.core_fp64 ? 1 : 0;
      info->a_scale = H.op.a_scale;
      info->a_fp64 = H.op.a_fp64 ? 1 : 0;
    }
    if (!std::isfinite(r.loglik)) return fail(Error{FSA_ERR_NAN, "non-finite log-likelihood"});
    if (!r.converged) return fail(Error{FSA_ERR_NO_CONVERGENCE, "CG iteration limit reached"});
    return FSA_OK;
  } catch (const Error& e) {
    cudaGetLastError();
    cudaMemsetAsync(H.err, 0, sizeof(unsigned), H.stream);
    return fail(e);
  } catch (const std::exception& e) {
    cudaGetLastError();
    cudaMemsetAsync(H.err, 0, sizeof(unsigned), H.stream);
    return fail_host_exception("fsa_loglik_grad", e);
  }
}

fsa_status fsa_matvec(fsa_handle* h, const fsa_theta* theta, int32_t precision, int32_t which, const double* v,
                      int32_t k, double* out) {
  if (!h || !v || !out || k < 1 || which < 0 || which > 2) return fail(Error{FSA_ERR_ARG, "bad argument"});
  if (!theta_ok(theta)) return fail(Error{FSA_ERR_ARG, "theta must be finite and > 0"});
  if (precision < FSA_FP64 || precision > FSA_MIXED_BF16X2) return fail(Error{FSA_ERR_ARG, "bad precision"});
  Handle& H = h->h;
  AllocStreamScope scope(H.stream);
  TraceRange trace("fsa_matvec");
  H.vec_pieces = 2;
  try {
    ensure_operator(H, *theta, precision);
    size_t nk = (size_t)H.n * k;
    DevPtr<double> a(nk), b(nk), c(nk);
    FSA_CUDA(cudaMemcpyAsync(a.p, v, sizeof(double) * nk, cudaMemcpyHostToDevice, H.stream));
    to_internal(H, k, a.p, b.p);
    apply_operator(H, which, b.p, k, c.p);
    to_original(H, k, c.p, a.p);
    FSA_CUDA(cudaMemcpyAsync(out, a.p, sizeof(double) * nk, cudaMemcpyDeviceToHost, H.stream));
    FSA_CUDA(cudaStreamSynchronize(H.stream));
    check_err(H);
    return FSA_OK;
  } catch (const Error& e) {
    cudaGetLastError();
    return fail(e);
  } catch (const std::exception& e) {
    cudaGetLastError();
    return fail_host_exception("fsa_matvec", e);
  }
}

fsa_status fsa_logdet_precond(fsa_handle* h, const fsa_theta* theta, int32_t precision, double* out) {
  if (!h || !out) return fail(Error{FSA_ERR_ARG, "NULL argument"});
  if (!theta_ok(theta)) return fail(Error{FSA_ERR_ARG, "theta must be finite and > 0"});
  if (precision < FSA_FP64 || precision > FSA_MIXED_BF16X2) return fail(Error{FSA_ERR_ARG, "bad precision"});
  Handle& H = h->h;
  AllocStreamScope scope(H.stream);
  try {
    ensure_operator(H, *theta, precision);
    double sc[3];
    FSA_CUDA(cudaMemcpyAsync(sc, H.op.scal.p, sizeof(sc), cudaMemcpyDeviceToHost, H.stream));
    FSA_CUDA(cudaStreamSynchronize(H.stream));
    *out = sc[2];
    return FSA_OK;
  } catch (const Error& e) {
    cudaGetLastError();
    return fail(e);
  } catch (const std::exception& e) {
    cudaGetLastError();
    return fail_host_exception("fsa_logdet_precond", e);
  }
}

fsa_status fsa_predict(fsa_handle* h, const double* y, const fsa_theta* theta, const fsa_opts* opts,
                       const double* pred_locs, int64_t n_p, int32_t num_var_samples, double* mean, double* var,
                       fsa_info* info) {
  if (!h || !y || !pred_locs || !mean || n_p < 1) return fail(Error{FSA_ERR_ARG, "NULL argument or n_p < 1"});
  if (!theta_ok(theta)) return fail(Error{FSA_ERR_ARG, "theta must be finite and > 0"});
  if (var && (num_var_samples < 1 || num_var_samples > 4096))
    return fail(Error{FSA_ERR_ARG, "num_var_samples must be in [1, 4096]"});
  fsa_opts o = resolve_opts(opts);
  if (o.cg_max_iter > 8000) return fail(Error{FSA_ERR_ARG, "cg_max_iter must be <= 8000"});
  if (o.precision < FSA_FP64 || o.precision > FSA_MIXED_BF16X2) return fail(Error{FSA_ERR_ARG, "bad precision"});
  if (o.pred_control_variate < 0 || o.pred_control_variate > 2)
    return fail(Error{FSA_ERR_ARG, "pred_control_variate must be 0, 1 or 2"});
  if (o.pred_exact_var && (o.precision != FSA_FP64 || !var))
    return fail(Error{FSA_ERR_ARG, "pred_exact_var needs the FP64 form and a variance output"});
  Handle& H = h->h;
  AllocStreamScope scope(H.stream);
  TraceRange trace("fsa_predict");
  try {
    FSA_CUDA(cudaEventRecord(H.ev0, H.stream));
    H.y.ensure(H.n);
    {
      const double* ydev = y;
      DevPtr<double> tmp;
      if (!o.y_on_device) {
        tmp.alloc(H.n);
        FSA_CUDA(cudaMemcpyAsync(tmp.p, y, sizeof(double) * H.n, cudaMemcpyHostToDevice, H.stream));
        ydev = tmp.p;
      }
      k_gather_y<<<grid_for(H.n, 256), 256, 0, H.stream>>>(H.n, H.perm.p, ydev, H.y.p, H.err);
      FSA_CHECK_LAUNCH();
      check_err(H);
    }
    H.vec_pieces = o.vec_pieces == 3 ? 3 : 2;
    ensure_operator(H, *theta, o.precision);
    PredResult r = o.precision == FSA_FP64
                       ? run_predict_fp64(H, *theta, o, pred_locs, n_p, num_var_samples, mean, var)
                       : run_predict_mixed(H, *theta, o, pred_locs, n_p, num_var_samples, mean, var);
    FSA_CUDA(cudaEventRecord(H.ev1, H.stream));
    FSA_CUDA(cudaEventSynchronize(H.ev1));
    float ms = 0;
    cudaEventElapsedTime(&ms, H.ev0, H.ev1);
    if (info) {
      std::memset(info, 0, sizeof(*info));
      info->iters_y = r.iters_u;
      info->iters_max = std::max(r.iters_u, r.iters_sparse);
      info->converged = r.converged ? 1 : 0;
      info->num_probes = num_var_samples;
      info->nnz = H.nnz;
      info->time_ms = ms;
      info->core_scale = H.op.core_scale;
      info->core_fp64 = H.op.core_fp64 ? 1 : 0;
      info->a_scale = H.op.a_scale;
      info->a_fp64 = H.op.a_fp64 ? 1 : 0;
    }
    if (!r.converged) return fail(Error{FSA_ERR_NO_CONVERGENCE, "CG iteration limit reached"});
    return FSA_OK;
  } catch (const Error& e) {
    cudaGetLastError();
    cudaMemsetAsync(H.err, 0, sizeof(unsigned), H.stream);
    return fail(e);
  } catch (const std::exception& e) {
    cudaGetLastError();
    cudaMemsetAsync(H.err, 0, sizeof(unsigned), H.stream);
    return fail_host_exception("fsa_predict", e);
  }
}

void fsa_free(fsa_handle* h) {
  if (!h) return;
  fsa::free_handle(h, true);
}

int64_t fsa_footprint_bytes(int64_t n, int32_t m, int64_t nnz, int32_t num_probes, int32_t precision) {
  // peak of one fsa_build + fsa_loglik_grad: pattern and coordinates, m x m
  // matrices, the n x m operator with its build or gradient temporaries
  // (whichever is larger), and the n x ldc CG block; plus 25 % and a fixed
  // allowance for split-K partials and scratch.  The SpMM row groups' union
  // entries (32 bytes of sources, and in the mixed forms 32 bytes of values)
  // number at most nnz.
  const int64_t c = (int64_t)num_probes + 1, ldc = (c + 7) / 8 * 8, mp = ((int64_t)m + 63) / 64 * 64;
  int64_t b = 64 * n + 52 * nnz + 128 * (int64_t)m * m + ((int64_t)64 << 20);
  if (precision == FSA_FP64)
    b += 32 * n * (int64_t)m + 72 * n * ldc;
  else
    b += (precision == FSA_MIXED_BF16X2 ? 20 : 16) * n * mp + 40 * n * ldc + 32 * nnz;
  return b + b / 4;
}

}  // extern "C"
