// Fisher information of theta = (sigma1^2, rho, nugget) by stochastic trace
// estimation (appendix "Fisher scoring"):
//     I_kj = 1/2 Tr(Sigma_dag^-1 dSigma_k Sigma_dag^-1 dSigma_j)
//          ~ 1/2 (1/l) sum_i (dSigma_k Sigma_dag^-1 z_i)^T (Sigma_dag^-1 dSigma_j z_i),
// z_i with E[z z^T] = I (Rademacher or Gaussian; SplitMix64 stream 7).
// The solves Sigma_dag^-1 z_i and Sigma_dag^-1 dSigma_j z_i (j = sigma1^2,
// rho; dSigma_nugget = I needs none) run as one block of 3 l right-hand sides
// of the FITC-preconditioned CG of Appendix A.  With V = Sigma_dag^-1 Z and
// X_j = Sigma_dag^-1 dSigma_j Z (X_nugget = V) the estimate is
//     I_kj = 1/2 (1/l) sum_i (dSigma_k V_i)^T X_j,i,
// not symmetric for finite l; fsa_fisher returns its symmetric part and, on
// request, the estimate as it stands.
#include <algorithm>
#include <cstring>
#include <vector>

#include "fsa_grad.cuh"
#include "fsa_kernels.cuh"
#include "fsa_mixed.cuh"
#include "fsa_vec.cuh"

namespace fsa {

constexpr uint64_t kStreamFisher = 7;

// X (n x ldc): probe z_i in column i < l (counter i n + original index), zero elsewhere
template <typename T>
__global__ void k_fisher_probes(int64_t n, int l, int ldc, int kind, uint64_t key, const int64_t* __restrict__ perm,
                                T* __restrict__ X) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * ldc; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / ldc;
    const int c = (int)(t - i * ldc);
    X[t] = c < l ? (T)probe_at(kind, key, (uint64_t)c * n + perm[i]) : (T)0;
  }
}

// R = [Z, dSigma_0 Z, dSigma_1 Z] from the first l columns of Z, D0, D1
template <typename T>
__global__ void k_fisher_rhs(int64_t n, int l, int ldc, const T* __restrict__ Z, const T* __restrict__ D0,
                             const T* __restrict__ D1, T* __restrict__ R) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * ldc; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / ldc;
    const int c = (int)(t - i * ldc);
    const int64_t r = i * ldc;
    R[t] = c < l ? Z[r + c] : c < 2 * l ? D0[r + c - l] : c < 3 * l ? D1[r + c - 2 * l] : (T)0;
  }
}

// V = the first l columns of U (the solves Sigma_dag^-1 z_i), zero elsewhere
template <typename T>
__global__ void k_fisher_take(int64_t n, int l, int ldc, const T* __restrict__ U, T* __restrict__ V) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * ldc; t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t % ldc);
    V[t] = c < l ? U[t] : (T)0;
  }
}

// per block and probe i: s[k][j] = sum over the block's rows of (dSigma_k V_i) . X_j,i
// (dSigma_2 V = V, X_0 = U[:, l + i], X_1 = U[:, 2 l + i], X_2 = V), FP64 sums
template <typename T>
__global__ void k_fisher_dots(int64_t n, int l, int ldc, int64_t chunk, const T* __restrict__ D0,
                              const T* __restrict__ D1, const T* __restrict__ V, const T* __restrict__ U,
                              double* __restrict__ part) {
  const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = r0 + chunk < n ? r0 + chunk : n;
  for (int i = threadIdx.x; i < l; i += blockDim.x) {
    double s[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t r = r0; r < r1; ++r) {
      const int64_t o = r * ldc;
      const double d[3] = {(double)D0[o + i], (double)D1[o + i], (double)V[o + i]};
      const double x[3] = {(double)U[o + l + i], (double)U[o + 2 * l + i], (double)V[o + i]};
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) s[3 * k + j] = fma(d[k], x[j], s[3 * k + j]);
    }
    for (int q = 0; q < 9; ++q) part[((int64_t)blockIdx.x * 9 + q) * l + i] = s[q];
  }
}

// raw[k][j] = 1/2 (1/l) sum_i sum_blocks part (fixed order)
__global__ void k_fisher_final(int nblk, int l, const double* __restrict__ part, double* __restrict__ raw) {
  const int q = threadIdx.x;
  if (q >= 9) return;
  double s = 0.0;
  for (int i = 0; i < l; ++i) {
    double t = 0.0;
    for (int b = 0; b < nblk; ++b) t += part[((int64_t)b * 9 + q) * l + i];
    s += t;
  }
  raw[q] = 0.5 * s / l;
}

struct FisherRun {
  int iters_max = 0;
  bool converged = true;
};

template <typename T>
static void fisher_dots(Handle& H, int l, int ldc, const T* D0, const T* D1, const T* V, const T* U, double* raw) {
  const int nblk = 152 * 4;
  const int64_t chunk = (H.n + nblk - 1) / nblk;
  DevPtr<double> part((size_t)nblk * 9 * l);
  k_fisher_dots<T><<<nblk, 64, 0, H.stream>>>(H.n, l, ldc, chunk, D0, D1, V, U, part.p);
  FSA_CHECK_LAUNCH();
  k_fisher_final<<<1, 32, 0, H.stream>>>(nblk, l, part.p, raw);
  FSA_CHECK_LAUNCH();
  FSA_CUDA(cudaStreamSynchronize(H.stream));
}

static FisherRun fisher_status(Handle& H, int c) {
  CGState& g = H.cg;
  FisherRun r;
  std::vector<int32_t> iters(c);
  int32_t nact = 0;
  FSA_CUDA(cudaMemcpyAsync(iters.data(), g.iters.p, sizeof(int32_t) * c, cudaMemcpyDeviceToHost, H.stream));
  FSA_CUDA(cudaMemcpyAsync(&nact, g.num_active.p, sizeof(int32_t), cudaMemcpyDeviceToHost, H.stream));
  FSA_CUDA(cudaStreamSynchronize(H.stream));
  check_err(H);
  for (int k = 0; k < c; ++k) r.iters_max = std::max(r.iters_max, (int)iters[k]);
  r.converged = nact == 0;
  return r;
}

static FisherRun run_fisher_mixed(Handle& H, const fsa_theta& th, const fsa_opts& o, double* raw_dev) {
  cudaStream_t s = H.stream;
  CGState& g = H.cg;
  const int64_t n = H.n;
  const int l = o.num_probes, c = 3 * l;
  FSA_REQUIRE(c <= 127, FSA_ERR_UNSUPPORTED, "mixed-precision Fisher information supports at most 42 probes");
  const int L = o.fixed_iters > 0 ? o.fixed_iters : (o.cg_max_iter > 0 ? o.cg_max_iter : 1000);
  CGLayout lay;
  lay.setup(n, c, L, mixed_ldc(c, H.vec_pieces));
  ensure_cg(H, lay, false);
  const int ldc = lay.ldc;
  const size_t nc = (size_t)n * ldc;
  g.U32.ensure(nc); g.R32.ensure(nc); g.Z32.ensure(nc); g.H32.ensure(nc); g.V32.ensure(nc);
  g.S32.ensure(nc); g.W032.ensure(nc);
  MixedCtx C;
  mixed_ctx_setup(H, C, n, c, ldc);
  DevPtr<float> wpart((size_t)C.splits_w * C.m_pad * ldc);
  C.wpart = wpart.p;
  DerivMixed Dv;
  build_deriv_mixed(H, C, th, Dv);
  DevPtr<float> X(nc), D0(nc), D1(nc);
  k_fisher_probes<float><<<grid_for((int64_t)nc, 256), 256, 0, s>>>(n, l, ldc, o.probe, rng_key(o.seed, kStreamFisher),
                                                                    H.perm.p, X.p);
  FSA_CHECK_LAUNCH();
  apply_dsigma_mixed(H, C, Dv, th, X.p, D0.p, D1.p);
  k_fisher_rhs<float><<<grid_for((int64_t)nc, 256), 256, 0, s>>>(n, l, ldc, X.p, D0.p, D1.p, g.R32.p);
  FSA_CHECK_LAUNCH();
  pcg_mixed_run(H, C, lay, o, L);
  k_fisher_take<float><<<grid_for((int64_t)nc, 256), 256, 0, s>>>(n, l, ldc, g.U32.p, X.p);
  FSA_CHECK_LAUNCH();
  apply_dsigma_mixed(H, C, Dv, th, X.p, D0.p, D1.p);
  fisher_dots<float>(H, l, ldc, D0.p, D1.p, X.p, g.U32.p, raw_dev);
  FisherRun r = fisher_status(H, c);
  r.converged = r.converged || o.fixed_iters > 0;
  return r;
}

static FisherRun run_fisher_fp64(Handle& H, const fsa_theta& th, const fsa_opts& o, double* raw_dev) {
  cudaStream_t s = H.stream;
  CGState& g = H.cg;
  const int64_t n = H.n;
  const int l = o.num_probes, c = 3 * l;
  const int L = o.fixed_iters > 0 ? o.fixed_iters : (o.cg_max_iter > 0 ? o.cg_max_iter : 1000);
  CGLayout lay;
  lay.setup(n, c, L);
  ensure_cg(H, lay, true);
  const int ldc = lay.ldc;
  const size_t nc = (size_t)n * ldc;
  DerivF64 Dv;
  build_deriv_f64(H, th, Dv);
  DevPtr<double> X(nc), D0(nc), D1(nc);
  k_fisher_probes<double><<<grid_for((int64_t)nc, 256), 256, 0, s>>>(n, l, ldc, o.probe,
                                                                     rng_key(o.seed, kStreamFisher), H.perm.p, X.p);
  FSA_CHECK_LAUNCH();
  apply_dsigma_f64(H, Dv, th, X.p, l, ldc, D0.p, D1.p);
  k_fisher_rhs<double><<<grid_for((int64_t)nc, 256), 256, 0, s>>>(n, l, ldc, X.p, D0.p, D1.p, g.R.p);
  FSA_CHECK_LAUNCH();
  pcg_fp64_run(H, lay, o, L);
  k_fisher_take<double><<<grid_for((int64_t)nc, 256), 256, 0, s>>>(n, l, ldc, g.U.p, X.p);
  FSA_CHECK_LAUNCH();
  apply_dsigma_f64(H, Dv, th, X.p, l, ldc, D0.p, D1.p);
  fisher_dots<double>(H, l, ldc, D0.p, D1.p, X.p, g.U.p, raw_dev);
  FisherRun r = fisher_status(H, c);
  r.converged = r.converged || o.fixed_iters > 0;
  return r;
}

}  // namespace fsa

using namespace fsa;

extern "C" fsa_status fsa_fisher(fsa_handle* h, const fsa_theta* theta, const fsa_opts* opts, double* fisher,
                                 double* fisher_raw, fsa_info* info) {
  if (!h || !theta || !fisher) {
    set_error("fsa_fisher: NULL argument");
    return FSA_ERR_ARG;
  }
  if (!(theta->sigma1_sq > 0 && theta->rho > 0 && theta->nugget > 0) || !std::isfinite(theta->sigma1_sq) ||
      !std::isfinite(theta->rho) || !std::isfinite(theta->nugget)) {
    set_error("fsa_fisher: theta must be finite and > 0");
    return FSA_ERR_ARG;
  }
  fsa_opts o;
  if (opts) o = *opts;
  else fsa_default_opts(&o);
  if (o.num_probes < 1 || o.num_probes > 300) {
    set_error("fsa_fisher: num_probes must be in [1, 300]");
    return FSA_ERR_ARG;
  }
  if (o.precision < FSA_FP64 || o.precision > FSA_MIXED_BF16X2 || o.cg_max_iter > 8000 || o.fixed_iters > 8000 ||
      o.fixed_iters < 0 || !(o.cg_tol >= 0.0) || (o.probe != FSA_PROBE_RADEMACHER && o.probe != FSA_PROBE_GAUSSIAN)) {
    set_error("fsa_fisher: bad option (precision, probe, cg_tol or iteration limits)");
    return FSA_ERR_ARG;
  }
  Handle& H = h->h;
  AllocStreamScope scope(H.stream);
  TraceRange trace("fsa_fisher");
  try {
    FSA_CUDA(cudaEventRecord(H.ev0, H.stream));
    H.vec_pieces = o.vec_pieces == 3 ? 3 : 2;
    ensure_operator(H, *theta, o.precision);
    DevPtr<double> raw(9);
    FisherRun r = o.precision == FSA_FP64 ? run_fisher_fp64(H, *theta, o, raw.p) : run_fisher_mixed(H, *theta, o, raw.p);
    double F[9];
    FSA_CUDA(cudaMemcpyAsync(F, raw.p, sizeof(F), cudaMemcpyDeviceToHost, H.stream));
    FSA_CUDA(cudaEventRecord(H.ev1, H.stream));
    FSA_CUDA(cudaEventSynchronize(H.ev1));
    float ms = 0;
    cudaEventElapsedTime(&ms, H.ev0, H.ev1);
    for (int k = 0; k < 3; ++k)
      for (int j = 0; j < 3; ++j) fisher[3 * k + j] = 0.5 * (F[3 * k + j] + F[3 * j + k]);
    if (fisher_raw)
      for (int q = 0; q < 9; ++q) fisher_raw[q] = F[q];
    if (info) {
      std::memset(info, 0, sizeof(*info));
      info->iters_max = r.iters_max;
      info->converged = r.converged ? 1 : 0;
      info->num_probes = o.num_probes;
      info->nnz = H.nnz;
      info->time_ms = ms;
    }
    for (int q = 0; q < 9; ++q)
      if (!std::isfinite(F[q])) {
        set_error("fsa_fisher: non-finite estimate");
        return FSA_ERR_NAN;
      }
    if (!r.converged) {
      set_error("fsa_fisher: CG iteration limit reached");
      return FSA_ERR_NO_CONVERGENCE;
    }
    return FSA_OK;
  } catch (const Error& e) {
    cudaGetLastError();
    cudaMemsetAsync(H.err, 0, sizeof(unsigned), H.stream);
    set_error(e.msg);
    return e.code;
  } catch (const std::exception& e) {
    cudaGetLastError();
    set_error(std::string("fsa_fisher: host exception: ") + e.what());
    return FSA_ERR_CUDA;
  }
}
