// theta-dependent operator build, probes, block PCG with Lanczos tridiagonals,
// SLQ log-determinant and STE gradient of the FSA log-likelihood.
//
//   operator (§2.1, §3.1):  Sigma_dag = Sigma_s~ + A A^T,  A = Sigma_nm L_m^-T
//   FITC preconditioner (Eq. eqfitcp): P_hat = D_s + A A^T, D_s = diag(Sigma_s~)
//     P_hat^-1 r = D^-1 r - D^-1 A M^-1 A^T D^-1 r,  M = I + A^T D^-1 A
//     (the paper's core Sigma_m + Sigma_mn D^-1 Sigma_nm with L_m factored out)
//     log det P_hat = log det M + sum log D_i   (Sylvester)
//   probes z = A eps1 + D^1/2 eps2 ~ (0, P_hat)   (appendix "Runtime of the FITC
//     preconditioner", Gardner et al. reparameterisation)
//   PCG with T~ (Appendix A); log det = (n/l) sum e1^T log T~ e1 + log det P_hat
//   STE gradient (§3.3) with U = Sigma_dag^-1 Z, W = P_hat^-1 Z.
//
// Per CG iteration the m-space projections are arranged so that A is read
// twice:  w = A^T (D^-1 r) ;  q = M^-1 w ;  s = A q = A A^T z ;
// z = D^-1 (r - s) ;  Sigma_dag z = Sigma_s~ z + s ;  v_{l+1} = Sigma_dag z + beta v_l
// (v = Sigma_dag h follows from h = z + beta h by linearity).
#include "fsa_grad.cuh"
#include "fsa_kernels.cuh"
#include "fsa_solver.cuh"
#include "fsa_vec.cuh"

namespace fsa {

// ---------------------------------------------------------------------------
// covariance evaluation
// ---------------------------------------------------------------------------
// out[i*ld + k] = s1 * r(|p_i - q_k|)  (deriv: s1 * dr/drho)
__global__ void k_cov_cross(int64_t np, int nq, const double* __restrict__ px, const double* __restrict__ py,
                            const double* __restrict__ qx, const double* __restrict__ qy, int cov, double s1,
                            double rho, int deriv, double* __restrict__ out, int64_t ld) {
  int64_t total = np * nq;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = t / nq;
    int k = (int)(t - i * nq);
    double d = sqrt(sqdist_rn(px[i], py[i], qx[k], qy[k]));
    out[i * ld + k] = s1 * (deriv ? matern_dr(cov, d, rho) : matern_r(cov, d, rho));
  }
}

void cov_cross(Handle& H, int64_t np, const double* px, const double* py, int nq, const double* qx,
               const double* qy, const fsa_theta& th, int deriv, double* out, int64_t ld) {
  k_cov_cross<<<grid_for(np * nq, 256), 256, 0, H.stream>>>(np, nq, px, py, qx, qy, H.cov, th.sigma1_sq,
                                                              th.rho, deriv, out, ld);
  FSA_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// tapered residual values and D_s (§2.1, Eq. eqfitcp): warp per row
//   val_ij = (s1 r(d_ij) - a_i.a_j) T(d_ij),  val_ii = max(s1 - |a_i|^2, 0) + nugget
// ---------------------------------------------------------------------------
__global__ void k_csr_values_f64(int64_t n, int m, const int64_t* __restrict__ rowptr,
                                 const int32_t* __restrict__ col, const double* __restrict__ xs,
                                 const double* __restrict__ ys, const double* __restrict__ A, int64_t lda, int cov,
                                 double s1, double rho, double nug, double gamma, double* __restrict__ vals,
                                 double* __restrict__ D) {
  int lane = threadIdx.x & 31;
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nwarps) {
    const double* ai = A + i * lda;
    double xi = xs[i], yi = ys[i];
    for (int64_t t = rowptr[i]; t < rowptr[i + 1]; ++t) {
      int j = col[t];
      const double* aj = A + (int64_t)j * lda;
      double s = 0.0;
      for (int k = lane; k < m; k += 32) s += ai[k] * aj[k];
      s = warp_sum(s);
      if (lane == 0) {
        double v;
        if (j == i) {
          v = fmax(s1 - s, 0.0) + nug;
          D[i] = v;
        } else {
          double d = sqrt(sqdist_rn(xi, yi, xs[j], ys[j]));
          v = (s1 * matern_r(cov, d, rho) - s) * wendland(d, gamma);
        }
        vals[t] = v;
      }
    }
  }
}

template <typename T>
__global__ void k_reciprocal(int64_t n, const double* __restrict__ D, T* __restrict__ Dinv, unsigned* err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double d = D[i];
    if (!(d > 0.0) || !isfinite(d)) atomicOr(err, kErrNotPD);
    Dinv[i] = (T)(1.0 / d);
  }
}

__global__ void k_sum_log(int64_t n, const double* __restrict__ D, double* __restrict__ part) {
  __shared__ double sh[256];
  double v = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v += log(D[i]);
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// scal[1] = sum of parts; scal[2] = scal[0] + scal[1]
__global__ void k_logdetP_final(const double* __restrict__ part, int np, double* __restrict__ scal) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < np; ++b) s += part[b];
  scal[1] = s;
  scal[2] = scal[0] + s;
}

__global__ void k_set_identity_plus(double* __restrict__ M, int m) {
  int64_t total = (int64_t)m * m;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x)
    M[t] = ((t / m) == (t % m)) ? 1.0 : 0.0;
}

void sum_log_D(Handle& H, const double* D, double* scal) {
  const int nb = 256;
  double* part = H.ws.scratch_f64(nb);
  k_sum_log<<<nb, 256, 0, H.stream>>>(H.n, D, part);
  FSA_CHECK_LAUNCH();
  k_logdetP_final<<<1, 32, 0, H.stream>>>(part, nb, scal);
  FSA_CHECK_LAUNCH();
}

// m-space part shared by both precisions: Sigma_m, L_m, L_m^-1
void build_mspace(Handle& H, const fsa_theta& th) {
  Operator& op = H.op;
  int m = H.m;
  op.Sm.ensure((size_t)m * m);
  op.Lmi.ensure((size_t)m * m);
  cov_cross(H, m, H.ind_x.p, H.ind_y.p, m, H.ind_x.p, H.ind_y.p, th, 0, op.Sm.p, m);
  cholesky(op.Sm.p, m, m, H.err, H.stream);
  unsigned e = read_err(H);
  FSA_REQUIRE(!(e & kErrNotPD), FSA_ERR_NOT_PD, "Sigma_m is not positive definite (Cholesky pivot <= 0)");
  lower_inverse(H.ws, op.Sm.p, m, op.Lmi.p, H.stream);
}

// Woodbury core from A^T D^-1 A already in op.Mp (M = I + ...): factor, log det, inverse
void finish_core(Handle& H) {
  Operator& op = H.op;
  int m = H.m;
  op.scal.ensure(4);
  cholesky(op.Mp.p, m, m, H.err, H.stream);
  unsigned e = read_err(H);
  FSA_REQUIRE(!(e & kErrNotPD), FSA_ERR_NOT_PD, "Woodbury core I + A^T D^-1 A is not positive definite");
  logdet_from_cholesky(op.Mp.p, m, op.scal.p, H.stream);
  sum_log_D(H, op.D.p, op.scal.p);
  DevPtr<double> Lpi((size_t)m * m);
  lower_inverse(H.ws, op.Mp.p, m, Lpi.p, H.stream);
  op.Minv.ensure((size_t)m * m);
  dgemm(H.ws, H.stream, true, false, m, m, m, 1.0, Lpi.p, m, Lpi.p, m, 0.0, op.Minv.p, m, nullptr,
        kTriA_KgeI | kTriB_KgeJ | kTriSymLower);   // M^-1 = L^-T L^-1
  FSA_CUDA(cudaStreamSynchronize(H.stream));
}

void build_operator_fp64(Handle& H, const fsa_theta& th) {
  Operator& op = H.op;
  int64_t n = H.n;
  int m = H.m;
  build_mspace(H, th);
  // A = Sigma_nm L_m^-T  (n x m)
  {
    DevPtr<double> Knm((size_t)n * m);
    cov_cross(H, n, H.xs.p, H.ys.p, m, H.ind_x.p, H.ind_y.p, th, 0, Knm.p, m);
    op.A.ensure((size_t)n * m);
    dgemm(H.ws, H.stream, false, true, (int)n, m, m, 1.0, Knm.p, m, op.Lmi.p, m, 0.0, op.A.p, m, nullptr,
          kTriB_KleJ);
    FSA_CUDA(cudaStreamSynchronize(H.stream));
  }
  op.vals.ensure(H.nnz);
  op.D.ensure(n);
  op.Dinv.ensure(n);
  k_csr_values_f64<<<grid_for(n * 32, 256, 152 * 64), 256, 0, H.stream>>>(
      n, m, H.rowptr.p, H.col.p, H.xs.p, H.ys.p, op.A.p, m, H.cov, th.sigma1_sq, th.rho, th.nugget, H.gamma,
      op.vals.p, op.D.p);
  FSA_CHECK_LAUNCH();
  k_reciprocal<double><<<grid_for(n, 256), 256, 0, H.stream>>>(n, op.D.p, op.Dinv.p, H.err);
  FSA_CHECK_LAUNCH();
  // M = I + A^T D^-1 A
  op.Mp.ensure((size_t)m * m);
  k_set_identity_plus<<<grid_for((int64_t)m * m, 256), 256, 0, H.stream>>>(op.Mp.p, m);
  FSA_CHECK_LAUNCH();
  dgemm(H.ws, H.stream, true, false, m, m, (int)n, 1.0, op.A.p, m, op.A.p, m, 1.0, op.Mp.p, m, op.Dinv.p);
  finish_core(H);
  op.theta = th;
  op.precision = FSA_FP64;
  op.valid = true;
}

// ---------------------------------------------------------------------------
// probes (stream 5: eps1 on the m inducing points; stream 4: eps2 on the n
// data points, counter = column * rows + ORIGINAL row index)
// ---------------------------------------------------------------------------
__global__ void k_eps1(int m, int l, int kind, uint64_t key, double* __restrict__ E, int64_t lde) {
  int64_t total = (int64_t)m * l;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int k = (int)(t / l), p = (int)(t % l);
    E[(int64_t)k * lde + p] = probe_at(kind, key, (uint64_t)p * m + k);
  }
}

// B[:,0] = y (internal order), B[:,1+p] += sqrt(D_i) eps2
template <typename T>
__global__ void k_probe_finish(int64_t n, int l, int ldc, int kind, uint64_t key, const int64_t* __restrict__ perm,
                               const double* __restrict__ y_int, const double* __restrict__ D, T* __restrict__ B) {
  int64_t total = n * ldc;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = t / ldc;
    int c = (int)(t - i * ldc);
    if (c == 0) B[t] = (T)y_int[i];
    else if (c <= l) B[t] = (T)((double)B[t] + sqrt(D[i]) * probe_at(kind, key, (uint64_t)(c - 1) * n + perm[i]));
    else B[t] = (T)0;
  }
}

__global__ void k_gather_y(int64_t n, const int64_t* __restrict__ perm, const double* __restrict__ y,
                           double* __restrict__ y_int, unsigned* __restrict__ err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double v = y[perm[i]];
    if (!isfinite(v)) atomicOr(err, kErrNaN);
    y_int[i] = v;
  }
}

// ---------------------------------------------------------------------------
// final assembly of the log-likelihood and log det (the gradient's slots are
// written by grad_final)
// outs: [0] loglik [1] logdet [2] yu [6] logdet_se [7] logdetP
__global__ void k_assemble(int64_t n, int c, int exact_weight, const double* __restrict__ quads,
                           const double* __restrict__ rz0, const double* __restrict__ scal,
                           const double* __restrict__ part_yu, int nblk_yu, int ldc, double* __restrict__ outs) {
  if (threadIdx.x != 0) return;
  int l = c - 1;
  double mean = 0.0;
  for (int k = 1; k < c; ++k) mean += (exact_weight ? rz0[k] : (double)n) * quads[k];
  mean /= l;
  double var = 0.0;
  for (int k = 1; k < c; ++k) {
    double t = (exact_weight ? rz0[k] : (double)n) * quads[k] - mean;
    var += t * t;
  }
  double se = l > 1 ? sqrt(var / (l - 1) / l) : 0.0;
  double logdet = mean + scal[2];
  double yu = 0.0;
  for (int b = 0; b < nblk_yu; ++b) yu += part_yu[(int64_t)b * ldc];
  outs[0] = -0.5 * (n * 1.8378770664093453 + logdet + yu);
  outs[1] = logdet;
  outs[2] = yu;
  outs[6] = se;
  outs[7] = scal[2];
}

// ---------------------------------------------------------------------------
// CG block set-up
// ---------------------------------------------------------------------------
void CGLayout::setup(int64_t n_, int c_, int L_, int ldc_) {
  n = n_;
  c = c_;
  ldc = ldc_ > 0 ? ldc_ : (c + 7) / 8 * 8;
  L = L_;
  threads = (ldc + 31) / 32 * 32;
  int64_t nb = (n + 127) / 128;
  if (nb > 152 * 8) nb = 152 * 8;
  if (nb < 1) nb = 1;
  nblk = (int)nb;
  chunk = (n + nblk - 1) / nblk;
  rpb = 256 / ldc;
  if (rpb < 1) rpb = 1;
  ethreads = rpb * ldc;
}

void ensure_cg(Handle& H, const CGLayout& lay, bool fp64) {
  CGState& g = H.cg;
  size_t nc = (size_t)lay.n * lay.ldc;
  if (fp64) {
    g.U.ensure(nc); g.R.ensure(nc); g.Z.ensure(nc); g.H.ensure(nc); g.V.ensure(nc);
    g.S.ensure(nc); g.W0.ensure(nc); g.X.ensure(nc);
  }
  size_t mc = (size_t)H.m * lay.ldc;
  g.w.ensure(mc);
  g.q.ensure(mc);
  size_t cc = lay.ldc;
  g.rho.ensure(cc); g.alpha.ensure(cc); g.beta.ensure(cc); g.alpha_prev.ensure(cc); g.beta_prev.ensure(cc);
  g.rnorm.ensure(cc); g.rz0.ensure(cc); g.active.ensure(cc); g.iters.ensure(cc); g.stop.ensure(cc);
  g.tdiag.ensure((size_t)lay.ldc * lay.L);
  g.toff.ensure((size_t)lay.ldc * lay.L);
  g.part.ensure((size_t)lay.nblk * lay.ldc);
  g.quads.ensure(cc);
  g.qlwork.ensure((size_t)lay.ldc * 3 * lay.L);
  g.num_active.ensure(1);
  if (!g.ticket.p) {
    g.ticket.alloc(1);
    FSA_CUDA(cudaMemsetAsync(g.ticket.p, 0, sizeof(unsigned), H.stream));
  }
}

CGScalars make_scalars(Handle& H, const fsa_opts& o, int L) {
  CGState& g = H.cg;
  CGScalars q;
  q.rho = g.rho.p; q.rz0 = g.rz0.p; q.alpha = g.alpha.p; q.beta = g.beta.p;
  q.alpha_prev = g.alpha_prev.p; q.beta_prev = g.beta_prev.p; q.rnorm = g.rnorm.p;
  q.tdiag = g.tdiag.p; q.toff = g.toff.p;
  q.active = g.active.p; q.iters = g.iters.p; q.stop = g.stop.p; q.num_active = g.num_active.p;
  q.err = H.err;
  q.ticket = g.ticket.p;
  q.tol = o.cg_tol;
  q.fixed = o.fixed_iters > 0 ? 1 : 0;
  q.L = L;
  q.nrows = H.n;
  return q;
}

}  // namespace fsa

// ===========================================================================
// drivers
// ===========================================================================
namespace fsa {

unsigned read_err(Handle& H) {
  unsigned e = 0;
  FSA_CUDA(cudaMemcpyAsync(&e, H.err, sizeof(unsigned), cudaMemcpyDeviceToHost, H.stream));
  FSA_CUDA(cudaStreamSynchronize(H.stream));
  return e;
}

void check_err(Handle& H) {
  unsigned e = read_err(H);
  if (e) {
    FSA_CUDA(cudaMemsetAsync(H.err, 0, sizeof(unsigned), H.stream));
    if (e & kErrNotPD) throw Error{FSA_ERR_NOT_PD, "a Cholesky pivot or D_s entry was not positive"};
    if (e & kErrTimeout) throw Error{FSA_ERR_TIMEOUT, "a bounded device wait ran out"};
    if (e & kErrBounds) throw Error{FSA_ERR_BOUNDS, "a device index check of the checked build failed"};
    if (e & kErrNaN) throw Error{FSA_ERR_NAN, "non-finite value in the computation"};
    throw Error{FSA_ERR_CUDA, "device error flag " + std::to_string(e)};
  }
}

void ensure_operator(Handle& H, const fsa_theta& th, int precision) {
  Operator& op = H.op;
  if (op.valid && op.precision == precision && op.theta.sigma1_sq == th.sigma1_sq && op.theta.rho == th.rho &&
      op.theta.nugget == th.nugget)
    return;
  op.valid = false;
  TraceRange trace("operator_build");
  ProfScope phase("phase_build", 0.0, H.stream);
  if (precision == FSA_FP64) build_operator_fp64(H, th);
  else build_operator_mixed(H, th, precision);
  check_err(H);
}

// S = A M^-1 A^T X   (FP64 form; X, S are n x ldc)
static void lowrank_fp64(Handle& H, const CGLayout& lay, const double* X, double* S) {
  Operator& op = H.op;
  CGState& g = H.cg;
  int m = H.m;
  dgemm(H.ws, H.stream, true, false, m, lay.c, (int)lay.n, 1.0, op.A.p, m, X, lay.ldc, 0.0, g.w.p, lay.ldc, nullptr);
  dgemm(H.ws, H.stream, false, false, m, lay.c, m, 1.0, op.Minv.p, m, g.w.p, lay.ldc, 0.0, g.q.p, lay.ldc, nullptr);
  dgemm(H.ws, H.stream, false, false, (int)lay.n, lay.c, m, 1.0, op.A.p, m, g.q.p, lay.ldc, 0.0, S, lay.ldc,
        nullptr);
}

// Block PCG of Appendix A, FP64 form, on the right-hand sides in H.cg.R
// (n x ldc, columns >= c zero): U receives Sigma_dag^-1 R, W0 the first
// preconditioner apply P_hat^-1 R, the per-column scalars the Lanczos
// tridiagonals, iteration counts and residual norms.
void pcg_fp64_run(Handle& H, const CGLayout& lay, const fsa_opts& o, int L) {
  cudaStream_t s = H.stream;
  Operator& op = H.op;
  CGState& g = H.cg;
  const int64_t n = H.n;
  const int ldc = lay.ldc;
  const size_t nc = (size_t)n * ldc;
  dim3 cgrid(lay.nblk), eblk(lay.ethreads);
  const size_t vsm = (size_t)lay.ethreads * sizeof(double);
  FSA_CUDA(cudaMemsetAsync(g.U.p, 0, nc * sizeof(double), s));
  FSA_CUDA(cudaMemsetAsync(g.V.p, 0, nc * sizeof(double), s));
  FSA_CUDA(cudaMemsetAsync(g.H.p, 0, nc * sizeof(double), s));
  // z0 = P^-1 r0 (scalars: rho, rz0, alpha_0 = 1, beta_0 = 0 fused into the z update)
  CGScalars q = make_scalars(H, o, L);
  kv_row_scale<double><<<cgrid, eblk, 0, s>>>(n, lay.c, ldc, lay.rpb, g.R.p, op.Dinv.p, g.X.p);
  FSA_CHECK_LAUNCH();
  lowrank_fp64(H, lay, g.X.p, g.S.p);
  kv_z_update<double><<<cgrid, eblk, vsm, s>>>(n, lay.c, ldc, lay.rpb, g.R.p, g.S.p, op.Dinv.p, g.Z.p, g.part.p,
                                               kStepInit, 0, q);
  FSA_CHECK_LAUNCH();
  FSA_CUDA(cudaMemcpyAsync(g.W0.p, g.Z.p, nc * sizeof(double), cudaMemcpyDeviceToDevice, s));
  // h0 = z0, v0 = Sigma_dag h0, alpha_1 = rho / h^T v
  launch_spmm_fused<double, double>(lay, s, H.rowptr.p, H.col.p, op.vals.p, g.Z.p, g.S.p, g.V.p, g.H.p, g.beta.p,
                                    g.part.p, kStepAlpha, q);
  int32_t* pin_active = reinterpret_cast<int32_t*>(H.host_pinned);
  for (int it = 0; it < L; ++it) {
    // u += alpha h ; r -= alpha v ; ||r|| and the stop test
    kv_ur_update<double><<<cgrid, eblk, vsm, s>>>(n, lay.c, ldc, lay.rpb, g.U.p, g.R.p, g.H.p, g.V.p, op.Dinv.p,
                                                  g.X.p, g.alpha.p, g.active.p, g.part.p, kStepResid, it, q);
    FSA_CHECK_LAUNCH();
    lowrank_fp64(H, lay, g.X.p, g.S.p);
    // z = P^-1 r ; beta ; Lanczos T~ entries
    kv_z_update<double><<<cgrid, eblk, vsm, s>>>(n, lay.c, ldc, lay.rpb, g.R.p, g.S.p, op.Dinv.p, g.Z.p, g.part.p,
                                                 kStepBeta, it, q);
    FSA_CHECK_LAUNCH();
    // h = z + beta h ; v = Sigma_dag z + beta v ; next alpha
    launch_spmm_fused<double, double>(lay, s, H.rowptr.p, H.col.p, op.vals.p, g.Z.p, g.S.p, g.V.p, g.H.p,
                                      g.beta.p, g.part.p, kStepAlpha, q);
    if (o.fixed_iters <= 0 && should_poll(it)) {
      FSA_CUDA(cudaMemcpyAsync(pin_active, g.num_active.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      FSA_CUDA(cudaStreamSynchronize(s));
      if (*pin_active == 0) break;
    }
  }
}

LoglikResult run_loglik_grad_fp64(Handle& H, const fsa_theta& th, const fsa_opts& o) {
  cudaStream_t s = H.stream;
  Operator& op = H.op;
  CGState& g = H.cg;
  int64_t n = H.n;
  int m = H.m;
  int l = o.num_probes;
  CGLayout lay;
  int L = o.fixed_iters > 0 ? o.fixed_iters : (o.cg_max_iter > 0 ? o.cg_max_iter : 1000);
  lay.setup(n, l + 1, L);
  ensure_cg(H, lay, true);
  int ldc = lay.ldc;
  size_t nc = (size_t)n * ldc;
  // probes: R = [y, A eps1 + D^1/2 eps2]
  {
    DevPtr<double> E1((size_t)m * l);
    k_eps1<<<grid_for((int64_t)m * l, 256), 256, 0, s>>>(m, l, o.probe, rng_key(o.seed, kStreamEps1), E1.p, l);
    FSA_CHECK_LAUNCH();
    dgemm(H.ws, s, false, false, (int)n, l, m, 1.0, op.A.p, m, E1.p, l, 0.0, g.R.p + 1, ldc, nullptr);
    FSA_CUDA(cudaStreamSynchronize(s));
    k_probe_finish<double><<<grid_for((int64_t)nc, 256), 256, 0, s>>>(n, l, ldc, o.probe,
                                                                       rng_key(o.seed, kStreamEps2), H.perm.p,
                                                                       H.y.p, op.D.p, g.R.p);
    FSA_CHECK_LAUNCH();
  }
  pcg_fp64_run(H, lay, o, L);
  // SLQ
  launch_slq(lay.c, L, g.iters.p, g.tdiag.p, g.toff.p, g.quads.p, H.err, s);
  // y^T u
  k_dot_col0<double><<<lay.nblk, 32, 0, s>>>(n, ldc, lay.chunk, H.y.p, g.U.p, g.part.p);
  FSA_CHECK_LAUNCH();
  H.outs.ensure(kOutCount);
  if (o.want_grad) {
    // X = U (u in column 0), Y = W with u in column 0 (stored in Z)
    FSA_CUDA(cudaMemcpyAsync(g.Z.p, g.W0.p, nc * sizeof(double), cudaMemcpyDeviceToDevice, s));
    k_copy_col0<double><<<grid_for(n, 256), 256, 0, s>>>(n, ldc, g.U.p, g.Z.p);
    FSA_CHECK_LAUNCH();
    int c = lay.c;
    size_t mc = (size_t)m * ldc;
    DevPtr<double> AX(mc), AY(mc), BX(mc), BY(mc), EAY(mc);
    dgemm(H.ws, s, true, false, m, c, (int)n, 1.0, op.A.p, m, g.U.p, ldc, 0.0, AX.p, ldc, nullptr);
    dgemm(H.ws, s, true, false, m, c, (int)n, 1.0, op.A.p, m, g.Z.p, ldc, 0.0, AY.p, ldc, nullptr);
    DerivF64 Dv;
    build_deriv_f64(H, th, Dv);
    dgemm(H.ws, s, true, false, m, c, (int)n, 1.0, Dv.B.p, m, g.U.p, ldc, 0.0, BX.p, ldc, nullptr);
    dgemm(H.ws, s, true, false, m, c, (int)n, 1.0, Dv.B.p, m, g.Z.p, ldc, 0.0, BY.p, ldc, nullptr);
    dgemm(H.ws, s, false, false, m, c, m, 1.0, Dv.E.p, m, AY.p, ldc, 0.0, EAY.p, ldc, nullptr);
    // sparse terms per column (range derivative of the residual values, one gather)
    const int nb = coldots_blocks();
    DevPtr<double> part((size_t)nb * kColTerms * ldc), lr((size_t)3 * ldc);
    grad_coldots<double, double, double>(H, c, ldc, op.vals.p, Dv.dv.p, g.U.p, g.Z.p, part.p, nb);
    grad_lowrank_cols(H, m, c, ldc, AX.p, AY.p, BX.p, BY.p, EAY.p, lr.p);
    DevPtr<double> cv, mtr;
    int ncv = 0;
    if (o.grad_control_variate != kCvNone) {
      ncv = cv_blocks();
      cv.alloc((size_t)ncv * kCvTerms);
      mtr.alloc(2);
      DevPtr<double> AM((size_t)n * m);
      dgemm(H.ws, s, false, false, (int)n, m, m, 1.0, op.A.p, m, op.Minv.p, m, 0.0, AM.p, m, nullptr);
      cv_rowdots_f64(H, m, AM.p, op.A.p, Dv.B.p, op.D.p, Dv.dD.p, cv.p, ncv);
      mspace_traces(H, m, Dv.E.p, op.Minv.p, mtr.p);
    }
    k_assemble<<<1, 32, 0, s>>>(n, lay.c, o.slq_exact_weight, g.quads.p, g.rz0.p, op.scal.p, g.part.p, lay.nblk,
                                ldc, H.outs.p);
    FSA_CHECK_LAUNCH();
    H.gterms.ensure((size_t)6 * l);
    H.gterms_l = l;
    grad_final(H, c, ldc, part.p, nb, lr.p, cv.p, ncv, mtr.p, th, o.grad_control_variate, H.gterms.p);
    FSA_CUDA(cudaStreamSynchronize(s));
  } else {
    k_assemble<<<1, 32, 0, s>>>(n, lay.c, o.slq_exact_weight, g.quads.p, g.rz0.p, op.scal.p, g.part.p, lay.nblk,
                                ldc, H.outs.p);
    FSA_CHECK_LAUNCH();
  }
  LoglikResult res;
  double outs[kOutCount];
  FSA_CUDA(cudaMemcpyAsync(outs, H.outs.p, sizeof(outs), cudaMemcpyDeviceToHost, s));
  std::vector<int32_t> iters(lay.c);
  std::vector<double> rn(lay.c);
  FSA_CUDA(cudaMemcpyAsync(iters.data(), g.iters.p, sizeof(int32_t) * lay.c, cudaMemcpyDeviceToHost, s));
  FSA_CUDA(cudaMemcpyAsync(rn.data(), g.rnorm.p, sizeof(double) * lay.c, cudaMemcpyDeviceToHost, s));
  int32_t nact = 0;
  FSA_CUDA(cudaMemcpyAsync(&nact, g.num_active.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  FSA_CUDA(cudaStreamSynchronize(s));
  check_err(H);
  res.loglik = outs[0];
  res.logdet = outs[1];
  res.yu = outs[2];
  for (int q = 0; q < 3; ++q) {
    res.grad[q] = outs[kOutGrad + q];
    res.trace[q] = outs[kOutTrace + q];
    res.quad[q] = outs[kOutQuad + q];
    res.traceP[q] = outs[kOutTraceP + q];
    res.cv_c[q] = outs[kOutCvC + q];
  }
  res.se = outs[6];
  res.logdetP = outs[7];
  res.iters_y = iters[0];
  res.resid_y = rn[0];
  for (int k = 0; k < lay.c; ++k) res.iters_max = std::max(res.iters_max, (int)iters[k]);
  res.converged = o.fixed_iters > 0 || nact == 0;
  return res;
}

LoglikResult run_loglik_grad_mixed(Handle& H, const fsa_theta& th, const fsa_opts& o);

LoglikResult run_loglik_grad(Handle& H, const fsa_theta& th, const fsa_opts& o) {
  ensure_operator(H, th, o.precision);
  if (o.precision == FSA_FP64) {
    TraceRange trace("loglik_grad_fp64");
    return run_loglik_grad_fp64(H, th, o);
  }
  return run_loglik_grad_mixed(H, th, o);
}

// out = Sigma_dag v (0), P_hat^-1 v (1), Sigma_s~ v (2), FP64 operator
void apply_operator_mixed(Handle& H, int which, const double* v, int k, double* out);

void apply_operator(Handle& H, int which, const double* v, int k, double* out) {
  if (H.op.precision != FSA_FP64) return apply_operator_mixed(H, which, v, k, out);
  Operator& op = H.op;
  cudaStream_t s = H.stream;
  int64_t n = H.n;
  int m = H.m;
  CGLayout lay;
  lay.setup(n, k, 1);
  if (which == 2 || which == 0) {
    k_spmm<double, double><<<dim3(lay.nblk, 1), 128, 0, s>>>(n, k, k, lay.chunk, H.rowptr.p, H.col.p, op.vals.p, v,
                                                              out, k);
    FSA_CHECK_LAUNCH();
    if (which == 2) return;
    DevPtr<double> w((size_t)m * k);
    dgemm(H.ws, s, true, false, m, k, (int)n, 1.0, op.A.p, m, v, k, 0.0, w.p, k, nullptr);
    dgemm(H.ws, s, false, false, (int)n, k, m, 1.0, op.A.p, m, w.p, k, 1.0, out, k, nullptr);
    FSA_CUDA(cudaStreamSynchronize(s));
    return;
  }
  // P^-1 v = D^-1 (v - A M^-1 A^T D^-1 v)
  DevPtr<double> X((size_t)n * k), w((size_t)m * k), q((size_t)m * k), S((size_t)n * k);
  lay.setup(n, k, 1);
  lay.ldc = k;
  lay.threads = (k + 31) / 32 * 32;
  k_row_scale<double><<<lay.nblk, lay.threads, 0, s>>>(n, k, k, lay.chunk, v, op.Dinv.p, X.p);
  FSA_CHECK_LAUNCH();
  dgemm(H.ws, s, true, false, m, k, (int)n, 1.0, op.A.p, m, X.p, k, 0.0, w.p, k, nullptr);
  dgemm(H.ws, s, false, false, m, k, m, 1.0, op.Minv.p, m, w.p, k, 0.0, q.p, k, nullptr);
  dgemm(H.ws, s, false, false, (int)n, k, m, 1.0, op.A.p, m, q.p, k, 0.0, S.p, k, nullptr);
  DevPtr<double> part((size_t)lay.nblk * k);
  k_z_update<double><<<lay.nblk, lay.threads, 0, s>>>(n, k, k, lay.chunk, v, S.p, op.Dinv.p, out, part.p);
  FSA_CHECK_LAUNCH();
  FSA_CUDA(cudaStreamSynchronize(s));
}

}  // namespace fsa
