// Predictive distribution of the FSA (paper §2.3) with simulation-based
// predictive variances (Algorithm 1, Proposition 1), FP64 form.
//
//   mean_p = Sigma^l_{p,n} Sigma_dag^-1 y + (S u)_p = ap_p . (A^T u) + (S u)_p,
//            u = Sigma_dag^-1 y,  ap_p = L_m^-1 k(s*, s^p_p),
//   S (n_p x n sparse, rows = prediction points) = Sigma^s_{n,np}^T with
//            S_pi = (s1 r(d_pi) - ap_p . a_i) T(d_pi)
//   D1_p = g_p^T (Sigma_mn W1) g_p,  g_p = Sigma_m^-1 k_p  (g_p^T = ap_p^T L_m^-1)
//   D2_p = sum_i S_pi (W1 g_p)_i
//   D3_p = v_p M^-1 v_p^T,          v_p = sum_i S_pi W2[i, :]
//   Dl_p = (1/s) sum_k z_pk (S Sigma_s~^-1 S^T z_k)_p
//   var_p = s1 + nugget - D1 - 2 D2 + D3 - Dl
// with W2 = Sigma_s~^-1 Sigma_mn^T (block CG on Sigma_s~, D_s preconditioner,
// solved together with Sigma_s~^-1 S^T Z), M = Sigma_m + Sigma_mn W2 and the
// exact Woodbury identity W1 = Sigma_dag^-1 Sigma_mn^T = W2 M^-1 Sigma_m
// (one sparse solve instead of a second, FITC-preconditioned, m-column solve).
#include <algorithm>

#include "fsa_kernels.cuh"
#include "fsa_solver.cuh"
#include "fsa_vec.cuh"

namespace fsa {

// ---------------------------------------------------------------------------
// generic FP64 block PCG (Appendix A without the tridiagonals' use):
// lowrank = 1: Sigma_dag with the FITC preconditioner; 0: Sigma_s~ with D_s.
// B (n x c, ld ldb) -> U (n x c, ld ldu); columns processed in chunks of <= 128.
// ---------------------------------------------------------------------------
struct PcgStats {
  int iters_max = 0;
  bool converged = true;
};

PcgStats pcg_fp64(Handle& H, const double* B, int64_t ldb, int c, double* U, int64_t ldu, double tol, int L,
                  bool lowrank) {
  cudaStream_t s = H.stream;
  Operator& op = H.op;
  const int64_t n = H.n;
  const int m = H.m;
  PcgStats st;
  for (int c0 = 0; c0 < c; c0 += 128) {
    const int cc = std::min(128, c - c0);
    CGLayout lay;
    lay.setup(n, cc, L);
    const int ldc = lay.ldc;
    const size_t nc = (size_t)n * ldc;
    DevPtr<double> Uc(nc), R(nc), Z(nc), Hh(nc), V(nc), S(nc), X(nc), w((size_t)m * ldc), q((size_t)m * ldc);
    DevPtr<double> rho(ldc), rz0(ldc), alpha(ldc), beta(ldc), ap(ldc), bp(ldc), rn(ldc), td((size_t)ldc * L),
        tof((size_t)ldc * L), part((size_t)lay.nblk * ldc);
    DevPtr<int32_t> active(ldc), iters(ldc), stop(ldc), nact(1);
    DevPtr<unsigned> ticket(1);
    FSA_CUDA(cudaMemsetAsync(ticket.p, 0, sizeof(unsigned), s));
    FSA_CUDA(cudaMemsetAsync(Uc.p, 0, nc * sizeof(double), s));
    FSA_CUDA(cudaMemsetAsync(V.p, 0, nc * sizeof(double), s));
    FSA_CUDA(cudaMemsetAsync(Hh.p, 0, nc * sizeof(double), s));
    FSA_CUDA(cudaMemsetAsync(S.p, 0, nc * sizeof(double), s));
    FSA_CUDA(cudaMemsetAsync(R.p, 0, nc * sizeof(double), s));
    FSA_CUDA(cudaMemcpy2DAsync(R.p, ldc * sizeof(double), B + c0, ldb * sizeof(double), cc * sizeof(double), n,
                               cudaMemcpyDeviceToDevice, s));
    CGScalars qs;
    qs.rho = rho.p; qs.rz0 = rz0.p; qs.alpha = alpha.p; qs.beta = beta.p; qs.alpha_prev = ap.p;
    qs.beta_prev = bp.p; qs.rnorm = rn.p; qs.tdiag = td.p; qs.toff = tof.p; qs.active = active.p;
    qs.iters = iters.p; qs.stop = stop.p; qs.num_active = nact.p; qs.err = H.err; qs.ticket = ticket.p;
    qs.tol = tol; qs.fixed = 0; qs.L = L;
    dim3 cgrid(lay.nblk), eblk(lay.ethreads);
    const size_t vsm = (size_t)lay.ethreads * sizeof(double);
    auto lowrank_apply = [&](const double* Xin, double* Sout) {
      dgemm(H.ws, s, true, false, m, cc, (int)n, 1.0, op.A.p, m, Xin, ldc, 0.0, w.p, ldc, nullptr);
      dgemm(H.ws, s, false, false, m, cc, m, 1.0, op.Minv.p, m, w.p, ldc, 0.0, q.p, ldc, nullptr);
      dgemm(H.ws, s, false, false, (int)n, cc, m, 1.0, op.A.p, m, q.p, ldc, 0.0, Sout, ldc, nullptr);
    };
    if (lowrank) {
      kv_row_scale<double><<<cgrid, eblk, 0, s>>>(n, cc, ldc, lay.rpb, R.p, op.Dinv.p, X.p);
      FSA_CHECK_LAUNCH();
      lowrank_apply(X.p, S.p);
    }
    kv_z_update<double><<<cgrid, eblk, vsm, s>>>(n, cc, ldc, lay.rpb, R.p, S.p, op.Dinv.p, Z.p, part.p, kStepInit,
                                                 0, qs);
    FSA_CHECK_LAUNCH();
    launch_spmm_fused<double, double>(lay, s, H.rowptr.p, H.col.p, op.vals.p, Z.p, S.p, V.p, Hh.p, beta.p, part.p,
                                      kStepAlpha, qs);
    int32_t* pin = reinterpret_cast<int32_t*>(H.host_pinned);
    int done = 0;
    for (int it = 0; it < L; ++it) {
      kv_ur_update<double><<<cgrid, eblk, vsm, s>>>(n, cc, ldc, lay.rpb, Uc.p, R.p, Hh.p, V.p, op.Dinv.p,
                                                    lowrank ? X.p : nullptr, alpha.p, active.p, part.p, kStepResid,
                                                    it, qs);
      FSA_CHECK_LAUNCH();
      if (lowrank) lowrank_apply(X.p, S.p);
      kv_z_update<double><<<cgrid, eblk, vsm, s>>>(n, cc, ldc, lay.rpb, R.p, S.p, op.Dinv.p, Z.p, part.p,
                                                   kStepBeta, it, qs);
      FSA_CHECK_LAUNCH();
      launch_spmm_fused<double, double>(lay, s, H.rowptr.p, H.col.p, op.vals.p, Z.p, S.p, V.p, Hh.p, beta.p,
                                        part.p, kStepAlpha, qs);
      FSA_CUDA(cudaMemcpyAsync(pin, nact.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      FSA_CUDA(cudaStreamSynchronize(s));
      done = it + 1;
      if (*pin == 0) break;
    }
    if (*pin != 0) st.converged = false;
    st.iters_max = std::max(st.iters_max, done);
    FSA_CUDA(cudaMemcpy2DAsync(U + c0, ldu * sizeof(double), Uc.p, ldc * sizeof(double), cc * sizeof(double), n,
                               cudaMemcpyDeviceToDevice, s));
    FSA_CUDA(cudaStreamSynchronize(s));
  }
  return st;
}

// ---------------------------------------------------------------------------
// prediction kernels
// ---------------------------------------------------------------------------
__global__ void k_split_xy(int64_t np, const double* __restrict__ pts, double* __restrict__ px,
                           double* __restrict__ py, unsigned* __restrict__ err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
    double x = pts[2 * i], y = pts[2 * i + 1];
    if (!isfinite(x) || !isfinite(y)) atomicOr(err, kErrNaN);
    px[i] = x;
    py[i] = y;
  }
}

// S_pi = (s1 r(d) - ap_p . a_i) T(d): warp per prediction row
__global__ void k_cross_values(int64_t np, int m, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                               const double* __restrict__ px, const double* __restrict__ py,
                               const double* __restrict__ xs, const double* __restrict__ ys,
                               const double* __restrict__ Ap, const double* __restrict__ A, int cov, double s1,
                               double rho, double gamma, double* __restrict__ vals) {
  int lane = threadIdx.x & 31;
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p = warp; p < np; p += nwarps) {
    const double* a = Ap + p * m;
    for (int64_t t = rowptr[p]; t < rowptr[p + 1]; ++t) {
      int i = col[t];
      const double* b = A + (int64_t)i * m;
      double sd = 0.0;
      for (int k = lane; k < m; k += 32) sd += a[k] * b[k];
      sd = warp_sum(sd);
      if (lane == 0) {
        double d = sqrt(sqdist_rn(px[p], py[p], xs[i], ys[i]));
        vals[t] = (s1 * matern_r(cov, d, rho) - sd) * wendland(d, gamma);
      }
    }
  }
}

// out[p] = sum_i S_pi (W1[i,:] . g_p)   (warp per prediction row)
__global__ void k_d2(int64_t np, int m, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                     const double* __restrict__ vals, const double* __restrict__ W1, const double* __restrict__ Gt,
                     double* __restrict__ out) {
  int lane = threadIdx.x & 31;
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p = warp; p < np; p += nwarps) {
    const double* g = Gt + p * m;
    double acc = 0.0;
    for (int64_t t = rowptr[p]; t < rowptr[p + 1]; ++t) {
      const double* w = W1 + (int64_t)col[t] * m;
      double sd = 0.0;
      for (int k = lane; k < m; k += 32) sd += w[k] * g[k];
      acc += vals[t] * warp_sum(sd);
    }
    if (lane == 0) out[p] = acc;
  }
}

// Y (np x k, ld ldy) = S X  (S: CSR by prediction rows; X rows = training points)
__global__ void k_cross_spmm(int64_t np, int k, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                             const double* __restrict__ vals, const double* __restrict__ X, int64_t ldx,
                             double* __restrict__ Y, int64_t ldy) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < np * k; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t p = t / k;
    int j = (int)(t % k);
    double s = 0.0;
    for (int64_t e = rowptr[p]; e < rowptr[p + 1]; ++e) s += vals[e] * X[(int64_t)col[e] * ldx + j];
    Y[p * ldy + j] = s;
  }
}

// transpose of the cross CSR: rows = training points (internal order), columns
// ascending prediction index (deterministic: counts, scan, fill, per-row sort)
__global__ void k_col_counts(int64_t nnz, const int32_t* __restrict__ col, int64_t* __restrict__ cnt) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nnz; t += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(reinterpret_cast<unsigned long long*>(&cnt[col[t]]), 1ull);
}

__global__ void k_transpose_fill(int64_t np, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                 const int64_t* __restrict__ trow, int64_t* __restrict__ cursor,
                                 int32_t* __restrict__ tcol, int64_t* __restrict__ tsrc) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x)
    for (int64_t e = rowptr[p]; e < rowptr[p + 1]; ++e) {
      int i = col[e];
      int64_t pos = trow[i] + (int64_t)atomicAdd(reinterpret_cast<unsigned long long*>(&cursor[i]), 1ull);
      tcol[pos] = (int32_t)p;
      tsrc[pos] = e;
    }
}

__global__ void k_transpose_sort(int64_t n, const int64_t* __restrict__ trow, int32_t* __restrict__ tcol,
                                 int64_t* __restrict__ tsrc) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = trow[i], e = trow[i + 1];
    for (int64_t k = b + 1; k < e; ++k) {
      int32_t c = tcol[k];
      int64_t sidx = tsrc[k];
      int64_t j = k - 1;
      while (j >= b && tcol[j] > c) { tcol[j + 1] = tcol[j]; tsrc[j + 1] = tsrc[j]; --j; }
      tcol[j + 1] = c;
      tsrc[j + 1] = sidx;
    }
  }
}

// RHS[i][m + k] = sum_p S_pi Z[p][k]  (rows of S^T Z, S^T in CSR by training points)
__global__ void k_st_z(int64_t n, int s, const int64_t* __restrict__ trow, const int32_t* __restrict__ tcol,
                       const int64_t* __restrict__ tsrc, const double* __restrict__ vals,
                       const double* __restrict__ Zp, double* __restrict__ out, int64_t ldo) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * s; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = t / s;
    int k = (int)(t % s);
    double acc = 0.0;
    for (int64_t e = trow[i]; e < trow[i + 1]; ++e) acc += vals[tsrc[e]] * Zp[(int64_t)tcol[e] * s + k];
    out[i * ldo + k] = acc;
  }
}

__global__ void k_pred_probes(int64_t np, int s, int kind, uint64_t key, double* __restrict__ Z) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < np * s; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t p = t / s;
    int k = (int)(t % s);
    Z[t] = probe_at(kind, key, (uint64_t)k * np + p);
  }
}

// out[p] = sum_k X[p][k] Y[p][k]   (row dots)
__global__ void k_rowdot(int64_t np, int k, const double* __restrict__ X, int64_t ldx, const double* __restrict__ Y,
                         int64_t ldy, double scale, double* __restrict__ out) {
  int lane = threadIdx.x & 31;
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p = warp; p < np; p += nwarps) {
    double s = 0.0;
    for (int j = lane; j < k; j += 32) s += X[p * ldx + j] * Y[p * ldy + j];
    s = warp_sum(s);
    if (lane == 0) out[p] = scale * s;
  }
}

__global__ void k_pred_assemble(int64_t np, double s1, double nug, const double* __restrict__ mean_lr,
                                const double* __restrict__ su, const double* __restrict__ D1,
                                const double* __restrict__ D2, const double* __restrict__ D3,
                                const double* __restrict__ Dl, double* __restrict__ mean, double* __restrict__ var) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
    mean[p] = mean_lr[p] + su[p];
    if (var) var[p] = s1 + nug - D1[p] - 2.0 * D2[p] + D3[p] - Dl[p];
  }
}

// dst (n x k) = D^-1 o src (n x k, leading dimension lds)
__global__ void k_scale_rows(int64_t n, int k, const double* __restrict__ Dv, const double* __restrict__ src,
                             int64_t lds, double* __restrict__ dst) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * k; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / k;
    const int j = (int)(t - i * k);
    dst[t] = src[i * lds + j] / Dv[i];
  }
}

// D_l with the diagonal preconditioner P_s = D_s as control variate
// (appendix "Preconditioner as control variate"), per prediction point p:
//   a_k = z_pk (S Sigma_s~^-1 S^T z_k)_p,  b_k = z_pk (S D_s^-1 S^T z_k)_p,
//   D_l = (1/s) sum_k (a_k - c b_k) + c sum_j S_pj^2 / D_j,
// c = sum_k (a_k - mean a) b_k / sum_k b_k^2 (mode 1; 0 where the
// denominator vanishes) or c = 1 (mode 2)
__global__ void k_dl_control_variate(int64_t np, int s, int mode, const double* __restrict__ Zp,
                                     const double* __restrict__ SY, const double* __restrict__ SU,
                                     const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                     const double* __restrict__ vals, const double* __restrict__ Dv,
                                     double* __restrict__ Dl) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
    const double* z = Zp + p * s;
    const double* ty = SY + p * s;
    const double* tu = SU + p * s;
    double sa = 0.0;
    for (int k = 0; k < s; ++k) sa += z[k] * ty[k];
    const double abar = sa / s;
    double c = 1.0;
    if (mode == 1) {
      double num = 0.0, den = 0.0;
      for (int k = 0; k < s; ++k) {
        const double b = z[k] * tu[k];
        num += (z[k] * ty[k] - abar) * b;
        den += b * b;
      }
      c = den > 0.0 ? num / den : 0.0;
    }
    double sd = 0.0;
    for (int k = 0; k < s; ++k) sd += z[k] * ty[k] - c * (z[k] * tu[k]);
    double eb = 0.0;
    for (int64_t e = rowptr[p]; e < rowptr[p + 1]; ++e) eb += vals[e] * vals[e] / Dv[col[e]];
    Dl[p] = sd / s + c * eb;
  }
}

// ---------------------------------------------------------------------------
// driver
// ---------------------------------------------------------------------------
PredResult run_predict_fp64(Handle& H, const fsa_theta& th, const fsa_opts& o, const double* pred_host, int64_t np,
                            int s, double* mean_host, double* var_host) {
  cudaStream_t st = H.stream;
  Operator& op = H.op;
  const int64_t n = H.n;
  const int m = H.m;
  const int L = o.cg_max_iter > 0 ? o.cg_max_iter : 1000;
  PredResult res;
  // prediction points (caller order; no reordering)
  DevPtr<double> pts(2 * np), px(np), py(np);
  FSA_CUDA(cudaMemcpyAsync(pts.p, pred_host, sizeof(double) * 2 * np, cudaMemcpyHostToDevice, st));
  k_split_xy<<<grid_for(np, 256), 256, 0, st>>>(np, pts.p, px.p, py.p, H.err);
  FSA_CHECK_LAUNCH();
  check_err(H);
  // cross pattern S (rows = prediction points)
  DevPtr<int64_t> srow;
  DevPtr<int32_t> scol;
  int64_t snnz = 0;
  build_cross_structure(H, px.p, py.p, np, srow, scol, snnz);
  // ap_p = L^-1 k_p (np x m), g_p^T = ap_p^T L^-1
  DevPtr<double> Ap((size_t)np * m), Gt((size_t)np * m);
  {
    DevPtr<double> Kp((size_t)np * m);
    cov_cross(H, np, px.p, py.p, m, H.ind_x.p, H.ind_y.p, th, 0, Kp.p, m);
    dgemm(H.ws, st, false, true, (int)np, m, m, 1.0, Kp.p, m, op.Lmi.p, m, 0.0, Ap.p, m, nullptr);
    dgemm(H.ws, st, false, false, (int)np, m, m, 1.0, Ap.p, m, op.Lmi.p, m, 0.0, Gt.p, m, nullptr);
    FSA_CUDA(cudaStreamSynchronize(st));
  }
  DevPtr<double> svals(snnz > 0 ? snnz : 1);
  if (snnz > 0) {
    k_cross_values<<<grid_for(np * 32, 256, 152 * 64), 256, 0, st>>>(np, m, srow.p, scol.p, px.p, py.p, H.xs.p,
                                                                       H.ys.p, Ap.p, op.A.p, H.cov, th.sigma1_sq,
                                                                       th.rho, H.gamma, svals.p);
    FSA_CHECK_LAUNCH();
  }
  // u = Sigma_dag^-1 y (FITC-PCG) and the mean
  DevPtr<double> u(n), Atu(m), mlr(np), su(np);
  {
    PcgStats ps = pcg_fp64(H, H.y.p, 1, 1, u.p, 1, o.cg_tol, L, true);
    res.iters_u = ps.iters_max;
    res.converged = ps.converged;
    dgemm(H.ws, st, true, false, m, 1, (int)n, 1.0, op.A.p, m, u.p, 1, 0.0, Atu.p, 1, nullptr);
    dgemm(H.ws, st, false, false, (int)np, 1, m, 1.0, Ap.p, m, Atu.p, 1, 0.0, mlr.p, 1, nullptr);
    k_cross_spmm<<<grid_for(np, 256), 256, 0, st>>>(np, 1, srow.p, scol.p, svals.p, u.p, 1, su.p, 1);
    FSA_CHECK_LAUNCH();
  }
  DevPtr<double> mean(np), var(np);
  if (var_host) {
    // sparse block solve: [Sigma_mn^T | S^T Z] (n x (m + s)) with Sigma_s~, D_s preconditioner
    const int cb = m + s;
    DevPtr<double> RHS((size_t)n * cb), X((size_t)n * cb), Zp((size_t)np * s);
    cov_cross(H, n, H.xs.p, H.ys.p, m, H.ind_x.p, H.ind_y.p, th, 0, RHS.p, cb);
    k_pred_probes<<<grid_for(np * s, 256), 256, 0, st>>>(np, s, o.probe, rng_key(o.seed, kStreamPred), Zp.p);
    FSA_CHECK_LAUNCH();
    {
      DevPtr<int64_t> cnt(n + 1), trow(n + 1), cursor(n), tsrc(snnz > 0 ? snnz : 1);
      DevPtr<int32_t> tcol(snnz > 0 ? snnz : 1);
      FSA_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int64_t) * (n + 1), st));
      FSA_CUDA(cudaMemsetAsync(cursor.p, 0, sizeof(int64_t) * n, st));
      if (snnz > 0) {
        k_col_counts<<<grid_for(snnz, 256), 256, 0, st>>>(snnz, scol.p, cnt.p);
        FSA_CHECK_LAUNCH();
      }
      exclusive_scan<int64_t>(cnt.p, trow.p, n + 1, st);
      if (snnz > 0) {
        k_transpose_fill<<<grid_for(np, 256), 256, 0, st>>>(np, srow.p, scol.p, trow.p, cursor.p, tcol.p, tsrc.p);
        FSA_CHECK_LAUNCH();
        k_transpose_sort<<<grid_for(n, 256), 256, 0, st>>>(n, trow.p, tcol.p, tsrc.p);
        FSA_CHECK_LAUNCH();
      }
      k_st_z<<<grid_for(n * s, 256), 256, 0, st>>>(n, s, trow.p, tcol.p, tsrc.p, svals.p, Zp.p, RHS.p + m, cb);
      FSA_CHECK_LAUNCH();
      FSA_CUDA(cudaStreamSynchronize(st));
    }
    PcgStats ps = pcg_fp64(H, RHS.p, cb, cb, X.p, cb, o.cg_tol, L, false);
    res.iters_sparse = ps.iters_max;
    res.converged = res.converged && ps.converged;
    const double* W2 = X.p;      // n x m, ld cb
    const double* Ys = X.p + m;  // n x s, ld cb
    // M = Sigma_m + Sigma_mn W2 ; Yms = M^-1 Sigma_m ; W1 = W2 Yms
    DevPtr<double> Mm((size_t)m * m), Minv((size_t)m * m), Sm((size_t)m * m), Yms((size_t)m * m);
    cov_cross(H, m, H.ind_x.p, H.ind_y.p, m, H.ind_x.p, H.ind_y.p, th, 0, Mm.p, m);
    FSA_CUDA(cudaMemcpyAsync(Sm.p, Mm.p, sizeof(double) * m * m, cudaMemcpyDeviceToDevice, st));
    dgemm(H.ws, st, true, false, m, m, (int)n, 1.0, RHS.p, cb, W2, cb, 1.0, Mm.p, m, nullptr);
    cholesky(Mm.p, m, m, H.err, st);
    {
      DevPtr<double> Li((size_t)m * m);
      lower_inverse(H.ws, Mm.p, m, Li.p, st);
      dgemm(H.ws, st, true, false, m, m, m, 1.0, Li.p, m, Li.p, m, 0.0, Minv.p, m, nullptr);
      FSA_CUDA(cudaStreamSynchronize(st));
    }
    check_err(H);
    dgemm(H.ws, st, false, false, m, m, m, 1.0, Minv.p, m, Sm.p, m, 0.0, Yms.p, m, nullptr);
    DevPtr<double> W1((size_t)n * m), C1((size_t)m * m), T((size_t)np * m), V((size_t)np * m);
    dgemm(H.ws, st, false, false, (int)n, m, m, 1.0, W2, cb, Yms.p, m, 0.0, W1.p, m, nullptr);
    // D1 = diag(G^T (Sigma_mn W1) G)
    dgemm(H.ws, st, true, false, m, m, (int)n, 1.0, RHS.p, cb, W1.p, m, 0.0, C1.p, m, nullptr);
    dgemm(H.ws, st, false, false, (int)np, m, m, 1.0, Gt.p, m, C1.p, m, 0.0, T.p, m, nullptr);
    DevPtr<double> D1(np), D2(np), D3(np), Dl(np);
    k_rowdot<<<grid_for(np * 32, 256, 152 * 64), 256, 0, st>>>(np, m, T.p, m, Gt.p, m, 1.0, D1.p);
    FSA_CHECK_LAUNCH();
    // D2 = sum_i S_pi (W1 g_p)_i
    k_d2<<<grid_for(np * 32, 256, 152 * 64), 256, 0, st>>>(np, m, srow.p, scol.p, svals.p, W1.p, Gt.p, D2.p);
    FSA_CHECK_LAUNCH();
    // D3 = diag(V M^-1 V^T), V = S W2
    k_cross_spmm<<<grid_for(np * m, 256), 256, 0, st>>>(np, m, srow.p, scol.p, svals.p, W2, cb, V.p, m);
    FSA_CHECK_LAUNCH();
    dgemm(H.ws, st, false, false, (int)np, m, m, 1.0, V.p, m, Minv.p, m, 0.0, T.p, m, nullptr);
    k_rowdot<<<grid_for(np * 32, 256, 152 * 64), 256, 0, st>>>(np, m, T.p, m, V.p, m, 1.0, D3.p);
    FSA_CHECK_LAUNCH();
    // Dl = (1/s) sum_k z_pk (S Ys)_pk, or its control-variate form
    {
      DevPtr<double> SY((size_t)np * s);
      k_cross_spmm<<<grid_for(np * s, 256), 256, 0, st>>>(np, s, srow.p, scol.p, svals.p, Ys, cb, SY.p, s);
      FSA_CHECK_LAUNCH();
      if (o.pred_control_variate == 0) {
        k_rowdot<<<grid_for(np * 32, 256, 152 * 64), 256, 0, st>>>(np, s, Zp.p, s, SY.p, s, 1.0 / s, Dl.p);
        FSA_CHECK_LAUNCH();
      } else {
        // S D_s^-1 S^T Z from the probe right-hand sides S^T Z (columns m.. of RHS)
        DevPtr<double> DZ((size_t)n * s), SU((size_t)np * s);
        k_scale_rows<<<grid_for(n * s, 256), 256, 0, st>>>(n, s, op.D.p, RHS.p + m, cb, DZ.p);
        FSA_CHECK_LAUNCH();
        k_cross_spmm<<<grid_for(np * s, 256), 256, 0, st>>>(np, s, srow.p, scol.p, svals.p, DZ.p, s, SU.p, s);
        FSA_CHECK_LAUNCH();
        k_dl_control_variate<<<grid_for(np, 128), 128, 0, st>>>(np, s, o.pred_control_variate, Zp.p, SY.p, SU.p,
                                                               srow.p, scol.p, svals.p, op.D.p, Dl.p);
        FSA_CHECK_LAUNCH();
      }
      k_pred_assemble<<<grid_for(np, 256), 256, 0, st>>>(np, th.sigma1_sq, th.nugget, mlr.p, su.p, D1.p, D2.p, D3.p,
                                                         Dl.p, mean.p, var.p);
      FSA_CHECK_LAUNCH();
      FSA_CUDA(cudaStreamSynchronize(st));
    }
  } else {
    k_pred_assemble<<<grid_for(np, 256), 256, 0, st>>>(np, th.sigma1_sq, th.nugget, mlr.p, su.p, nullptr, nullptr,
                                                       nullptr, nullptr, mean.p, nullptr);
    FSA_CHECK_LAUNCH();
  }
  FSA_CUDA(cudaMemcpyAsync(mean_host, mean.p, sizeof(double) * np, cudaMemcpyDeviceToHost, st));
  if (var_host) FSA_CUDA(cudaMemcpyAsync(var_host, var.p, sizeof(double) * np, cudaMemcpyDeviceToHost, st));
  FSA_CUDA(cudaStreamSynchronize(st));
  check_err(H);
  return res;
}

}  // namespace fsa
