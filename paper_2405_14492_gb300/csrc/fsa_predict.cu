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
#include "fsa_mixed.cuh"
#include "fsa_tcd.cuh"
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
template <typename TW>
__global__ void k_d2(int64_t np, int m, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                     const double* __restrict__ vals, const TW* __restrict__ W1, int64_t ldw,
                     const double* __restrict__ Gt, double* __restrict__ out) {
  int lane = threadIdx.x & 31;
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p = warp; p < np; p += nwarps) {
    const double* g = Gt + p * m;
    double acc = 0.0;
    for (int64_t t = rowptr[p]; t < rowptr[p + 1]; ++t) {
      const TW* w = W1 + (int64_t)col[t] * ldw;
      double sd = 0.0;
      for (int k = lane; k < m; k += 32) sd += (double)w[k] * g[k];
      acc += vals[t] * warp_sum(sd);
    }
    if (lane == 0) out[p] = acc;
  }
}

// Y (np x k, ld ldy) = S X  (S: CSR by prediction rows; X rows = training points)
template <typename TX, typename TY>
__global__ void k_cross_spmm(int64_t np, int k, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                             const double* __restrict__ vals, const TX* __restrict__ X, int64_t ldx,
                             TY* __restrict__ Y, int64_t ldy) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < np * k; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t p = t / k;
    int j = (int)(t % k);
    double s = 0.0;
    for (int64_t e = rowptr[p]; e < rowptr[p + 1]; ++e) s += vals[e] * (double)X[(int64_t)col[e] * ldx + j];
    Y[p * ldy + j] = (TY)s;
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

// out[i][p] = S_pi (dense rows of S^T, n x np, ld ldo) from S^T in CSR by training points
__global__ void k_st_dense(int64_t n, int64_t np, const int64_t* __restrict__ trow, const int32_t* __restrict__ tcol,
                           const int64_t* __restrict__ tsrc, const double* __restrict__ vals, double* __restrict__ out,
                           int64_t ldo) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double* o = out + i * ldo;
    for (int64_t p = 0; p < np; ++p) o[p] = 0.0;
    for (int64_t e = trow[i]; e < trow[i + 1]; ++e) o[tcol[e]] = vals[tsrc[e]];
  }
}

// out[p] = sum_i S_pi Y[i][p]  (the diagonal of S Y for Y = Sigma_s~^-1 S^T)
__global__ void k_cross_diag(int64_t np, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                             const double* __restrict__ vals, const double* __restrict__ Y, int64_t ldy,
                             double* __restrict__ out) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int64_t e = rowptr[p]; e < rowptr[p + 1]; ++e) acc += vals[e] * Y[(int64_t)col[e] * ldy + p];
    out[p] = acc;
  }
}

__global__ void k_pred_probes(int64_t np, int s, int kind, uint64_t key, double* __restrict__ Z) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < np * s; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t p = t / s;
    int k = (int)(t % s);
    Z[t] = probe_at(kind, key, (uint64_t)k * np + p);
  }
}

// out[p] = sum_k X[p][k] Y[p][k]   (row dots, FP64 sums)
template <typename TX, typename TY>
__global__ void k_rowdot(int64_t np, int k, const TX* __restrict__ X, int64_t ldx, const TY* __restrict__ Y,
                         int64_t ldy, double scale, double* __restrict__ out) {
  int lane = threadIdx.x & 31;
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p = warp; p < np; p += nwarps) {
    double s = 0.0;
    for (int j = lane; j < k; j += 32) s += (double)X[p * ldx + j] * (double)Y[p * ldy + j];
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
    dgemm(H.ws, st, false, true, (int)np, m, m, 1.0, Kp.p, m, op.Lmi.p, m, 0.0, Ap.p, m, nullptr, kTriB_KleJ);
    dgemm(H.ws, st, false, false, (int)np, m, m, 1.0, Ap.p, m, op.Lmi.p, m, 0.0, Gt.p, m, nullptr, kTriB_KgeJ);
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
    k_cross_spmm<double, double><<<grid_for(np, 256), 256, 0, st>>>(np, 1, srow.p, scol.p, svals.p, u.p, 1, su.p, 1);
    FSA_CHECK_LAUNCH();
  }
  DevPtr<double> mean(np), var(np);
  if (var_host) {
    // sparse block solve: [Sigma_mn^T | S^T Z] (n x (m + s)) with Sigma_s~, D_s
    // preconditioner; for the exact variances [Sigma_mn^T | S^T] (n x (m + np))
    const bool exact = o.pred_exact_var != 0;
    const int cb = exact ? m + (int)np : m + s;
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
      if (exact)
        k_st_dense<<<grid_for(n, 128), 128, 0, st>>>(n, np, trow.p, tcol.p, tsrc.p, svals.p, RHS.p + m, cb);
      else
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
      dgemm(H.ws, st, true, false, m, m, m, 1.0, Li.p, m, Li.p, m, 0.0, Minv.p, m, nullptr,
            kTriA_KgeI | kTriB_KgeJ | kTriSymLower);
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
    k_rowdot<double, double><<<grid_for(np * 32, 256, 152 * 64), 256, 0, st>>>(np, m, T.p, m, Gt.p, m, 1.0, D1.p);
    FSA_CHECK_LAUNCH();
    // D2 = sum_i S_pi (W1 g_p)_i
    k_d2<double><<<grid_for(np * 32, 256, 152 * 64), 256, 0, st>>>(np, m, srow.p, scol.p, svals.p, W1.p, m, Gt.p,
                                                                 D2.p);
    FSA_CHECK_LAUNCH();
    // D3 = diag(V M^-1 V^T), V = S W2
    k_cross_spmm<double, double><<<grid_for(np * m, 256), 256, 0, st>>>(np, m, srow.p, scol.p, svals.p, W2, cb, V.p, m);
    FSA_CHECK_LAUNCH();
    dgemm(H.ws, st, false, false, (int)np, m, m, 1.0, V.p, m, Minv.p, m, 0.0, T.p, m, nullptr);
    k_rowdot<double, double><<<grid_for(np * 32, 256, 152 * 64), 256, 0, st>>>(np, m, T.p, m, V.p, m, 1.0, D3.p);
    FSA_CHECK_LAUNCH();
    // Dl = (1/s) sum_k z_pk (S Ys)_pk, its control-variate form, or exactly diag(S Sigma_s~^-1 S^T)
    {
      DevPtr<double> SY((size_t)np * s);
      if (!exact) {
        k_cross_spmm<double, double><<<grid_for(np * s, 256), 256, 0, st>>>(np, s, srow.p, scol.p, svals.p, Ys, cb,
                                                                            SY.p, s);
        FSA_CHECK_LAUNCH();
      }
      if (exact) {
        k_cross_diag<<<grid_for(np, 256), 256, 0, st>>>(np, srow.p, scol.p, svals.p, Ys, cb, Dl.p);
        FSA_CHECK_LAUNCH();
      } else if (o.pred_control_variate == 0) {
        k_rowdot<double, double><<<grid_for(np * 32, 256, 152 * 64), 256, 0, st>>>(np, s, Zp.p, s, SY.p, s, 1.0 / s, Dl.p);
        FSA_CHECK_LAUNCH();
      } else {
        // S D_s^-1 S^T Z from the probe right-hand sides S^T Z (columns m.. of RHS)
        DevPtr<double> DZ((size_t)n * s), SU((size_t)np * s);
        k_scale_rows<<<grid_for(n * s, 256), 256, 0, st>>>(n, s, op.D.p, RHS.p + m, cb, DZ.p);
        FSA_CHECK_LAUNCH();
        k_cross_spmm<double, double><<<grid_for(np * s, 256), 256, 0, st>>>(np, s, srow.p, scol.p, svals.p, DZ.p, s, SU.p, s);
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

// ---------------------------------------------------------------------------
// mixed form (FSA_MIXED_BF16X2 / FSA_MIXED_BF16): the operator of the mixed
// log-likelihood (A~ as BF16, FP32 residual values), FP32 block CG for the
// sparse solves, the m-column products on the tensor cores (tc_dgemm), the
// m x m factorisations and the diagonals' sums in FP64
// ---------------------------------------------------------------------------
// S_pi = (s1 r(d) - ap_p . a~_i) T(d), ap FP64 (np x m), A~ as BF16 hi (+ lo)
// in the blocked K-major layout: warp per prediction row
__global__ void k_cross_values_pairs(int64_t np, int64_t n, int m, int m_pad, const int64_t* __restrict__ rowptr,
                                     const int32_t* __restrict__ col, const double* __restrict__ px,
                                     const double* __restrict__ py, const double* __restrict__ xs,
                                     const double* __restrict__ ys, const double* __restrict__ Ap,
                                     const __nv_bfloat16* __restrict__ A, const __nv_bfloat16* __restrict__ Alo,
                                     int cov, double s1, double rho, double gamma, double* __restrict__ vals) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p = warp; p < np; p += nwarps) {
    const double* a = Ap + p * m;
    for (int64_t t = rowptr[p]; t < rowptr[p + 1]; ++t) {
      const int64_t i = col[t];
      double sd = 0.0;
      for (int kb = 0; kb < m_pad / 64; ++kb) {
        const int k = kb * 64 + 2 * lane;
        const int64_t o = ((int64_t)kb * n + i) * 64 + 2 * lane;
        float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(A + o));
        if (Alo) {
          const float2 w = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(Alo + o));
          v.x += w.x;
          v.y += w.y;
        }
        if (k < m) sd += a[k] * (double)v.x;
        if (k + 1 < m) sd += a[k + 1] * (double)v.y;
      }
      sd = warp_sum(sd);
      if (lane == 0) {
        const double d = sqrt(sqdist_rn(px[p], py[p], xs[i], ys[i]));
        vals[t] = (s1 * matern_r(cov, d, rho) - sd) * wendland(d, gamma);
      }
    }
  }
}

template <typename TS, typename TD>
__global__ void k_convert(int64_t total, const TS* __restrict__ src, TD* __restrict__ dst) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
    dst[t] = (TD)src[t];
}

// dst (n x k FP64) = the first k columns of src (n x lds FP32)
__global__ void k_take_cols_f64(int64_t n, int k, const float* __restrict__ src, int64_t lds, double* __restrict__ dst) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * k; t += (int64_t)gridDim.x * blockDim.x)
    dst[t] = (double)src[(t / k) * lds + t % k];
}

// R (n x ldc FP32): y in column 0, zeros elsewhere
__global__ void k_rhs_col0(int64_t n, int ldc, const double* __restrict__ y, float* __restrict__ R) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * ldc; t += (int64_t)gridDim.x * blockDim.x)
    R[t] = (t % ldc) == 0 ? (float)y[t / ldc] : 0.f;
}

// u (FP64) = column 0 of U (n x ldc FP32)
__global__ void k_col0_f64(int64_t n, int ldc, const float* __restrict__ U, double* __restrict__ u) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    u[i] = (double)U[i * ldc];
}

// FP32 block PCG on Sigma_s~ (the mixed operator's residual values) with the
// D_s preconditioner (Algorithm 1's sparse solves, Appendix A): B (n x c
// FP32, ld ldb) -> U (n x c FP32, ld ldu), columns in chunks of at most 128
PcgStats pcg_sparse_f32(Handle& H, const float* B, int64_t ldb, int c, float* U, int64_t ldu, const fsa_opts& o,
                        int L) {
  cudaStream_t s = H.stream;
  Operator& op = H.op;
  CGState& g = H.cg;
  const int64_t n = H.n;
  fsa_opts oc = o;
  oc.fixed_iters = 0;
  PcgStats st;
  int32_t* pin = reinterpret_cast<int32_t*>(H.host_pinned);
  for (int c0 = 0; c0 < c; c0 += 128) {
    const int cc = std::min(128, c - c0);
    CGLayout lay;
    lay.setup(n, cc, L, (cc + 3) / 4 * 4);
    ensure_cg(H, lay, false);
    const int ldc = lay.ldc;
    const size_t nc = (size_t)n * ldc;
    g.U32.ensure(nc); g.R32.ensure(nc); g.Z32.ensure(nc); g.H32.ensure(nc); g.V32.ensure(nc); g.S32.ensure(nc);
    FSA_CUDA(cudaMemsetAsync(g.U32.p, 0, nc * sizeof(float), s));
    FSA_CUDA(cudaMemsetAsync(g.V32.p, 0, nc * sizeof(float), s));
    FSA_CUDA(cudaMemsetAsync(g.H32.p, 0, nc * sizeof(float), s));
    FSA_CUDA(cudaMemsetAsync(g.S32.p, 0, nc * sizeof(float), s));   // no low-rank part
    FSA_CUDA(cudaMemsetAsync(g.R32.p, 0, nc * sizeof(float), s));
    FSA_CUDA(cudaMemcpy2DAsync(g.R32.p, ldc * sizeof(float), B + c0, ldb * sizeof(float), cc * sizeof(float), n,
                               cudaMemcpyDeviceToDevice, s));
    CGScalars q = make_scalars(H, oc, L);
    const Vec4Launch v4 = vec4_launch(lay, reinterpret_cast<const void*>(kv4_ur_update));
    const Vec4Launch v4z = vec4_launch(lay, reinterpret_cast<const void*>(kv4_z_update));
    const StagedLaunch sl = staged_launch(H, ldc);
    kv4_z_update<<<v4z.blocks, v4z.threads, v4z.smem, s>>>(n, cc, ldc, v4z.rpb, g.R32.p, g.S32.p, op.Dinv32.p,
                                                          g.Z32.p, g.part.p, kStepInit, 0, q);
    FSA_CHECK_LAUNCH();
    launch_spmm_f32(H, lay, sl, s, op.vals32.p, g.Z32.p, g.S32.p, g.V32.p, g.H32.p, g.beta.p, g.part.p, kStepAlpha, q);
    int done = 0;
    *pin = 1;
    for (int it = 0; it < L; ++it) {
      kv4_ur_update<<<v4.blocks, v4.threads, v4.smem, s>>>(n, cc, ldc, v4.rpb, g.U32.p, g.R32.p, g.H32.p, g.V32.p,
                                                           g.alpha.p, g.active.p, g.part.p, kStepResid, it, q);
      FSA_CHECK_LAUNCH();
      kv4_z_update<<<v4z.blocks, v4z.threads, v4z.smem, s>>>(n, cc, ldc, v4z.rpb, g.R32.p, g.S32.p, op.Dinv32.p,
                                                            g.Z32.p, g.part.p, kStepBeta, it, q);
      FSA_CHECK_LAUNCH();
      launch_spmm_f32(H, lay, sl, s, op.vals32.p, g.Z32.p, g.S32.p, g.V32.p, g.H32.p, g.beta.p, g.part.p,
                      kStepAlpha, q);
      FSA_CUDA(cudaMemcpyAsync(pin, g.num_active.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      FSA_CUDA(cudaStreamSynchronize(s));
      done = it + 1;
      if (*pin == 0) break;
    }
    if (*pin != 0) st.converged = false;
    st.iters_max = std::max(st.iters_max, done);
    FSA_CUDA(cudaMemcpy2DAsync(U + c0, ldu * sizeof(float), g.U32.p, ldc * sizeof(float), cc * sizeof(float), n,
                               cudaMemcpyDeviceToDevice, s));
  }
  FSA_CUDA(cudaStreamSynchronize(s));
  return st;
}

PredResult run_predict_mixed(Handle& H, const fsa_theta& th, const fsa_opts& o, const double* pred_host, int64_t np,
                             int s, double* mean_host, double* var_host) {
  cudaStream_t st = H.stream;
  Operator& op = H.op;
  CGState& g = H.cg;
  const int64_t n = H.n;
  const int m = H.m, m_pad = op.m_pad;
  const int L = o.cg_max_iter > 0 ? o.cg_max_iter : 1000;
  const __nv_bfloat16* Alo = op.has_lo ? op.Ab_lo.p : nullptr;
  PredResult res;
  // prediction points (caller order) and the cross pattern S (rows = prediction points)
  DevPtr<double> pts(2 * np), px(np), py(np);
  FSA_CUDA(cudaMemcpyAsync(pts.p, pred_host, sizeof(double) * 2 * np, cudaMemcpyHostToDevice, st));
  k_split_xy<<<grid_for(np, 256), 256, 0, st>>>(np, pts.p, px.p, py.p, H.err);
  FSA_CHECK_LAUNCH();
  check_err(H);
  DevPtr<int64_t> srow;
  DevPtr<int32_t> scol;
  int64_t snnz = 0;
  build_cross_structure(H, px.p, py.p, np, srow, scol, snnz);
  // ap_p = L^-1 k_p and g_p^T = ap_p^T L^-1 (np x m) on the tensor cores
  DevPtr<double> Ap((size_t)np * m), Gt((size_t)np * m);
  {
    DevPtr<double> Kp((size_t)np * m);
    cov_cross(H, np, px.p, py.p, m, H.ind_x.p, H.ind_y.p, th, 0, Kp.p, m);
    tc_dgemm<double, double>(H, false, true, (int)np, m, m, Kp.p, m, op.Lmi.p, m, Ap.p, m, false, nullptr, "predict");
    tc_dgemm<double, double>(H, false, false, (int)np, m, m, Ap.p, m, op.Lmi.p, m, Gt.p, m, false, nullptr, "predict");
    FSA_CUDA(cudaStreamSynchronize(st));
  }
  DevPtr<double> svals(snnz > 0 ? snnz : 1);
  if (snnz > 0) {
    k_cross_values_pairs<<<grid_for(np * 32, 256, 152 * 64), 256, 0, st>>>(
        np, n, m, m_pad, srow.p, scol.p, px.p, py.p, H.xs.p, H.ys.p, Ap.p, op.Ab.p, Alo, H.cov, th.sigma1_sq, th.rho,
        H.gamma, svals.p);
    FSA_CHECK_LAUNCH();
  }
  // u = Sigma_dag^-1 y by the mixed FITC-PCG, and the mean ap_p . (A~^T u) + (S u)_p
  DevPtr<double> u(n), Atu(m), mlr(np), su(np);
  {
    CGLayout lay;
    lay.setup(n, 1, L, mixed_ldc(1, H.vec_pieces));
    ensure_cg(H, lay, false);
    const int ldc = lay.ldc;
    const size_t nc = (size_t)n * ldc;
    g.U32.ensure(nc); g.R32.ensure(nc); g.Z32.ensure(nc); g.H32.ensure(nc); g.V32.ensure(nc);
    g.S32.ensure(nc); g.W032.ensure(nc);
    MixedCtx C;
    mixed_ctx_setup(H, C, n, 1, ldc);
    DevPtr<float> wpart((size_t)C.splits_w * C.m_pad * ldc);
    C.wpart = wpart.p;
    k_rhs_col0<<<grid_for((int64_t)nc, 256), 256, 0, st>>>(n, ldc, H.y.p, g.R32.p);
    FSA_CHECK_LAUNCH();
    fsa_opts ou = o;
    ou.fixed_iters = 0;
    pcg_mixed_run(H, C, lay, ou, L);
    int32_t it0 = 0, nact = 0;
    FSA_CUDA(cudaMemcpyAsync(&it0, g.iters.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    FSA_CUDA(cudaMemcpyAsync(&nact, g.num_active.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    DevPtr<double> w((size_t)m * ldc);
    mixed_AtX(H, C, g.U32.p, nullptr, w.p, "predict");
    k_col0_f64<<<grid_for(n, 256), 256, 0, st>>>(n, ldc, g.U32.p, u.p);
    FSA_CHECK_LAUNCH();
    FSA_CUDA(cudaStreamSynchronize(st));
    res.iters_u = it0;
    res.converged = nact == 0;
    // A~^T u is column 0 of w (m x ldc FP64)
    FSA_CUDA(cudaMemcpy2DAsync(Atu.p, sizeof(double), w.p, ldc * sizeof(double), sizeof(double), m,
                               cudaMemcpyDeviceToDevice, st));
    dgemm(H.ws, st, false, false, (int)np, 1, m, 1.0, Ap.p, m, Atu.p, 1, 0.0, mlr.p, 1, nullptr);
    k_cross_spmm<double, double><<<grid_for(np, 256), 256, 0, st>>>(np, 1, srow.p, scol.p, svals.p, u.p, 1, su.p, 1);
    FSA_CHECK_LAUNCH();
  }
  DevPtr<double> mean(np), var(np);
  if (var_host) {
    // sparse block solve [Sigma_mn^T | S^T Z] (n x (m + s)) with Sigma_s~ and the
    // D_s preconditioner, in FP32
    const int cb = m + s;
    DevPtr<float> RHS32((size_t)n * cb), X((size_t)n * cb);
    DevPtr<double> Knm((size_t)n * m), Zp((size_t)np * s), StZ((size_t)n * s);
    {
      DevPtr<double> RHS((size_t)n * cb);
      cov_cross(H, n, H.xs.p, H.ys.p, m, H.ind_x.p, H.ind_y.p, th, 0, RHS.p, cb);
      cov_cross(H, n, H.xs.p, H.ys.p, m, H.ind_x.p, H.ind_y.p, th, 0, Knm.p, m);
      k_pred_probes<<<grid_for(np * s, 256), 256, 0, st>>>(np, s, o.probe, rng_key(o.seed, kStreamPred), Zp.p);
      FSA_CHECK_LAUNCH();
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
      k_st_z<<<grid_for(n * s, 256), 256, 0, st>>>(n, s, trow.p, tcol.p, tsrc.p, svals.p, Zp.p, StZ.p, s);
      FSA_CHECK_LAUNCH();
      FSA_CUDA(cudaMemcpy2DAsync(RHS.p + m, cb * sizeof(double), StZ.p, s * sizeof(double), s * sizeof(double), n,
                                 cudaMemcpyDeviceToDevice, st));
      k_convert<double, float><<<grid_for((int64_t)n * cb, 256), 256, 0, st>>>((int64_t)n * cb, RHS.p, RHS32.p);
      FSA_CHECK_LAUNCH();
      FSA_CUDA(cudaStreamSynchronize(st));
    }
    PcgStats ps = pcg_sparse_f32(H, RHS32.p, cb, cb, X.p, cb, o, L);
    res.iters_sparse = ps.iters_max;
    res.converged = res.converged && ps.converged;
    const float* W2 = X.p;       // n x m, ld cb
    const float* Ys = X.p + m;   // n x s, ld cb
    // M = Sigma_m + Sigma_mn W2 ; Yms = M^-1 Sigma_m ; W1 = W2 Yms
    DevPtr<double> Mm((size_t)m * m), Minv((size_t)m * m), Sm((size_t)m * m), Yms((size_t)m * m);
    cov_cross(H, m, H.ind_x.p, H.ind_y.p, m, H.ind_x.p, H.ind_y.p, th, 0, Mm.p, m);
    FSA_CUDA(cudaMemcpyAsync(Sm.p, Mm.p, sizeof(double) * m * m, cudaMemcpyDeviceToDevice, st));
    {
      // the core Sigma_m + Sigma_mn W2 in FP64: its small eigenvalues sit far
      // below its largest entries (of order n sigma1^4 / nugget), which FP32
      // sums on the tensor cores would not resolve
      DevPtr<double> W2d((size_t)n * m);
      FSA_CUDA(cudaMemsetAsync(W2d.p, 0, sizeof(double) * (size_t)n * m, st));
      k_take_cols_f64<<<grid_for((int64_t)n * m, 256), 256, 0, st>>>(n, m, W2, cb, W2d.p);
      FSA_CHECK_LAUNCH();
      dgemm(H.ws, st, true, false, m, m, (int)n, 1.0, Knm.p, m, W2d.p, m, 1.0, Mm.p, m, nullptr);
      FSA_CUDA(cudaStreamSynchronize(st));
    }
    cholesky(Mm.p, m, m, H.err, st);
    {
      DevPtr<double> Li((size_t)m * m);
      lower_inverse(H.ws, Mm.p, m, Li.p, st);
      dgemm(H.ws, st, true, false, m, m, m, 1.0, Li.p, m, Li.p, m, 0.0, Minv.p, m, nullptr,
            kTriA_KgeI | kTriB_KgeJ | kTriSymLower);
      FSA_CUDA(cudaStreamSynchronize(st));
    }
    check_err(H);
    dgemm(H.ws, st, false, false, m, m, m, 1.0, Minv.p, m, Sm.p, m, 0.0, Yms.p, m, nullptr);
    DevPtr<float> W1((size_t)n * m), T32((size_t)np * m), V32((size_t)np * m);
    DevPtr<double> C1((size_t)m * m);
    tc_dgemm<float, double>(H, false, false, (int)n, m, m, W2, cb, Yms.p, m, nullptr, m, false, W1.p, "predict");
    // D1 = diag(G^T (Sigma_mn W1) G)
    tc_dgemm<double, float>(H, true, false, m, m, (int)n, Knm.p, m, W1.p, m, C1.p, m, false, nullptr, "predict");
    tc_dgemm<double, double>(H, false, false, (int)np, m, m, Gt.p, m, C1.p, m, nullptr, m, false, T32.p, "predict");
    DevPtr<double> D1(np), D2(np), D3(np), Dl(np);
    k_rowdot<float, double><<<grid_for(np * 32, 256, 152 * 64), 256, 0, st>>>(np, m, T32.p, m, Gt.p, m, 1.0, D1.p);
    FSA_CHECK_LAUNCH();
    // D2 = sum_i S_pi (W1 g_p)_i
    k_d2<float><<<grid_for(np * 32, 256, 152 * 64), 256, 0, st>>>(np, m, srow.p, scol.p, svals.p, W1.p, m, Gt.p,
                                                                D2.p);
    FSA_CHECK_LAUNCH();
    // D3 = diag(V M^-1 V^T), V = S W2
    k_cross_spmm<float, float><<<grid_for(np * m, 256), 256, 0, st>>>(np, m, srow.p, scol.p, svals.p, W2, cb, V32.p,
                                                                      m);
    FSA_CHECK_LAUNCH();
    tc_dgemm<float, double>(H, false, false, (int)np, m, m, V32.p, m, Minv.p, m, nullptr, m, false, T32.p, "predict");
    k_rowdot<float, float><<<grid_for(np * 32, 256, 152 * 64), 256, 0, st>>>(np, m, T32.p, m, V32.p, m, 1.0, D3.p);
    FSA_CHECK_LAUNCH();
    // Dl = (1/s) sum_k z_pk (S Ys)_pk, or its control-variate form
    {
      DevPtr<double> SY((size_t)np * s);
      k_cross_spmm<float, double><<<grid_for(np * s, 256), 256, 0, st>>>(np, s, srow.p, scol.p, svals.p, Ys, cb,
                                                                         SY.p, s);
      FSA_CHECK_LAUNCH();
      if (o.pred_control_variate == 0) {
        k_rowdot<double, double><<<grid_for(np * 32, 256, 152 * 64), 256, 0, st>>>(np, s, Zp.p, s, SY.p, s, 1.0 / s,
                                                                                   Dl.p);
        FSA_CHECK_LAUNCH();
      } else {
        DevPtr<double> DZ((size_t)n * s), SU((size_t)np * s);
        k_scale_rows<<<grid_for(n * s, 256), 256, 0, st>>>(n, s, op.D.p, StZ.p, s, DZ.p);
        FSA_CHECK_LAUNCH();
        k_cross_spmm<double, double><<<grid_for(np * s, 256), 256, 0, st>>>(np, s, srow.p, scol.p, svals.p, DZ.p, s,
                                                                            SU.p, s);
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
