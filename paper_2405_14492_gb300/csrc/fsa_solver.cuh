// Declarations shared by the solver translation units.
#pragma once
#include "fsa_internal.cuh"

namespace fsa {

struct CGLayout {
  int64_t n = 0;
  int c = 0, ldc = 0, L = 0, threads = 32, nblk = 1;
  int64_t chunk = 1;      // rows per block (row-chunk kernels): nblk * chunk >= n
  int rpb = 1;            // rows per block step of the flat element-wise kernels
  int ethreads = 32;      // rpb * ldc threads per block
  void setup(int64_t n_, int c_, int L_, int ldc_ = 0);   // ldc_ = 0: c rounded up to 8
};

struct LoglikResult {
  double loglik = 0, logdet = 0, yu = 0, grad[3] = {0, 0, 0}, se = 0, logdetP = 0;
  // gradient parts: trace estimate, quadratic term u^T dSigma u, Tr(P^-1 dP)
  // and the control variate's coefficient, per parameter
  double trace[3] = {0, 0, 0}, quad[3] = {0, 0, 0}, traceP[3] = {0, 0, 0}, cv_c[3] = {0, 0, 0};
  int iters_max = 0, iters_y = 0;
  double resid_y = 0;
  bool converged = true;
  float ms = 0;
};

void cov_cross(Handle& H, int64_t np, const double* px, const double* py, int nq, const double* qx,
               const double* qy, const fsa_theta& th, int deriv, double* out, int64_t ld);
void build_mspace(Handle& H, const fsa_theta& th);
void finish_core(Handle& H);
void build_operator_fp64(Handle& H, const fsa_theta& th);
void build_operator_mixed(Handle& H, const fsa_theta& th, int precision);
void ensure_operator(Handle& H, const fsa_theta& th, int precision);
void ensure_cg(Handle& H, const CGLayout& lay, bool fp64);
void sum_log_D(Handle& H, const double* D, double* scal);

LoglikResult run_loglik_grad(Handle& H, const fsa_theta& th, const fsa_opts& o);
// block PCG (Appendix A), FP64 form, on the right-hand sides in H.cg.R
void pcg_fp64_run(Handle& H, const CGLayout& lay, const fsa_opts& o, int L);

struct PredResult {
  int iters_u = 0, iters_sparse = 0;
  bool converged = true;
};
PredResult run_predict_fp64(Handle& H, const fsa_theta& th, const fsa_opts& o, const double* pred_host, int64_t np,
                            int s, double* mean_host, double* var_host);
PredResult run_predict_mixed(Handle& H, const fsa_theta& th, const fsa_opts& o, const double* pred_host, int64_t np,
                            int s, double* mean_host, double* var_host);
void apply_operator(Handle& H, int which, const double* v_dev_internal, int k, double* out_dev_internal);

// kernels used across units
__global__ void k_eps1(int m, int l, int kind, uint64_t key, double* __restrict__ E, int64_t lde);
__global__ void k_gather_y(int64_t n, const int64_t* __restrict__ perm, const double* __restrict__ y,
                           double* __restrict__ y_int, unsigned* __restrict__ err);
template <typename T>
__global__ void k_probe_finish(int64_t n, int l, int ldc, int kind, uint64_t key, const int64_t* __restrict__ perm,
                               const double* __restrict__ y_int, const double* __restrict__ D, T* __restrict__ B);
// tile form of the mixed residual values (shared-memory staging of A~ over
// the cell-grid tiles); false when the handle has no tiles or the shapes do
// not fit, and the caller runs the row form.  cap_rows_max > 0 caps the
// staged rows per tile (tiles above it run from global memory).
bool csr_values_tiles(Handle& H, const fsa_theta& th, const __nv_bfloat16* A, const __nv_bfloat16* Alo, int m_pad,
                      int cap_rows_max = 0);
// row form (one warp per row, global gathers) of the same product
void csr_values_rows(Handle& H, const fsa_theta& th, const __nv_bfloat16* A, const __nv_bfloat16* Alo, int m_pad);
__global__ void k_assemble(int64_t n, int c, int exact_weight, const double* __restrict__ quads,
                           const double* __restrict__ rz0, const double* __restrict__ scal,
                           const double* __restrict__ part_yu, int nblk_yu, int ldc, double* __restrict__ outs);

}  // namespace fsa
