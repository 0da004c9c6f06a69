// CG scalar steps of the block PCG (Appendix A), fused into the kernels that
// produce the dot products they need (element-wise CG kernels, the SpMM and
// the tensor-core epilogue of S = A~ q).
#pragma once
#include "fsa_internal.cuh"

namespace fsa {

// ---------------------------------------------------------------------------
// CG scalars fused into the producing kernels (Appendix A).  The last block
// to finish (ticket counter) sums the per-block partials of every column in
// a fixed order and applies the per-column scalar step, so results do not
// depend on which block finishes last.
// ---------------------------------------------------------------------------
struct CGScalars {
  double *rho, *rz0, *alpha, *beta, *alpha_prev, *beta_prev, *rnorm, *tdiag, *toff;
  int32_t *active, *iters, *stop, *num_active;
  unsigned* err;
  unsigned* ticket;
  double tol;
  int fixed, L;
  int64_t nrows;   // rows of the CG block (the index checks of the checked build)
};

enum ScalarStep : int { kStepNone = 0, kStepInit = 1, kStepAlpha = 2, kStepResid = 3, kStepBeta = 4 };

__device__ __forceinline__ void scalar_step(int step, int col, int c, double v, int l, CGScalars& q) {
  if (col >= c) return;
  if (step == kStepInit) {
    if (!isfinite(v)) atomicOr(q.err, kErrNaN);
    q.rho[col] = v;
    q.rz0[col] = v;
    q.alpha_prev[col] = 1.0;   // alpha_0 = 1
    q.beta_prev[col] = 0.0;    // beta_0 = 0
    q.beta[col] = 0.0;
    q.active[col] = v > 0.0 ? 1 : 0;
    q.iters[col] = 0;
    q.stop[col] = 0;
  } else if (step == kStepAlpha) {
    double a = 0.0;
    if (q.active[col]) {
      a = q.rho[col] / v;
      if (!isfinite(a) || !(v > 0.0)) { atomicOr(q.err, kErrNaN); a = 0.0; }
    }
    q.alpha[col] = a;
  } else if (step == kStepResid) {
    if (q.active[col]) {
      double rn = sqrt(v);
      q.rnorm[col] = rn;
      q.stop[col] = (!q.fixed && rn < q.tol) ? 1 : 0;
    }
  } else if (step == kStepBeta) {
    if (q.active[col]) {
      double b = v / q.rho[col];
      double a = q.alpha[col];
      if (l < q.L) {   // Lanczos tridiagonal from the CG coefficients (Appendix A)
        q.tdiag[(int64_t)col * q.L + l] = 1.0 / a + q.beta_prev[col] / q.alpha_prev[col];
        if (l > 0) q.toff[(int64_t)col * q.L + l - 1] = sqrt(q.beta_prev[col]) / q.alpha_prev[col];
      }
      q.iters[col] = l + 1;
      q.alpha_prev[col] = a;
      q.beta_prev[col] = b;
      q.rho[col] = v;
      if (!isfinite(b)) { atomicOr(q.err, kErrNaN); b = 0.0; }
      q.beta[col] = b;
      if (q.stop[col] || v <= 0.0) q.active[col] = 0;
    } else {
      q.beta[col] = 0.0;
    }
  }
}

// called by every thread of every block after part[blockIdx.x][*] is written;
// red: shared scratch of at least blockDim.x doubles
__device__ __forceinline__ void finish_scalars(int step, const double* __restrict__ part, int ldc, int c, int l,
                                               CGScalars& q, double* __restrict__ red) {
  if (step == kStepNone) return;
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = atomicAdd(q.ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  // coalesced fixed-order sum of the nb partial rows: thread (group g, column
  // col) adds rows g, g + RG, ... in order (four running sums); the RG group
  // sums are then added in group order
  const int nb = (int)gridDim.x;
  const int RG = ((int)blockDim.x / ldc) > 1 ? (int)blockDim.x / ldc : 1;
  for (int t = threadIdx.x; t < RG * ldc; t += blockDim.x) {
    const int col = t % ldc, g = t / ldc;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int b = g;
    // sixteen independent loads in flight per step (the reduction tail is a
    // chain of L2 round trips), added to the four running sums in a fixed order
    for (; b + 15 * RG < nb; b += 16 * RG) {
      double v[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] = __ldcg(&part[(int64_t)(b + k * RG) * ldc + col]);
#pragma unroll
      for (int k = 0; k < 16; k += 4) {
        s0 += v[k];
        s1 += v[k + 1];
        s2 += v[k + 2];
        s3 += v[k + 3];
      }
    }
    for (; b + 3 * RG < nb; b += 4 * RG) {
      s0 += __ldcg(&part[(int64_t)b * ldc + col]);
      s1 += __ldcg(&part[(int64_t)(b + RG) * ldc + col]);
      s2 += __ldcg(&part[(int64_t)(b + 2 * RG) * ldc + col]);
      s3 += __ldcg(&part[(int64_t)(b + 3 * RG) * ldc + col]);
    }
    for (; b < nb; b += RG) s0 += __ldcg(&part[(int64_t)b * ldc + col]);
    red[t] = (s0 + s1) + (s2 + s3);
  }
  __syncthreads();
  for (int col = threadIdx.x; col < ldc; col += blockDim.x) {
    double v = 0.0;
    for (int g = 0; g < RG; ++g) v += red[g * ldc + col];
    scalar_step(step, col, c, v, l, q);
  }
  if (step == kStepBeta) {
    __syncthreads();
    if (threadIdx.x == 0) {
      int s = 0;
      for (int k = 0; k < c; ++k) s += q.active[k];
      *q.num_active = s;
    }
  }
  if (threadIdx.x == 0) *q.ticket = 0u;
}

}  // namespace fsa
