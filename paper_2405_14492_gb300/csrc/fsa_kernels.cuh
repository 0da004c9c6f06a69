// Element-wise, sparse and reduction kernels of the FSA solver, templated on
// the vector type (double: FP64 form; float: mixed form).
//
// Block-vector layout: n x ldc row-major (row = point in internal order,
// column = right-hand side: 0 is y, 1..l the probes).  Column kernels use
// one thread per column and one block per chunk of rows: each thread owns one
// column, so every per-column dot product is reduced in a fixed order
// (per-block partials [nblk][ldc], then a fixed-order sum) and results are
// bit-reproducible run to run.
#pragma once
#include "fsa_internal.cuh"

namespace fsa {

template <typename T> struct AccOf { using type = double; };
template <> struct AccOf<float> { using type = float; };

// Products in T; partial sums of up to 32 rows in T, then carried in FP64.
#define FSA_ROWLOOP_BEGIN                                                  \
  int col = threadIdx.x;                                                   \
  if (col >= ldc) return;                                                  \
  int64_t r0 = (int64_t)blockIdx.x * chunk;                                \
  int64_t r1 = r0 + chunk < n ? r0 + chunk : n;                            \
  double acc = 0.0;                                                        \
  typename AccOf<T>::type sub = 0;                                         \
  int cnt = 0;

#define FSA_ACC(v)                    \
  do {                                \
    sub += (v);                       \
    if (++cnt == 32) { acc += (double)sub; sub = 0; cnt = 0; } \
  } while (0)

#define FSA_ROWLOOP_END                       \
  acc += (double)sub;                         \
  part[(int64_t)blockIdx.x * ldc + col] = acc;

// X = R * Dinv (row scale)
template <typename T>
__global__ void k_row_scale(int64_t n, int c, int ldc, int64_t chunk, const T* __restrict__ R,
                            const T* __restrict__ Dinv, T* __restrict__ X) {
  int col = threadIdx.x;
  if (col >= ldc) return;
  int64_t r0 = (int64_t)blockIdx.x * chunk;
  int64_t r1 = r0 + chunk < n ? r0 + chunk : n;
  for (int64_t i = r0; i < r1; ++i) {
    int64_t idx = i * ldc + col;
    X[idx] = col < c ? R[idx] * Dinv[i] : (T)0;
  }
}

// U += a H; R -= a V; X = R Dinv; part = ||R||^2 per column
template <typename T>
__global__ void k_ur_update(int64_t n, int c, int ldc, int64_t chunk, T* __restrict__ U, T* __restrict__ R,
                            const T* __restrict__ H, const T* __restrict__ V, const T* __restrict__ Dinv,
                            T* __restrict__ X, const double* __restrict__ alpha,
                            const int32_t* __restrict__ active, double* __restrict__ part) {
  FSA_ROWLOOP_BEGIN
  T a = (col < c && active[col]) ? (T)alpha[col] : (T)0;
  for (int64_t i = r0; i < r1; ++i) {
    int64_t idx = i * ldc + col;
    if (col < c) {
      T r = R[idx];
      if (a != (T)0) {
        U[idx] = U[idx] + a * H[idx];
        r = r - a * V[idx];
        R[idx] = r;
      }
      if (X) X[idx] = r * Dinv[i];
      FSA_ACC(r * r);
    } else if (X) {
      X[idx] = (T)0;
    }
  }
  FSA_ROWLOOP_END
}

// Z = (R - S) Dinv (the Woodbury correction applied); part = r^T z
template <typename T>
__global__ void k_z_update(int64_t n, int c, int ldc, int64_t chunk, const T* __restrict__ R,
                           const T* __restrict__ S, const T* __restrict__ Dinv, T* __restrict__ Z,
                           double* __restrict__ part) {
  FSA_ROWLOOP_BEGIN
  for (int64_t i = r0; i < r1; ++i) {
    int64_t idx = i * ldc + col;
    if (col < c) {
      T r = R[idx];
      T z = (r - S[idx]) * Dinv[i];
      Z[idx] = z;
      FSA_ACC(r * z);
    } else {
      Z[idx] = (T)0;
    }
  }
  FSA_ROWLOOP_END
}

// V = Sigma_s~ Z + S + beta V ; H = Z + beta H ; part = h^T v
template <typename T, typename VT>
__global__ void k_spmm_fused(int64_t n, int c, int ldc, int64_t chunk, const int64_t* __restrict__ rowptr,
                             const int32_t* __restrict__ colidx, const VT* __restrict__ vals,
                             const T* __restrict__ Z, const T* __restrict__ S, T* __restrict__ V,
                             T* __restrict__ H, const double* __restrict__ beta, double* __restrict__ part) {
  FSA_ROWLOOP_BEGIN
  T b = col < c ? (T)beta[col] : (T)0;
  for (int64_t i = r0; i < r1; ++i) {
    int64_t idx = i * ldc + col;
    int64_t e = rowptr[i + 1];
    T s = 0;
    for (int64_t t = rowptr[i]; t < e; ++t) s += (T)vals[t] * Z[(int64_t)colidx[t] * ldc + col];
    if (col < c) {
      T v = s + S[idx] + (b != (T)0 ? b * V[idx] : (T)0);
      T h = Z[idx] + (b != (T)0 ? b * H[idx] : (T)0);
      V[idx] = v;
      H[idx] = h;
      FSA_ACC(h * v);
    } else {
      V[idx] = (T)0;
      H[idx] = (T)0;
    }
  }
  FSA_ROWLOOP_END
}

// Y = Sigma_s~ X (plain SpMM, any column count)
template <typename T, typename VT>
__global__ void k_spmm(int64_t n, int c, int ldx, int64_t chunk, const int64_t* __restrict__ rowptr,
                       const int32_t* __restrict__ colidx, const VT* __restrict__ vals, const T* __restrict__ X,
                       T* __restrict__ Y, int ldy) {
  int64_t r0 = (int64_t)blockIdx.x * chunk;
  int64_t r1 = r0 + chunk < n ? r0 + chunk : n;
  for (int col = blockIdx.y * blockDim.x + threadIdx.x; col < c; col += gridDim.y * blockDim.x) {
    for (int64_t i = r0; i < r1; ++i) {
      T s = 0;
      for (int64_t t = rowptr[i]; t < rowptr[i + 1]; ++t) s += (T)vals[t] * X[(int64_t)colidx[t] * ldx + col];
      Y[i * ldy + col] = s;
    }
  }
}

// part = X[:, col]^T Y[:, col] for every column
template <typename T>
__global__ void k_coldot(int64_t n, int c, int ldc, int64_t chunk, const T* __restrict__ X,
                         const T* __restrict__ Y, double* __restrict__ part) {
  FSA_ROWLOOP_BEGIN
  for (int64_t i = r0; i < r1; ++i) {
    int64_t idx = i * ldc + col;
    if (col < c) FSA_ACC(X[idx] * Y[idx]);
  }
  FSA_ROWLOOP_END
}

// part[blk * ldc] = sum over the block's rows of y_i U[i][0]
template <typename T>
__global__ void k_dot_col0(int64_t n, int ldc, int64_t chunk, const double* __restrict__ y,
                           const T* __restrict__ U, double* __restrict__ part) {
  if (threadIdx.x != 0) return;
  int64_t r0 = (int64_t)blockIdx.x * chunk;
  int64_t r1 = r0 + chunk < n ? r0 + chunk : n;
  double s = 0.0;
  for (int64_t i = r0; i < r1; ++i) s += y[i] * (double)U[i * ldc];
  part[(int64_t)blockIdx.x * ldc] = s;
}

template <typename T>
__global__ void k_copy_col0(int64_t n, int ldc, const T* __restrict__ src, T* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i * ldc] = src[i * ldc];
}

#undef FSA_ROWLOOP_BEGIN
#undef FSA_ROWLOOP_END
#undef FSA_ACC

// ---------------------------------------------------------------------------
// per-column CG scalars (Appendix A): one block, one thread per column
// ---------------------------------------------------------------------------
__device__ __forceinline__ double sum_part(const double* part, int nblk, int ldc, int col) {
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * ldc + col];
  return s;
}

static __global__ void k_cg_init(int c, int ldc, int nblk, const double* __restrict__ part, double* __restrict__ rho,
                          double* __restrict__ rz0, double* __restrict__ alpha_prev, double* __restrict__ beta_prev,
                          double* __restrict__ beta, int32_t* __restrict__ active, int32_t* __restrict__ iters,
                          int32_t* __restrict__ stop, unsigned* __restrict__ err) {
  int col = threadIdx.x;
  if (col >= ldc) return;
  double r = col < c ? sum_part(part, nblk, ldc, col) : 0.0;
  if (col < c && !isfinite(r)) atomicOr(err, kErrNaN);
  rho[col] = r;
  rz0[col] = r;
  alpha_prev[col] = 1.0;   // alpha_0 = 1
  beta_prev[col] = 0.0;    // beta_0 = 0
  beta[col] = 0.0;
  active[col] = (col < c && r > 0.0) ? 1 : 0;
  iters[col] = 0;
  stop[col] = 0;
}

static __global__ void k_cg_alpha(int c, int ldc, int nblk, const double* __restrict__ part, const double* __restrict__ rho,
                           double* __restrict__ alpha, const int32_t* __restrict__ active, unsigned* __restrict__ err) {
  int col = threadIdx.x;
  if (col >= ldc) return;
  double a = 0.0;
  if (col < c && active[col]) {
    double hv = sum_part(part, nblk, ldc, col);
    a = rho[col] / hv;
    if (!isfinite(a) || !(hv > 0.0)) { atomicOr(err, kErrNaN); a = 0.0; }
  }
  alpha[col] = a;
}

static __global__ void k_cg_resid(int c, int ldc, int nblk, const double* __restrict__ part, double* __restrict__ rnorm,
                           const int32_t* __restrict__ active, int32_t* __restrict__ stop, double tol, int fixed) {
  int col = threadIdx.x;
  if (col >= ldc || col >= c || !active[col]) return;
  double rn = sqrt(sum_part(part, nblk, ldc, col));
  rnorm[col] = rn;
  stop[col] = (!fixed && rn < tol) ? 1 : 0;
}

static __global__ void k_cg_beta(int c, int ldc, int nblk, int l, int L, const double* __restrict__ part,
                          double* __restrict__ rho, const double* __restrict__ alpha, double* __restrict__ beta,
                          double* __restrict__ alpha_prev, double* __restrict__ beta_prev,
                          int32_t* __restrict__ active, int32_t* __restrict__ iters, const int32_t* __restrict__ stop,
                          double* __restrict__ tdiag, double* __restrict__ toff, int32_t* __restrict__ num_active,
                          unsigned* __restrict__ err) {
  __shared__ int cnt[32];
  int col = threadIdx.x;
  int still = 0;
  if (col < c && active[col]) {
    double rz = sum_part(part, nblk, ldc, col);
    double b = rz / rho[col];
    double a = alpha[col];
    // Lanczos tridiagonal from the CG coefficients (Appendix A)
    if (l < L) {
      tdiag[(int64_t)col * L + l] = 1.0 / a + beta_prev[col] / alpha_prev[col];
      if (l > 0) toff[(int64_t)col * L + l - 1] = sqrt(beta_prev[col]) / alpha_prev[col];
    }
    iters[col] = l + 1;
    alpha_prev[col] = a;
    beta_prev[col] = b;
    rho[col] = rz;
    if (!isfinite(b)) { atomicOr(err, kErrNaN); b = 0.0; }
    beta[col] = b;
    if (stop[col] || rz <= 0.0) active[col] = 0;
    else still = 1;
  } else if (col < ldc) {
    beta[col] = 0.0;
  }
  // count active columns
  unsigned ballot = __ballot_sync(0xffffffffu, still);
  if ((threadIdx.x & 31) == 0) cnt[threadIdx.x >> 5] = __popc(ballot);
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < (int)((blockDim.x + 31) / 32); ++w) s += cnt[w];
    *num_active = s;
  }
}

// ---------------------------------------------------------------------------
// stochastic Lanczos quadrature (§3.1): e1^T log(T) e1 = sum_j q_1j^2 log lambda_j
// for each probe's tridiagonal, by the implicit symmetric QL iteration with
// Wilkinson-type shifts (Bowdler, Martin, Reinsch & Wilkinson 1968; EISPACK
// tql1/tql2), carrying only the first row of the eigenvector matrix.
// ---------------------------------------------------------------------------
// One block per probe column (blockIdx.x + 1); the rotation chain is
// sequential, so one thread works on d, e, z held in shared memory.
static __global__ void k_slq(int c, int L, const int32_t* __restrict__ iters, const double* __restrict__ tdiag,
                      const double* __restrict__ toff, double* __restrict__ work, double* __restrict__ quads,
                      unsigned* __restrict__ err) {
  extern __shared__ double qlsh[];
  int col = 1 + blockIdx.x;   // probe columns 1..c-1
  if (col >= c || threadIdx.x != 0) return;
  (void)work;
  int k = iters[col];
  if (k <= 0) { quads[col] = 0.0; return; }
  double* d = qlsh;
  double* e = d + L;
  double* z = e + L;
  for (int i = 0; i < k; ++i) {
    d[i] = tdiag[(int64_t)col * L + i];
    e[i] = (i + 1 < k) ? toff[(int64_t)col * L + i] : 0.0;
    z[i] = (i == 0) ? 1.0 : 0.0;
  }
  for (int l = 0; l < k; ++l) {
    int it = 0;
    while (true) {
      int mm = l;
      for (; mm < k - 1; ++mm) {
        double dd = fabs(d[mm]) + fabs(d[mm + 1]);
        if (fabs(e[mm]) + dd == dd) break;
      }
      if (mm == l) break;
      if (++it > 100) { atomicOr(err, kErrNaN); break; }
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = sqrt(g * g + 1.0);
      g = d[mm] - d[l] + e[l] / (g + copysign(r, g));
      double s = 1.0, cs = 1.0, p = 0.0;
      bool deflated = false;
      for (int i = mm - 1; i >= l; --i) {
        double f = s * e[i], b = cs * e[i];
        // r = |(f, g)| and 1/r from one reciprocal square root (the FP64
        // divide and square root are long dependent chains on this path)
        const double hh = f * f + g * g;
        const double rinv = hh > 0.0 ? rsqrt(hh) : 0.0;
        r = hh * rinv;
        e[i + 1] = r;
        if (r == 0.0) {   // split: the rotation chain stops early
          d[i + 1] -= p;
          e[mm] = 0.0;
          deflated = true;
          break;
        }
        s = f * rinv;
        cs = g * rinv;
        g = d[i + 1] - p;
        r = (d[i] - g) * s + 2.0 * cs * b;
        p = s * r;
        d[i + 1] = g + p;
        g = cs * r - b;
        double zf = z[i + 1];
        z[i + 1] = s * z[i] + cs * zf;
        z[i] = cs * z[i] - s * zf;
      }
      if (deflated) continue;
      d[l] -= p;
      e[l] = g;
      e[mm] = 0.0;
    }
  }
  double q = 0.0;
  for (int j = 0; j < k; ++j) {
    if (!(d[j] > 0.0)) { atomicOr(err, kErrNaN); continue; }
    q += z[j] * z[j] * log(d[j]);
  }
  quads[col] = q;
}

// e1^T log(T) e1 for every probe column (L <= 8000 iterations)
static inline void launch_slq(int c, int L, const int32_t* iters, const double* tdiag, const double* toff,
                              double* quads, unsigned* err, cudaStream_t s) {
  static const bool attr_done =
      cudaFuncSetAttribute(k_slq, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) == cudaSuccess;
  (void)attr_done;
  if (c < 2) return;
  k_slq<<<c - 1, 32, (size_t)3 * L * sizeof(double), s>>>(c, L, iters, tdiag, toff, nullptr, quads, err);
  FSA_CHECK_LAUNCH();
}

}  // namespace fsa
