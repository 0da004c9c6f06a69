// STE gradient of the log-likelihood (§3.3, Eq. NEGLLDNEGLLFSA), split per
// CG column, and the preconditioner as control variate for its trace term
// (appendix "Preconditioner as control variate", Eq. Troptc).
//
// With X = U (u = Sigma_dag^-1 y in column 0, U_k = Sigma_dag^-1 z_k) and
// Y = W (u in column 0, W_k = P_hat^-1 z_k), every parameter j has per column k
//     e_jk = X_k^T dSigma_dag/dtheta_j Y_k,
// so that e_j0 = u^T dSigma_j u is the quadratic term and e_jk (k >= 1) are the
// per-probe terms of the stochastic trace estimate of Tr(Sigma_dag^-1 dSigma_j):
//     dl/dtheta_j = -1/2 [ (1/l) sum_k e_jk - e_j0 ].
// dSigma_dag is (§2.2)
//     sigma1^2:  (Sigma_dag - nugget I) / sigma1^2     (degree-one homogeneity)
//     rho:       dSigma_s~/drho + B A~^T + A~ B^T - A~ E A~^T,
//                B = dK L^-T, E = L^-1 dSigma_m L^-T,  dSigma_s~ per nonzero
//     nugget:    I.
// The sparse parts are sums over the taper pattern, evaluated per row with one
// gather of the neighbour rows of Y for both the values and their range
// derivative (k_grad_coldots); the low-rank parts are m-space dots of the
// products A~^T X, A~^T Y, B^T X, B^T Y and E A~^T Y (k_grad_lowrank_cols).
//
// Control variate: b_jk = W_k^T dP_hat/dtheta_j W_k with
//     sigma1^2:  (z_k^T W_k - nugget |W_k|^2) / sigma1^2,
//     rho:       sum_i dD_i W_ik^2 + 2 (B^T W_k).(A~^T W_k) - (A~^T W_k)^T E (A~^T W_k),
//     nugget:    |W_k|^2,
// and Tr(P_hat^-1 dP_hat_j) through the Woodbury form P_hat^-1 =
// D^-1 - D^-1 A~ M^-1 A~^T D^-1 (M = I + A~^T D^-1 A~), with h_i = a_i M^-1 a_i^T
// and g_i = a_i M^-1 b_i^T:
//     Tr(P_hat^-1)        = sum 1/D_i - sum h_i / D_i^2
//     Tr(P_hat^-1 dP_rho) = sum dD_i/D_i - sum dD_i h_i / D_i^2 + 2 sum g_i / D_i
//                           - Tr(E) + Tr(E M^-1)
//     Tr(P_hat^-1 dP_s1)  = (n - nugget Tr(P_hat^-1)) / sigma1^2,
// the O(n m^2) cost the appendix "Runtime of the FITC preconditioner" states
// (one n x m x m product A~ M^-1 and row dots).
#include "fsa_grad.cuh"
#include "fsa_kernels.cuh"
#include "fsa_tc.cuh"
#include "fsa_vec.cuh"

namespace fsa {

constexpr int kCdWarps = 8, kCdThreads = 32 * kCdWarps, kCdPerLane = 4, kCdCols = 32 * kCdPerLane;

// per block partials part[(block * kColTerms + q) * ldc + col], columns
// [cb, cb + 128) of this launch:
//   q = 0: X_k^T Sigma_s~ Y_k     q = 1: X_k^T dSigma_s~/drho Y_k
//   q = 2: X_k^T Y_k              q = 3: Y_k^T Y_k        q = 4: sum_i dD_i Y_ik^2
// one warp per row; lane L owns columns cb + L + 32 r.  A row's gathers are
// summed in the vectors' precision (FP32 in the mixed form, as the CG's own
// SpMM), the per-row products and the sums over rows in FP64.
template <typename T, typename VT, typename DT>
__global__ void __launch_bounds__(kCdThreads) k_grad_coldots(int64_t n, int c, int ldc, int cb,
                                                              const int64_t* __restrict__ rowptr,
                                                              const int32_t* __restrict__ col,
                                                              const VT* __restrict__ vals, const DT* __restrict__ dvals,
                                                              const T* __restrict__ X, const T* __restrict__ Y,
                                                              double* __restrict__ part) {
  __shared__ double red[kCdWarps][kColTerms][kCdCols];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  double acc[kColTerms][kCdPerLane];
#pragma unroll
  for (int q = 0; q < kColTerms; ++q)
#pragma unroll
    for (int r = 0; r < kCdPerLane; ++r) acc[q][r] = 0.0;
  bool on[kCdPerLane];
#pragma unroll
  for (int r = 0; r < kCdPerLane; ++r) on[r] = cb + lane + 32 * r < c;
  const int64_t nwarps = (int64_t)gridDim.x * kCdWarps;
  for (int64_t i = (int64_t)blockIdx.x * kCdWarps + wib; i < n; i += nwarps) {
    using Acc = typename AccOf<T>::type;
    Acc ts[kCdPerLane] = {0, 0, 0, 0}, td[kCdPerLane] = {0, 0, 0, 0};
    double dDi = 0.0;
    const int64_t rb = rowptr[i], re = rowptr[i + 1];
    for (int64_t base = rb; base < re; base += 32) {
      const int cnt = (int)((re - base) < 32 ? (re - base) : 32);
      const int myj = lane < cnt ? col[base + lane] : 0;
      const Acc myv = lane < cnt ? (Acc)vals[base + lane] : (Acc)0;
      const Acc myd = lane < cnt ? (Acc)dvals[base + lane] : (Acc)0;
      for (int t = 0; t < cnt; ++t) {
        const int j = __shfl_sync(0xffffffffu, myj, t);
        const Acc v = __shfl_sync(0xffffffffu, myv, t);
        const Acc dv = __shfl_sync(0xffffffffu, myd, t);
        if (j == i) dDi = (double)dv;
        const T* yj = Y + (int64_t)j * ldc + cb + lane;
#pragma unroll
        for (int r = 0; r < kCdPerLane; ++r)
          if (on[r]) {
            const Acc y = (Acc)yj[32 * r];
            ts[r] = fma(v, y, ts[r]);
            td[r] = fma(dv, y, td[r]);
          }
      }
    }
    const T* xi = X + i * ldc + cb + lane;
    const T* yi = Y + i * ldc + cb + lane;
#pragma unroll
    for (int r = 0; r < kCdPerLane; ++r)
      if (on[r]) {
        const double x = (double)xi[32 * r], y = (double)yi[32 * r];
        acc[0][r] = fma(x, (double)ts[r], acc[0][r]);
        acc[1][r] = fma(x, (double)td[r], acc[1][r]);
        acc[2][r] = fma(x, y, acc[2][r]);
        acc[3][r] = fma(y, y, acc[3][r]);
        acc[4][r] = fma(dDi * y, y, acc[4][r]);
      }
  }
#pragma unroll
  for (int q = 0; q < kColTerms; ++q)
#pragma unroll
    for (int r = 0; r < kCdPerLane; ++r) red[wib][q][lane + 32 * r] = acc[q][r];
  __syncthreads();
  for (int t = threadIdx.x; t < kColTerms * kCdCols; t += kCdThreads) {
    const int q = t / kCdCols, cc = t % kCdCols;
    if (cb + cc >= ldc) continue;
    double s = 0.0;
    for (int w = 0; w < kCdWarps; ++w) s += red[w][q][cc];
    part[((int64_t)blockIdx.x * kColTerms + q) * ldc + cb + cc] = s;
  }
}

int coldots_blocks() {
  static const int blocks = [] {
    int dev = 0, sms = 152, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_grad_coldots<float, float, float>, kCdThreads, 0);
    return sms * (per > 0 ? per : 1);
  }();
  return blocks;
}

template <typename T, typename VT, typename DT>
void grad_coldots(Handle& H, int c, int ldc, const VT* vals, const DT* dvals, const T* X, const T* Y, double* part,
                  int nblk) {
  for (int cb = 0; cb < c; cb += kCdCols) {
    k_grad_coldots<T, VT, DT><<<nblk, kCdThreads, 0, H.stream>>>(H.n, c, ldc, cb, H.rowptr.p, H.col.p, vals, dvals,
                                                                 X, Y, part);
    FSA_CHECK_LAUNCH();
  }
}
template void grad_coldots<float, float, float>(Handle&, int, int, const float*, const float*, const float*,
                                                const float*, double*, int);
template void grad_coldots<double, double, double>(Handle&, int, int, const double*, const double*, const double*,
                                                   const double*, double*, int);

// per column k (m x ldc FP64 products):
//   lr[0][k] = (A~^T X_k).(A~^T Y_k)
//   lr[1][k] = (B^T X_k).(A~^T Y_k) + (A~^T X_k).(B^T Y_k) - (A~^T X_k).(E A~^T Y_k)
//   lr[2][k] = 2 (B^T Y_k).(A~^T Y_k) - (A~^T Y_k).(E A~^T Y_k)
__global__ void k_grad_lowrank_cols(int m, int c, int ldc, const double* __restrict__ AX,
                                    const double* __restrict__ AY, const double* __restrict__ BX,
                                    const double* __restrict__ BY, const double* __restrict__ EAY,
                                    double* __restrict__ lr) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ldc; k += gridDim.x * blockDim.x) {
    double t0 = 0.0, t1 = 0.0, t2 = 0.0;
    if (k < c)
      for (int a = 0; a < m; ++a) {
        const int64_t x = (int64_t)a * ldc + k;
        t0 += AX[x] * AY[x];
        t1 += BX[x] * AY[x] + AX[x] * BY[x] - AX[x] * EAY[x];
        t2 += 2.0 * BY[x] * AY[x] - AY[x] * EAY[x];
      }
    lr[k] = t0;
    lr[ldc + k] = t1;
    lr[2 * ldc + k] = t2;
  }
}

void grad_lowrank_cols(Handle& H, int m, int c, int ldc, const double* AX, const double* AY, const double* BX,
                       const double* BY, const double* EAY, double* lr) {
  k_grad_lowrank_cols<<<(ldc + 127) / 128, 128, 0, H.stream>>>(m, c, ldc, AX, AY, BX, BY, EAY, lr);
  FSA_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// control variate: row dots of A~ M^-1 with a_i and b_i, weighted sums
// ---------------------------------------------------------------------------
// per block partials cv[block * kCvTerms + q]:
//   q = 0: sum h_i / D_i^2    q = 1: sum dD_i h_i / D_i^2    q = 2: sum g_i / D_i
//   q = 3: sum 1 / D_i        q = 4: sum dD_i / D_i
// h_i = (A~ M^-1)_i . a_i, g_i = (A~ M^-1)_i . b_i.  Mixed form: AM row-major
// FP32 (n x m_pad); a, b BF16 hi + lo pairs in the blocked K-major layout.
constexpr int kCvWarps = 8;
__device__ __forceinline__ void cv_accumulate(int lane, double h, double g, double D, double dD, double* acc) {
  h = warp_sum(h);
  g = warp_sum(g);
  if (lane == 0) {
    const double id = 1.0 / D;
    acc[0] += h * id * id;
    acc[1] += dD * h * id * id;
    acc[2] += g * id;
    acc[3] += id;
    acc[4] += dD * id;
  }
}

__device__ __forceinline__ void cv_block_store(int lane, int wib, const double* acc, double* __restrict__ cv) {
  __shared__ double red[kCvWarps][kCvTerms];
  if (lane == 0)
    for (int q = 0; q < kCvTerms; ++q) red[wib][q] = acc[q];
  __syncthreads();
  if (threadIdx.x < kCvTerms) {
    double s = 0.0;
    for (int w = 0; w < kCvWarps; ++w) s += red[w][threadIdx.x];
    cv[(int64_t)blockIdx.x * kCvTerms + threadIdx.x] = s;
  }
}

__global__ void __launch_bounds__(32 * kCvWarps) k_cv_rowdots_mixed(
    int64_t n, int m_pad, const float* __restrict__ AM, const __nv_bfloat16* __restrict__ A,
    const __nv_bfloat16* __restrict__ Alo, const __nv_bfloat16* __restrict__ B, const __nv_bfloat16* __restrict__ Blo,
    const float* __restrict__ D32, const float* __restrict__ dD, double* __restrict__ cv) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  double acc[kCvTerms] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const int nkb = m_pad / 64;
  for (int64_t i = (int64_t)blockIdx.x * kCvWarps + wib; i < n; i += (int64_t)gridDim.x * kCvWarps) {
    float h = 0.f, g = 0.f;
    for (int kb = 0; kb < nkb; ++kb) {
      const int64_t o = ((int64_t)kb * n + i) * 64 + 2 * lane;
      const float2 am = *reinterpret_cast<const float2*>(AM + i * m_pad + kb * 64 + 2 * lane);
      const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(A + o));
      const float2 al = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(Alo + o));
      const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(B + o));
      const float2 bl = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(Blo + o));
      h = fmaf(am.x, a.x + al.x, fmaf(am.y, a.y + al.y, h));
      g = fmaf(am.x, b.x + bl.x, fmaf(am.y, b.y + bl.y, g));
    }
    cv_accumulate(lane, (double)h, (double)g, (double)D32[i], (double)dD[i], acc);
  }
  cv_block_store(lane, wib, acc, cv);
}

// FP64 form: AM, A, B row-major n x m (FP64)
__global__ void __launch_bounds__(32 * kCvWarps) k_cv_rowdots_f64(int64_t n, int m, const double* __restrict__ AM,
                                                                 const double* __restrict__ A,
                                                                 const double* __restrict__ B,
                                                                 const double* __restrict__ D,
                                                                 const double* __restrict__ dD,
                                                                 double* __restrict__ cv) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  double acc[kCvTerms] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * kCvWarps + wib; i < n; i += (int64_t)gridDim.x * kCvWarps) {
    double h = 0.0, g = 0.0;
    for (int k = lane; k < m; k += 32) {
      const double am = AM[i * m + k];
      h = fma(am, A[i * m + k], h);
      g = fma(am, B[i * m + k], g);
    }
    cv_accumulate(lane, h, g, D[i], dD[i], acc);
  }
  cv_block_store(lane, wib, acc, cv);
}

// mtr[0] = Tr(E), mtr[1] = Tr(E M^-1) = sum_ab E_ab Minv_ab (both symmetric), FP64
__global__ void k_mspace_traces(int m, const double* __restrict__ E, const double* __restrict__ Minv,
                                double* __restrict__ mtr) {
  __shared__ double red[2][256];
  double t0 = 0.0, t1 = 0.0;
  for (int64_t x = threadIdx.x; x < (int64_t)m * m; x += blockDim.x) {
    const int a = (int)(x / m), b = (int)(x % m);
    if (a == b) t0 += E[x];
    t1 += E[x] * Minv[(int64_t)b * m + a];
  }
  red[0][threadIdx.x] = t0;
  red[1][threadIdx.x] = t1;
  __syncthreads();
  if (threadIdx.x < 2) {
    double s = 0.0;
    for (int t = 0; t < (int)blockDim.x; ++t) s += red[threadIdx.x][t];
    mtr[threadIdx.x] = s;
  }
}

int cv_blocks() {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms * 4;
}

void cv_rowdots_mixed(Handle& H, int m_pad, const float* AM, const __nv_bfloat16* A, const __nv_bfloat16* Alo,
                      const __nv_bfloat16* B, const __nv_bfloat16* Blo, const float* D32, const float* dD, double* cv,
                      int nblk) {
  FSA_REQUIRE(m_pad % 64 == 0 && Alo && Blo, FSA_ERR_UNSUPPORTED, "control variate needs BF16 pairs, m_pad % 64 == 0");
  k_cv_rowdots_mixed<<<nblk, 32 * kCvWarps, 0, H.stream>>>(H.n, m_pad, AM, A, Alo, B, Blo, D32, dD, cv);
  FSA_CHECK_LAUNCH();
}

void cv_rowdots_f64(Handle& H, int m, const double* AM, const double* A, const double* B, const double* D,
                    const double* dD, double* cv, int nblk) {
  k_cv_rowdots_f64<<<nblk, 32 * kCvWarps, 0, H.stream>>>(H.n, m, AM, A, B, D, dD, cv);
  FSA_CHECK_LAUNCH();
}

void mspace_traces(Handle& H, int m, const double* E, const double* Minv, double* mtr) {
  k_mspace_traces<<<1, 256, 0, H.stream>>>(m, E, Minv, mtr);
  FSA_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// final assembly (one block): fixed-order sums of the partials, the per-probe
// terms, the control variate and the gradient
// ---------------------------------------------------------------------------
__global__ void k_grad_final(int64_t n, int c, int ldc, const double* __restrict__ part, int nblk,
                             const double* __restrict__ lr, const double* __restrict__ cv, int ncv,
                             const double* __restrict__ mtr, const double* __restrict__ rz0, double s1, double nug,
                             int cv_kind, double* __restrict__ outs, double* __restrict__ terms) {
  extern __shared__ double Et[];   // kColTerms x ldc column sums
  for (int t = threadIdx.x; t < kColTerms * ldc; t += blockDim.x) {
    const int q = t / ldc, k = t % ldc;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[((int64_t)b * kColTerms + q) * ldc + k];
    Et[t] = s;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const int l = c - 1;
  const double* Es = Et;              // X^T Sigma_s~ Y
  const double* Ed = Et + ldc;        // X^T dSigma_s~/drho Y
  const double* Exy = Et + 2 * ldc;   // X^T Y
  const double* Eyy = Et + 3 * ldc;   // Y^T Y
  const double* Edy = Et + 4 * ldc;   // sum dD Y^2
  auto e = [&](int j, int k) {
    if (j == 0) return (Es[k] + lr[k] - nug * Exy[k]) / s1;
    if (j == 1) return Ed[k] + lr[ldc + k];
    return Exy[k];
  };
  auto bterm = [&](int j, int k) {
    if (j == 0) return (rz0[k] - nug * Eyy[k]) / s1;
    if (j == 1) return Edy[k] + lr[2 * ldc + k];
    return Eyy[k];
  };
  double trP[3] = {0.0, 0.0, 0.0};
  if (cv_kind != kCvNone) {
    double S[kCvTerms] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int b = 0; b < ncv; ++b)
      for (int q = 0; q < kCvTerms; ++q) S[q] += cv[(int64_t)b * kCvTerms + q];
    const double trPinv = S[3] - S[0];
    trP[0] = ((double)n - nug * trPinv) / s1;
    trP[1] = S[4] - S[1] + 2.0 * S[2] - mtr[0] + mtr[1];
    trP[2] = trPinv;
  }
  for (int j = 0; j < 3; ++j) {
    double ma = 0.0, mb = 0.0;
    for (int k = 1; k <= l; ++k) {
      const double a = e(j, k), b = cv_kind != kCvNone ? bterm(j, k) : 0.0;
      terms[(int64_t)j * l + k - 1] = a;
      terms[(int64_t)(3 + j) * l + k - 1] = b;
      ma += a;
      mb += b;
    }
    ma /= l;
    mb /= l;
    double cc = 0.0;
    if (cv_kind == kCvOne) {
      cc = 1.0;
    } else if (cv_kind == kCvOptPrinted || cv_kind == kCvOptCentred) {
      double num = 0.0, den = 0.0;
      for (int k = 1; k <= l; ++k) {
        const double a = e(j, k), b = bterm(j, k);
        const double bb = cv_kind == kCvOptCentred ? b - mb : b;
        num += (a - ma) * bb;
        den += bb * bb;
      }
      cc = den > 0.0 ? num / den : 0.0;
    }
    const double tr = ma - cc * mb + cc * trP[j];
    const double qf = e(j, 0);
    outs[kOutGrad + j] = -0.5 * (tr - qf);
    outs[kOutTrace + j] = tr;
    outs[kOutQuad + j] = qf;
    outs[kOutTraceP + j] = trP[j];
    outs[kOutCvC + j] = cc;
  }
}

void grad_final(Handle& H, int c, int ldc, const double* part, int nblk, const double* lr, const double* cv, int ncv,
                const double* mtr, const fsa_theta& th, int cv_kind, double* terms) {
  const size_t smem = (size_t)kColTerms * ldc * sizeof(double);
  if (smem > 48 * 1024)
    FSA_CUDA(cudaFuncSetAttribute(k_grad_final, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_grad_final<<<1, 256, smem, H.stream>>>(H.n, c, ldc, part, nblk, lr, cv, ncv, mtr, H.cg.rz0.p, th.sigma1_sq,
                                           th.nugget, cv_kind, H.outs.p, terms);
  FSA_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// FP64 form: range derivative of the residual values, one warp per row
// ---------------------------------------------------------------------------
__global__ void k_dvals_f64(int64_t n, int m, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                            const double* __restrict__ xs, const double* __restrict__ ys, const double* __restrict__ A,
                            const double* __restrict__ B, const double* __restrict__ F, int cov, double s1,
                            double rho, double gamma, double* __restrict__ dvals, double* __restrict__ dD) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nwarps) {
    const double* ai = A + i * m;
    const double* bi = B + i * m;
    for (int64_t t = rowptr[i]; t < rowptr[i + 1]; ++t) {
      const int64_t j = col[t];
      const double* aj = A + j * m;
      const double* bj = B + j * m;
      const double* fj = F + j * m;
      double dl = 0.0;
      for (int k = lane; k < m; k += 32) dl += bi[k] * aj[k] + ai[k] * bj[k] - ai[k] * fj[k];
      dl = warp_sum(dl);
      if (lane == 0) {
        if (j == i) {
          dvals[t] = -dl;
          dD[i] = -dl;
        } else {
          const double d = sqrt(sqdist_rn(xs[i], ys[i], xs[j], ys[j]));
          dvals[t] = (s1 * matern_dr(cov, d, rho) - dl) * wendland(d, gamma);
        }
      }
    }
  }
}

void dvals_f64(Handle& H, const fsa_theta& th, int m, const double* A, const double* B, const double* F,
               double* dvals, double* dD) {
  k_dvals_f64<<<152 * 8, 256, 0, H.stream>>>(H.n, m, H.rowptr.p, H.col.p, H.xs.p, H.ys.p, A, B, F, H.cov,
                                             th.sigma1_sq, th.rho, H.gamma, dvals, dD);
  FSA_CHECK_LAUNCH();
}

void build_deriv_f64(Handle& H, const fsa_theta& th, DerivF64& Dv) {
  cudaStream_t s = H.stream;
  Operator& op = H.op;
  const int64_t n = H.n;
  const int m = H.m;
  Dv.B.alloc((size_t)n * m);
  Dv.F.alloc((size_t)n * m);
  Dv.E.alloc((size_t)m * m);
  {
    DevPtr<double> dK((size_t)n * m);
    cov_cross(H, n, H.xs.p, H.ys.p, m, H.ind_x.p, H.ind_y.p, th, 1, dK.p, m);
    dgemm(H.ws, s, false, true, (int)n, m, m, 1.0, dK.p, m, op.Lmi.p, m, 0.0, Dv.B.p, m, nullptr, kTriB_KleJ);
    FSA_CUDA(cudaStreamSynchronize(s));
  }
  {
    DevPtr<double> dSm((size_t)m * m), T1((size_t)m * m);
    cov_cross(H, m, H.ind_x.p, H.ind_y.p, m, H.ind_x.p, H.ind_y.p, th, 1, dSm.p, m);
    dgemm(H.ws, s, false, false, m, m, m, 1.0, op.Lmi.p, m, dSm.p, m, 0.0, T1.p, m, nullptr, kTriA_KleI);
    dgemm(H.ws, s, false, true, m, m, m, 1.0, T1.p, m, op.Lmi.p, m, 0.0, Dv.E.p, m, nullptr,
          kTriB_KleJ | kTriSymLower);
    FSA_CUDA(cudaStreamSynchronize(s));
  }
  dgemm(H.ws, s, false, false, (int)n, m, m, 1.0, op.A.p, m, Dv.E.p, m, 0.0, Dv.F.p, m, nullptr);
  Dv.dv.alloc(H.nnz);
  Dv.dD.alloc(n);
  dvals_f64(H, th, m, op.A.p, Dv.B.p, Dv.F.p, Dv.dv.p, Dv.dD.p);
}

// out0 = (out0 + T0 - nugget X) / sigma1^2; out1 += T1 + T2 (n x k blocks of leading dimension ld)
__global__ void k_dsigma_combine_f64(int64_t n, int k, int ld, double s1, double nug, const double* __restrict__ X,
                                     const double* __restrict__ T0, const double* __restrict__ T1,
                                     const double* __restrict__ T2, double* __restrict__ out0,
                                     double* __restrict__ out1) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * k; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = (t / k) * ld + t % k;
    out0[x] = (out0[x] + T0[x] - nug * X[x]) / s1;
    out1[x] = out1[x] + T1[x] + T2[x];
  }
}

void apply_dsigma_f64(Handle& H, DerivF64& Dv, const fsa_theta& th, const double* X, int k, int ldx, double* out0,
                      double* out1) {
  cudaStream_t s = H.stream;
  Operator& op = H.op;
  const int64_t n = H.n;
  const int m = H.m;
  CGLayout lay;
  lay.setup(n, k, 1);
  k_spmm<double, double><<<dim3(lay.nblk, 1), 128, 0, s>>>(n, k, ldx, lay.chunk, H.rowptr.p, H.col.p, op.vals.p, X,
                                                            out0, ldx);
  FSA_CHECK_LAUNCH();
  k_spmm<double, double><<<dim3(lay.nblk, 1), 128, 0, s>>>(n, k, ldx, lay.chunk, H.rowptr.p, H.col.p, Dv.dv.p, X,
                                                            out1, ldx);
  FSA_CHECK_LAUNCH();
  const size_t mk = (size_t)m * k, nk = (size_t)n * ldx;
  DevPtr<double> AX(mk), BX(mk), T0(nk), T1(nk), T2(nk);
  dgemm(H.ws, s, true, false, m, k, (int)n, 1.0, op.A.p, m, X, ldx, 0.0, AX.p, k, nullptr);
  dgemm(H.ws, s, true, false, m, k, (int)n, 1.0, Dv.B.p, m, X, ldx, 0.0, BX.p, k, nullptr);
  dgemm(H.ws, s, false, false, m, k, m, -1.0, Dv.E.p, m, AX.p, k, 1.0, BX.p, k, nullptr);
  dgemm(H.ws, s, false, false, (int)n, k, m, 1.0, op.A.p, m, AX.p, k, 0.0, T0.p, ldx, nullptr);
  dgemm(H.ws, s, false, false, (int)n, k, m, 1.0, op.A.p, m, BX.p, k, 0.0, T1.p, ldx, nullptr);
  dgemm(H.ws, s, false, false, (int)n, k, m, 1.0, Dv.B.p, m, AX.p, k, 0.0, T2.p, ldx, nullptr);
  k_dsigma_combine_f64<<<grid_for(n * k, 256), 256, 0, s>>>(n, k, ldx, th.sigma1_sq, th.nugget, X, T0.p, T1.p, T2.p,
                                                            out0, out1);
  FSA_CHECK_LAUNCH();
  FSA_CUDA(cudaStreamSynchronize(s));
}

}  // namespace fsa
