// Bandwidth-oriented block-vector kernels of the CG loop.
//
// Layout: n x ldc row-major.  Element-wise kernels run a flat grid-stride
// loop whose stride (blocks x rows-per-block x ldc) is a multiple of ldc, so
// every thread always touches the same column: loads and stores are fully
// coalesced, and each thread keeps the partial dot product of its column.
// Block partials are reduced over the block's row slots in a fixed order and
// written to part[block][col]; the per-column CG scalars then sum the nblk
// partials in a fixed order, so every dot product is bit-reproducible.
//
// The SpMM (tapered residual Sigma_s~ times the block) runs one warp per row:
// the row's column indices and values are loaded once, coalesced, into the
// lanes and broadcast with shuffles, so the gathers of neighbour rows are
// independent and several stay in flight per lane.
#pragma once
#include <algorithm>
#include <type_traits>

#include "fsa_internal.cuh"
#include "fsa_solver.cuh"
#include "fsa_tc.cuh"

namespace fsa {

template <typename T> struct VAcc { using type = double; };
template <> struct VAcc<float> { using type = float; };

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

// block reduction of per-thread column partials -> part[blockIdx.x][col]
__device__ __forceinline__ void vec_block_partials(double acc, int ldc, int rpb, double* __restrict__ red,
                                                   double* __restrict__ part) {
  red[threadIdx.x] = acc;
  __syncthreads();
  if ((int)threadIdx.x < ldc) {
    double s = 0.0;
    for (int r = 0; r < rpb; ++r) s += red[r * ldc + threadIdx.x];
    part[(int64_t)blockIdx.x * ldc + threadIdx.x] = s;
  }
}

#define FSA_VEC_BEGIN                                                          \
  extern __shared__ double red[];                                              \
  const int col = threadIdx.x % ldc;                                           \
  const int64_t row0 = (int64_t)blockIdx.x * rpb + threadIdx.x / ldc;          \
  const int64_t rstride = (int64_t)gridDim.x * rpb;                            \
  double acc = 0.0;                                                            \
  typename VAcc<T>::type sub = 0;                                              \
  int cnt = 0;

#define FSA_VEC_ACC(v)                                              \
  do {                                                              \
    sub += (v);                                                     \
    if (++cnt == 32) { acc += (double)sub; sub = 0; cnt = 0; }      \
  } while (0)

#define FSA_VEC_END                      \
  acc += (double)sub;                    \
  vec_block_partials(acc, ldc, rpb, red, part); \
  finish_scalars(step, part, ldc, c, l, q, red);

// U += a H ; R -= a V ; (X = R Dinv) ; part = ||R||^2
template <typename T>
__global__ void kv_ur_update(int64_t n, int c, int ldc, int rpb, T* __restrict__ U, T* __restrict__ R,
                             const T* __restrict__ H, const T* __restrict__ V, const T* __restrict__ Dinv,
                             T* __restrict__ X, const double* __restrict__ alpha, const int32_t* __restrict__ active,
                             double* __restrict__ part, int step, int l, CGScalars q) {
  FSA_VEC_BEGIN
  const T a = (col < c && active[col]) ? (T)alpha[col] : (T)0;
  for (int64_t i = row0; i < n; i += rstride) {
    const int64_t idx = i * ldc + col;
    if (col < c) {
      T r = R[idx];
      if (a != (T)0) {
        U[idx] = U[idx] + a * H[idx];
        r = r - a * V[idx];
        R[idx] = r;
      }
      if (X) X[idx] = r * Dinv[i];
      FSA_VEC_ACC(r * r);
    } else if (X) {
      X[idx] = (T)0;
    }
  }
  FSA_VEC_END
}

// Z = (R - S) Dinv ; part = r^T z
template <typename T>
__global__ void kv_z_update(int64_t n, int c, int ldc, int rpb, const T* __restrict__ R, const T* __restrict__ S,
                            const T* __restrict__ Dinv, T* __restrict__ Z, double* __restrict__ part, int step,
                            int l, CGScalars q) {
  FSA_VEC_BEGIN
  for (int64_t i = row0; i < n; i += rstride) {
    const int64_t idx = i * ldc + col;
    if (col < c) {
      T r = R[idx];
      T z = (r - S[idx]) * Dinv[i];
      Z[idx] = z;
      FSA_VEC_ACC(r * z);
    } else {
      Z[idx] = (T)0;
    }
  }
  FSA_VEC_END
}

// X = R Dinv
template <typename T>
__global__ void kv_row_scale(int64_t n, int c, int ldc, int rpb, const T* __restrict__ R, const T* __restrict__ Dinv,
                             T* __restrict__ X) {
  const int col = threadIdx.x % ldc;
  const int64_t row0 = (int64_t)blockIdx.x * rpb + threadIdx.x / ldc;
  const int64_t rstride = (int64_t)gridDim.x * rpb;
  for (int64_t i = row0; i < n; i += rstride) {
    const int64_t idx = i * ldc + col;
    X[idx] = col < c ? R[idx] * Dinv[i] : (T)0;
  }
}

#undef FSA_VEC_BEGIN
#undef FSA_VEC_ACC
#undef FSA_VEC_END

// V = Sigma_s~ Z + S + beta V ; H = Z + beta H ; part = h^T v
// NS 32-column slots per lane (ldc <= 32 NS); 8 warps per block.
template <typename T, typename VT, int NS>
__global__ void __launch_bounds__(256) kv_spmm_fused(int64_t n, int c, int ldc, const int64_t* __restrict__ rowptr,
                                                     const int32_t* __restrict__ colidx,
                                                     const VT* __restrict__ vals, const T* __restrict__ Z,
                                                     const T* __restrict__ S, T* __restrict__ V, T* __restrict__ H,
                                                     const double* __restrict__ beta, double* __restrict__ part,
                                                     int step, CGScalars q) {
  __shared__ double red[8][NS * 32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t nwarps = (int64_t)gridDim.x * 8;
  T b[NS];
  double dot[NS];
  typename VAcc<T>::type sub[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    int col = lane + 32 * s;
    b[s] = col < c ? (T)beta[col] : (T)0;
    dot[s] = 0.0;
    sub[s] = 0;
  }
  int cnt = 0;
  for (int64_t i = (int64_t)blockIdx.x * 8 + wib; i < n; i += nwarps) {
    const int64_t rb = rowptr[i], re = rowptr[i + 1];
    T acc[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) acc[s] = 0;
    for (int64_t base = rb; base < re; base += 32) {
      const int m = (int)((re - base) < 32 ? (re - base) : 32);
      const int myc = lane < m ? colidx[base + lane] : 0;
      const T myv = lane < m ? (T)vals[base + lane] : (T)0;
#pragma unroll 4
      for (int t = 0; t < m; ++t) {
        const int j = __shfl_sync(0xffffffffu, myc, t);
        const T v = __shfl_sync(0xffffffffu, myv, t);
        const T* zr = Z + (int64_t)j * ldc;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
          int col = lane + 32 * s;
          if (col < ldc) acc[s] += v * zr[col];
        }
      }
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      int col = lane + 32 * s;
      if (col >= ldc) continue;
      int64_t idx = i * ldc + col;
      if (col < c) {
        T v = acc[s] + S[idx] + (b[s] != (T)0 ? b[s] * V[idx] : (T)0);
        T h = Z[idx] + (b[s] != (T)0 ? b[s] * H[idx] : (T)0);
        V[idx] = v;
        H[idx] = h;
        sub[s] += h * v;
      } else {
        V[idx] = (T)0;
        H[idx] = (T)0;
      }
    }
    if (++cnt == 32) {
#pragma unroll
      for (int s = 0; s < NS; ++s) { dot[s] += (double)sub[s]; sub[s] = 0; }
      cnt = 0;
    }
  }
#pragma unroll
  for (int s = 0; s < NS; ++s) red[wib][lane + 32 * s] = dot[s] + (double)sub[s];
  __syncthreads();
  for (int col = threadIdx.x; col < ldc; col += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w][col];
    part[(int64_t)blockIdx.x * ldc + col] = t;
  }
  finish_scalars(step, part, ldc, c, 0, q, &red[0][0]);
}

// FP32 form: lane L owns columns 4L..4L+3 (ldc <= 128, ldc % 4 == 0), so one
// 16-byte load per active lane gathers a whole neighbour row.
static __global__ void __launch_bounds__(256) kv_spmm_fused_f4(int64_t n, int c, int ldc, const int64_t* __restrict__ rowptr,
                                                        const int32_t* __restrict__ colidx,
                                                        const float* __restrict__ vals, const float* __restrict__ Z,
                                                        const float* __restrict__ S, float* __restrict__ V,
                                                        float* __restrict__ H, const double* __restrict__ beta,
                                                        double* __restrict__ part, int step, CGScalars q) {
  __shared__ double red[8][128];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t nwarps = (int64_t)gridDim.x * 8;
  const int c4 = ldc >> 2;
  const bool act = lane < c4;
  const int col0 = 4 * lane;
  float b[4];
  float sub[4] = {0.f, 0.f, 0.f, 0.f};
  double dot[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int k = 0; k < 4; ++k) b[k] = (act && col0 + k < c) ? (float)beta[col0 + k] : 0.f;
  const bool use_b = (b[0] != 0.f) || (b[1] != 0.f) || (b[2] != 0.f) || (b[3] != 0.f);
  int cnt = 0;
  for (int64_t i = (int64_t)blockIdx.x * 8 + wib; i < n; i += nwarps) {
    const int64_t rb = rowptr[i], re = rowptr[i + 1];
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    // the row's own operands are loaded up front, in flight with the gathers
    const int64_t idx = i * ldc + col0;
    float4 sv = make_float4(0.f, 0.f, 0.f, 0.f), zi = sv, vv = sv, hh = sv;
    if (act) {
      sv = *reinterpret_cast<const float4*>(S + idx);
      zi = *reinterpret_cast<const float4*>(Z + idx);
      if (use_b) {
        vv = *reinterpret_cast<const float4*>(V + idx);
        hh = *reinterpret_cast<const float4*>(H + idx);
      }
    }
    for (int64_t base = rb; base < re; base += 32) {
      const int m = (int)((re - base) < 32 ? (re - base) : 32);
      const int myc = lane < m ? colidx[base + lane] : 0;
      const float myv = lane < m ? vals[base + lane] : 0.f;
#pragma unroll 8
      for (int t = 0; t < m; ++t) {
        const int j = __shfl_sync(0xffffffffu, myc, t);
        const float v = __shfl_sync(0xffffffffu, myv, t);
        if (act) {
          const float4 z = *reinterpret_cast<const float4*>(Z + (int64_t)j * ldc + col0);
          acc.x = fmaf(v, z.x, acc.x);
          acc.y = fmaf(v, z.y, acc.y);
          acc.z = fmaf(v, z.z, acc.z);
          acc.w = fmaf(v, z.w, acc.w);
        }
      }
    }
    if (act) {
      float4 vo = make_float4(acc.x + sv.x, acc.y + sv.y, acc.z + sv.z, acc.w + sv.w);
      float4 ho = zi;
      if (use_b) {
        vo.x += b[0] * vv.x; vo.y += b[1] * vv.y; vo.z += b[2] * vv.z; vo.w += b[3] * vv.w;
        ho.x += b[0] * hh.x; ho.y += b[1] * hh.y; ho.z += b[2] * hh.z; ho.w += b[3] * hh.w;
      }
      // columns >= c hold zeros in Z and S and get zero beta, so they stay zero
      *reinterpret_cast<float4*>(V + idx) = vo;
      *reinterpret_cast<float4*>(H + idx) = ho;
      sub[0] += ho.x * vo.x; sub[1] += ho.y * vo.y; sub[2] += ho.z * vo.z; sub[3] += ho.w * vo.w;
    }
    if (++cnt == 32) {
#pragma unroll
      for (int k = 0; k < 4; ++k) { dot[k] += (double)sub[k]; sub[k] = 0.f; }
      cnt = 0;
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) red[wib][(4 * lane + k) & 127] = act ? dot[k] + (double)sub[k] : 0.0;
  __syncthreads();
  for (int col = threadIdx.x; col < ldc; col += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w][col];
    part[(int64_t)blockIdx.x * ldc + col] = t;
  }
  finish_scalars(step, part, ldc, c, 0, q, &red[0][0]);
}

// FP32 form over the cell-grid tiles with shared-memory staging: a block
// copies its tile's three neighbour ranges of Z (contiguous runs of rows) and
// the tile's (staged column, value) pairs into shared memory with coalesced
// loads, then each warp runs its rows from shared memory: per nonzero one
// broadcast load of the pair, one 16-byte load of the neighbour's columns per
// lane and four FMAs (lane L owns columns 4L..4L+3).  A tile that exceeds the
// staging capacity, or holds a column outside its ranges (the cell-grid
// pattern produces none), runs the row kernel's global gathers instead.
static __global__ void __launch_bounds__(256, 3) kv_spmm_staged(
    int ntiles, const int64_t* __restrict__ tiles, const int32_t* __restrict__ tile_bad, int cap_rows, int cap_nnz,
    int cap_trows, int c, int ldc, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
    const int32_t* __restrict__ scol, const float* __restrict__ vals, const float* __restrict__ Z,
    const float* __restrict__ S, float* __restrict__ V, float* __restrict__ H, const double* __restrict__ beta,
    double* __restrict__ part, int step, CGScalars q) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int c4 = ldc >> 2;
  float4* zs = reinterpret_cast<float4*>(smraw);                               // cap_rows x c4
  int2* prs = reinterpret_cast<int2*>(smraw + (size_t)cap_rows * c4 * 16);    // cap_nnz pairs
  int* ro = reinterpret_cast<int*>(prs + cap_nnz);                             // cap_trows + 1 offsets
  __shared__ int64_t td[8];
  __shared__ int bad_sh;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  // lane -> (row slot, chunk pair): L lanes per row, R rows per warp step;
  // the lane owns float4 chunks q0 = ch and q1 = ch + L of its row, so that
  // the L lanes of a row read L consecutive 16-byte words (no bank conflicts
  // within a row)
  const int L = (c4 + 1) >> 1, R = 32 / L;
  const int slot = lane / L, ch = lane - (lane / L) * L;
  const bool lane_on = slot < R;
  const int q0 = ch, q1 = ch + L;
  const bool has1 = q1 < c4;
  const float4* Z4 = reinterpret_cast<const float4*>(Z);
  __shared__ float bsh[136];   // beta per column (0 beyond c), 8 spare for the odd-c4 chunk
  __shared__ int any_b;
  float sub[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  double dot[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  if (threadIdx.x == 0) any_b = 0;
  __syncthreads();
  for (int col = threadIdx.x; col < 136; col += blockDim.x) {
    const float bv = col < c ? (float)beta[col] : 0.f;
    bsh[col] = bv;
    if (bv != 0.f) any_b = 1;
  }
  __syncthreads();
  const bool use_b = any_b != 0;
  int cnt = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    __syncthreads();   // the previous tile's reads of shared memory are done
    if (threadIdx.x < 8) td[threadIdx.x] = tiles[(int64_t)tile * 8 + threadIdx.x];
    if (threadIdx.x == 0) bad_sh = tile_bad[tile];
    __syncthreads();
    const int64_t p0 = td[0], p1 = td[1];
    const int64_t e0 = rowptr[p0], e1 = rowptr[p1];
    const int nr = (int)(p1 - p0), ne = (int)(e1 - e0);
    const int r0b = (int)td[2], r1b = (int)td[4], r2b = (int)td[6];
    const int n0 = (int)(td[3] - td[2]), n1 = (int)(td[5] - td[4]), n2 = (int)(td[7] - td[6]);
    const bool staged = !bad_sh && n0 + n1 + n2 <= cap_rows && ne <= cap_nnz && nr <= cap_trows;
    if (staged) {
      const int x0 = n0 * c4, x1 = x0 + n1 * c4, x2 = x1 + n2 * c4;
      for (int x = threadIdx.x; x < x2; x += blockDim.x) {
        const int64_t src = x < x0 ? (int64_t)r0b * c4 + x
                                   : (x < x1 ? (int64_t)r1b * c4 + (x - x0) : (int64_t)r2b * c4 + (x - x1));
        zs[x] = Z4[src];
      }
      for (int x = threadIdx.x; x < ne; x += blockDim.x)
        prs[x] = make_int2(scol[e0 + x], __float_as_int(vals[e0 + x]));
      for (int x = threadIdx.x; x <= nr; x += blockDim.x) ro[x] = (int)(rowptr[p0 + x] - e0);
    }
    __syncthreads();
    for (int rbase = wib * R; rbase < nr; rbase += 8 * R) {
      const int r = rbase + slot;
      const bool on = lane_on && r < nr;
      const int64_t i = p0 + r;
      const int64_t i0 = i * c4;
      float4 sv0 = make_float4(0.f, 0.f, 0.f, 0.f), sv1 = sv0, zi0 = sv0, zi1 = sv0;
      if (on) {   // the row's own operand S is loaded up front, in flight with the row's products
        const float4* S4 = reinterpret_cast<const float4*>(S);
        sv0 = S4[i0 + q0];
        if (has1) sv1 = S4[i0 + q1];
      }
      float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
      if (on) {
        if (staged) {
          const int tb = ro[r], te = ro[r + 1];
          // q1 may run one chunk past the row for odd c4: it reads the next
          // staged row (in bounds: one spare row is allocated; kept off the output)
#pragma unroll 4
          for (int t = tb; t < te; ++t) {
            const int2 pv = prs[t];
            const float v = __int_as_float(pv.y);
            const float4 z0 = zs[pv.x * c4 + q0];
            const float4 z1 = zs[pv.x * c4 + q1];
            a0.x = fmaf(v, z0.x, a0.x); a0.y = fmaf(v, z0.y, a0.y);
            a0.z = fmaf(v, z0.z, a0.z); a0.w = fmaf(v, z0.w, a0.w);
            a1.x = fmaf(v, z1.x, a1.x); a1.y = fmaf(v, z1.y, a1.y);
            a1.z = fmaf(v, z1.z, a1.z); a1.w = fmaf(v, z1.w, a1.w);
          }
          const int zr = (n0 + (int)(i - r1b)) * c4;
          zi0 = zs[zr + q0];
          if (has1) zi1 = zs[zr + q1];
        } else {
          zi0 = Z4[i0 + q0];
          if (has1) zi1 = Z4[i0 + q1];
          const int64_t rb = rowptr[i], re = rowptr[i + 1];
          for (int64_t t = rb; t < re; ++t) {
            const int64_t j = colidx[t];
            const float v = vals[t];
            const float4 z0 = Z4[j * c4 + q0];
            const float4 z1 = has1 ? Z4[j * c4 + q1] : make_float4(0.f, 0.f, 0.f, 0.f);
            a0.x = fmaf(v, z0.x, a0.x); a0.y = fmaf(v, z0.y, a0.y);
            a0.z = fmaf(v, z0.z, a0.z); a0.w = fmaf(v, z0.w, a0.w);
            a1.x = fmaf(v, z1.x, a1.x); a1.y = fmaf(v, z1.y, a1.y);
            a1.z = fmaf(v, z1.z, a1.z); a1.w = fmaf(v, z1.w, a1.w);
          }
        }
        float4 vo0 = make_float4(a0.x + sv0.x, a0.y + sv0.y, a0.z + sv0.z, a0.w + sv0.w);
        float4 vo1 = make_float4(a1.x + sv1.x, a1.y + sv1.y, a1.z + sv1.z, a1.w + sv1.w);
        float4 ho0 = zi0, ho1 = zi1;
        if (use_b) {
          const float4* V4 = reinterpret_cast<const float4*>(V);
          const float4* H4 = reinterpret_cast<const float4*>(H);
          const float* b = bsh + 4 * q0;
          const float4 vv0 = V4[i0 + q0], hh0 = H4[i0 + q0];
          vo0.x += b[0] * vv0.x; vo0.y += b[1] * vv0.y; vo0.z += b[2] * vv0.z; vo0.w += b[3] * vv0.w;
          ho0.x += b[0] * hh0.x; ho0.y += b[1] * hh0.y; ho0.z += b[2] * hh0.z; ho0.w += b[3] * hh0.w;
          if (has1) {
            const float* b1 = bsh + 4 * q1;
            const float4 vv1 = V4[i0 + q1], hh1 = H4[i0 + q1];
            vo1.x += b1[0] * vv1.x; vo1.y += b1[1] * vv1.y; vo1.z += b1[2] * vv1.z; vo1.w += b1[3] * vv1.w;
            ho1.x += b1[0] * hh1.x; ho1.y += b1[1] * hh1.y; ho1.z += b1[2] * hh1.z; ho1.w += b1[3] * hh1.w;
          }
        }
        float4* Vw = reinterpret_cast<float4*>(V);
        float4* Hw = reinterpret_cast<float4*>(H);
        Vw[i0 + q0] = vo0;
        Hw[i0 + q0] = ho0;
        sub[0] += ho0.x * vo0.x; sub[1] += ho0.y * vo0.y; sub[2] += ho0.z * vo0.z; sub[3] += ho0.w * vo0.w;
        if (has1) {
          Vw[i0 + q1] = vo1;
          Hw[i0 + q1] = ho1;
          sub[4] += ho1.x * vo1.x; sub[5] += ho1.y * vo1.y; sub[6] += ho1.z * vo1.z; sub[7] += ho1.w * vo1.w;
        }
      }
      if (++cnt == 32) {
#pragma unroll
        for (int k = 0; k < 8; ++k) { dot[k] += (double)sub[k]; sub[k] = 0.f; }
        cnt = 0;
      }
    }
  }
  // fixed-order sum over the warp's row slots (lanes ch, ch + L, ...), then
  // over the 8 warps in the (now free) staging buffer
#pragma unroll
  for (int k = 0; k < 8; ++k) dot[k] += (double)sub[k];
  for (int sl = 1; sl < R; ++sl) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const double o = __shfl_sync(0xffffffffu, dot[k], (ch + sl * L) & 31);
      if (slot == 0) dot[k] += o;
    }
  }
  double* red = reinterpret_cast<double*>(smraw);
  __syncthreads();
  if (slot == 0) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int col = k < 4 ? 4 * q0 + k : 4 * q1 + (k - 4);
      if (col < 128) red[wib * 128 + col] = (col < ldc) ? dot[k] : 0.0;
    }
  }
  __syncthreads();
  for (int col = threadIdx.x; col < ldc; col += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w * 128 + col];
    part[(int64_t)blockIdx.x * ldc + col] = t;
  }
  finish_scalars(step, part, ldc, c, 0, q, red);
}

// launch shape of kv_spmm_staged for a block width: staging capacities
// (rows of Z within kStageBytes, the largest tile's nonzeros and rows) and a
// one-wave grid
struct StagedLaunch {
  int blocks = 0, cap_rows = 0, cap_nnz = 0, cap_trows = 0;
  size_t smem = 0;
};
constexpr size_t kStageBytes = 56 * 1024;
constexpr size_t kStageMaxSmem = 100 * 1024;
static inline StagedLaunch staged_launch(const Handle& Hd, int ldc) {
  static const bool attr =
      cudaFuncSetAttribute(kv_spmm_staged, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStageMaxSmem) ==
      cudaSuccess;
  (void)attr;
  StagedLaunch L;
  const int64_t cap = (int64_t)(kStageBytes / ((size_t)ldc * sizeof(float)));
  L.cap_rows = (int)std::min<int64_t>(cap, std::max<int64_t>(Hd.max_staged, 1));
  L.cap_nnz = (int)std::min<int64_t>(2048, std::max<int64_t>(Hd.max_tile_nnz, 1));
  L.cap_trows = (int)std::min<int64_t>(512, std::max<int64_t>(Hd.max_tile_rows, 1));
  size_t bytes = (size_t)(L.cap_rows + 1) * ldc * sizeof(float) + (size_t)L.cap_nnz * 8 +
                 (size_t)(L.cap_trows + 1) * 4;
  L.smem = std::max<size_t>((bytes + 15) / 16 * 16, 8 * 128 * sizeof(double));
  int dev = 0, sms = 152, per = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kv_spmm_staged, 256, L.smem);
  L.blocks = std::max(1, std::min(Hd.ntiles, sms * std::max(per, 1)));
  return L;
}

// ---------------------------------------------------------------------------
// FP32 element-wise kernels with 16-byte accesses: thread -> 4 consecutive
// columns (c4 = ldc/4 threads per row, rpb rows per block step), row loop
// unrolled so that several independent loads are in flight per thread.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void vec4_block_partials(const double (&acc)[4], int ldc, int c4, int rpb,
                                                    double* __restrict__ red, double* __restrict__ part) {
#pragma unroll
  for (int k = 0; k < 4; ++k) red[threadIdx.x * 4 + k] = acc[k];
  __syncthreads();
  for (int col = threadIdx.x; col < ldc; col += blockDim.x) {
    double s = 0.0;
    for (int r = 0; r < rpb; ++r) s += red[(r * c4 + col / 4) * 4 + (col & 3)];
    part[(int64_t)blockIdx.x * ldc + col] = s;
  }
}

// U += a H ; R -= a V ; part = ||R||^2
static __global__ void kv4_ur_update(int64_t n, int c, int ldc, int rpb, float* __restrict__ U, float* __restrict__ R,
                                     const float* __restrict__ H, const float* __restrict__ V,
                                     const double* __restrict__ alpha, const int32_t* __restrict__ active,
                                     double* __restrict__ part, int step, int l, CGScalars q) {
  extern __shared__ double red4[];
  const int c4 = ldc >> 2;
  const int cq = threadIdx.x % c4, col0 = 4 * cq;
  const int64_t row0 = (int64_t)blockIdx.x * rpb + threadIdx.x / c4;
  const int64_t rstride = (int64_t)gridDim.x * rpb;
  float a[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) a[k] = (col0 + k < c && active[col0 + k]) ? (float)alpha[col0 + k] : 0.f;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  float sub[4] = {0.f, 0.f, 0.f, 0.f};
  int cnt = 0;
#pragma unroll 4
  for (int64_t i = row0; i < n; i += rstride) {
    const int64_t idx = i * ldc + col0;
    float4 r = *reinterpret_cast<const float4*>(R + idx);
    const float4 h = *reinterpret_cast<const float4*>(H + idx);
    const float4 v = *reinterpret_cast<const float4*>(V + idx);
    float4 u = *reinterpret_cast<const float4*>(U + idx);
    u.x = fmaf(a[0], h.x, u.x); u.y = fmaf(a[1], h.y, u.y); u.z = fmaf(a[2], h.z, u.z); u.w = fmaf(a[3], h.w, u.w);
    r.x = fmaf(-a[0], v.x, r.x); r.y = fmaf(-a[1], v.y, r.y); r.z = fmaf(-a[2], v.z, r.z); r.w = fmaf(-a[3], v.w, r.w);
    *reinterpret_cast<float4*>(U + idx) = u;
    *reinterpret_cast<float4*>(R + idx) = r;
    sub[0] += r.x * r.x; sub[1] += r.y * r.y; sub[2] += r.z * r.z; sub[3] += r.w * r.w;
    if (++cnt == 32) {
#pragma unroll
      for (int k = 0; k < 4; ++k) { acc[k] += (double)sub[k]; sub[k] = 0.f; }
      cnt = 0;
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) acc[k] += (double)sub[k];
  vec4_block_partials(acc, ldc, c4, rpb, red4, part);
  finish_scalars(step, part, ldc, c, l, q, red4);
}

// Z = (R - S) Dinv ; part = r^T z
static __global__ void kv4_z_update(int64_t n, int c, int ldc, int rpb, const float* __restrict__ R,
                                    const float* __restrict__ S, const float* __restrict__ Dinv,
                                    float* __restrict__ Z, double* __restrict__ part, int step, int l, CGScalars q) {
  extern __shared__ double red4[];
  const int c4 = ldc >> 2;
  const int cq = threadIdx.x % c4, col0 = 4 * cq;
  const int64_t row0 = (int64_t)blockIdx.x * rpb + threadIdx.x / c4;
  const int64_t rstride = (int64_t)gridDim.x * rpb;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  float sub[4] = {0.f, 0.f, 0.f, 0.f};
  int cnt = 0;
#pragma unroll 4
  for (int64_t i = row0; i < n; i += rstride) {
    const int64_t idx = i * ldc + col0;
    const float4 r = *reinterpret_cast<const float4*>(R + idx);
    const float4 sv = *reinterpret_cast<const float4*>(S + idx);
    const float d = Dinv[i];
    // columns >= c hold zeros in R and S, so Z is zero there
    float4 z = make_float4((r.x - sv.x) * d, (r.y - sv.y) * d, (r.z - sv.z) * d, (r.w - sv.w) * d);
    *reinterpret_cast<float4*>(Z + idx) = z;
    sub[0] += r.x * z.x; sub[1] += r.y * z.y; sub[2] += r.z * z.z; sub[3] += r.w * z.w;
    if (++cnt == 32) {
#pragma unroll
      for (int k = 0; k < 4; ++k) { acc[k] += (double)sub[k]; sub[k] = 0.f; }
      cnt = 0;
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) acc[k] += (double)sub[k];
  vec4_block_partials(acc, ldc, c4, rpb, red4, part);
  finish_scalars(step, part, ldc, c, l, q, red4);
}

struct Vec4Launch {
  int blocks, threads, rpb;
  size_t smem;
};
static inline Vec4Launch vec4_launch(const CGLayout& lay) {
  Vec4Launch v;
  const int c4 = lay.ldc / 4;
  v.rpb = std::max(1, 256 / c4);
  v.threads = v.rpb * c4;
  v.blocks = lay.nblk;
  v.smem = (size_t)v.threads * 4 * sizeof(double);
  return v;
}

// grid of one full wave: SM count x resident blocks of the kernel
static inline int spmm_f4_blocks() {
  static const int blocks = [] {
    int dev = 0, sms = 152, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kv_spmm_fused_f4, 256, 0);
    return sms * (per > 0 ? per : 1);
  }();
  return blocks;
}

CGScalars make_scalars(Handle& H, const fsa_opts& o, int L);

// the host reads the active-column count after every iteration
inline bool should_poll(int /*it*/) { return true; }

template <typename T, typename VT>
inline void launch_spmm_fused(const CGLayout& lay, cudaStream_t s, const int64_t* rowptr, const int32_t* col,
                              const VT* vals, const T* Z, const T* S, T* V, T* H, const double* beta,
                              double* part, int step, const CGScalars& q) {
  if constexpr (std::is_same<T, float>::value && std::is_same<VT, float>::value) {
    if (lay.ldc % 4 == 0 && lay.ldc <= 128) {
      const int nb = std::min(lay.nblk, spmm_f4_blocks());
      kv_spmm_fused_f4<<<nb, 256, 0, s>>>(lay.n, lay.c, lay.ldc, rowptr, col, vals, Z, S, V, H, beta, part, step, q);
      FSA_CHECK_LAUNCH();
      return;
    }
  }
  const int ns = (lay.ldc + 31) / 32;
  switch (ns) {
    case 1: kv_spmm_fused<T, VT, 1><<<lay.nblk, 256, 0, s>>>(lay.n, lay.c, lay.ldc, rowptr, col, vals, Z, S, V, H, beta, part, step, q); break;
    case 2: kv_spmm_fused<T, VT, 2><<<lay.nblk, 256, 0, s>>>(lay.n, lay.c, lay.ldc, rowptr, col, vals, Z, S, V, H, beta, part, step, q); break;
    case 3: kv_spmm_fused<T, VT, 3><<<lay.nblk, 256, 0, s>>>(lay.n, lay.c, lay.ldc, rowptr, col, vals, Z, S, V, H, beta, part, step, q); break;
    case 4: kv_spmm_fused<T, VT, 4><<<lay.nblk, 256, 0, s>>>(lay.n, lay.c, lay.ldc, rowptr, col, vals, Z, S, V, H, beta, part, step, q); break;
    default: throw Error{FSA_ERR_UNSUPPORTED, "block of more than 128 columns"};
  }
  FSA_CHECK_LAUNCH();
}

// FP32 SpMM of the CG loop: the staged tile kernel when the handle has tiles,
// the row kernel otherwise
inline void launch_spmm_f32(const Handle& Hd, const CGLayout& lay, const StagedLaunch& L, cudaStream_t s,
                            const float* vals, const float* Z, const float* S, float* V, float* Hv,
                            const double* beta, double* part, int step, const CGScalars& q) {
  if (Hd.ntiles > 0 && lay.ldc % 4 == 0 && lay.ldc <= 128 && L.blocks > 0) {
    // timed under the profiling hooks (tag pcg_spmm); algorithmic bytes: the
    // pattern (staged column + value per nonzero, row pointers), Z and S read
    // once, V and H read and written once
    const bool prof = profile_on() && step != kStepNone;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (prof) {
      e0 = profile_event();
      e1 = profile_event();
      FSA_CUDA(cudaEventRecord(e0, s));
    }
    kv_spmm_staged<<<std::min(L.blocks, lay.nblk), 256, L.smem, s>>>(
        Hd.ntiles, Hd.tiles.p, Hd.tile_bad.p, L.cap_rows, L.cap_nnz, L.cap_trows, lay.c, lay.ldc, Hd.rowptr.p,
        Hd.col.p, Hd.scol.p, vals, Z, S, V, Hv, beta, part, step, q);
    FSA_CHECK_LAUNCH();
    if (prof) {
      FSA_CUDA(cudaEventRecord(e1, s));
      const double nb = (double)Hd.n * lay.ldc * sizeof(float);
      profile_record("pcg_spmm", e0, e1, (double)Hd.nnz * 8.0 + (double)(Hd.n + 1) * 8.0 + 6.0 * nb);
    }
    return;
  }
  launch_spmm_fused<float, float>(lay, s, Hd.rowptr.p, Hd.col.p, vals, Z, S, V, Hv, beta, part, step, q);
}

}  // namespace fsa
