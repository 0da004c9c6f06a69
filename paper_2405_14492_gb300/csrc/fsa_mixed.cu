// Mixed-precision form of the FSA operator, preconditioner and block PCG.
//
//   A = Sigma_nm L_m^-T is formed on the tensor cores from hi/lo BF16 splits
//   of Sigma_nm (FP32 kernel values) and of L_m^-1 (FP64), three products
//   (hi.hi + hi.lo + lo.hi) with FP32 accumulation, then rounded once to BF16:
//   that rounded A~ DEFINES the operator Sigma_dag = Sigma_s~ + A~ A~^T, and the
//   same A~ is used in the residual values (a_i . a_j), in D_s, in the
//   Woodbury core M = I + A~^T D^-1 A~, in log det P_hat and in the probes, so
//   the preconditioner applied is the one whose log-determinant is added
//   (paper §3.3: log det Sigma = log det(P^-1/2 Sigma P^-1/2) + log det P).
//   Vector operands of the tensor-core products are split hi/lo BF16 (stacked
//   along N, summed in the epilogue) so that each product is linear in the
//   vector to ~2^-16 relative.  Vectors are FP32; CG scalars, dot-product
//   accumulation, the m x m Cholesky factors / inverse and the Lanczos
//   eigen-quadrature are FP64.
#include <memory>

#include "fsa_grad.cuh"
#include "fsa_kernels.cuh"
#include "fsa_mixed.cuh"
#include "fsa_solver.cuh"
#include "fsa_tc.cuh"
#include "fsa_vec.cuh"

namespace fsa {

// k-blocks (64 rows each) of one FP32 accumulation span of the Woodbury core
// on the tensor cores (512 rows; the spans are reduced in FP64)
constexpr int kCoreSpanBlocks = 8;
constexpr int kCoreSpans = 64;      // spans per launch
// 2^-24 |M - I|_inf above which the core is formed in FP64 (M's identity part
// would be resolved to worse than about 1e-5 by the FP32 span sums)
constexpr double kCoreFp64Above = 1e-3;
// 2^-16 sigma1 |L_m^-1|_inf above which A = Sigma_nm L_m^-T is formed in FP64:
// the split products of the tensor cores round each term of the sum to about
// 2^-16 of |k| |L_m^-1|, and a badly conditioned Sigma_m (long range, close
// inducing points) makes those terms far larger than the entries of A
constexpr double kAFp64Above = 1e-4;



// coordinates as FP32 hi/lo pairs: x = x_hi + x_lo to ~2^-48 relative
__global__ void k_coord_split(int64_t n, const double* __restrict__ xs, const double* __restrict__ ys,
                              float4* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float xh = (float)xs[i], yh = (float)ys[i];
    out[i] = make_float4(xh, (float)(xs[i] - (double)xh), yh, (float)(ys[i] - (double)yh));
  }
}

// 8 FP32 values -> their BF16 hi (and lo) pieces, packed for one 16-byte store each
__device__ __forceinline__ void split8(const float (&v)[8], uint4& h, uint4& l) {
  uint32_t wh[4], wl[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    __nv_bfloat16 h0, l0, h1, l1;
    split_bf16(v[2 * k], h0, l0);
    split_bf16(v[2 * k + 1], h1, l1);
    wh[k] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
    wl[k] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
  }
  h = make_uint4(wh[0], wh[1], wh[2], wh[3]);
  l = make_uint4(wl[0], wl[1], wl[2], wl[3]);
}

// Sigma_nm (deriv = 0) or its rho-derivative in FP32, split hi/lo BF16,
// row-major n x m_pad (columns m .. m_pad - 1 zero).  The coordinate
// differences come from the FP32 hi/lo pairs, (x_hi,i - x_hi,k) + (x_lo,i -
// x_lo,k), each within a rounding of the exact difference, so no FP64
// arithmetic is needed per element.  A thread keeps the coordinates of 8
// consecutive inducing points in registers and takes the rows blockIdx.x,
// blockIdx.x + gridDim.x, ...: one 16-byte store per piece and row.
__global__ void k_cov_nm_split(int64_t n, int m, int m_pad, const float4* __restrict__ pxy,
                               const float4* __restrict__ ixy, int cov, float s1, float rho, int deriv,
                               __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  const int k0 = 8 * (blockIdx.y * blockDim.x + threadIdx.x);
  if (k0 >= m_pad) return;
  float4 q[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) q[j] = k0 + j < m ? ixy[k0 + j] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float irho = 1.0f / rho;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    const float4 p = pxy[i];
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      float x = 0.f;
      if (k0 + j < m) {
        const float dx = (p.x - q[j].x) + (p.y - q[j].y), dy = (p.z - q[j].z) + (p.w - q[j].w);
        const float d = sqrtf(dx * dx + dy * dy);
        if (cov == 0) {
          const float e = expf(-d * irho);
          x = deriv ? s1 * (d * irho * irho) * e : s1 * e;
        } else {
          const float t = 1.7320508f * d * irho;
          const float e = expf(-t);
          x = deriv ? s1 * (t * t * irho) * e : s1 * (1.f + t) * e;
        }
      }
      v[j] = x;
    }
    uint4 h, l;
    split8(v, h, l);
    *reinterpret_cast<uint4*>(hi + i * m_pad + k0) = h;
    *reinterpret_cast<uint4*>(lo + i * m_pad + k0) = l;
  }
}

static void cov_nm_split(Handle& H, int m_pad, const fsa_theta& th, int deriv, __nv_bfloat16* hi,
                         __nv_bfloat16* lo) {
  cudaStream_t s = H.stream;
  if (!H.xy32.p || H.xy32.n < (size_t)H.n) {
    H.xy32.alloc(H.n);
    H.ixy32.alloc(H.m);
    k_coord_split<<<grid_for(H.n, 256), 256, 0, s>>>(H.n, H.xs.p, H.ys.p, H.xy32.p);
    k_coord_split<<<grid_for(H.m, 256), 256, 0, s>>>(H.m, H.ind_x.p, H.ind_y.p, H.ixy32.p);
    FSA_CHECK_LAUNCH();
  }
  FSA_REQUIRE(m_pad % 8 == 0, FSA_ERR_ARG, "inducing-point padding must be a multiple of 8");
  const int chunks = m_pad / 8, threads = std::min(256, (chunks + 31) / 32 * 32);
  const unsigned gy = (unsigned)((chunks + threads - 1) / threads);
  dim3 grid((unsigned)std::min<int64_t>(H.n, (int64_t)152 * 16 * 256 / threads), gy);
  k_cov_nm_split<<<grid, threads, 0, s>>>(H.n, H.m, m_pad, H.xy32.p, H.ixy32.p, H.cov, (float)th.sigma1_sq,
                                          (float)th.rho, deriv, hi, lo);
  FSA_CHECK_LAUNCH();
}

// FP64 rows x cols (ld) -> BF16 hi/lo rows_pad x cols_pad (zero padded)
__global__ void k_split_f64(int rows, int cols, const double* __restrict__ src, int64_t lds, int rows_pad,
                            int cols_pad, __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  int64_t total = (int64_t)rows_pad * cols_pad;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int r = (int)(t / cols_pad), c = (int)(t % cols_pad);
    double v = (r < rows && c < cols) ? src[(int64_t)r * lds + c] : 0.0;
    __nv_bfloat16 h = __double2bfloat16(v);
    hi[t] = h;
    lo[t] = __double2bfloat16(v - (double)__bfloat162float(h));
  }
}

// a BF16 pair (hi + lo, lo optional) of element pair k as two FP32 values
__device__ __forceinline__ float2 ld_pair(const __nv_bfloat162* hi, const __nv_bfloat162* lo, int k) {
  float2 a = __bfloat1622float2(hi[k]);
  if (lo) {
    float2 b = __bfloat1622float2(lo[k]);
    a.x += b.x;
    a.y += b.y;
  }
  return a;
}

// src (n x m_pad FP32, row-major) -> its BF16 pieces in the blocked K-major
// layout of both orientations: hi/lo with rows n and K = m_pad (the A operand
// of A~ q) and hiT/loT with rows m_pad and K = n_pad (the A operand of A~^T X),
// the points n .. n_pad - 1 of the latter written as zeros; lo = loT = nullptr
// writes the single rounded piece.  Persistent: a block takes 64 x 64 tiles in
// turn.  16-byte loads of the rows; the row-major pieces are written from
// registers, the tile goes through shared memory (row stride 65 words) for the
// transposed ones (a thread: 8 consecutive points of one column, one 16-byte
// store per piece).
constexpr int kSBT = 64;
__global__ void __launch_bounds__(256) k_split_both(int64_t n, int m_pad, int64_t n_pad, const float* __restrict__ src,
                                                    __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                                                    __nv_bfloat16* __restrict__ hiT, __nv_bfloat16* __restrict__ loT) {
  __shared__ float tf[kSBT][kSBT + 1];
  const int ktiles = m_pad / kSBT;
  const int64_t ntiles = (n_pad / kSBT) * ktiles;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t rt = t / ktiles;
    const int kt = (int)(t - rt * ktiles);
    const int64_t r0 = rt * kSBT;
    const int k0 = kt * kSBT;
    for (int f = threadIdx.x; f < kSBT * 8; f += blockDim.x) {
      const int rr = f >> 3, q = f & 7;   // row rr, columns 8q .. 8q + 7 of the tile
      const int64_t r = r0 + rr;
      float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (r < n) {
        const float4 a = *reinterpret_cast<const float4*>(src + r * m_pad + k0 + 8 * q);
        const float4 b = *reinterpret_cast<const float4*>(src + r * m_pad + k0 + 8 * q + 4);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
        uint4 h, l;
        split8(v, h, l);
        const int64_t d = blocked_index(r, k0 + 8 * q, n);
        if (lo) {
          *reinterpret_cast<uint4*>(hi + d) = h;
          *reinterpret_cast<uint4*>(lo + d) = l;
        } else {
          uint32_t w[4];
#pragma unroll
          for (int k = 0; k < 4; ++k)
            w[k] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v[2 * k])) |
                   ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v[2 * k + 1])) << 16);
          *reinterpret_cast<uint4*>(hi + d) = make_uint4(w[0], w[1], w[2], w[3]);
        }
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) tf[rr][8 * q + k] = v[k];
    }
    __syncthreads();
    for (int f = threadIdx.x; f < kSBT * 8; f += blockDim.x) {
      const int g = f & 7, kk = f >> 3;   // column kk, points 8g .. 8g + 7 of the tile
      float v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = tf[8 * g + k][kk];
      const int64_t d = blocked_index(k0 + kk, r0 + 8 * g, m_pad);
      if (loT) {
        uint4 h, l;
        split8(v, h, l);
        *reinterpret_cast<uint4*>(hiT + d) = h;
        *reinterpret_cast<uint4*>(loT + d) = l;
      } else {
        uint32_t w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
          w[k] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v[2 * k])) |
                 ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v[2 * k + 1])) << 16);
        *reinterpret_cast<uint4*>(hiT + d) = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
    __syncthreads();   // the tile is rewritten by the next one
  }
}

// one full wave of k_split_both (SM count x resident blocks)
static int split_both_blocks(int64_t ntiles) {
  static const int wave = [] {
    int dev = 0, sms = 152, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_split_both, 256, 0) != cudaSuccess) {
      cudaGetLastError();
      per = 0;
    }
    return sms * std::max(per, 1);
  }();
  return (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, wave));
}

// residual values from the BF16 A~ (FP32 products of BF16 values are exact;
// FP32 accumulation), values kept in FP64 and FP32; D rounded to FP32 once so
// that every consumer sees the same diagonal
__global__ void k_csr_values_mixed(int64_t n, int m_pad, const int64_t* __restrict__ rowptr,
                                   const int32_t* __restrict__ col, const double* __restrict__ xs,
                                   const double* __restrict__ ys, const __nv_bfloat16* __restrict__ A,
                                   const __nv_bfloat16* __restrict__ Alo, int cov,
                                   double s1, double rho, double nug, double gamma, double* __restrict__ vals,
                                   float* __restrict__ vals32, double* __restrict__ D, float* __restrict__ D32,
                                   float* __restrict__ Dinv32) {
  int lane = threadIdx.x & 31;
  int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int np2 = m_pad / 2;
  // A~ (and its low half) in the blocked K-major layout: pair k of row i is
  // pair (k & 31) of 64-element block k >> 5 at ((k >> 5) n + i) 64
  const __nv_bfloat162* A2 = reinterpret_cast<const __nv_bfloat162*>(A);
  const __nv_bfloat162* A2l = Alo ? reinterpret_cast<const __nv_bfloat162*>(Alo) : nullptr;
  for (int64_t i = warp; i < n; i += nwarps) {
    double xi = xs[i], yi = ys[i];
    for (int64_t t = rowptr[i]; t < rowptr[i + 1]; ++t) {
      int j = col[t];
      float s = 0.f;
      for (int k = lane; k < np2; k += 32) {
        const int64_t bi = ((int64_t)(k >> 5) * n + i) * 32 + (k & 31);
        const int64_t bj = ((int64_t)(k >> 5) * n + j) * 32 + (k & 31);
        float2 a = ld_pair(A2 + bi, A2l ? A2l + bi : nullptr, 0);
        float2 b = ld_pair(A2 + bj, A2l ? A2l + bj : nullptr, 0);
        s = fmaf(a.x, b.x, s);
        s = fmaf(a.y, b.y, s);
      }
      s = warp_sum(s);
      if (lane == 0) {
        double v;
        if (j == i) {
          float dv = (float)(fmax(s1 - (double)s, 0.0) + nug);
          v = (double)dv;
          D[i] = v;
          D32[i] = dv;
          Dinv32[i] = 1.0f / dv;
        } else {
          double d = sqrt(sqdist_rn(xi, yi, xs[j], ys[j]));
          v = (s1 * matern_r(cov, d, rho) - (double)s) * wendland(d, gamma);
        }
        vals[t] = v;
        vals32[t] = (float)v;
      }
    }
  }
}

// Y^T = (D^-1 A~)^T split hi/lo, from A~^T (m_pad x n_pad)
// (all four in the blocked K-major layout: element t holds point (t / (64 m_pad)) 64 + t % 64);
// a thread takes 8 consecutive elements (8 consecutive points of one row)
__global__ void k_scale_cols_split(int m_pad, int64_t n, int64_t n_pad, const __nv_bfloat16* __restrict__ At,
                                   const __nv_bfloat16* __restrict__ At_lo, const float* __restrict__ Dinv,
                                   __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  const int64_t total8 = (int64_t)m_pad * n_pad / 8;
  for (int64_t t8 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t8 < total8;
       t8 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = 8 * t8;
    const int64_t i = (t / (64 * (int64_t)m_pad)) * 64 + (t & 63);
    const uint4 ah = *reinterpret_cast<const uint4*>(At + t);
    uint4 al = make_uint4(0u, 0u, 0u, 0u);
    if (At_lo) al = *reinterpret_cast<const uint4*>(At_lo + t);
    const uint32_t wh[4] = {ah.x, ah.y, ah.z, ah.w}, wl[4] = {al.x, al.y, al.z, al.w};
    float v[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float a0 = __uint_as_float(wh[k] << 16) + (At_lo ? __uint_as_float(wl[k] << 16) : 0.f);
      const float a1 = __uint_as_float(wh[k] & 0xffff0000u) + (At_lo ? __uint_as_float(wl[k] & 0xffff0000u) : 0.f);
      v[2 * k] = i + 2 * k < n ? a0 * Dinv[i + 2 * k] : 0.f;
      v[2 * k + 1] = i + 2 * k + 1 < n ? a1 * Dinv[i + 2 * k + 1] : 0.f;
    }
    uint4 h, l;
    split8(v, h, l);
    *reinterpret_cast<uint4*>(hi + t) = h;
    *reinterpret_cast<uint4*>(lo + t) = l;
  }
}

__global__ void k_f32_to_f64(int64_t n, const float* __restrict__ src, double* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (double)src[i];
}

__global__ void k_f64_to_f32(int64_t n, const double* __restrict__ src, float* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

// out[0] = max_r sum_c |L_rc| (the infinity norm of an m x m matrix), one block
__global__ void k_inf_norm(int m, const double* __restrict__ L, double* __restrict__ out) {
  __shared__ double red[256];
  double mx = 0.0;
  for (int r = threadIdx.x; r < m; r += blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < m; ++c) s += fabs(L[(int64_t)r * m + c]);
    mx = fmax(mx, s);
  }
  red[threadIdx.x] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int t = 0; t < (int)blockDim.x; ++t) v = fmax(v, red[t]);
    out[0] = v;
  }
}

__global__ void k_set_identity(int m, double* __restrict__ M) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)m * m;
       t += (int64_t)gridDim.x * blockDim.x)
    M[t] = (t / m == t % m) ? 1.0 : 0.0;
}

// out[0] = max_r sum_c |M_rc - [r == c]|  (the infinity norm of M - I), one block
__global__ void k_core_norm(int m, const double* __restrict__ M, double* __restrict__ out) {
  __shared__ double red[256];
  double mx = 0.0;
  for (int r = threadIdx.x; r < m; r += blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < m; ++c) s += fabs(M[(int64_t)r * m + c] - (r == c ? 1.0 : 0.0));
    mx = fmax(mx, s);
  }
  red[threadIdx.x] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int t = 0; t < (int)blockDim.x; ++t) v = fmax(v, red[t]);
    out[0] = v;
  }
}

// A (FP64, n x m row-major) = the BF16 pair (hi + lo, blocked K-major, m_pad columns)
__global__ void k_pair_to_f64(int64_t n, int m, const __nv_bfloat16* __restrict__ hi,
                              const __nv_bfloat16* __restrict__ lo, double* __restrict__ A) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * m; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / m;
    const int k = (int)(t - i * m);
    const int64_t b = blocked_index(i, k, n);
    A[t] = (double)__bfloat162float(hi[b]) + (lo ? (double)__bfloat162float(lo[b]) : 0.0);
  }
}

// out[r][c] = sum_s part[s][r][c] (+1 on the diagonal), FP64; with mirror,
// the entries above the diagonal are read from below it (symmetric products
// whose upper tiles were not computed)
__global__ void k_reduce_splits(int splits, int rows, int cols, const float* __restrict__ part, int64_t ldp,
                                int64_t split_stride, double* __restrict__ out, int64_t ldo, int add_identity,
                                int accumulate = 0, int mirror = 0) {
  int64_t total = (int64_t)rows * cols;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int r = (int)(t / cols), c = (int)(t % cols);
    double s = accumulate ? out[(int64_t)r * ldo + c] : ((add_identity && r == c) ? 1.0 : 0.0);
    const int pr = mirror && c > r ? c : r, pc = mirror && c > r ? r : c;
    for (int z = 0; z < splits; ++z) s += (double)part[(int64_t)z * split_stride + (int64_t)pr * ldp + pc];
    out[(int64_t)r * ldo + c] = s;
  }
}

// v = sum of nsplit BF16 pieces (2: ~16 significant bits, 3: the full FP32 24);
// FP32 arithmetic (the pieces of an FP32 value are exact differences)
__device__ __forceinline__ void split_n(float v, int nsplit, __nv_bfloat16* out) {
  __nv_bfloat16 h = __float2bfloat16_rn(v);
  out[0] = h;
  float r = v - __bfloat162float(h);
  __nv_bfloat16 mid = __float2bfloat16_rn(r);
  out[1] = mid;
  if (nsplit == 3) out[2] = __float2bfloat16_rn(r - __bfloat162float(mid));
}

// src (n x ldc FP32) optionally scaled by rowscale -> dst (nsplit ldc x n_pad BF16,
// blocked K-major layout): plane p (rows p ldc .. p ldc + ldc - 1) holds the
// p-th BF16 piece; K = the point index, for the B operand of A^T X.  A block transposes a tile
// of kSTRows points: coalesced 16-byte loads of the FP32 rows into shared
// memory (row stride ldc + 1 words against bank conflicts), then each thread
// splits 8 consecutive points of one column and writes each piece as one
// 16-byte store (8 threads cover 128 contiguous bytes of a column).
constexpr int kSTRows = 64;
__global__ void __launch_bounds__(256) k_split_transpose(int64_t n, int c, int ldc, int nsplit,
                                                         const float* __restrict__ src,
                                                         const float* __restrict__ rowscale, int64_t n_pad,
                                                         __nv_bfloat16* __restrict__ dst) {
  extern __shared__ float tf[];   // [kSTRows][ldc + 1] then rowscale[kSTRows]
  const int ls = ldc + 1;
  float* rs = tf + kSTRows * ls;
  const int64_t r0 = (int64_t)blockIdx.x * kSTRows;
  const int c4 = ldc >> 2;
  for (int t = threadIdx.x; t < kSTRows * c4; t += blockDim.x) {
    const int rr = t / c4, q = t - (t / c4) * c4;
    const int64_t r = r0 + rr;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r < n) v = *reinterpret_cast<const float4*>(src + r * ldc + 4 * q);
    float* d = tf + rr * ls + 4 * q;
    d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
  }
  for (int t = threadIdx.x; t < kSTRows; t += blockDim.x) {
    const int64_t r = r0 + t;
    rs[t] = (r < n) ? (rowscale ? rowscale[r] : 1.f) : 0.f;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < ldc * (kSTRows / 8); t += blockDim.x) {
    const int g = t & 7, cc = t >> 3;
    if (r0 + 8 * g >= n_pad) continue;
    uint32_t w[3][4];   // 8 BF16 per piece, packed in pairs
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
      __nv_bfloat16 e[3], o[3];
      const float ve = cc < c ? tf[(8 * g + k) * ls + cc] * rs[8 * g + k] : 0.f;
      const float vo = cc < c ? tf[(8 * g + k + 1) * ls + cc] * rs[8 * g + k + 1] : 0.f;
      split_n(ve, nsplit, e);
      split_n(vo, nsplit, o);
      if (nsplit != 3) { e[2] = e[1]; o[2] = o[1]; }
#pragma unroll
      for (int p = 0; p < 3; ++p)
        w[p][k / 2] = (uint32_t)__bfloat16_as_ushort(e[p]) | ((uint32_t)__bfloat16_as_ushort(o[p]) << 16);
    }
    // blocked K-major output: this tile is K block blockIdx.x, rows p ldc + cc
    const int64_t ns = (int64_t)nsplit * ldc;
    const int64_t base = ((int64_t)blockIdx.x * ns + cc) * 64 + 8 * g;
    *reinterpret_cast<uint4*>(dst + base) = make_uint4(w[0][0], w[0][1], w[0][2], w[0][3]);
    *reinterpret_cast<uint4*>(dst + base + (int64_t)ldc * 64) = make_uint4(w[1][0], w[1][1], w[1][2], w[1][3]);
    if (nsplit == 3)
      *reinterpret_cast<uint4*>(dst + base + (int64_t)2 * ldc * 64) = make_uint4(w[2][0], w[2][1], w[2][2], w[2][3]);
  }
}

// One CG step's U += a H, R -= a V and ||R||^2 (as kv4_ur_update, with the
// kStepResid scalar step) fused with the split of D^-1 R into the blocked
// K-major BF16 pieces of the next A~^T X (as k_split_transpose, bit for bit):
// the block keeps its tile of updated R rows in shared memory for the
// transpose, so R is read once per iteration instead of twice.  Persistent:
// the blocks take the kSTRows-point tiles in turn.  rpb x c4 threads (c4 =
// ldc / 4); a thread keeps one float4 column chunk and takes the tile rows
// tid / c4 + k rpb, two at a time with both rows' loads issued first.
__global__ void __launch_bounds__(256, 4) k_ur_split(int64_t n, int c, int ldc, int rpb, int nsplit, int64_t n_pad,
                                                  float* __restrict__ U, float* __restrict__ R,
                                                  const float* __restrict__ Hm, const float* __restrict__ V,
                                                  const float* __restrict__ rowscale,
                                                  const double* __restrict__ alpha, const int32_t* __restrict__ active,
                                                  __nv_bfloat16* __restrict__ dst, double* __restrict__ part,
                                                  int step, int l, CGScalars q) {
  extern __shared__ __align__(16) unsigned char ursm[];
  float* tf = reinterpret_cast<float*>(ursm);   // [kSTRows][ldc + 1] then rowscale[kSTRows]
  const int ls = ldc + 1;
  float* rs = tf + kSTRows * ls;
  const int c4 = ldc >> 2;
  const int cq = threadIdx.x % c4, col0 = 4 * cq, rr0 = threadIdx.x / c4;
  float a[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) a[k] = (col0 + k < c && active[col0 + k]) ? (float)alpha[col0 + k] : 0.f;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  float sub[4] = {0.f, 0.f, 0.f, 0.f};
  int cnt = 0;
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  // updated row -> U, R in global memory, R into the tile, its squares into sub
  auto urow = [&](float4 r, const float4 h, const float4 v, float4 u, const int64_t idx, float* trow) {
    u.x = fmaf(a[0], h.x, u.x); u.y = fmaf(a[1], h.y, u.y); u.z = fmaf(a[2], h.z, u.z); u.w = fmaf(a[3], h.w, u.w);
    r.x = fmaf(-a[0], v.x, r.x); r.y = fmaf(-a[1], v.y, r.y); r.z = fmaf(-a[2], v.z, r.z); r.w = fmaf(-a[3], v.w, r.w);
    *reinterpret_cast<float4*>(U + idx) = u;
    *reinterpret_cast<float4*>(R + idx) = r;
    sub[0] += r.x * r.x; sub[1] += r.y * r.y; sub[2] += r.z * r.z; sub[3] += r.w * r.w;
    trow[0] = r.x; trow[1] = r.y; trow[2] = r.z; trow[3] = r.w;
  };
  auto zrow = [&](float* trow) { trow[0] = 0.f; trow[1] = 0.f; trow[2] = 0.f; trow[3] = 0.f; };
  const int64_t ntiles = (n_pad + kSTRows - 1) / kSTRows;
  const int64_t ns = (int64_t)nsplit * ldc;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t r0 = t * kSTRows;
    for (int rr = rr0; rr < kSTRows; rr += 2 * rpb) {
      const int rb = rr + rpb;
      const int64_t ra_i = r0 + rr, rb_i = r0 + rb;
      const bool va = ra_i < n, vb = rb < kSTRows && rb_i < n;
      const int64_t ia = ra_i * ldc + col0, ib = rb_i * ldc + col0;
      float4 ra = zero4, ha = zero4, vva = zero4, ua = zero4, rbv = zero4, hb = zero4, vvb = zero4, ub = zero4;
      if (va) {
        ra = *reinterpret_cast<const float4*>(R + ia);
        ha = *reinterpret_cast<const float4*>(Hm + ia);
        vva = *reinterpret_cast<const float4*>(V + ia);
        ua = *reinterpret_cast<const float4*>(U + ia);
      }
      if (vb) {
        rbv = *reinterpret_cast<const float4*>(R + ib);
        hb = *reinterpret_cast<const float4*>(Hm + ib);
        vvb = *reinterpret_cast<const float4*>(V + ib);
        ub = *reinterpret_cast<const float4*>(U + ib);
      }
      if (va) urow(ra, ha, vva, ua, ia, tf + rr * ls + col0);
      else zrow(tf + rr * ls + col0);
      if (vb) urow(rbv, hb, vvb, ub, ib, tf + rb * ls + col0);
      else if (rb < kSTRows) zrow(tf + rb * ls + col0);
      if (++cnt == 16) {
#pragma unroll
        for (int k = 0; k < 4; ++k) { acc[k] += (double)sub[k]; sub[k] = 0.f; }
        cnt = 0;
      }
    }
    for (int k = threadIdx.x; k < kSTRows; k += blockDim.x) {
      const int64_t r = r0 + k;
      rs[k] = (r < n) ? (rowscale ? rowscale[r] : 1.f) : 0.f;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < ldc * (kSTRows / 8); k += blockDim.x) {
      const int g = k & 7, cc = k >> 3;
      if (r0 + 8 * g >= n_pad) continue;
      uint32_t w[3][4];   // 8 BF16 per piece, packed in pairs
#pragma unroll
      for (int j = 0; j < 8; j += 2) {
        __nv_bfloat16 e[3], o[3];
        const float ve = cc < c ? tf[(8 * g + j) * ls + cc] * rs[8 * g + j] : 0.f;
        const float vo = cc < c ? tf[(8 * g + j + 1) * ls + cc] * rs[8 * g + j + 1] : 0.f;
        split_n(ve, nsplit, e);
        split_n(vo, nsplit, o);
        if (nsplit != 3) { e[2] = e[1]; o[2] = o[1]; }
#pragma unroll
        for (int p = 0; p < 3; ++p)
          w[p][j / 2] = (uint32_t)__bfloat16_as_ushort(e[p]) | ((uint32_t)__bfloat16_as_ushort(o[p]) << 16);
      }
      const int64_t base = (t * ns + cc) * 64 + 8 * g;
      *reinterpret_cast<uint4*>(dst + base) = make_uint4(w[0][0], w[0][1], w[0][2], w[0][3]);
      *reinterpret_cast<uint4*>(dst + base + (int64_t)ldc * 64) = make_uint4(w[1][0], w[1][1], w[1][2], w[1][3]);
      if (nsplit == 3)
        *reinterpret_cast<uint4*>(dst + base + (int64_t)2 * ldc * 64) = make_uint4(w[2][0], w[2][1], w[2][2], w[2][3]);
    }
    __syncthreads();   // the tile buffer is rewritten by the next tile
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) acc[k] += (double)sub[k];
  double* red4 = reinterpret_cast<double*>(ursm);   // the tile buffer is free now
  vec4_block_partials(acc, ldc, c4, rpb, red4, part);
  finish_scalars(step, part, ldc, c, l, q, red4);
}

// q (m x ldc FP64) -> (nsplit ldc x m_pad) BF16 pieces, K-major (q transposed)
__global__ void k_split_q(int m, int c, int ldc, int nsplit, int m_pad, const double* __restrict__ q,
                          __nv_bfloat16* __restrict__ dst) {
  int64_t total = (int64_t)ldc * m_pad;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int cc = (int)(t / m_pad), k = (int)(t % m_pad);
    float v = (cc < c && k < m) ? (float)q[(int64_t)k * ldc + cc] : 0.f;
    __nv_bfloat16 pc[3];
    split_n(v, nsplit, pc);
    for (int p = 0; p < nsplit; ++p) dst[(int64_t)(p * ldc + cc) * m_pad + k] = pc[p];
  }
}

// eps1^T (l16 x m_pad) hi/lo BF16 (Rademacher values are exact in BF16)
__global__ void k_eps1_split(int m, int l, int l16, int m_pad, int kind, uint64_t key, __nv_bfloat16* __restrict__ hi,
                             __nv_bfloat16* __restrict__ lo) {
  int64_t total = (int64_t)l16 * m_pad;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int p = (int)(t / m_pad), k = (int)(t % m_pad);
    float v = (p < l && k < m) ? (float)probe_at(kind, key, (uint64_t)p * m + k) : 0.f;
    split_bf16(v, hi[t], lo[t]);
  }
}

// R[:,0] = y; R[:,1+p] = (A~ eps1)[:,p] + sqrt(D_i) eps2
__global__ void k_probe_finish_mixed(int64_t n, int l, int ldc, int ldz, int kind, uint64_t key,
                                     const int64_t* __restrict__ perm, const double* __restrict__ y_int,
                                     const float* __restrict__ D32, const float* __restrict__ Zp,
                                     float* __restrict__ R) {
  int64_t total = n * ldc;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = t / ldc;
    int c = (int)(t - i * ldc);
    float v = 0.f;
    if (c == 0) v = (float)y_int[i];
    else if (c <= l)
      v = (float)((double)Zp[i * ldz + (c - 1)] +
                  sqrt((double)D32[i]) * probe_at(kind, key, (uint64_t)(c - 1) * n + perm[i]));
    R[t] = v;
  }
}

// values of the SpMM row groups' union entries (one block per tile): entry
// word 0 the staged column, word 1 + g the FP32 value of the group's row g in
// that column (bits), or 0 where the column is not one of its neighbours
__global__ void k_grp_values(const int32_t* __restrict__ ptile, const int4* __restrict__ src,
                             const float* __restrict__ vals32, int4* __restrict__ ent, unsigned* __restrict__ err) {
  const int t = blockIdx.x;
  const int32_t* rec = ptile + (int64_t)t * kTileWords;
  if (rec[15]) return;   // bad tile: no union entries
  const int64_t e0 = (int64_t)(uint32_t)rec[8] | ((int64_t)rec[9] << 32);
  const int64_t eb = (int64_t)(uint32_t)rec[12] | ((int64_t)rec[13] << 32);
  const int ne = rec[14], tnnz = rec[10];
  auto val = [&](int r) {
    if (r < 0) return 0;
    if (!FSA_INDEX_OK(r < tnnz, err)) return 0;   // a source inside the tile's nonzeros (checked build)
    return __float_as_int(vals32[e0 + r]);
  };
  for (int i = threadIdx.x; i < ne; i += blockDim.x) {
    const int64_t x = kEntVec * (eb + i);
    const int4 a = src[x];
    ent[x] = make_int4(a.x, val(a.y), val(a.z), val(a.w));
    if (kEntVec == 2) {
      const int4 b = src[x + 1];
      ent[x + 1] = make_int4(val(b.x), val(b.y), val(b.z), val(b.w));
    }
  }
}

// hi + lo BF16 pair of a - b (FP32 rows x cols, row-major), in the blocked
// K-major layout with K = the column; a thread takes 8 consecutive columns
// (cols a multiple of 8)
__global__ void k_sub_split(int64_t rows, int cols, const float* __restrict__ a, const float* __restrict__ b,
                            __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  const int64_t total8 = rows * cols / 8;
  for (int64_t t8 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t8 < total8;
       t8 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = 8 * t8;
    const int64_t r = t / cols;
    const int k = (int)(t - r * cols);
    const float4 a0 = *reinterpret_cast<const float4*>(a + t), a1 = *reinterpret_cast<const float4*>(a + t + 4);
    const float4 b0 = *reinterpret_cast<const float4*>(b + t), b1 = *reinterpret_cast<const float4*>(b + t + 4);
    const float v[8] = {a0.x - b0.x, a0.y - b0.y, a0.z - b0.z, a0.w - b0.w,
                        a1.x - b1.x, a1.y - b1.y, a1.z - b1.z, a1.w - b1.w};
    uint4 h, l;
    split8(v, h, l);
    const int64_t d = blocked_index(r, k, rows);
    *reinterpret_cast<uint4*>(hi + d) = h;
    *reinterpret_cast<uint4*>(lo + d) = l;
  }
}

__device__ __forceinline__ float dot8_bf16(const uint4& x, const uint4& y) {
  const __nv_bfloat162* a = reinterpret_cast<const __nv_bfloat162*>(&x);
  const __nv_bfloat162* b = reinterpret_cast<const __nv_bfloat162*>(&y);
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    float2 u = __bfloat1622float2(a[k]), v = __bfloat1622float2(b[k]);
    s = fmaf(u.x, v.x, s);
    s = fmaf(u.y, v.y, s);
  }
  return s;
}

void csr_values_rows(Handle& H, const fsa_theta& th, const __nv_bfloat16* A, const __nv_bfloat16* Alo, int m_pad) {
  Operator& op = H.op;
  k_csr_values_mixed<<<grid_for(H.n * 32, 256, 152 * 64), 256, 0, H.stream>>>(
      H.n, m_pad, H.rowptr.p, H.col.p, H.xs.p, H.ys.p, A, Alo, H.cov, th.sigma1_sq, th.rho, th.nugget, H.gamma,
      op.vals.p, op.vals32.p, op.D.p, op.D32.p, op.Dinv32.p);
  FSA_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// operator build
// ---------------------------------------------------------------------------
static inline int round_up(int v, int a) { return (v + a - 1) / a * a; }

__global__ void k_f64_to_f32_pad(int64_t n, int k, int ldk, const double* __restrict__ src, float* __restrict__ dst);

void build_operator_mixed(Handle& H, const fsa_theta& th, int precision) {
  Operator& op = H.op;
  cudaStream_t s = H.stream;
  int64_t n = H.n;
  int m = H.m;
  int m_pad = round_up(m, 64);
  int64_t n_pad = ((n + 63) / 64) * 64;
  const bool lo = precision == FSA_MIXED_BF16X2;
  op.m_pad = m_pad;
  op.n_pad = n_pad;
  op.has_lo = lo;
  build_mspace(H, th);
  size_t nm = (size_t)n * m_pad;
  // A = Sigma_nm L^-T with the split products, rounded once to BF16 (or a BF16 hi + lo pair)
  {
    DevPtr<__nv_bfloat16> Khi(nm), Klo(nm), Lhi((size_t)m_pad * m_pad), Llo((size_t)m_pad * m_pad);
    DevPtr<float> A32(nm);
    {
      DevPtr<double> nrm(1);
      k_inf_norm<<<1, 256, 0, s>>>(m, op.Lmi.p, nrm.p);
      FSA_CHECK_LAUNCH();
      double h = 0.0;
      FSA_CUDA(cudaMemcpyAsync(&h, nrm.p, sizeof(double), cudaMemcpyDeviceToHost, s));
      FSA_CUDA(cudaStreamSynchronize(s));
      op.a_scale = 0x1p-16 * sqrt(th.sigma1_sq) * h;
      op.a_fp64 = op.a_scale > kAFp64Above;
    }
    if (op.a_fp64) {
      // A = Sigma_nm L_m^-T in FP64, then rounded like the tensor-core result
      DevPtr<double> K64((size_t)n * m), A64((size_t)n * m);
      cov_cross(H, n, H.xs.p, H.ys.p, m, H.ind_x.p, H.ind_y.p, th, 0, K64.p, m);
      dgemm(H.ws, s, false, true, (int)n, m, m, 1.0, K64.p, m, op.Lmi.p, m, 0.0, A64.p, m, nullptr, kTriB_KleJ);
      k_f64_to_f32_pad<<<grid_for((int64_t)n * m_pad, 256), 256, 0, s>>>(n, m, m_pad, A64.p, A32.p);
      FSA_CHECK_LAUNCH();
      FSA_CUDA(cudaStreamSynchronize(s));
    } else {
      cov_nm_split(H, m_pad, th, 0, Khi.p, Klo.p);
      k_split_f64<<<grid_for((int64_t)m_pad * m_pad, 256), 256, 0, s>>>(m, m, op.Lmi.p, m, m_pad, m_pad, Lhi.p,
                                                                         Llo.p);
      FSA_CHECK_LAUNCH();
      TmaMap mKh = make_tma_bf16(Khi.p, n, m_pad, m_pad, 128), mKl = make_tma_bf16(Klo.p, n, m_pad, m_pad, 128);
      TmaMap mLh = make_tma_bf16(Lhi.p, m_pad, m_pad, m_pad, 128),
             mLl = make_tma_bf16(Llo.p, m_pad, m_pad, m_pad, 128);
      TcGemm g;
      g.a[0] = &mKh; g.a[1] = &mKl; g.num_a = 2;
      g.b[0] = &mLh; g.b[1] = &mLl; g.num_b = 2;
      g.pairs = 1u | 2u | 4u;   // hi.hi + hi.lo + lo.hi
      g.M = (int)n; g.N = m_pad; g.K = m_pad; g.bn = 128;
      g.out = A32.p; g.ldo = m_pad;
      g.tag = "build";
      tc_gemm(g, H.err, s);
    }
    // the GEMM's operands are freed (stream-ordered) before the pieces are allocated
    Khi.release(); Klo.release(); Lhi.release(); Llo.release();
    // A~ as BF16 pieces in both orientations: A~ (rows n, K = m_pad) for A~ q and
    // A~^T (rows m_pad, K = n_pad, zero past n) for A~^T X, from one pass over A32
    op.Ab.ensure(nm);
    op.Atb.ensure((size_t)m_pad * n_pad);
    if (lo) {
      op.Ab_lo.ensure(nm);
      op.Atb_lo.ensure((size_t)m_pad * n_pad);
    }
    {
      ProfScope ps("build_split", 4.0 * n * m_pad + (lo ? 8.0 : 4.0) * n * m_pad, s);   // A32 read; pieces twice
      const int64_t nt = (n_pad / kSBT) * (m_pad / kSBT);
      k_split_both<<<split_both_blocks(nt), 256, 0, s>>>(n, m_pad, n_pad, A32.p, op.Ab.p, lo ? op.Ab_lo.p : nullptr,
                                                          op.Atb.p, lo ? op.Atb_lo.p : nullptr);
      FSA_CHECK_LAUNCH();
    }
    FSA_CUDA(cudaStreamSynchronize(s));
  }
  const __nv_bfloat16* Alo = lo ? op.Ab_lo.p : nullptr;
  const __nv_bfloat16* Atlo = lo ? op.Atb_lo.p : nullptr;
  // residual values, D
  op.vals.ensure(H.nnz);
  op.vals32.ensure(H.nnz + 4);   // spare entries: the SpMM copies in 16-byte units
  op.D.ensure(n);
  op.D32.ensure(n);
  op.Dinv32.ensure(n);
  if (!csr_values_tiles(H, th, op.Ab.p, Alo, m_pad)) csr_values_rows(H, th, op.Ab.p, Alo, m_pad);
  // the values of the SpMM row groups' union entries, read by one bulk copy per tile
  op.grp_ent.ensure((size_t)std::max<int64_t>(H.grp_entries, 1) * kEntVec);
  if (H.sp_ntiles > 0 && H.grp_entries > 0) {
    k_grp_values<<<H.sp_ntiles, 128, 0, s>>>(H.sp_ptile.p, H.grp_src.p, op.vals32.p, op.grp_ent.p, H.err);
    FSA_CHECK_LAUNCH();
  }
  // Woodbury core M = I + A^T D^-1 A on the tensor cores (split-K, FP64 reduction)
  {
    size_t mn = (size_t)m_pad * n_pad;
    DevPtr<__nv_bfloat16> Yhi(mn), Ylo(mn);
    k_scale_cols_split<<<grid_for((int64_t)mn / 8, 256), 256, 0, s>>>(m_pad, n, n_pad, op.Atb.p, Atlo, op.Dinv32.p,
                                                                        Yhi.p, Ylo.p);
    FSA_CHECK_LAUNCH();
    TmaMap mAt = make_tma_bf16_blocked(op.Atb.p, m_pad, n_pad, 128);
    TmaMap mAtl = lo ? make_tma_bf16_blocked(op.Atb_lo.p, m_pad, n_pad, 128) : mAt;
    TmaMap mYh = make_tma_bf16_blocked(Yhi.p, m_pad, n_pad, 128), mYl = make_tma_bf16_blocked(Ylo.p, m_pad, n_pad, 128);
    TcGemm g;
    g.a[0] = &mAt; g.a[1] = &mAtl; g.num_a = lo ? 2 : 1;
    g.b[0] = &mYh; g.b[1] = &mYl; g.num_b = 2;
    g.pairs = lo ? (1u | 2u | 4u) : (1u | 2u);
    g.M = m_pad; g.N = m_pad; g.bn = 128;
    g.lower = true;   // symmetric: the tiles on and below the diagonal, mirrored in the reduction
    // M - I = A~^T D^-1 A~ has entries up to n / min(D) while the identity is
    // what the small eigenvalues of M keep: FP32 accumulation runs over spans
    // of kCoreSpanBlocks k-blocks only and the spans are summed in FP64, in
    // launches of kCoreSpans spans (bounded partial buffer), in a fixed order
    const int kb = (int)((n + 63) / 64);
    const int spans = std::min(kCoreSpans, (kb + kCoreSpanBlocks - 1) / kCoreSpanBlocks);
    DevPtr<float> part((size_t)spans * m_pad * m_pad);
    op.Mp.ensure((size_t)m * m);
    g.out = part.p; g.ldo = m_pad; g.split_stride = (int64_t)m_pad * m_pad;
    g.tag = "build";
    for (int b0 = 0, first = 1; b0 < kb; b0 += spans * kCoreSpanBlocks, first = 0) {
      const int nb = std::min(kb - b0, spans * kCoreSpanBlocks);
      g.k0 = b0 * 64;
      g.K = nb * 64;
      g.splits = (nb + kCoreSpanBlocks - 1) / kCoreSpanBlocks;
      tc_gemm(g, H.err, s);
      k_reduce_splits<<<grid_for((int64_t)m * m, 256), 256, 0, s>>>(g.splits, m, m, part.p, m_pad, g.split_stride,
                                                                    op.Mp.p, m, 1, first ? 0 : 1, 1);
      FSA_CHECK_LAUNCH();
    }
    FSA_CUDA(cudaStreamSynchronize(s));
  }
  // The FP32 sums above round each span at about 2^-24 of its size, which is
  // bounded by |M - I|.  Where that is not small against the identity (a long
  // range with a small nugget puts entries of order n / nugget beside it), the
  // small eigenvalues of M, and with them log det P and the identity
  // A~^T z = q of the two-pass CG iteration, would be lost: M - I is then
  // formed in FP64 from the same A~ and D.
  {
    DevPtr<double> nrm(1);
    k_core_norm<<<1, 256, 0, s>>>(m, op.Mp.p, nrm.p);
    FSA_CHECK_LAUNCH();
    double h = 0.0;
    FSA_CUDA(cudaMemcpyAsync(&h, nrm.p, sizeof(double), cudaMemcpyDeviceToHost, s));
    FSA_CUDA(cudaStreamSynchronize(s));
    op.core_scale = h * 0x1p-24;
    op.core_fp64 = op.core_scale > kCoreFp64Above;
    if (op.core_fp64) {
      DevPtr<double> A64((size_t)n * m), Dinv64(n);
      k_pair_to_f64<<<grid_for((int64_t)n * m, 256), 256, 0, s>>>(n, m, op.Ab.p, lo ? op.Ab_lo.p : nullptr, A64.p);
      FSA_CHECK_LAUNCH();
      // the D^-1 the CG applies (FP32), so that A~^T z = q holds for its iterates
      k_f32_to_f64<<<grid_for(n, 256), 256, 0, s>>>(n, op.Dinv32.p, Dinv64.p);
      FSA_CHECK_LAUNCH();
      k_set_identity<<<grid_for((int64_t)m * m, 256), 256, 0, s>>>(m, op.Mp.p);
      FSA_CHECK_LAUNCH();
      dgemm(H.ws, s, true, false, m, m, (int)n, 1.0, A64.p, m, A64.p, m, 1.0, op.Mp.p, m, Dinv64.p);
      FSA_CUDA(cudaStreamSynchronize(s));
    }
  }
  check_err(H);
  finish_core(H);
  op.theta = th;
  op.precision = precision;
  op.valid = true;
}

// ---------------------------------------------------------------------------
// per-iteration products on the tensor cores
// ---------------------------------------------------------------------------

// vector-operand split: two BF16 pieces (~16 significant bits) by default;
// three (the full FP32 24) when the call asks for them (fsa_opts.vec_pieces)
// and the stacked block fits one N tile (3 ldc <= 256, ldc a multiple of 16
// so that 3 ldc is a multiple of the MMA's N granule)
static inline int pick_nsplit(int ldc, int pieces) { return pieces == 3 && 3 * ldc <= 256 && ldc % 16 == 0 ? 3 : 2; }
int mixed_ldc(int c, int pieces) {
  int l16 = (c + 15) / 16 * 16;
  return pieces == 3 && 3 * l16 <= 256 ? l16 : (c + 7) / 8 * 8;
}

static void set_operator_maps(const Operator& op, int64_t n, MixedCtx& C);

void mixed_ctx_setup(Handle& H, MixedCtx& C, int64_t n, int c, int ldc) {
  Operator& op = H.op;
  CGState& g = H.cg;
  C.ldc = ldc; C.c = c; C.m_pad = op.m_pad; C.n = n; C.n_pad = op.n_pad;
  C.nsplit = pick_nsplit(ldc, H.vec_pieces);
  const int ns = C.nsplit * ldc;
  FSA_REQUIRE(ns <= 256, FSA_ERR_UNSUPPORTED, "block too wide for the tensor-core products");
  g.Xb.ensure((size_t)ns * C.n_pad);
  g.qb.ensure((size_t)ns * C.m_pad);
  set_operator_maps(op, n, C);
  C.mX = make_tma_bf16_blocked(g.Xb.p, ns, C.n_pad, ns);
  C.mQ = make_tma_bf16(g.qb.p, ns, C.m_pad, C.m_pad, ns);
  C.splits_w = tc_pick_splits(C.m_pad, ns, (int)n, ns);
}

static void set_operator_maps(const Operator& op, int64_t n, MixedCtx& C) {
  C.mAt = make_tma_bf16_blocked(op.Atb.p, C.m_pad, C.n_pad, 128);
  C.mA = make_tma_bf16_blocked(op.Ab.p, n, C.m_pad, 128);
  C.lo = op.has_lo;
  if (C.lo) {
    C.mAt_lo = make_tma_bf16_blocked(op.Atb_lo.p, C.m_pad, C.n_pad, 128);
    C.mA_lo = make_tma_bf16_blocked(op.Ab_lo.p, n, C.m_pad, 128);
  }
}

static void mixed_AtX_pieces(Handle& H, MixedCtx& C, double* w, const char* tag);

// w (FP64, m x ldc) = A~^T X  where X = rows of `src` (scaled by rowscale), split hi/lo
void mixed_AtX(Handle& H, MixedCtx& C, const float* src, const float* rowscale, double* w,
                      const char* tag) {
  cudaStream_t s = H.stream;
  CGState& g = H.cg;
  int ldc = C.ldc;
  size_t smem = (size_t)(kSTRows * (ldc + 1) + kSTRows) * sizeof(float);
  {
    // FP32 block read once, nsplit BF16 pieces written
    ProfScope ps("pcg_split", (double)C.n * C.c * (4.0 + 2.0 * C.nsplit), s, tag && tag[0] == 'p');
    k_split_transpose<<<(unsigned)((C.n_pad + kSTRows - 1) / kSTRows), 256, smem, s>>>(C.n, C.c, ldc, C.nsplit,
                                                                                      src, rowscale, C.n_pad, g.Xb.p);
    FSA_CHECK_LAUNCH();
  }
  mixed_AtX_pieces(H, C, w, tag);
}

// w (FP64, m x ldc) = A~^T X with X already split into the blocked pieces (H.cg.Xb)
static void mixed_AtX_pieces(Handle& H, MixedCtx& C, double* w, const char* tag) {
  cudaStream_t s = H.stream;
  const int ldc = C.ldc;
  TcGemm t;
  t.a[0] = &C.mAt; t.a[1] = &C.mAt_lo; t.num_a = C.lo ? 2 : 1;
  t.b[0] = &C.mX; t.num_b = 1;
  t.pairs = C.lo ? (1u | 4u) : 1u;
  t.M = C.m_pad; t.N = C.nsplit * ldc; t.K = (int)C.n; t.bn = C.nsplit * ldc;
  t.stack = C.nsplit;
  t.splits = C.splits_w;
  int kb = (t.K + 63) / 64, per = (kb + t.splits - 1) / t.splits, splits = (kb + per - 1) / per;
  t.out = C.wpart; t.ldo = ldc; t.split_stride = (int64_t)C.m_pad * ldc;
  t.tag = tag;
  t.alg_bytes = t.num_a * (double)H.m * C.n * 2.0 + (double)C.nsplit * C.c * C.n * 2.0 +
                (double)splits * H.m * C.c * 4.0;
  tc_gemm(t, H.err, s);
  {
    // split-K partials read once (FP32), w written once (FP64)
    ProfScope ps("pcg_reduce", (double)H.m * C.c * (4.0 * splits + 8.0), s, tag && tag[0] == 'p');
    k_reduce_splits<<<grid_for((int64_t)H.m * ldc, 256), 256, 0, s>>>(splits, H.m, ldc, C.wpart, ldc,
                                                                      t.split_stride, w, ldc, 0);
    FSA_CHECK_LAUNCH();
  }
}

// S (FP32 n x ldc) = A~ q, q FP64 m x ldc
void mixed_Aq(Handle& H, MixedCtx& C, const double* q, float* S, const char* tag) {
  cudaStream_t s = H.stream;
  CGState& g = H.cg;
  int ldc = C.ldc;
  k_split_q<<<grid_for((int64_t)ldc * C.m_pad, 256), 256, 0, s>>>(H.m, C.c, ldc, C.nsplit, C.m_pad, q, g.qb.p);
  FSA_CHECK_LAUNCH();
  TcGemm t;
  t.a[0] = &C.mA; t.a[1] = &C.mA_lo; t.num_a = C.lo ? 2 : 1;
  t.b[0] = &C.mQ; t.num_b = 1;
  t.pairs = C.lo ? (1u | 4u) : 1u;
  t.M = (int)C.n; t.N = C.nsplit * ldc; t.K = C.m_pad; t.bn = C.nsplit * ldc;
  t.stack = C.nsplit;
  t.out = S; t.ldo = ldc;
  t.tag = tag;
  t.alg_bytes = t.num_a * (double)C.n * H.m * 2.0 + (double)C.nsplit * C.c * H.m * 2.0 + (double)C.n * C.c * 4.0;
  tc_gemm(t, H.err, s);
}

// S = A~ M^-1 w  (w = A~^T (D^-1 R) in H.cg.w)
static void lowrank_mixed_tail(Handle& H, MixedCtx& C, float* S) {
  CGState& g = H.cg;
  Operator& op = H.op;
  {
    // FP64 q = M^-1 w: m x m core read once, w read, q written
    ProfScope ps("pcg_q", 8.0 * ((double)H.m * H.m + 2.0 * H.m * C.c), H.stream);
    dgemm_tall(H.ws, H.stream, H.m, C.ldc, H.m, op.Minv.p, H.m, g.w.p, C.ldc, g.q.p, C.ldc);
  }
  mixed_Aq(H, C, g.q.p, S, "pcg_Aq");
}

// S = A~ M^-1 A~^T (D^-1 R)
static void lowrank_mixed(Handle& H, MixedCtx& C, const float* R, float* S) {
  mixed_AtX(H, C, R, H.op.Dinv32.p, H.cg.w.p, "pcg_AtX");
  lowrank_mixed_tail(H, C, S);
}

// launch shape of k_ur_split: one full wave (SM count x resident blocks, at
// most the layout's partial rows and the tile count)
struct URSplitLaunch {
  int blocks = 1, threads = 32, rpb = 1;
  size_t smem = 0;
};
static URSplitLaunch ur_split_launch(const CGLayout& lay, int64_t n_pad) {
  URSplitLaunch u;
  const int ldc = lay.ldc, c4 = ldc / 4;
  u.rpb = std::max(1, 256 / c4);
  u.threads = u.rpb * c4;
  u.smem = std::max((size_t)(kSTRows * (ldc + 1) + kSTRows) * sizeof(float), (size_t)u.threads * 4 * sizeof(double));
  int dev = 0, sms = 152, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_ur_split, u.threads, u.smem) != cudaSuccess) {
    cudaGetLastError();
    per = 0;
  }
  const int64_t ntiles = std::max<int64_t>((n_pad + kSTRows - 1) / kSTRows, 1);
  int64_t b = std::min<int64_t>(ntiles, (int64_t)sms * std::max(per, 1));
  u.blocks = (int)std::max<int64_t>(1, std::min<int64_t>(b, lay.nblk));
  return u;
}

// Block PCG of Appendix A on the right-hand sides in H.cg.R32 (n x ldc FP32,
// columns >= c zero) with the mixed operator and the FITC preconditioner:
// U receives Sigma_dag^-1 R, W0 the first preconditioner apply P_hat^-1 R, and
// the per-column scalars the Lanczos tridiagonals, iteration counts and
// residual norms.  Runs L iterations (opts.fixed_iters) or until every column
// meets cg_tol.
void pcg_mixed_run(Handle& H, MixedCtx& C, const CGLayout& lay, const fsa_opts& o, int L) {
  cudaStream_t s = H.stream;
  Operator& op = H.op;
  CGState& g = H.cg;
  const int64_t n = H.n;
  const int ldc = lay.ldc;
  const size_t nc = (size_t)n * ldc;
  FSA_REQUIRE(ldc % 4 == 0 && ldc == C.ldc, FSA_ERR_ARG, "block layout and tensor-core context disagree");
  const URSplitLaunch us = ur_split_launch(lay, C.n_pad);
  const Vec4Launch v4z = vec4_launch(lay, reinterpret_cast<const void*>(kv4_z_update));
  FSA_CUDA(cudaMemsetAsync(g.U32.p, 0, nc * sizeof(float), s));
  FSA_CUDA(cudaMemsetAsync(g.V32.p, 0, nc * sizeof(float), s));
  FSA_CUDA(cudaMemsetAsync(g.H32.p, 0, nc * sizeof(float), s));
  CGScalars q = make_scalars(H, o, L);
  const ZBulkLaunch zb = zbulk_launch(lay);
  // Z = D^-1 (R - S) with its r^T z step: the bulk-copy stream where its
  // shared memory is granted, else the register form
  auto z_update = [&](int step, int l) {
    if (zb.blocks > 0)
      kz_bulk<<<zb.blocks, zb.threads, zb.smem, s>>>(n, lay.c, ldc, zb.rpb, g.R32.p, g.S32.p, op.Dinv32.p, g.Z32.p,
                                                     g.part.p, step, l, q);
    else
      kv4_z_update<<<v4z.blocks, v4z.threads, v4z.smem, s>>>(n, lay.c, ldc, v4z.rpb, g.R32.p, g.S32.p, op.Dinv32.p,
                                                            g.Z32.p, g.part.p, step, l, q);
    FSA_CHECK_LAUNCH();
  };
  lowrank_mixed(H, C, g.R32.p, g.S32.p);
  z_update(kStepInit, 0);
  FSA_CUDA(cudaMemcpyAsync(g.W032.p, g.Z32.p, nc * sizeof(float), cudaMemcpyDeviceToDevice, s));
  const StagedLaunch sl = staged_launch(H, ldc);
  launch_spmm_f32(H, lay, sl, s, op.vals32.p, g.Z32.p, g.S32.p, g.V32.p, g.H32.p, g.beta.p, g.part.p, kStepAlpha, q);
  int32_t* pin_active = reinterpret_cast<int32_t*>(H.host_pinned);
  const double blk_bytes = (double)n * lay.c * sizeof(float);   // algorithmic: the c columns, not the padding
  for (int it = 0; it < L; ++it) {
    {
      // U, R read and written; H, V read; the nsplit BF16 pieces of D^-1 R written; D^-1
      ProfScope ps("pcg_ur", (6.0 + 0.5 * C.nsplit) * blk_bytes + 4.0 * n, s);
      k_ur_split<<<us.blocks, us.threads, us.smem, s>>>(n, lay.c, ldc, us.rpb, C.nsplit, C.n_pad, g.U32.p, g.R32.p,
                                                        g.H32.p, g.V32.p, op.Dinv32.p, g.alpha.p, g.active.p, g.Xb.p,
                                                        g.part.p, kStepResid, it, q);
      FSA_CHECK_LAUNCH();
    }
    mixed_AtX_pieces(H, C, g.w.p, "pcg_AtX");
    lowrank_mixed_tail(H, C, g.S32.p);
    {
      ProfScope ps("pcg_z", 3.0 * blk_bytes + 4.0 * n, s);   // R, S read, Z written; D^-1
      z_update(kStepBeta, it);
    }
    launch_spmm_f32(H, lay, sl, s, op.vals32.p, g.Z32.p, g.S32.p, g.V32.p, g.H32.p, g.beta.p, g.part.p, kStepAlpha,
                    q);
    if (o.fixed_iters <= 0 && should_poll(it)) {
      FSA_CUDA(cudaMemcpyAsync(pin_active, g.num_active.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      FSA_CUDA(cudaStreamSynchronize(s));
      if (*pin_active == 0) break;
    }
  }
}

// ---------------------------------------------------------------------------
// range derivative of the mixed operator
// ---------------------------------------------------------------------------
void build_deriv_mixed(Handle& H, const MixedCtx& C, const fsa_theta& th, DerivMixed& Dv) {
  cudaStream_t s = H.stream;
  Operator& op = H.op;
  const int64_t n = H.n;
  const int m = H.m, m_pad = C.m_pad;
  const size_t nm = (size_t)n * m_pad, mm_pad = (size_t)m_pad * m_pad;
  Dv.Alo = op.Ab_lo.p;
  if (!op.has_lo) {
    Dv.zero_lo.alloc(nm);
    FSA_CUDA(cudaMemsetAsync(Dv.zero_lo.p, 0, nm * sizeof(__nv_bfloat16), s));
    Dv.Alo = Dv.zero_lo.p;
  }
  Dv.E.alloc((size_t)m * m);
  {
    // order: F = A~ E, then B = dK L^-T, so that the n x m temporaries peak at
    // four of them (B32, the pieces of q, of B and of B^T)
    DevPtr<__nv_bfloat16> Lhi(mm_pad), Llo(mm_pad);
    TmaMap mLh = make_tma_bf16(Lhi.p, m_pad, m_pad, m_pad, 128), mLl = make_tma_bf16(Llo.p, m_pad, m_pad, m_pad, 128);
    // E = L^-1 dSigma_m L^-T (FP64), F = A~ E (split products)
    {
      DevPtr<double> dSm((size_t)m * m), T1((size_t)m * m);
      cov_cross(H, m, H.ind_x.p, H.ind_y.p, m, H.ind_x.p, H.ind_y.p, th, 1, dSm.p, m);
      dgemm(H.ws, s, false, false, m, m, m, 1.0, op.Lmi.p, m, dSm.p, m, 0.0, T1.p, m, nullptr, kTriA_KleI);
      dgemm(H.ws, s, false, true, m, m, m, 1.0, T1.p, m, op.Lmi.p, m, 0.0, Dv.E.p, m, nullptr,
            kTriB_KleJ | kTriSymLower);
    }
    k_split_f64<<<grid_for((int64_t)mm_pad, 256), 256, 0, s>>>(m, m, Dv.E.p, m, m_pad, m_pad, Lhi.p, Llo.p);
    FSA_CHECK_LAUNCH();
    DevPtr<float> F32(nm);
    {
      TcGemm f;
      f.a[0] = &C.mA; f.a[1] = &C.mA_lo; f.num_a = C.lo ? 2 : 1;
      f.b[0] = &mLh; f.b[1] = &mLl; f.num_b = 2;
      f.pairs = C.lo ? (1u | 2u | 4u) : (1u | 2u);
      f.M = (int)n; f.N = m_pad; f.K = m_pad; f.bn = 128;
      f.out = F32.p; f.ldo = m_pad;
      f.tag = "grad";
      tc_gemm(f, H.err, s);
    }
    // B = dK L^-T (the pieces of L^-1 replace those of E once F is done: same stream)
    DevPtr<float> B32(nm);
    {
      DevPtr<__nv_bfloat16> Khi(nm), Klo(nm);
      cov_nm_split(H, m_pad, th, 1, Khi.p, Klo.p);
      k_split_f64<<<grid_for((int64_t)mm_pad, 256), 256, 0, s>>>(m, m, op.Lmi.p, m, m_pad, m_pad, Lhi.p, Llo.p);
      FSA_CHECK_LAUNCH();
      TmaMap mKh = make_tma_bf16(Khi.p, n, m_pad, m_pad, 128), mKl = make_tma_bf16(Klo.p, n, m_pad, m_pad, 128);
      TcGemm t;
      t.a[0] = &mKh; t.a[1] = &mKl; t.num_a = 2;
      t.b[0] = &mLh; t.b[1] = &mLl; t.num_b = 2;
      t.pairs = 1u | 2u | 4u;
      t.M = (int)n; t.N = m_pad; t.K = m_pad; t.bn = 128;
      t.out = B32.p; t.ldo = m_pad;
      t.tag = "grad";
      tc_gemm(t, H.err, s);
    }
    // q = b - F as a BF16 pair
    Dv.Qh.alloc(nm); Dv.Ql.alloc(nm);
    k_sub_split<<<grid_for((int64_t)nm / 8, 256), 256, 0, s>>>(n, m_pad, B32.p, F32.p, Dv.Qh.p, Dv.Ql.p);
    FSA_CHECK_LAUNCH();
    F32.release();
    // B as a BF16 pair in both orientations: B (rows n) for B q, B^T (blocked,
    // K = the point, zero past n) for B^T X
    const size_t mn = (size_t)m_pad * C.n_pad;
    Dv.Bh.alloc(nm); Dv.Bl.alloc(nm); Dv.Bth.alloc(mn); Dv.Btl.alloc(mn);
    const int64_t nt = (C.n_pad / kSBT) * (m_pad / kSBT);
    k_split_both<<<split_both_blocks(nt), 256, 0, s>>>(n, m_pad, C.n_pad, B32.p, Dv.Bh.p, Dv.Bl.p, Dv.Bth.p, Dv.Btl.p);
    FSA_CHECK_LAUNCH();
    FSA_CUDA(cudaStreamSynchronize(s));
  }
  Dv.CBt = C;
  Dv.CBt.mAt = make_tma_bf16_blocked(Dv.Bth.p, m_pad, C.n_pad, 128);
  Dv.CBt.mAt_lo = make_tma_bf16_blocked(Dv.Btl.p, m_pad, C.n_pad, 128);
  Dv.CBt.lo = true;
  Dv.CB = C;
  Dv.CB.mA = make_tma_bf16_blocked(Dv.Bh.p, n, m_pad, 128);
  Dv.CB.mA_lo = make_tma_bf16_blocked(Dv.Bl.p, n, m_pad, 128);
  Dv.CB.lo = true;
  // the range derivative of the residual values (per nonzero) and of D_s
  Dv.dv.alloc(H.nnz + 4);
  Dv.dD.alloc(n);
  dvals_mixed(H, th, m_pad, op.Ab.p, Dv.Alo, Dv.Bh.p, Dv.Bl.p, Dv.Qh.p, Dv.Ql.p, Dv.dv.p, Dv.dD.p);
}

// out0 = Sigma_s~ X, out1 = dSigma_s~/drho X (FP32 blocks, lane L owns columns 4L .. 4L + 3)
static __global__ void __launch_bounds__(256) kv_spmm2_f4(int64_t n, int ldc, const int64_t* __restrict__ rowptr,
                                                          const int32_t* __restrict__ colidx,
                                                          const float* __restrict__ vals,
                                                          const float* __restrict__ dvals, const float* __restrict__ X,
                                                          float* __restrict__ out0, float* __restrict__ out1) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t nwarps = (int64_t)gridDim.x * 8;
  const bool act = lane < (ldc >> 2);
  for (int64_t i = (int64_t)blockIdx.x * 8 + wib; i < n; i += nwarps) {
    const int64_t rb = rowptr[i], re = rowptr[i + 1];
    float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
    for (int64_t base = rb; base < re; base += 32) {
      const int cnt = (int)((re - base) < 32 ? (re - base) : 32);
      const int myc = lane < cnt ? colidx[base + lane] : 0;
      const float myv = lane < cnt ? vals[base + lane] : 0.f;
      const float myd = lane < cnt ? dvals[base + lane] : 0.f;
      for (int t = 0; t < cnt; ++t) {
        const int j = __shfl_sync(0xffffffffu, myc, t);
        const float v = __shfl_sync(0xffffffffu, myv, t), d = __shfl_sync(0xffffffffu, myd, t);
        if (act) {
          const float4 x = *reinterpret_cast<const float4*>(X + (int64_t)j * ldc + 4 * lane);
          a0.x = fmaf(v, x.x, a0.x); a0.y = fmaf(v, x.y, a0.y); a0.z = fmaf(v, x.z, a0.z); a0.w = fmaf(v, x.w, a0.w);
          a1.x = fmaf(d, x.x, a1.x); a1.y = fmaf(d, x.y, a1.y); a1.z = fmaf(d, x.z, a1.z); a1.w = fmaf(d, x.w, a1.w);
        }
      }
    }
    if (act) {
      *reinterpret_cast<float4*>(out0 + i * ldc + 4 * lane) = a0;
      *reinterpret_cast<float4*>(out1 + i * ldc + 4 * lane) = a1;
    }
  }
}

// out0 = (out0 + T0 - nugget X) / sigma1^2; out1 += T1 + T2
static __global__ void k_dsigma_combine(int64_t total, double s1, double nug, const float* __restrict__ X,
                                        const float* __restrict__ T0, const float* __restrict__ T1,
                                        const float* __restrict__ T2, float* __restrict__ out0,
                                        float* __restrict__ out1) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    out0[t] = (float)(((double)out0[t] + (double)T0[t] - nug * (double)X[t]) / s1);
    out1[t] = out1[t] + T1[t] + T2[t];
  }
}

void apply_dsigma_mixed(Handle& H, MixedCtx& C, DerivMixed& Dv, const fsa_theta& th, const float* X, float* out0,
                        float* out1) {
  cudaStream_t s = H.stream;
  const int64_t n = H.n;
  const int m = H.m, ldc = C.ldc;
  FSA_REQUIRE(ldc % 4 == 0 && ldc <= 128, FSA_ERR_UNSUPPORTED, "derivative apply needs ldc % 4 == 0, ldc <= 128");
  kv_spmm2_f4<<<spmm_f4_blocks(), 256, 0, s>>>(n, ldc, H.rowptr.p, H.col.p, H.op.vals32.p, Dv.dv.p, X, out0, out1);
  FSA_CHECK_LAUNCH();
  const size_t mc = (size_t)m * ldc, nc = (size_t)n * ldc;
  DevPtr<double> AX(mc), BX(mc);
  mixed_AtX(H, C, X, nullptr, AX.p, "fisher");
  mixed_AtX(H, Dv.CBt, X, nullptr, BX.p, "fisher");
  // BX - E A~^T X (E symmetric)
  dgemm(H.ws, s, false, false, m, ldc, m, -1.0, Dv.E.p, m, AX.p, ldc, 1.0, BX.p, ldc, nullptr);
  DevPtr<float> T0(nc), T1(nc), T2(nc);
  mixed_Aq(H, C, AX.p, T0.p, "fisher");
  mixed_Aq(H, C, BX.p, T1.p, "fisher");
  mixed_Aq(H, Dv.CB, AX.p, T2.p, "fisher");
  k_dsigma_combine<<<grid_for((int64_t)nc, 256), 256, 0, s>>>((int64_t)nc, th.sigma1_sq, th.nugget, X, T0.p, T1.p,
                                                              T2.p, out0, out1);
  FSA_CHECK_LAUNCH();
}

LoglikResult run_loglik_grad_mixed(Handle& H, const fsa_theta& th, const fsa_opts& o) {
  cudaStream_t s = H.stream;
  Operator& op = H.op;
  CGState& g = H.cg;
  int64_t n = H.n;
  int m = H.m;
  int l = o.num_probes;
  FSA_REQUIRE(l + 1 <= 128, FSA_ERR_UNSUPPORTED, "mixed precision supports at most 127 probes");
  CGLayout lay;
  int L = o.fixed_iters > 0 ? o.fixed_iters : (o.cg_max_iter > 0 ? o.cg_max_iter : 1000);
  lay.setup(n, l + 1, L, mixed_ldc(l + 1, H.vec_pieces));
  ensure_cg(H, lay, false);
  int ldc = lay.ldc;
  size_t nc = (size_t)n * ldc;
  g.U32.ensure(nc); g.R32.ensure(nc); g.Z32.ensure(nc); g.H32.ensure(nc); g.V32.ensure(nc);
  g.S32.ensure(nc); g.W032.ensure(nc);
  MixedCtx C;
  mixed_ctx_setup(H, C, n, lay.c, ldc);
  DevPtr<float> wpart_buf((size_t)C.splits_w * C.m_pad * ldc);
  C.wpart = wpart_buf.p;
  FSA_REQUIRE(ldc % 4 == 0 && ldc <= 128, FSA_ERR_UNSUPPORTED, "mixed block width must be a multiple of 4, at most 128");
  // probes: R = [y, A~ eps1 + D^1/2 eps2]
  {
    TraceRange trace("probes");
    ProfScope phase("phase_probes", 0.0, s);
    int l16 = round_up(l, 16);
    DevPtr<__nv_bfloat16> Ehi((size_t)l16 * C.m_pad), Elo((size_t)l16 * C.m_pad);
    DevPtr<float> Zp((size_t)n * l16);
    k_eps1_split<<<grid_for((int64_t)l16 * C.m_pad, 256), 256, 0, s>>>(m, l, l16, C.m_pad, o.probe,
                                                                       rng_key(o.seed, kStreamEps1), Ehi.p, Elo.p);
    FSA_CHECK_LAUNCH();
    TmaMap mEh = make_tma_bf16(Ehi.p, l16, C.m_pad, C.m_pad, l16), mEl = make_tma_bf16(Elo.p, l16, C.m_pad, C.m_pad, l16);
    TcGemm t;
    t.a[0] = &C.mA; t.a[1] = &C.mA_lo; t.num_a = C.lo ? 2 : 1;
    t.b[0] = &mEh; t.b[1] = &mEl; t.num_b = 2;
    t.pairs = C.lo ? (1u | 2u | 4u) : (1u | 2u);
    t.M = (int)n; t.N = l16; t.K = C.m_pad; t.bn = l16;
    t.out = Zp.p; t.ldo = l16;
    t.tag = "build";
    tc_gemm(t, H.err, s);
    k_probe_finish_mixed<<<grid_for((int64_t)nc, 256), 256, 0, s>>>(n, l, ldc, l16, o.probe,
                                                                    rng_key(o.seed, kStreamEps2), H.perm.p, H.y.p,
                                                                    op.D32.p, Zp.p, g.R32.p);
    FSA_CHECK_LAUNCH();
    FSA_CUDA(cudaStreamSynchronize(s));
  }
  auto pcg_trace = std::make_unique<TraceRange>("pcg");
  auto pcg_phase = std::make_unique<ProfScope>("phase_pcg", 0.0, s);
  pcg_mixed_run(H, C, lay, o, L);
  pcg_phase.reset();
  pcg_trace.reset();
  TraceRange slq_grad_trace("slq_gradient");
  auto grad_phase = std::make_unique<ProfScope>("phase_grad", 0.0, s);
  // the Lanczos eigen-quadrature depends only on the tridiagonals: it runs on
  // the side stream (one thread per probe column) beside the gradient work
  if (!H.side) {
    FSA_CUDA(cudaStreamCreateWithFlags(&H.side, cudaStreamNonBlocking));
    FSA_CUDA(cudaEventCreateWithFlags(&H.ev_fork, cudaEventDisableTiming));
    FSA_CUDA(cudaEventCreateWithFlags(&H.ev_join, cudaEventDisableTiming));
  }
  FSA_CUDA(cudaEventRecord(H.ev_fork, s));
  FSA_CUDA(cudaStreamWaitEvent(H.side, H.ev_fork, 0));
  launch_slq(lay.c, L, g.iters.p, g.tdiag.p, g.toff.p, g.quads.p, H.err, H.side);
  FSA_CUDA(cudaEventRecord(H.ev_join, H.side));
  DevPtr<double> ypart((size_t)lay.nblk * ldc);
  k_dot_col0<float><<<lay.nblk, 32, 0, s>>>(n, ldc, lay.chunk, H.y.p, g.U32.p, ypart.p);
  FSA_CHECK_LAUNCH();
  H.outs.ensure(kOutCount);
  if (o.want_grad) {
    // X = U (u in column 0), Y = W with u in column 0
    FSA_CUDA(cudaMemcpyAsync(g.Z32.p, g.W032.p, nc * sizeof(float), cudaMemcpyDeviceToDevice, s));
    k_copy_col0<float><<<grid_for(n, 256), 256, 0, s>>>(n, ldc, g.U32.p, g.Z32.p);
    FSA_CHECK_LAUNCH();
    const int c = lay.c;
    const int m_pad = C.m_pad;
    const size_t mc = (size_t)m * ldc, nm = (size_t)n * m_pad, mm_pad = (size_t)m_pad * m_pad;
    DevPtr<double> AX(mc), AY(mc), BX(mc), BY(mc), EAY(mc);
    mixed_AtX(H, C, g.U32.p, nullptr, AX.p, "grad");
    mixed_AtX(H, C, g.Z32.p, nullptr, AY.p, "grad");
    DerivMixed Dv;
    build_deriv_mixed(H, C, th, Dv);
    mixed_AtX(H, Dv.CBt, g.U32.p, nullptr, BX.p, "grad");
    mixed_AtX(H, Dv.CBt, g.Z32.p, nullptr, BY.p, "grad");
    dgemm(H.ws, s, false, false, m, c, m, 1.0, Dv.E.p, m, AY.p, ldc, 0.0, EAY.p, ldc, nullptr);
    // sparse terms per column: one gather of Y's neighbour rows for the
    // residual values and their range derivative
    const int nb = coldots_blocks();
    DevPtr<double> part((size_t)nb * kColTerms * ldc), lr((size_t)3 * ldc);
    grad_coldots<float, float, float>(H, c, ldc, op.vals32.p, Dv.dv.p, g.U32.p, g.Z32.p, part.p, nb);
    grad_lowrank_cols(H, m, c, ldc, AX.p, AY.p, BX.p, BY.p, EAY.p, lr.p);
    // control variate: A~ M^-1 on the tensor cores, row dots, m-space traces
    DevPtr<double> cv, mtr;
    int ncv = 0;
    if (o.grad_control_variate != kCvNone) {
      ncv = cv_blocks();
      cv.alloc((size_t)ncv * kCvTerms);
      mtr.alloc(2);
      DevPtr<__nv_bfloat16> Mh(mm_pad), Ml(mm_pad);
      k_split_f64<<<grid_for((int64_t)mm_pad, 256), 256, 0, s>>>(m, m, op.Minv.p, m, m_pad, m_pad, Mh.p, Ml.p);
      FSA_CHECK_LAUNCH();
      TmaMap mMh = make_tma_bf16(Mh.p, m_pad, m_pad, m_pad, 128), mMl = make_tma_bf16(Ml.p, m_pad, m_pad, m_pad, 128);
      DevPtr<float> AM(nm);
      TcGemm t;
      t.a[0] = &C.mA; t.a[1] = &C.mA_lo; t.num_a = C.lo ? 2 : 1;
      t.b[0] = &mMh; t.b[1] = &mMl; t.num_b = 2;
      t.pairs = C.lo ? (1u | 2u | 4u) : (1u | 2u);
      t.M = (int)n; t.N = m_pad; t.K = m_pad; t.bn = 128;
      t.out = AM.p; t.ldo = m_pad;
      t.tag = "grad";
      tc_gemm(t, H.err, s);
      cv_rowdots_mixed(H, m_pad, AM.p, op.Ab.p, Dv.Alo, Dv.Bh.p, Dv.Bl.p, op.D32.p, Dv.dD.p, cv.p, ncv);
      mspace_traces(H, m, Dv.E.p, op.Minv.p, mtr.p);
    }
    FSA_CUDA(cudaStreamWaitEvent(s, H.ev_join, 0));
    k_assemble<<<1, 32, 0, s>>>(n, lay.c, o.slq_exact_weight, g.quads.p, g.rz0.p, op.scal.p, ypart.p, lay.nblk, ldc,
                                H.outs.p);
    FSA_CHECK_LAUNCH();
    H.gterms.ensure((size_t)6 * l);
    H.gterms_l = l;
    grad_final(H, c, ldc, part.p, nb, lr.p, cv.p, ncv, mtr.p, th, o.grad_control_variate, H.gterms.p);
    FSA_CUDA(cudaStreamSynchronize(s));
  } else {
    FSA_CUDA(cudaStreamWaitEvent(s, H.ev_join, 0));
    k_assemble<<<1, 32, 0, s>>>(n, lay.c, o.slq_exact_weight, g.quads.p, g.rz0.p, op.scal.p, ypart.p, lay.nblk, ldc,
                                H.outs.p);
    FSA_CHECK_LAUNCH();
  }
  grad_phase.reset();
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

__global__ void k_f64_to_f32_pad(int64_t n, int k, int ldk, const double* __restrict__ src, float* __restrict__ dst) {
  int64_t total = n * ldk;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = t / ldk;
    int c = (int)(t - i * ldk);
    dst[t] = c < k ? (float)src[i * k + c] : 0.f;
  }
}

__global__ void k_f32_to_f64_unpad(int64_t n, int k, int ldk, const float* __restrict__ src, double* __restrict__ dst) {
  int64_t total = n * k;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = t / k;
    int c = (int)(t - i * k);
    dst[t] = (double)src[i * ldk + c];
  }
}

// mixed-precision operator on vectors in internal order (n x k FP64):
// 0: Sigma_dag v = Sigma_s~ v + A~ (A~^T v); 1: P_hat^-1 v; 2: Sigma_s~ v
void apply_operator_mixed(Handle& H, int which, const double* v, int k, double* out) {
  cudaStream_t s = H.stream;
  Operator& op = H.op;
  CGState& g = H.cg;
  int64_t n = H.n;
  int m = H.m;
  FSA_REQUIRE(k <= 128, FSA_ERR_UNSUPPORTED, "mixed matvec supports at most 128 columns");
  CGLayout lay;
  lay.setup(n, k, 1, mixed_ldc(k, H.vec_pieces));
  int ldc = lay.ldc;
  size_t nc = (size_t)n * ldc;
  DevPtr<float> V32(nc), S32(nc), O32(nc);
  k_f64_to_f32_pad<<<grid_for((int64_t)nc, 256), 256, 0, s>>>(n, k, ldc, v, V32.p);
  FSA_CHECK_LAUNCH();
  MixedCtx C;
  g.w.ensure((size_t)m * ldc);
  g.q.ensure((size_t)m * ldc);
  mixed_ctx_setup(H, C, n, k, ldc);
  DevPtr<float> wpart((size_t)C.splits_w * C.m_pad * ldc);
  C.wpart = wpart.p;
  DevPtr<double> part((size_t)lay.nblk * ldc), beta(ldc);
  FSA_CUDA(cudaMemsetAsync(beta.p, 0, sizeof(double) * ldc, s));
  if (which == 1) {
    lowrank_mixed(H, C, V32.p, S32.p);
    k_z_update<float><<<lay.nblk, lay.threads, 0, s>>>(n, k, ldc, lay.chunk, V32.p, S32.p, op.Dinv32.p, O32.p,
                                                       part.p);
    FSA_CHECK_LAUNCH();
  } else {
    if (which == 0) {
      mixed_AtX(H, C, V32.p, nullptr, g.w.p, nullptr);
      mixed_Aq(H, C, g.w.p, S32.p, nullptr);
    } else {
      FSA_CUDA(cudaMemsetAsync(S32.p, 0, nc * sizeof(float), s));
    }
    DevPtr<float> Hd(nc);
    FSA_CUDA(cudaMemsetAsync(Hd.p, 0, nc * sizeof(float), s));
    FSA_CUDA(cudaMemsetAsync(O32.p, 0, nc * sizeof(float), s));
    CGScalars none{};
    none.err = H.err;   // bounded waits in the SpMM report a timeout here
    launch_spmm_f32(H, lay, staged_launch(H, ldc), s, op.vals32.p, V32.p, S32.p, O32.p, Hd.p, beta.p, part.p,
                    kStepNone, none);
  }
  k_f32_to_f64_unpad<<<grid_for(n * k, 256), 256, 0, s>>>(n, k, ldc, O32.p, out);
  FSA_CHECK_LAUNCH();
  FSA_CUDA(cudaStreamSynchronize(s));
}

}  // namespace fsa
