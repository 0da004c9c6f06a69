// Tile kernels for the two sampled dense products of the mixed form (SDDMM-
// shaped work over the taper pattern, paper §2.1 and §2.2):
//
//   * the tapered residual values val_ij = (c(s_i, s_j) - a_i . a_j) T(d_ij)
//     and D_s,i = sigma1^2 - |a_i|^2 + nugget (Eq. eqfitcp), and
//   * the sparse part of the range derivative of the gradient (Eq.
//     NEGLLDNEGLLFSA with the derivative of Sigma_dag), whose low-rank piece
//     sum_ij w_ij (b_i . a_j + a_i . q_j) is evaluated row by row as
//     b_i . (sum_j w_ij a_j) + a_i . (sum_j w_ij q_j).
//
// Both run over the cell-grid tiles of the SpMM: the taper neighbours of a
// tile's rows lie in three contiguous row ranges, so the m-long rows a_j (and
// q_j) of those ranges are staged in shared memory one 64-column block at a
// time (cp.async, two stages) and every a_j is read from L2 once per tile
// instead of once per nonzero.  A~ is in the blocked K-major layout: the
// rows of one 64-column block are consecutive 128-byte runs.  One persistent
// block of 512 threads per SM; a tile whose ranges exceed the staging
// capacity (none in a cell-grid pattern of the sizes used here) is computed
// from global memory by the same per-nonzero arithmetic.
#include <algorithm>

#include "fsa_vec.cuh"

namespace fsa {

constexpr int kSdThreads = 512, kSdWarps = kSdThreads / 32, kSdPer = 4;   // nonzeros per thread <= 4
constexpr int kSdRowV = 72;   // staged row stride of the values kernel in BF16 (64 + 8: 144 B)
constexpr size_t kSdSmemMax = 200 * 1024;

struct TileRec {
  int p0, nr, r0b, n0, r1b, n1, r2b, n2, ne;
  int64_t e0;
  bool staged;
};

__device__ __forceinline__ TileRec load_tile(const int32_t* __restrict__ ptile, const int32_t* __restrict__ tile_bad,
                                             int tile, int cap_rows, int cap_nnz, int cap_trows) {
  const int32_t* r = ptile + (int64_t)tile * kTileWords;
  TileRec t;
  t.p0 = r[0]; t.nr = r[1];
  t.r0b = r[2]; t.n0 = r[3]; t.r1b = r[4]; t.n1 = r[5]; t.r2b = r[6]; t.n2 = r[7];
  t.e0 = (int64_t)(uint32_t)r[8] | ((int64_t)r[9] << 32);
  t.ne = r[10];
  t.staged = !tile_bad[tile] && t.n0 + t.n1 + t.n2 <= cap_rows && t.ne <= cap_nnz && t.nr <= cap_trows;
  return t;
}

// cp.async of 128-byte row pieces: rows [rb, rb + nrows) of a source whose
// row k starts at src + k * src_ld (elements), to dst rows starting at drow
// (dst_ld elements per row); 8 copies of 16 bytes per row
__device__ __forceinline__ void stage_rows(__nv_bfloat16* dst, int drow, int dst_ld, const __nv_bfloat16* src,
                                           int64_t src_ld, int rb, int nrows) {
  for (int x = threadIdx.x; x < nrows * 8; x += kSdThreads) {
    const int r = x >> 3, c = x & 7;
    cpa16(dst + (size_t)(drow + r) * dst_ld + c * 8, src + (int64_t)(rb + r) * src_ld + c * 8);
  }
}

// the row of each of the tile's nonzeros (srow) and its staged column (ssc)
__device__ __forceinline__ void tile_rows(const TileRec& T, const int64_t* __restrict__ rowptr,
                                          const int32_t* __restrict__ scol, int* srow, int* ssc) {
  for (int r = threadIdx.x; r < T.nr; r += kSdThreads) {
    const int tb = (int)(rowptr[T.p0 + r] - T.e0), te = (int)(rowptr[T.p0 + r + 1] - T.e0);
    for (int t = tb; t < te; ++t) srow[t] = r;
  }
  if (ssc)
    for (int t = threadIdx.x; t < T.ne; t += kSdThreads) ssc[t] = scol[T.e0 + t];
}

__device__ __forceinline__ float2 bf2f(uint32_t w) {
  return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}

// ---------------------------------------------------------------------------
// residual values
// ---------------------------------------------------------------------------
// the value of nonzero (i, j) from s = a_i . a_j (same arithmetic as the row form)
__device__ __forceinline__ void write_value(int64_t t, int64_t i, int64_t j, double s, const double* __restrict__ xs,
                                            const double* __restrict__ ys, int cov, double s1, double rho, double nug,
                                            double gamma, double* __restrict__ vals, float* __restrict__ vals32,
                                            double* __restrict__ D, float* __restrict__ D32,
                                            float* __restrict__ Dinv32) {
  double v;
  if (j == i) {
    const float dv = (float)(fmax(s1 - (double)s, 0.0) + nug);
    v = (double)dv;
    D[i] = v;
    D32[i] = dv;
    Dinv32[i] = 1.0f / dv;
  } else {
    const double d = sqrt(sqdist_rn(xs[i], ys[i], xs[j], ys[j]));
    v = (s1 * matern_r(cov, d, rho) - (double)s) * wendland(d, gamma);
  }
  vals[t] = v;
  vals32[t] = (float)v;
}

// a_i . a_j over one 64-column block: eight running FP32 sums of 8 products
// (one per 16-byte chunk), added pairwise within each half of four and the
// two halves added; the blocks are summed in FP64
__device__ __forceinline__ float dot_block(const uint4* __restrict__ hi_i, const uint4* __restrict__ hi_j,
                                           const uint4* __restrict__ lo_i, const uint4* __restrict__ lo_j) {
  float tot = 0.f;
#pragma unroll 1
  for (int h = 0; h < 2; ++h) {   // two halves of four chunks (bounds the loads in flight)
    float cs[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const uint4 ah = hi_i[4 * h + c], bh = hi_j[4 * h + c];
      const uint32_t wah[4] = {ah.x, ah.y, ah.z, ah.w}, wbh[4] = {bh.x, bh.y, bh.z, bh.w};
      uint32_t wal[4] = {0u, 0u, 0u, 0u}, wbl[4] = {0u, 0u, 0u, 0u};
      if (lo_i) {
        const uint4 al = lo_i[4 * h + c], bl = lo_j[4 * h + c];
        wal[0] = al.x; wal[1] = al.y; wal[2] = al.z; wal[3] = al.w;
        wbl[0] = bl.x; wbl[1] = bl.y; wbl[2] = bl.z; wbl[3] = bl.w;
      }
      float t = 0.f;
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        float2 a = bf2f(wah[w]), b = bf2f(wbh[w]);
        if (lo_i) {
          const float2 la = bf2f(wal[w]), lb = bf2f(wbl[w]);
          a.x += la.x; a.y += la.y; b.x += lb.x; b.y += lb.y;
        }
        t = fmaf(a.x, b.x, t);
        t = fmaf(a.y, b.y, t);
      }
      cs[c] = t;
    }
    tot += (cs[0] + cs[1]) + (cs[2] + cs[3]);
  }
  return tot;
}

// a_i . a_j from global memory (blocked layout, hi + lo)
__device__ __forceinline__ double dot_rows_global(const __nv_bfloat16* __restrict__ A,
                                                  const __nv_bfloat16* __restrict__ Alo, int64_t n, int m_pad,
                                                  int64_t i, int64_t j) {
  double s = 0.0;
  for (int kb = 0; kb < m_pad / 64; ++kb) {
    const int64_t oi = ((int64_t)kb * n + i) * 64, oj = ((int64_t)kb * n + j) * 64;
    s += (double)dot_block(reinterpret_cast<const uint4*>(A + oi), reinterpret_cast<const uint4*>(A + oj),
                           Alo ? reinterpret_cast<const uint4*>(Alo + oi) : nullptr,
                           Alo ? reinterpret_cast<const uint4*>(Alo + oj) : nullptr);
  }
  return s;
}

__global__ void __launch_bounds__(kSdThreads, 1) k_csr_values_tiles(
    int ntiles, const int32_t* __restrict__ ptile, const int32_t* __restrict__ tile_bad, int cap_rows, int cap_nnz,
    int cap_trows, int64_t n, int m_pad, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
    const int32_t* __restrict__ scol, const double* __restrict__ xs, const double* __restrict__ ys,
    const __nv_bfloat16* __restrict__ A, const __nv_bfloat16* __restrict__ Alo, int cov, double s1, double rho,
    double nug, double gamma, double* __restrict__ vals, float* __restrict__ vals32, double* __restrict__ D,
    float* __restrict__ D32, float* __restrict__ Dinv32) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int planes = Alo ? 2 : 1;
  const size_t plane = (size_t)cap_rows * kSdRowV;   // elements
  __nv_bfloat16* st = reinterpret_cast<__nv_bfloat16*>(smraw);   // 2 stages x planes x plane
  int* srow = reinterpret_cast<int*>(st + 2 * planes * plane);
  int* ssc = srow + cap_nnz;
  const int nkb = m_pad / 64;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const TileRec T = load_tile(ptile, tile_bad, tile, cap_rows, cap_nnz, cap_trows);
    if (!T.staged) {
      for (int t = threadIdx.x; t < T.ne; t += kSdThreads) {
        const int64_t e = T.e0 + t;
        int64_t i = T.p0;
        while (rowptr[i + 1] <= e) ++i;
        const int64_t j = col[e];
        write_value(e, i, j, dot_rows_global(A, Alo, n, m_pad, i, j), xs, ys, cov, s1, rho, nug, gamma, vals,
                    vals32, D, D32, Dinv32);
      }
      continue;
    }
    tile_rows(T, rowptr, scol, srow, ssc);
    auto issue = [&](int kb) {
      __nv_bfloat16* sb = st + (size_t)(kb & 1) * planes * plane;
      for (int p = 0; p < planes; ++p) {
        const __nv_bfloat16* src = (p == 0 ? A : Alo) + (int64_t)kb * n * 64;
        __nv_bfloat16* dst = sb + p * plane;
        stage_rows(dst, 0, kSdRowV, src, 64, T.r0b, T.n0);
        stage_rows(dst, T.n0, kSdRowV, src, 64, T.r1b, T.n1);
        stage_rows(dst, T.n0 + T.n1, kSdRowV, src, 64, T.r2b, T.n2);
      }
      cpa_commit();
    };
    issue(0);
    double acc[kSdPer] = {0.0, 0.0, 0.0, 0.0};
    for (int kb = 0; kb < nkb; ++kb) {
      if (kb + 1 < nkb) issue(kb + 1);
      else cpa_commit();
      cpa_wait<1>();
      __syncthreads();
      const __nv_bfloat16* sb = st + (size_t)(kb & 1) * planes * plane;
#pragma unroll
      for (int u = 0; u < kSdPer; ++u) {
        const int t = threadIdx.x + u * kSdThreads;
        if (t < T.ne) {
          const int ri = T.n0 + (T.p0 + srow[t] - T.r1b), rj = ssc[t];
          const uint4* hi_i = reinterpret_cast<const uint4*>(sb + (size_t)ri * kSdRowV);
          const uint4* hi_j = reinterpret_cast<const uint4*>(sb + (size_t)rj * kSdRowV);
          const uint4* lo_i = planes == 2 ? reinterpret_cast<const uint4*>(sb + plane + (size_t)ri * kSdRowV) : nullptr;
          const uint4* lo_j = planes == 2 ? reinterpret_cast<const uint4*>(sb + plane + (size_t)rj * kSdRowV) : nullptr;
          acc[u] += (double)dot_block(hi_i, hi_j, lo_i, lo_j);
        }
      }
      __syncthreads();   // stage kb & 1 is free for block kb + 2
    }
#pragma unroll
    for (int u = 0; u < kSdPer; ++u) {
      const int t = threadIdx.x + u * kSdThreads;
      if (t < T.ne) {
        const int64_t e = T.e0 + t;
        write_value(e, (int64_t)T.p0 + srow[t], col[e], acc[u], xs, ys, cov, s1, rho, nug, gamma, vals, vals32, D,
                    D32, Dinv32);
      }
    }
    __syncthreads();   // srow, ssc are rewritten by the next tile
  }
  cpa_wait<0>();
}

struct SdLaunch {
  int blocks = 0, cap_rows = 0, cap_nnz = 0, cap_trows = 0;
  size_t smem = 0;
};

// capacities: every tile's rows and nonzeros; staged rows as many as the
// shared-memory budget allows (up to the largest tile's)
static SdLaunch sd_launch(const Handle& H, size_t per_row, size_t per_trow, size_t fixed_per_nnz,
                          const void* kernel, int cap_rows_max) {
  SdLaunch L;
  L.cap_trows = (int)std::min<int64_t>(4096, std::max<int64_t>(H.max_tile_rows, 1));
  L.cap_nnz = (int)std::min<int64_t>((int64_t)kSdThreads * kSdPer, std::max<int64_t>(H.max_tile_nnz, 1));
  const size_t fixed = (size_t)L.cap_nnz * fixed_per_nnz + (size_t)(L.cap_trows + 1) * (4 + 2 * per_trow) + 64;
  if (fixed >= kSdSmemMax) return L;
  const int64_t fit = (int64_t)((kSdSmemMax - fixed) / (2 * per_row));
  L.cap_rows = (int)std::min<int64_t>(fit, std::max<int64_t>(H.max_staged, 1));
  if (cap_rows_max > 0) L.cap_rows = std::min(L.cap_rows, cap_rows_max);
  L.smem = 2 * ((size_t)L.cap_rows * per_row + (size_t)L.cap_trows * per_trow) + (size_t)L.cap_nnz * fixed_per_nnz +
           (size_t)(L.cap_trows + 1) * 4 + 64;
  int dev = 0, sms = 152, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSdSmemMax);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, kSdThreads, L.smem);
  L.blocks = (L.cap_rows > 0 && per > 0) ? std::min(H.ntiles, sms * per) : 0;
  return L;
}

bool csr_values_tiles(Handle& H, const fsa_theta& th, const __nv_bfloat16* A, const __nv_bfloat16* Alo, int m_pad,
                      int cap_rows_max) {
  if (H.ntiles <= 0 || m_pad % 64 != 0) return false;
  Operator& op = H.op;
  const size_t planes = Alo ? 2 : 1;
  const SdLaunch L = sd_launch(H, planes * kSdRowV * sizeof(__nv_bfloat16), 0, 2 * sizeof(int),
                               reinterpret_cast<const void*>(k_csr_values_tiles), cap_rows_max);
  if (L.blocks <= 0) return false;
  k_csr_values_tiles<<<L.blocks, kSdThreads, L.smem, H.stream>>>(
      H.ntiles, H.ptile.p, H.tile_bad.p, L.cap_rows, L.cap_nnz, L.cap_trows, H.n, m_pad, H.rowptr.p, H.col.p,
      H.scol.p, H.xs.p, H.ys.p, A, Alo, H.cov, th.sigma1_sq, th.rho, th.nugget, H.gamma, op.vals.p, op.vals32.p,
      op.D.p, op.D32.p, op.Dinv32.p);
  FSA_CHECK_LAUNCH();
  return true;
}

// ---------------------------------------------------------------------------
// gradient, sparse part
// ---------------------------------------------------------------------------
// Per nonzero (i, j): G_ij = sum_k X_ik Y_jk w_k (w_0 = -1, w_k = 1/l), then
//   s0 += dval/ds1 G = (val_ij - nugget [i = j]) / s1 G
//   sr += s1 r'(d) T(d) G  (j != i)            (the covariance part)
//   s2 += [i = j] G
// and the weight w_ij = T(d_ij) G_ij (T(0) = 1) of the low-rank part
//   sr -= sum_ij w_ij (b_i . a_j + a_i . q_j),  b = dK L^-T, q = b - A~ E.
__device__ __forceinline__ float grad_weight(int64_t i, int64_t j, int c, int ldc, const float* __restrict__ X,
                                             const float* __restrict__ Y, double val, const double* __restrict__ xs,
                                             const double* __restrict__ ys, int cov, double s1, double rho,
                                             double nug, double gamma, double& s0, double& sr, double& s2) {
  const float inv_l = c > 1 ? 1.0f / (float)(c - 1) : 0.f;
  const float4* x4 = reinterpret_cast<const float4*>(X + i * ldc);
  const float4* y4 = reinterpret_cast<const float4*>(Y + j * ldc);
  float gq[4] = {0.f, 0.f, 0.f, 0.f};   // four running sums (columns k mod 4), added pairwise
  for (int k4 = 0; k4 < ldc / 4; ++k4) {
    const float4 x = x4[k4], y = y4[k4];
    const float xv[4] = {x.x, x.y, x.z, x.w}, yv[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = 4 * k4 + q;
      if (k < c) gq[q] = fmaf(xv[q] * (k == 0 ? -1.0f : inv_l), yv[q], gq[q]);
    }
  }
  const float g = (gq[0] + gq[1]) + (gq[2] + gq[3]);
  const double gd = (double)g;
  if (j == i) {
    s0 += (val - nug) / s1 * gd;
    s2 += gd;
    return g;
  }
  const double d = sqrt(sqdist_rn(xs[i], ys[i], xs[j], ys[j]));
  const double tp = wendland(d, gamma);
  s0 += val / s1 * gd;
  sr += s1 * matern_dr(cov, d, rho) * tp * gd;
  return (float)(tp * gd);
}

__global__ void __launch_bounds__(kSdThreads, 1) k_grad_sparse_tiles(
    int ntiles, const int32_t* __restrict__ ptile, const int32_t* __restrict__ tile_bad, int cap_rows, int cap_nnz,
    int cap_trows, int64_t n, int m_pad, int c, int ldc, const int64_t* __restrict__ rowptr,
    const int32_t* __restrict__ col, const int32_t* __restrict__ scol, const double* __restrict__ vals,
    const double* __restrict__ xs, const double* __restrict__ ys, const float* __restrict__ X,
    const float* __restrict__ Y, const __nv_bfloat16* __restrict__ A, const __nv_bfloat16* __restrict__ B,
    const __nv_bfloat16* __restrict__ Q, int cov, double s1, double rho, double nug, double gamma,
    double* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double red[3][kSdThreads / 32];
  // per stage: A~ rows of the ranges | q rows of the ranges | b rows of the tile (64 BF16 each)
  const size_t sA = (size_t)cap_rows * 64, sB = (size_t)cap_trows * 64, sstage = 2 * sA + sB;
  __nv_bfloat16* st = reinterpret_cast<__nv_bfloat16*>(smraw);
  float* sw = reinterpret_cast<float*>(st + 2 * sstage);
  int* ssc = reinterpret_cast<int*>(sw + cap_nnz);
  int* srow = ssc + cap_nnz;
  int* srp = srow + cap_nnz;   // cap_trows + 1 row offsets
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int nkb = m_pad / 64;
  double s0 = 0.0, sr = 0.0, s2 = 0.0, sdl = 0.0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const TileRec T = load_tile(ptile, tile_bad, tile, cap_rows, cap_nnz, cap_trows);
    if (!T.staged) {
      for (int t = threadIdx.x; t < T.ne; t += kSdThreads) {
        const int64_t e = T.e0 + t;
        int64_t i = T.p0;
        while (rowptr[i + 1] <= e) ++i;
        const int64_t j = col[e];
        const float w = grad_weight(i, j, c, ldc, X, Y, vals[e], xs, ys, cov, s1, rho, nug, gamma, s0, sr, s2);
        float dl = 0.f;
        for (int kb = 0; kb < nkb; ++kb) {
          const uint32_t* aj = reinterpret_cast<const uint32_t*>(A + ((int64_t)kb * n + j) * 64);
          const uint32_t* ai = reinterpret_cast<const uint32_t*>(A + ((int64_t)kb * n + i) * 64);
          const uint32_t* bi = reinterpret_cast<const uint32_t*>(B + i * m_pad + kb * 64);
          const uint32_t* qj = reinterpret_cast<const uint32_t*>(Q + j * m_pad + kb * 64);
          for (int w2 = 0; w2 < 32; ++w2) {
            const float2 a = bf2f(aj[w2]), b = bf2f(bi[w2]), a2 = bf2f(ai[w2]), q = bf2f(qj[w2]);
            dl = fmaf(b.x, a.x, fmaf(b.y, a.y, dl));
            dl = fmaf(a2.x, q.x, fmaf(a2.y, q.y, dl));
          }
        }
        sdl += (double)(w * dl);
      }
      continue;
    }
    tile_rows(T, rowptr, scol, srow, ssc);
    for (int r = threadIdx.x; r <= T.nr; r += kSdThreads) srp[r] = (int)(rowptr[T.p0 + r] - T.e0);
    auto issue = [&](int kb) {
      __nv_bfloat16* sb = st + (size_t)(kb & 1) * sstage;
      const __nv_bfloat16* Ak = A + (int64_t)kb * n * 64;
      stage_rows(sb, 0, 64, Ak, 64, T.r0b, T.n0);
      stage_rows(sb, T.n0, 64, Ak, 64, T.r1b, T.n1);
      stage_rows(sb, T.n0 + T.n1, 64, Ak, 64, T.r2b, T.n2);
      const __nv_bfloat16* Qk = Q + kb * 64;
      stage_rows(sb + sA, 0, 64, Qk, m_pad, T.r0b, T.n0);
      stage_rows(sb + sA, T.n0, 64, Qk, m_pad, T.r1b, T.n1);
      stage_rows(sb + sA, T.n0 + T.n1, 64, Qk, m_pad, T.r2b, T.n2);
      stage_rows(sb + 2 * sA, 0, 64, B + kb * 64, m_pad, T.p0, T.nr);
      cpa_commit();
    };
    issue(0);
    __syncthreads();   // srow, ssc
    for (int t = threadIdx.x; t < T.ne; t += kSdThreads)
      sw[t] = grad_weight((int64_t)T.p0 + srow[t], col[T.e0 + t], c, ldc, X, Y, vals[T.e0 + t], xs, ys, cov, s1,
                          rho, nug, gamma, s0, sr, s2);
    for (int kb = 0; kb < nkb; ++kb) {
      if (kb + 1 < nkb) issue(kb + 1);
      else cpa_commit();
      cpa_wait<1>();
      __syncthreads();   // block kb staged by every thread; the weights written
      const uint32_t* sa = reinterpret_cast<const uint32_t*>(st + (size_t)(kb & 1) * sstage);
      const uint32_t* sq = sa + sA / 2;
      const uint32_t* sbr = sa + sA;
      for (int r = wib; r < T.nr; r += kSdWarps) {
        const int tb = srp[r], te = srp[r + 1];
        float px = 0.f, py = 0.f, qx = 0.f, qy = 0.f;
#pragma unroll 4
        for (int t = tb; t < te; ++t) {
          const float w = sw[t];
          const int rj = ssc[t];
          const float2 a = bf2f(sa[rj * 32 + lane]), q = bf2f(sq[rj * 32 + lane]);
          px = fmaf(w, a.x, px); py = fmaf(w, a.y, py);
          qx = fmaf(w, q.x, qx); qy = fmaf(w, q.y, qy);
        }
        const int ri = T.n0 + (T.p0 + r - T.r1b);
        const float2 ai = bf2f(sa[ri * 32 + lane]), bi = bf2f(sbr[r * 32 + lane]);
        sdl += (double)(bi.x * px + bi.y * py + ai.x * qx + ai.y * qy);
      }
      __syncthreads();   // stage kb & 1 is free for block kb + 2
    }
  }
  cpa_wait<0>();
  // fixed-order block reduction: warp sums, then the warps in order
  s0 = warp_sum(s0);
  s2 = warp_sum(s2);
  const double srt = warp_sum(sr - sdl);
  if (lane == 0) { red[0][wib] = s0; red[1][wib] = srt; red[2][wib] = s2; }
  __syncthreads();
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int w = 0; w < kSdThreads / 32; ++w) s += red[threadIdx.x][w];
    part[(int64_t)blockIdx.x * 3 + threadIdx.x] = s;
  }
}

int grad_sparse_tiles(Handle& H, int m_pad, int c, int ldc, const double* vals, const float* X, const float* Y,
                      const __nv_bfloat16* A, const __nv_bfloat16* B, const __nv_bfloat16* Q, const fsa_theta& th,
                      double* part, int max_blocks, int cap_rows_max) {
  if (H.ntiles <= 0 || m_pad % 64 != 0 || ldc % 4 != 0) return 0;
  const SdLaunch L = sd_launch(H, 2 * 64 * sizeof(__nv_bfloat16), 64 * sizeof(__nv_bfloat16),
                               3 * sizeof(int) + sizeof(float), reinterpret_cast<const void*>(k_grad_sparse_tiles),
                               cap_rows_max);
  if (L.blocks <= 0) return 0;
  const int blocks = std::min(L.blocks, max_blocks);
  k_grad_sparse_tiles<<<blocks, kSdThreads, L.smem, H.stream>>>(
      H.ntiles, H.ptile.p, H.tile_bad.p, L.cap_rows, L.cap_nnz, L.cap_trows, H.n, m_pad, c, ldc, H.rowptr.p, H.col.p,
      H.scol.p, vals, H.xs.p, H.ys.p, X, Y, A, B, Q, H.cov, th.sigma1_sq, th.rho, th.nugget, H.gamma, part);
  FSA_CHECK_LAUNCH();
  return blocks;
}

}  // namespace fsa
