// Tile kernels for the two sampled dense products of the mixed form (SDDMM-
// shaped work over the taper pattern, paper §2.1 and §2.2):
//
//   * the tapered residual values val_ij = (c(s_i, s_j) - a_i . a_j) T(d_ij)
//     and D_s,i = sigma1^2 - |a_i|^2 + nugget (Eq. eqfitcp), and
//   * the range derivative of those values (§2.2), with
//     d(a_i . a_j)/drho = b_i . a_j + a_i . q_j (b = dK L^-T, q = b - A~ E).
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

// the row of each of the tile's nonzeros (srow) and its staged column (ssc);
// err: the error word of the checked build's index checks
__device__ __forceinline__ void tile_rows(const TileRec& T, const int64_t* __restrict__ rowptr,
                                          const int32_t* __restrict__ scol, int* srow, int* ssc, unsigned* err) {
  for (int r = threadIdx.x; r < T.nr; r += kSdThreads) {
    const int tb = (int)(rowptr[T.p0 + r] - T.e0), te = (int)(rowptr[T.p0 + r + 1] - T.e0);
    if (!FSA_INDEX_OK(tb >= 0 && tb <= te && te <= T.ne, err)) continue;
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
    float* __restrict__ D32, float* __restrict__ Dinv32, unsigned* __restrict__ err) {
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
    tile_rows(T, rowptr, scol, srow, ssc, err);
    const int nst = T.n0 + T.n1 + T.n2;   // staged rows
    (void)nst;                            // read by the checked build only
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
          if (!FSA_INDEX_OK(ri >= 0 && ri < nst && rj >= 0 && rj < nst, err)) continue;
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
      op.D.p, op.D32.p, op.Dinv32.p, H.err);
  FSA_CHECK_LAUNCH();
  return true;
}

// ---------------------------------------------------------------------------
// range derivative of the tapered residual values (per nonzero)
// ---------------------------------------------------------------------------
// dval_ij = (s1 r'(d_ij) - dl_ij) T(d_ij) for j != i and -dl_ii on the
// diagonal (r(0) = 1 does not depend on rho, T(0) = 1), with
//   dl_ij = b_i . a_j + a_i . q_j = d(a_i . a_j)/drho,  b = dK L^-T, q = b - A~ E,
// every m-long row as a BF16 hi + lo pair (~2^-17).  The diagonal values are
// dD_s/drho.  Staged like the values kernel: per stage the A~ and q rows of
// the tile's three neighbour ranges and the b rows of its own rows.
__device__ __forceinline__ void write_dvalue(int64_t t, int64_t i, int64_t j, double dl,
                                             const double* __restrict__ xs, const double* __restrict__ ys, int cov,
                                             double s1, double rho, double gamma, float* __restrict__ dvals,
                                             float* __restrict__ dD) {
  if (j == i) {
    const float v = (float)(-dl);
    dvals[t] = v;
    dD[i] = v;
  } else {
    const double d = sqrt(sqdist_rn(xs[i], ys[i], xs[j], ys[j]));
    dvals[t] = (float)((s1 * matern_dr(cov, d, rho) - dl) * wendland(d, gamma));
  }
}

__device__ __forceinline__ double dl_rows_global(const __nv_bfloat16* __restrict__ A, const __nv_bfloat16* __restrict__ Alo,
                                                 const __nv_bfloat16* __restrict__ B, const __nv_bfloat16* __restrict__ Blo,
                                                 const __nv_bfloat16* __restrict__ Q, const __nv_bfloat16* __restrict__ Qlo,
                                                 int64_t n, int m_pad, int64_t i, int64_t j) {
  double s = 0.0;
  for (int kb = 0; kb < m_pad / 64; ++kb) {
    const int64_t oi = ((int64_t)kb * n + i) * 64, oj = ((int64_t)kb * n + j) * 64;
    s += (double)dot_block(reinterpret_cast<const uint4*>(B + oi), reinterpret_cast<const uint4*>(A + oj),
                           reinterpret_cast<const uint4*>(Blo + oi), reinterpret_cast<const uint4*>(Alo + oj));
    s += (double)dot_block(reinterpret_cast<const uint4*>(A + oi), reinterpret_cast<const uint4*>(Q + oj),
                           reinterpret_cast<const uint4*>(Alo + oi), reinterpret_cast<const uint4*>(Qlo + oj));
  }
  return s;
}

__global__ void __launch_bounds__(kSdThreads, 1) k_dvals_tiles(
    int ntiles, const int32_t* __restrict__ ptile, const int32_t* __restrict__ tile_bad, int cap_rows, int cap_nnz,
    int cap_trows, int64_t n, int m_pad, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
    const int32_t* __restrict__ scol, const double* __restrict__ xs, const double* __restrict__ ys,
    const __nv_bfloat16* __restrict__ A, const __nv_bfloat16* __restrict__ Alo, const __nv_bfloat16* __restrict__ B,
    const __nv_bfloat16* __restrict__ Blo, const __nv_bfloat16* __restrict__ Q, const __nv_bfloat16* __restrict__ Qlo,
    int cov, double s1, double rho, double gamma, float* __restrict__ dvals, float* __restrict__ dD,
    unsigned* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smraw[];
  // per stage: A hi, A lo, q hi, q lo of the ranges (cap_rows rows each), then b hi, b lo of the tile rows
  const size_t plane = (size_t)cap_rows * kSdRowV, tplane = (size_t)cap_trows * kSdRowV;
  const size_t sstage = 4 * plane + 2 * tplane;
  __nv_bfloat16* st = reinterpret_cast<__nv_bfloat16*>(smraw);
  int* srow = reinterpret_cast<int*>(st + 2 * sstage);
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
        write_dvalue(e, i, j, dl_rows_global(A, Alo, B, Blo, Q, Qlo, n, m_pad, i, j), xs, ys, cov, s1, rho, gamma,
                     dvals, dD);
      }
      continue;
    }
    tile_rows(T, rowptr, scol, srow, ssc, err);
    const int nst = T.n0 + T.n1 + T.n2;   // staged rows
    (void)nst;                            // read by the checked build only
    auto issue = [&](int kb) {
      __nv_bfloat16* sb = st + (size_t)(kb & 1) * sstage;
      const __nv_bfloat16* srcs[4] = {A, Alo, Q, Qlo};
      for (int p = 0; p < 4; ++p) {
        const __nv_bfloat16* src = srcs[p] + (int64_t)kb * n * 64;
        __nv_bfloat16* dst = sb + p * plane;
        stage_rows(dst, 0, kSdRowV, src, 64, T.r0b, T.n0);
        stage_rows(dst, T.n0, kSdRowV, src, 64, T.r1b, T.n1);
        stage_rows(dst, T.n0 + T.n1, kSdRowV, src, 64, T.r2b, T.n2);
      }
      stage_rows(sb + 4 * plane, 0, kSdRowV, B + (int64_t)kb * n * 64, 64, T.p0, T.nr);
      stage_rows(sb + 4 * plane + tplane, 0, kSdRowV, Blo + (int64_t)kb * n * 64, 64, T.p0, T.nr);
      cpa_commit();
    };
    issue(0);
    double acc[kSdPer] = {0.0, 0.0, 0.0, 0.0};
    for (int kb = 0; kb < nkb; ++kb) {
      if (kb + 1 < nkb) issue(kb + 1);
      else cpa_commit();
      cpa_wait<1>();
      __syncthreads();
      const __nv_bfloat16* sb = st + (size_t)(kb & 1) * sstage;
#pragma unroll
      for (int u = 0; u < kSdPer; ++u) {
        const int t = threadIdx.x + u * kSdThreads;
        if (t < T.ne) {
          const int r = srow[t];
          const int ri = T.n0 + (T.p0 + r - T.r1b), rj = ssc[t];
          if (!FSA_INDEX_OK(r >= 0 && r < T.nr && ri >= 0 && ri < nst && rj >= 0 && rj < nst, err)) continue;
          auto row = [&](int pl, int k) { return reinterpret_cast<const uint4*>(sb + pl * plane + (size_t)k * kSdRowV); };
          const uint4* bh = reinterpret_cast<const uint4*>(sb + 4 * plane + (size_t)r * kSdRowV);
          const uint4* bl = reinterpret_cast<const uint4*>(sb + 4 * plane + tplane + (size_t)r * kSdRowV);
          acc[u] += (double)dot_block(bh, row(0, rj), bl, row(1, rj));
          acc[u] += (double)dot_block(row(0, ri), row(2, rj), row(1, ri), row(3, rj));
        }
      }
      __syncthreads();   // stage kb & 1 is free for block kb + 2
    }
#pragma unroll
    for (int u = 0; u < kSdPer; ++u) {
      const int t = threadIdx.x + u * kSdThreads;
      if (t < T.ne) {
        const int64_t e = T.e0 + t;
        write_dvalue(e, (int64_t)T.p0 + srow[t], col[e], acc[u], xs, ys, cov, s1, rho, gamma, dvals, dD);
      }
    }
    __syncthreads();   // srow, ssc are rewritten by the next tile
  }
  cpa_wait<0>();
}

// one warp per nonzero, from global memory (handles without tiles)
__global__ void k_dvals_rows(int64_t n, int m_pad, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                             const double* __restrict__ xs, const double* __restrict__ ys,
                             const __nv_bfloat16* __restrict__ A, const __nv_bfloat16* __restrict__ Alo,
                             const __nv_bfloat16* __restrict__ B, const __nv_bfloat16* __restrict__ Blo,
                             const __nv_bfloat16* __restrict__ Q, const __nv_bfloat16* __restrict__ Qlo, int cov,
                             double s1, double rho, double gamma, float* __restrict__ dvals, float* __restrict__ dD) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e)
      write_dvalue(e, i, col[e], dl_rows_global(A, Alo, B, Blo, Q, Qlo, n, m_pad, i, col[e]), xs, ys, cov, s1, rho,
                   gamma, dvals, dD);
}

bool dvals_tiles(Handle& H, const fsa_theta& th, int m_pad, const __nv_bfloat16* A, const __nv_bfloat16* Alo,
                 const __nv_bfloat16* B, const __nv_bfloat16* Blo, const __nv_bfloat16* Q, const __nv_bfloat16* Qlo,
                 float* dvals, float* dD, int cap_rows_max) {
  if (H.ntiles <= 0 || m_pad % 64 != 0) return false;
  const SdLaunch L = sd_launch(H, 4 * kSdRowV * sizeof(__nv_bfloat16), 2 * kSdRowV * sizeof(__nv_bfloat16),
                               2 * sizeof(int), reinterpret_cast<const void*>(k_dvals_tiles), cap_rows_max);
  if (L.blocks <= 0) return false;
  k_dvals_tiles<<<L.blocks, kSdThreads, L.smem, H.stream>>>(
      H.ntiles, H.ptile.p, H.tile_bad.p, L.cap_rows, L.cap_nnz, L.cap_trows, H.n, m_pad, H.rowptr.p, H.col.p,
      H.scol.p, H.xs.p, H.ys.p, A, Alo, B, Blo, Q, Qlo, H.cov, th.sigma1_sq, th.rho, H.gamma, dvals, dD, H.err);
  FSA_CHECK_LAUNCH();
  return true;
}

void dvals_rows(Handle& H, const fsa_theta& th, int m_pad, const __nv_bfloat16* A, const __nv_bfloat16* Alo,
                const __nv_bfloat16* B, const __nv_bfloat16* Blo, const __nv_bfloat16* Q, const __nv_bfloat16* Qlo,
                float* dvals, float* dD) {
  k_dvals_rows<<<grid_for(H.n, 128), 128, 0, H.stream>>>(H.n, m_pad, H.rowptr.p, H.col.p, H.xs.p, H.ys.p, A, Alo,
                                                          B, Blo, Q, Qlo, H.cov, th.sigma1_sq, th.rho, H.gamma,
                                                          dvals, dD);
  FSA_CHECK_LAUNCH();
}

void dvals_mixed(Handle& H, const fsa_theta& th, int m_pad, const __nv_bfloat16* A, const __nv_bfloat16* Alo,
                 const __nv_bfloat16* B, const __nv_bfloat16* Blo, const __nv_bfloat16* Q, const __nv_bfloat16* Qlo,
                 float* dvals, float* dD) {
  FSA_REQUIRE(m_pad % 64 == 0 && A && Alo && B && Blo && Q && Qlo, FSA_ERR_UNSUPPORTED,
              "range derivative values need BF16 pairs of A~, b and q with m_pad % 64 == 0");
  if (!dvals_tiles(H, th, m_pad, A, Alo, B, Blo, Q, Qlo, dvals, dD, 0))
    dvals_rows(H, th, m_pad, A, Alo, B, Blo, Q, Qlo, dvals, dD);
}

}  // namespace fsa
