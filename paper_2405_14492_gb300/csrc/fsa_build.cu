// Taper-support neighbour structure (paper §2.1: the taper makes Sigma_s
// sparse; pairs with |s_i - s_j| >= gamma are zero).  Cell-grid binning with
// cell side >= gamma, a deterministic counting sort of the points by cell
// (internal order: cell id, then original index), and a two-pass CSR build
// (count, exclusive scan, fill) over the 3x3 cell stencil.
#include <algorithm>
#include <vector>

#include "fsa_internal.cuh"

namespace fsa {

// ---------------------------------------------------------------------------
// exclusive scan (multi-level, deterministic)
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 512;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename T>
__global__ void scan_tile_kernel(const T* __restrict__ in, T* __restrict__ out, int64_t n,
                                 T* __restrict__ block_sums) {
  __shared__ T warp_tot[kScanThreads / 32];
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  T v[kScanItems];
  T run = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + k;
    T x = (i < n) ? in[i] : (T)0;
    v[k] = run;
    run += x;
  }
  // inclusive scan of per-thread totals across the block
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    T w = (lane < kScanThreads / 32) ? warp_tot[lane] : (T)0;
    T wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = wi - w;  // exclusive warp offsets
  }
  __syncthreads();
  T offset = warp_tot[wid] + (incl - run);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + k;
    if (i < n) out[i] = v[k] + offset;
  }
  if (threadIdx.x == kScanThreads - 1 && block_sums) block_sums[blockIdx.x] = offset + run;
}

template <typename T>
__global__ void scan_add_kernel(T* __restrict__ out, int64_t n, const T* __restrict__ block_offsets) {
  int64_t i = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
  T add = block_offsets[blockIdx.x];
  for (int k = 0; k < kScanItems; ++k, i += kScanThreads)
    if (i < n) out[i] += add;
}

// out[i] = sum_{j<i} in[i]; returns total via *total_dev (device pointer, may be null)
template <typename T>
void exclusive_scan(const T* in, T* out, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  int64_t nb = (n + kScanTile - 1) / kScanTile;
  if (nb == 1) {
    scan_tile_kernel<T><<<1, kScanThreads, 0, s>>>(in, out, n, nullptr);
    FSA_CHECK_LAUNCH();
    return;
  }
  T* sums = nullptr;
  FSA_CUDA(cudaMallocAsync(&sums, sizeof(T) * nb * 2, s));
  scan_tile_kernel<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, sums);
  FSA_CHECK_LAUNCH();
  exclusive_scan<T>(sums, sums + nb, nb, s);
  scan_add_kernel<T><<<(unsigned)nb, kScanThreads, 0, s>>>(out, n, sums + nb);
  FSA_CHECK_LAUNCH();
  FSA_CUDA(cudaFreeAsync(sums, s));
}
template void exclusive_scan<int64_t>(const int64_t*, int64_t*, int64_t, cudaStream_t);
template void exclusive_scan<int32_t>(const int32_t*, int32_t*, int64_t, cudaStream_t);

// ---------------------------------------------------------------------------
// bounding box + finiteness
// ---------------------------------------------------------------------------
__global__ void bbox_partial_kernel(const double* __restrict__ pts, int64_t n, double* __restrict__ part,
                                    unsigned* __restrict__ err) {
  double mnx = INFINITY, mny = INFINITY, mxx = -INFINITY, mxy = -INFINITY;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double x = pts[2 * i], y = pts[2 * i + 1];
    if (!isfinite(x) || !isfinite(y)) atomicOr(err, kErrNaN);
    mnx = fmin(mnx, x); mxx = fmax(mxx, x);
    mny = fmin(mny, y); mxy = fmax(mxy, y);
  }
  __shared__ double sh[4][256];
  sh[0][threadIdx.x] = mnx; sh[1][threadIdx.x] = mny;
  sh[2][threadIdx.x] = mxx; sh[3][threadIdx.x] = mxy;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sh[0][threadIdx.x] = fmin(sh[0][threadIdx.x], sh[0][threadIdx.x + o]);
      sh[1][threadIdx.x] = fmin(sh[1][threadIdx.x], sh[1][threadIdx.x + o]);
      sh[2][threadIdx.x] = fmax(sh[2][threadIdx.x], sh[2][threadIdx.x + o]);
      sh[3][threadIdx.x] = fmax(sh[3][threadIdx.x], sh[3][threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 4; ++k) part[4 * blockIdx.x + k] = sh[k][0];
}

__global__ void bbox_final_kernel(const double* __restrict__ part, int nparts, double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double b[4] = {INFINITY, INFINITY, -INFINITY, -INFINITY};
  for (int p = 0; p < nparts; ++p) {
    b[0] = fmin(b[0], part[4 * p]); b[1] = fmin(b[1], part[4 * p + 1]);
    b[2] = fmax(b[2], part[4 * p + 2]); b[3] = fmax(b[3], part[4 * p + 3]);
  }
  for (int k = 0; k < 4; ++k) out[k] = b[k];
}

// ---------------------------------------------------------------------------
// binning and counting sort
// ---------------------------------------------------------------------------
__device__ __forceinline__ int cell_coord(double v, double lo, double h, int nc) {
  int c = (int)floor((v - lo) / h);
  return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

__global__ void cell_count_kernel(const double* __restrict__ pts, int64_t n, Grid g,
                                  int32_t* __restrict__ cell_of, int32_t* __restrict__ count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int cx = cell_coord(pts[2 * i], g.x0, g.hx, g.ncx);
    int cy = cell_coord(pts[2 * i + 1], g.y0, g.hy, g.ncy);
    int c = cy * g.ncx + cx;
    cell_of[i] = c;
    atomicAdd(&count[c], 1);
  }
}

__global__ void cell_scatter_kernel(const int32_t* __restrict__ cell_of, int64_t n,
                                    const int32_t* __restrict__ start, int32_t* __restrict__ cursor,
                                    int64_t* __restrict__ perm) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int c = cell_of[i];
    int pos = start[c] + atomicAdd(&cursor[c], 1);
    perm[pos] = i;
  }
}

// sort each cell's points by original index, so that the order inside a cell
// does not depend on the scatter's atomics
__global__ void cell_sort_kernel(const int32_t* __restrict__ start, const int32_t* __restrict__ count,
                                 int ncells, int64_t* __restrict__ perm) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x)
    heap_sort_thread(perm + start[c], (int64_t)count[c]);
}

__global__ void gather_points_kernel(const double* __restrict__ pts, const int64_t* __restrict__ perm,
                                     int64_t n, double* __restrict__ xs, double* __restrict__ ys,
                                     int64_t* __restrict__ iperm) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = perm[k];
    xs[k] = pts[2 * i];
    ys[k] = pts[2 * i + 1];
    iperm[i] = k;
  }
}

// ---------------------------------------------------------------------------
// neighbour count and fill over the 3x3 cell stencil (cells in ascending id
// order, so columns come out ascending in internal order)
// ---------------------------------------------------------------------------
template <bool kFill>
__global__ void neighbour_kernel(const double* __restrict__ qx, const double* __restrict__ qy, int64_t nq,
                                 const double* __restrict__ xs, const double* __restrict__ ys,
                                 const int32_t* __restrict__ cell_start, const int32_t* __restrict__ cell_count,
                                 Grid g, double gamma2, int64_t* __restrict__ counts,
                                 const int64_t* __restrict__ rowptr, int32_t* __restrict__ col) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq;
       i += (int64_t)gridDim.x * blockDim.x) {
    double xi = qx[i], yi = qy[i];
    int cx = cell_coord(xi, g.x0, g.hx, g.ncx);
    int cy = cell_coord(yi, g.y0, g.hy, g.ncy);
    int64_t cnt = 0;
    int64_t w = kFill ? rowptr[i] : 0;
    for (int dy = -1; dy <= 1; ++dy) {
      int yy = cy + dy;
      if (yy < 0 || yy >= g.ncy) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        int xx = cx + dx;
        if (xx < 0 || xx >= g.ncx) continue;
        int c = yy * g.ncx + xx;
        int b = cell_start[c], e = b + cell_count[c];
        for (int j = b; j < e; ++j) {
          double d2 = sqdist_rn(xi, yi, xs[j], ys[j]);
          if (d2 < gamma2) {
            if (kFill) col[w++] = j;
            else ++cnt;
          }
        }
      }
    }
    if (!kFill) counts[i] = cnt;
  }
}

// ---------------------------------------------------------------------------
// export of the pattern in the caller's order, columns ascending
// ---------------------------------------------------------------------------
__global__ void orig_counts_kernel(const int64_t* __restrict__ rowptr, const int64_t* __restrict__ iperm,
                                   int64_t n, int64_t* __restrict__ cnt) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    int64_t k = iperm[r];
    cnt[r] = rowptr[k + 1] - rowptr[k];
  }
}

__global__ void orig_fill_kernel(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                 const int64_t* __restrict__ perm, const int64_t* __restrict__ iperm,
                                 int64_t n, const int64_t* __restrict__ rowptr_o, int32_t* __restrict__ col_o) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    int64_t k = iperm[r];
    int64_t b = rowptr[k], e = rowptr[k + 1], o = rowptr_o[r];
    for (int64_t t = b; t < e; ++t) col_o[o + (t - b)] = (int32_t)perm[col[t]];
    heap_sort_thread(col_o + o, e - b);
  }
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
Grid make_grid(const double bb[4], double gamma, int64_t n) {
  Grid g;
  double ex = bb[2] - bb[0], ey = bb[3] - bb[1];
  double h = gamma * (1.0 + 1e-6);
  int64_t ncx = (int64_t)floor(ex / h), ncy = (int64_t)floor(ey / h);
  if (ncx < 1) ncx = 1;
  if (ncy < 1) ncy = 1;
  // cap the number of cells at ~4n (larger cells only add candidates)
  int64_t cap = 4 * n + 16;
  while (ncx * ncy > cap) {
    ncx = (ncx + 1) / 2;
    ncy = (ncy + 1) / 2;
  }
  g.ncx = (int)ncx; g.ncy = (int)ncy;
  g.x0 = bb[0]; g.y0 = bb[1];
  g.hx = ex > 0 ? ex / ncx : 1.0;
  g.hy = ey > 0 ? ey / ncy : 1.0;
  if (g.hx < h) g.hx = h;
  if (g.hy < h) g.hy = h;
  return g;
}

void build_tiles(Handle& H);

// per nonzero of a tile's rows: the row of its column within the tile's
// staged ranges (range 0, then 1, then 2), or -1 outside them
__global__ void k_tile_scol(const int64_t* __restrict__ tiles, const int64_t* __restrict__ rowptr,
                            const int32_t* __restrict__ col, int32_t* __restrict__ scol,
                            int32_t* __restrict__ bad) {
  const int64_t* d = tiles + (int64_t)blockIdx.x * 8;
  const int64_t e0 = rowptr[d[0]], e1 = rowptr[d[1]];
  const int64_t n0 = d[3] - d[2], n1 = d[5] - d[4], n2 = d[7] - d[6];
  for (int64_t t = e0 + threadIdx.x; t < e1; t += blockDim.x) {
    const int64_t j = col[t];
    int64_t r = -1;
    if (j >= d[4] && j < d[5]) r = n0 + (j - d[4]);
    else if (j >= d[2] && j < d[3]) r = j - d[2];
    else if (j >= d[6] && j < d[7]) r = n0 + n1 + (j - d[6]);
    (void)n2;
    scol[t] = (int32_t)r;
    if (r < 0) bad[blockIdx.x] = 1;
  }
}

// Row groups of the SpMM tiles.  A tile's rows p0 .. p1 - 1 are cut into
// groups of kGrpRows consecutive rows; the union list of a group holds every
// staged row that is a taper neighbour of one of its rows, in ascending order.
// The staged index grows with the column index (the ranges lie in ascending
// order), so each row's nonzeros appear in its list in CSR order.  Both passes
// mark the group's staged rows in a bitmap of the tile's staged rows in shared
// memory; tiles with more than kGrpMaxStaged staged rows are marked bad (the
// SpMM then gathers their rows from global memory).
constexpr int kGrpMaxStaged = 16384;

__device__ __forceinline__ void grp_mark(uint32_t* bits, int nw, int64_t eb, int64_t ee,
                                         const int32_t* __restrict__ scol) {
  for (int w = threadIdx.x; w < nw; w += blockDim.x) bits[w] = 0u;
  __syncthreads();
  for (int64_t e = eb + threadIdx.x; e < ee; e += blockDim.x) {
    const int sr = scol[e];
    atomicOr(&bits[sr >> 5], 1u << (sr & 31));
  }
  __syncthreads();
}

// pass 1: cnt[gbase[t] + j] = entries of group j of tile t
__global__ void k_grp_count(const int64_t* __restrict__ tiles, const int64_t* __restrict__ rowptr,
                            const int32_t* __restrict__ scol, int32_t* __restrict__ bad,
                            const int32_t* __restrict__ gbase, int32_t* __restrict__ cnt) {
  extern __shared__ uint32_t bits[];
  __shared__ int tot;
  const int t = blockIdx.x;
  const int64_t* d = tiles + (int64_t)t * 8;
  const int64_t p0 = d[0], p1 = d[1];
  const int64_t ns = (d[3] - d[2]) + (d[5] - d[4]) + (d[7] - d[6]);
  const int ng = (int)((p1 - p0 + kGrpRows - 1) / kGrpRows);
  const int32_t g0 = gbase[t];
  if (bad[t] || ns > kGrpMaxStaged) {
    __syncthreads();   // every thread has read bad[t] before it changes
    if (threadIdx.x == 0) bad[t] = 1;
    for (int j = threadIdx.x; j < ng; j += blockDim.x) cnt[g0 + j] = 0;
    return;
  }
  const int nw = (int)((ns + 31) / 32);
  for (int j = 0; j < ng; ++j) {
    const int64_t ra = p0 + (int64_t)j * kGrpRows, rz = min(p1, ra + kGrpRows);
    if (threadIdx.x == 0) tot = 0;
    grp_mark(bits, nw, rowptr[ra], rowptr[rz], scol);
    int c = 0;
    for (int w = threadIdx.x; w < nw; w += blockDim.x) c += __popc(bits[w]);
    c = warp_sum(c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&tot, c);
    __syncthreads();
    if (threadIdx.x == 0) cnt[g0 + j] = tot;
    __syncthreads();
  }
}

// pass 2: the entries (src, kEntWords int32 each, preset to -1): word 0 the staged
// row, word 1 + g the nonzero of the group's row g in that column, relative
// to the tile's first nonzero
__global__ void k_grp_fill(const int64_t* __restrict__ tiles, const int32_t* __restrict__ ptile,
                           const int64_t* __restrict__ rowptr, const int32_t* __restrict__ scol,
                           const int32_t* __restrict__ bad, const int32_t* __restrict__ gofs,
                           int32_t* __restrict__ src) {
  extern __shared__ uint32_t sm[];
  const int t = blockIdx.x;
  if (bad[t]) return;
  const int64_t* d = tiles + (int64_t)t * 8;
  const int32_t* rec = ptile + (int64_t)t * kTileWords;
  const int64_t p0 = d[0], p1 = d[1];
  const int64_t ns = (d[3] - d[2]) + (d[5] - d[4]) + (d[7] - d[6]);
  const int ng = (int)((p1 - p0 + kGrpRows - 1) / kGrpRows);
  const int nw = (int)((ns + 31) / 32);
  uint32_t* bits = sm;
  uint32_t* pre = sm + nw;
  const int64_t e0 = rowptr[p0];
  const int32_t* go = gofs + rec[11];
  const int64_t ent0 = (int64_t)(uint32_t)rec[12] | ((int64_t)rec[13] << 32);
  const int lane = threadIdx.x & 31;
  for (int j = 0; j < ng; ++j) {
    const int64_t ra = p0 + (int64_t)j * kGrpRows, rz = min(p1, ra + kGrpRows);
    grp_mark(bits, nw, rowptr[ra], rowptr[rz], scol);
    // exclusive prefix of the words' popcounts (first warp)
    if (threadIdx.x < 32) {
      uint32_t run = 0;
      for (int w0 = 0; w0 < nw; w0 += 32) {
        const int w = w0 + lane;
        const uint32_t own = w < nw ? (uint32_t)__popc(bits[w]) : 0u;
        uint32_t v = own;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
          if (lane >= o) v += y;
        }
        if (w < nw) pre[w] = run + v - own;
        run += __shfl_sync(0xffffffffu, v, 31);
      }
    }
    __syncthreads();
    const int64_t base = ent0 + go[j];
    auto rank = [&](int sr) {
      const uint32_t w = bits[sr >> 5];
      return (int64_t)pre[sr >> 5] + __popc(w & ((1u << (sr & 31)) - 1u));
    };
    for (int sr = threadIdx.x; sr < (int)ns; sr += blockDim.x)
      if ((bits[sr >> 5] >> (sr & 31)) & 1u) src[(base + rank(sr)) * kEntWords] = sr;
    for (int64_t r = ra; r < rz; ++r) {
      const int g = (int)(r - ra);
      for (int64_t e = rowptr[r] + threadIdx.x; e < rowptr[r + 1]; e += blockDim.x)
        src[(base + rank(scol[e])) * kEntWords + 1 + g] = (int32_t)(e - e0);
    }
    __syncthreads();
  }
}

void build_structure(Handle& H, const double* locs_host) {
  cudaStream_t s = H.stream;
  int64_t n = H.n;
  DevPtr<double> pts(2 * n);
  FSA_CUDA(cudaMemcpyAsync(pts.p, locs_host, sizeof(double) * 2 * n, cudaMemcpyHostToDevice, s));
  // bounding box
  const int nparts = 304;
  DevPtr<double> part(4 * nparts), bb(4);
  bbox_partial_kernel<<<nparts, 256, 0, s>>>(pts.p, n, part.p, H.err);
  FSA_CHECK_LAUNCH();
  bbox_final_kernel<<<1, 32, 0, s>>>(part.p, nparts, bb.p);
  FSA_CHECK_LAUNCH();
  double hb[4];
  FSA_CUDA(cudaMemcpyAsync(hb, bb.p, sizeof(hb), cudaMemcpyDeviceToHost, s));
  unsigned herr = 0;
  FSA_CUDA(cudaMemcpyAsync(&herr, H.err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  FSA_CUDA(cudaStreamSynchronize(s));
  FSA_REQUIRE(!(herr & kErrNaN), FSA_ERR_NAN, "non-finite location coordinates");
  H.grid = make_grid(hb, H.gamma, n);
  int ncells = H.grid.ncx * H.grid.ncy;
  // counting sort by cell
  DevPtr<int32_t> cell_of(n), count(ncells), cursor(ncells);
  H.cell_start.alloc(ncells);
  H.cell_count.alloc(ncells);
  FSA_CUDA(cudaMemsetAsync(count.p, 0, sizeof(int32_t) * ncells, s));
  FSA_CUDA(cudaMemsetAsync(cursor.p, 0, sizeof(int32_t) * ncells, s));
  unsigned gb = grid_for(n, 256);
  cell_count_kernel<<<gb, 256, 0, s>>>(pts.p, n, H.grid, cell_of.p, count.p);
  FSA_CHECK_LAUNCH();
  exclusive_scan<int32_t>(count.p, H.cell_start.p, ncells, s);
  FSA_CUDA(cudaMemcpyAsync(H.cell_count.p, count.p, sizeof(int32_t) * ncells, cudaMemcpyDeviceToDevice, s));
  H.perm.alloc(n);
  H.iperm.alloc(n);
  cell_scatter_kernel<<<gb, 256, 0, s>>>(cell_of.p, n, H.cell_start.p, cursor.p, H.perm.p);
  FSA_CHECK_LAUNCH();
  cell_sort_kernel<<<grid_for(ncells, 256), 256, 0, s>>>(H.cell_start.p, H.cell_count.p, ncells, H.perm.p);
  FSA_CHECK_LAUNCH();
  H.xs.alloc(n);
  H.ys.alloc(n);
  gather_points_kernel<<<gb, 256, 0, s>>>(pts.p, H.perm.p, n, H.xs.p, H.ys.p, H.iperm.p);
  FSA_CHECK_LAUNCH();
  // CSR: count, scan, fill
  DevPtr<int64_t> counts(n + 1);
  FSA_CUDA(cudaMemsetAsync(counts.p + n, 0, sizeof(int64_t), s));
  double g2 = H.gamma * H.gamma;
  neighbour_kernel<false><<<gb, 256, 0, s>>>(H.xs.p, H.ys.p, n, H.xs.p, H.ys.p, H.cell_start.p,
                                             H.cell_count.p, H.grid, g2, counts.p, nullptr, nullptr);
  FSA_CHECK_LAUNCH();
  H.rowptr.alloc(n + 2);   // one spare entry: the SpMM copies row pointers in 16-byte units
  exclusive_scan<int64_t>(counts.p, H.rowptr.p, n + 1, s);
  int64_t nnz = 0;
  FSA_CUDA(cudaMemcpyAsync(&nnz, H.rowptr.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  FSA_CUDA(cudaStreamSynchronize(s));
  FSA_REQUIRE(nnz < (int64_t)1 << 40, FSA_ERR_ARG, "taper pattern too large");
  H.nnz = nnz;
  H.col.alloc(nnz);
  neighbour_kernel<true><<<gb, 256, 0, s>>>(H.xs.p, H.ys.p, n, H.xs.p, H.ys.p, H.cell_start.p,
                                            H.cell_count.p, H.grid, g2, nullptr, H.rowptr.p, H.col.p);
  FSA_CHECK_LAUNCH();
  build_tiles(H);
  FSA_CUDA(cudaStreamSynchronize(s));
}

// Tiles of about `rows` points: each grid row of cells is cut into runs of
// cells holding at least that many points; the taper neighbours of a run's
// points lie in the run's cells widened by one on each side, in the rows
// above, at and below (cell side >= gamma), i.e. in three contiguous ranges of
// the internal order.  Per tile 8 int64: p0, p1, then [begin, end) of the
// three ranges.
static std::vector<int64_t> cut_tiles(const std::vector<int32_t>& start, const std::vector<int32_t>& count, int ncx,
                                      int ncy, int64_t rows, int64_t* max_staged) {
  auto range = [&](int cy, int cxa, int cxb, int64_t* out) {
    if (cy < 0 || cy >= ncy) { out[0] = out[1] = 0; return; }
    const int a = std::max(cxa - 1, 0), b = std::min(cxb + 1, ncx - 1);
    const int64_t c0 = (int64_t)cy * ncx + a, c1 = (int64_t)cy * ncx + b;
    out[0] = start[c0];
    out[1] = (int64_t)start[c1] + count[c1];
  };
  std::vector<int64_t> t;
  int64_t ms = 0;
  for (int cy = 0; cy < ncy; ++cy) {
    int cxa = 0;
    int64_t acc = 0;
    for (int cx = 0; cx < ncx; ++cx) {
      acc += count[(int64_t)cy * ncx + cx];
      if (acc >= rows || cx == ncx - 1) {
        if (acc > 0) {
          int64_t d[8];
          d[0] = start[(int64_t)cy * ncx + cxa];
          d[1] = (int64_t)start[(int64_t)cy * ncx + cx] + count[(int64_t)cy * ncx + cx];
          range(cy - 1, cxa, cx, d + 2);
          range(cy, cxa, cx, d + 4);
          range(cy + 1, cxa, cx, d + 6);
          ms = std::max(ms, (d[3] - d[2]) + (d[5] - d[4]) + (d[7] - d[6]));
          t.insert(t.end(), d, d + 8);
        }
        cxa = cx + 1;
        acc = 0;
      }
    }
  }
  if (max_staged) *max_staged = ms;
  return t;
}

// tile records (kTileWords int32; words 11-15 zero): p0, rows, (begin,
// length) of the three ranges, first nonzero (low, high 32 bits), nonzeros
static std::vector<int32_t> tile_records(const std::vector<int64_t>& t, const std::vector<int64_t>& rp) {
  const int nt = (int)(t.size() / 8);
  std::vector<int32_t> pt((size_t)std::max(nt, 1) * kTileWords, 0);
  for (int k = 0; k < nt; ++k) {
    const int64_t* d = &t[8 * (size_t)k];
    int32_t* o = &pt[kTileWords * (size_t)k];
    const int64_t e0 = rp[d[0]];
    o[0] = (int32_t)d[0];
    o[1] = (int32_t)(d[1] - d[0]);
    for (int r = 0; r < 3; ++r) {
      o[2 + 2 * r] = (int32_t)d[2 + 2 * r];
      o[3 + 2 * r] = (int32_t)(d[3 + 2 * r] - d[2 + 2 * r]);
    }
    o[8] = (int32_t)(uint32_t)((uint64_t)e0 & 0xffffffffu);
    o[9] = (int32_t)(e0 >> 32);
    o[10] = (int32_t)(rp[d[1]] - e0);
  }
  return pt;
}

// The SpMM's own tiling (kSpTileRows) and the row groups of its tiles: the
// records (words 11-15: offset of the tile's group offsets in gofs, first
// union entry, union entries, bad flag), the group offsets and the union
// entries' sources.  Its staged columns and bad flags are needed only here.
static void build_spmm_groups(Handle& H, const std::vector<int64_t>& t, const std::vector<int64_t>& rp) {
  cudaStream_t s = H.stream;
  const int nt = (int)(t.size() / 8);
  H.sp_ntiles = nt;
  std::vector<int32_t> pt = tile_records(t, rp);
  std::vector<int32_t> gbase(std::max(nt, 1), 0);
  int64_t ngroups = 0;
  for (int k = 0; k < nt; ++k) {
    gbase[k] = (int32_t)ngroups;
    ngroups += (pt[kTileWords * (size_t)k + 1] + kGrpRows - 1) / kGrpRows;
  }
  FSA_REQUIRE(ngroups + nt + 4 < ((int64_t)1 << 31), FSA_ERR_ARG, "too many SpMM row groups");
  H.grp_entries = 0;
  std::vector<int32_t> go((size_t)(ngroups + nt + 4), 0);
  DevPtr<int64_t> tiles(std::max<size_t>(t.size(), 8));
  DevPtr<int32_t> scol(H.nnz + 4), bad(std::max(nt, 1));
  if (nt > 0) {
    FSA_CUDA(cudaMemcpyAsync(tiles.p, t.data(), sizeof(int64_t) * t.size(), cudaMemcpyHostToDevice, s));
    FSA_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int32_t) * nt, s));
    k_tile_scol<<<nt, 256, 0, s>>>(tiles.p, H.rowptr.p, H.col.p, scol.p, bad.p);
    FSA_CHECK_LAUNCH();
    // union-list sizes of the row groups
    DevPtr<int32_t> gb(nt), cnt(std::max<int64_t>(ngroups, 1));
    FSA_CUDA(cudaMemcpyAsync(gb.p, gbase.data(), sizeof(int32_t) * nt, cudaMemcpyHostToDevice, s));
    const size_t bits_bytes = (size_t)(kGrpMaxStaged / 32) * sizeof(uint32_t);
    k_grp_count<<<nt, 256, bits_bytes, s>>>(tiles.p, H.rowptr.p, scol.p, bad.p, gb.p, cnt.p);
    FSA_CHECK_LAUNCH();
    std::vector<int32_t> gc((size_t)std::max<int64_t>(ngroups, 1)), hb(nt);
    FSA_CUDA(cudaMemcpyAsync(gc.data(), cnt.p, sizeof(int32_t) * gc.size(), cudaMemcpyDeviceToHost, s));
    FSA_CUDA(cudaMemcpyAsync(hb.data(), bad.p, sizeof(int32_t) * nt, cudaMemcpyDeviceToHost, s));
    FSA_CUDA(cudaStreamSynchronize(s));
    int64_t ent = 0;
    for (int k = 0; k < nt; ++k) {
      int32_t* o = &pt[kTileWords * (size_t)k];
      const int ng = (o[1] + kGrpRows - 1) / kGrpRows;
      const int64_t gob = (int64_t)gbase[k] + k;   // ng + 1 offsets from here
      int64_t rel = 0;
      for (int j = 0; j < ng; ++j) {
        go[(size_t)(gob + j)] = (int32_t)rel;
        rel += gc[(size_t)gbase[k] + j];
      }
      go[(size_t)(gob + ng)] = (int32_t)rel;
      FSA_REQUIRE(rel < ((int64_t)1 << 30), FSA_ERR_ARG, "SpMM tile with too many union entries");
      o[11] = (int32_t)gob;
      o[12] = (int32_t)(uint32_t)((uint64_t)ent & 0xffffffffu);
      o[13] = (int32_t)(ent >> 32);
      o[14] = (int32_t)rel;
      o[15] = hb[k] ? 1 : 0;
      ent += rel;
    }
    H.grp_entries = ent;
  }
  H.sp_ptile.alloc(pt.size());
  FSA_CUDA(cudaMemcpyAsync(H.sp_ptile.p, pt.data(), sizeof(int32_t) * pt.size(), cudaMemcpyHostToDevice, s));
  H.gofs.alloc(go.size());   // spare entries: the SpMM copies in 16-byte units
  FSA_CUDA(cudaMemcpyAsync(H.gofs.p, go.data(), sizeof(int32_t) * go.size(), cudaMemcpyHostToDevice, s));
  const size_t nv = (size_t)std::max<int64_t>(H.grp_entries, 1) * kEntVec;
  H.grp_src.alloc(nv);
  FSA_CUDA(cudaMemsetAsync(H.grp_src.p, 0xff, sizeof(int4) * nv, s));
  if (nt > 0 && H.grp_entries > 0) {
    const size_t sm_bytes = 2 * (size_t)(kGrpMaxStaged / 32) * sizeof(uint32_t);
    k_grp_fill<<<nt, 256, sm_bytes, s>>>(tiles.p, H.sp_ptile.p, H.rowptr.p, scol.p, bad.p, H.gofs.p,
                                         reinterpret_cast<int32_t*>(H.grp_src.p));
    FSA_CHECK_LAUNCH();
  }
  FSA_CUDA(cudaStreamSynchronize(s));   // the temporaries are freed on return
}

// Tiles of the tile-staged kernels: the SDDMM forms of the residual values and
// their range derivative (kTileRows points per tile) and the SpMM
// (kSpTileRows, its own tiling: its staged rows are Z rows of at most 512
// bytes, the SDDMM's are BF16 pairs of A~ blocks).
void build_tiles(Handle& H) {
  constexpr int64_t kTileRows = 24, kSpTileRows = 40;
  const int ncx = H.grid.ncx, ncy = H.grid.ncy;
  const int64_t ncells = (int64_t)ncx * ncy;
  std::vector<int32_t> start(ncells), count(ncells);
  std::vector<int64_t> rp(H.n + 1);
  FSA_CUDA(cudaMemcpyAsync(start.data(), H.cell_start.p, sizeof(int32_t) * ncells, cudaMemcpyDeviceToHost, H.stream));
  FSA_CUDA(cudaMemcpyAsync(count.data(), H.cell_count.p, sizeof(int32_t) * ncells, cudaMemcpyDeviceToHost, H.stream));
  FSA_CUDA(cudaMemcpyAsync(rp.data(), H.rowptr.p, sizeof(int64_t) * (H.n + 1), cudaMemcpyDeviceToHost, H.stream));
  FSA_CUDA(cudaStreamSynchronize(H.stream));
  FSA_REQUIRE(H.n < ((int64_t)1 << 31), FSA_ERR_ARG, "more than 2^31 - 1 points");
  int64_t max_staged = 0;
  const std::vector<int64_t> t = cut_tiles(start, count, ncx, ncy, kTileRows, &max_staged);
  H.ntiles = (int)(t.size() / 8);
  H.max_staged = max_staged;
  H.tiles.alloc(std::max<size_t>(t.size(), 8));
  if (!t.empty())
    FSA_CUDA(cudaMemcpyAsync(H.tiles.p, t.data(), sizeof(int64_t) * t.size(), cudaMemcpyHostToDevice, H.stream));
  // largest tile (rows, nonzeros) from the row pointers
  int64_t mr = 0, me = 0;
  for (int k = 0; k < H.ntiles; ++k) {
    mr = std::max(mr, t[8 * k + 1] - t[8 * k]);
    me = std::max(me, rp[t[8 * k + 1]] - rp[t[8 * k]]);
  }
  H.max_tile_rows = mr;
  H.max_tile_nnz = me;
  const std::vector<int32_t> pt = tile_records(t, rp);
  H.ptile.alloc(pt.size());
  FSA_CUDA(cudaMemcpyAsync(H.ptile.p, pt.data(), sizeof(int32_t) * pt.size(), cudaMemcpyHostToDevice, H.stream));
  H.scol.alloc(H.nnz + 4);   // spare entries: copies in 16-byte units
  H.tile_bad.alloc(std::max(H.ntiles, 1));
  FSA_CUDA(cudaMemsetAsync(H.tile_bad.p, 0, sizeof(int32_t) * std::max(H.ntiles, 1), H.stream));
  if (H.ntiles > 0) {
    k_tile_scol<<<H.ntiles, 256, 0, H.stream>>>(H.tiles.p, H.rowptr.p, H.col.p, H.scol.p, H.tile_bad.p);
    FSA_CHECK_LAUNCH();
  }
  build_spmm_groups(H, cut_tiles(start, count, ncx, ncy, kSpTileRows, nullptr), rp);
}

void build_cross_structure(Handle& H, const double* qx, const double* qy, int64_t nq,
                           DevPtr<int64_t>& rowptr, DevPtr<int32_t>& col, int64_t& nnz) {
  cudaStream_t s = H.stream;
  DevPtr<int64_t> counts(nq + 1);
  FSA_CUDA(cudaMemsetAsync(counts.p + nq, 0, sizeof(int64_t), s));
  double g2 = H.gamma * H.gamma;
  unsigned gb = grid_for(nq, 256);
  neighbour_kernel<false><<<gb, 256, 0, s>>>(qx, qy, nq, H.xs.p, H.ys.p, H.cell_start.p, H.cell_count.p,
                                             H.grid, g2, counts.p, nullptr, nullptr);
  FSA_CHECK_LAUNCH();
  rowptr.alloc(nq + 1);
  exclusive_scan<int64_t>(counts.p, rowptr.p, nq + 1, s);
  FSA_CUDA(cudaMemcpyAsync(&nnz, rowptr.p + nq, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  FSA_CUDA(cudaStreamSynchronize(s));
  col.alloc(nnz > 0 ? nnz : 1);
  neighbour_kernel<true><<<gb, 256, 0, s>>>(qx, qy, nq, H.xs.p, H.ys.p, H.cell_start.p, H.cell_count.p,
                                            H.grid, g2, nullptr, rowptr.p, col.p);
  FSA_CHECK_LAUNCH();
}

void export_csr(Handle& H, int64_t* rowptr_host, int32_t* col_host) {
  cudaStream_t s = H.stream;
  int64_t n = H.n;
  DevPtr<int64_t> cnt(n + 1), rp(n + 1);
  DevPtr<int32_t> co(H.nnz > 0 ? H.nnz : 1);
  FSA_CUDA(cudaMemsetAsync(cnt.p + n, 0, sizeof(int64_t), s));
  unsigned gb = grid_for(n, 256);
  orig_counts_kernel<<<gb, 256, 0, s>>>(H.rowptr.p, H.iperm.p, n, cnt.p);
  FSA_CHECK_LAUNCH();
  exclusive_scan<int64_t>(cnt.p, rp.p, n + 1, s);
  orig_fill_kernel<<<gb, 256, 0, s>>>(H.rowptr.p, H.col.p, H.perm.p, H.iperm.p, n, rp.p, co.p);
  FSA_CHECK_LAUNCH();
  FSA_CUDA(cudaMemcpyAsync(rowptr_host, rp.p, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, s));
  FSA_CUDA(cudaMemcpyAsync(col_host, co.p, sizeof(int32_t) * H.nnz, cudaMemcpyDeviceToHost, s));
  FSA_CUDA(cudaStreamSynchronize(s));
}

}  // namespace fsa
