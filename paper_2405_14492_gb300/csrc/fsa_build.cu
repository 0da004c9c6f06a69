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

// SpMM tiles (host): each grid row of cells is cut into runs of cells holding
// about kTileRows points; the taper neighbours of a run's points lie in the
// run's cells widened by one on each side, in the rows above, at and below
// (cell side >= gamma), i.e. in three contiguous ranges of the internal order.
void build_tiles(Handle& H) {
  constexpr int64_t kTileRows = 24;
  const int ncx = H.grid.ncx, ncy = H.grid.ncy;
  const int64_t ncells = (int64_t)ncx * ncy;
  std::vector<int32_t> start(ncells), count(ncells);
  FSA_CUDA(cudaMemcpyAsync(start.data(), H.cell_start.p, sizeof(int32_t) * ncells, cudaMemcpyDeviceToHost, H.stream));
  FSA_CUDA(cudaMemcpyAsync(count.data(), H.cell_count.p, sizeof(int32_t) * ncells, cudaMemcpyDeviceToHost, H.stream));
  FSA_CUDA(cudaStreamSynchronize(H.stream));
  auto range = [&](int cy, int cxa, int cxb, int64_t* out) {
    if (cy < 0 || cy >= ncy) { out[0] = out[1] = 0; return; }
    const int a = std::max(cxa - 1, 0), b = std::min(cxb + 1, ncx - 1);
    const int64_t c0 = (int64_t)cy * ncx + a, c1 = (int64_t)cy * ncx + b;
    out[0] = start[c0];
    out[1] = (int64_t)start[c1] + count[c1];
  };
  std::vector<int64_t> t;
  int64_t max_staged = 0;
  for (int cy = 0; cy < ncy; ++cy) {
    int cxa = 0;
    int64_t acc = 0;
    for (int cx = 0; cx < ncx; ++cx) {
      acc += count[(int64_t)cy * ncx + cx];
      if (acc >= kTileRows || cx == ncx - 1) {
        if (acc > 0) {
          int64_t d[8];
          d[0] = start[(int64_t)cy * ncx + cxa];
          d[1] = (int64_t)start[(int64_t)cy * ncx + cx] + count[(int64_t)cy * ncx + cx];
          range(cy - 1, cxa, cx, d + 2);
          range(cy, cxa, cx, d + 4);
          range(cy + 1, cxa, cx, d + 6);
          max_staged = std::max(max_staged, (d[3] - d[2]) + (d[5] - d[4]) + (d[7] - d[6]));
          t.insert(t.end(), d, d + 8);
        }
        cxa = cx + 1;
        acc = 0;
      }
    }
  }
  H.ntiles = (int)(t.size() / 8);
  H.max_staged = max_staged;
  H.tiles.alloc(std::max<size_t>(t.size(), 8));
  if (!t.empty())
    FSA_CUDA(cudaMemcpyAsync(H.tiles.p, t.data(), sizeof(int64_t) * t.size(), cudaMemcpyHostToDevice, H.stream));
  // largest tile (rows, nonzeros) from the row pointers
  std::vector<int64_t> rp(H.n + 1);
  FSA_CUDA(cudaMemcpyAsync(rp.data(), H.rowptr.p, sizeof(int64_t) * (H.n + 1), cudaMemcpyDeviceToHost, H.stream));
  FSA_CUDA(cudaStreamSynchronize(H.stream));
  int64_t mr = 0, me = 0;
  for (int k = 0; k < H.ntiles; ++k) {
    mr = std::max(mr, t[8 * k + 1] - t[8 * k]);
    me = std::max(me, rp[t[8 * k + 1]] - rp[t[8 * k]]);
  }
  H.max_tile_rows = mr;
  H.max_tile_nnz = me;
  // the pipelined SpMM's record: p0, rows, (begin, length) of the three
  // ranges, first nonzero (low, high 32 bits), nonzeros, unused
  FSA_REQUIRE(H.n < ((int64_t)1 << 31), FSA_ERR_ARG, "more than 2^31 - 1 points");
  std::vector<int32_t> pt((size_t)std::max(H.ntiles, 1) * 12, 0);
  for (int k = 0; k < H.ntiles; ++k) {
    const int64_t* d = &t[8 * (size_t)k];
    int32_t* o = &pt[12 * (size_t)k];
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
  H.ptile.alloc(pt.size());
  FSA_CUDA(cudaMemcpyAsync(H.ptile.p, pt.data(), sizeof(int32_t) * pt.size(), cudaMemcpyHostToDevice, H.stream));
  H.scol.alloc(H.nnz + 4);   // spare entries: the SpMM copies in 16-byte units
  H.tile_bad.alloc(std::max(H.ntiles, 1));
  FSA_CUDA(cudaMemsetAsync(H.tile_bad.p, 0, sizeof(int32_t) * std::max(H.ntiles, 1), H.stream));
  if (H.ntiles > 0) {
    k_tile_scol<<<H.ntiles, 256, 0, H.stream>>>(H.tiles.p, H.rowptr.p, H.col.p, H.scol.p, H.tile_bad.p);
    FSA_CHECK_LAUNCH();
  }
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
