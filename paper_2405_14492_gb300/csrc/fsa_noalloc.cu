// fsa_csr_noalloc: the taper-support neighbour structure (the CSR that
// fsa_build + fsa_get_csr produce) computed without allocating any memory.
//
// Some callers cannot allocate device memory: an application that owns the
// whole device pool (a custom allocator or a memory-capped serving process), a
// host library called inside a region where cudaMalloc is forbidden, or code
// whose allocator must not be re-entered.  This entry point takes device input
// and output buffers from the caller and keeps all of its temporaries in one
// file-scope __device__ array of fixed size, so it never calls cudaMalloc,
// cudaFree or an allocating library routine.  The array is part of the
// library image: every GPU that loads libfsa holds it (about 6 MB) until the
// process exits.
#include <cuda.h>
#include <mutex>

#include "fsa_internal.cuh"

namespace fsa {
namespace na {

constexpr int64_t kMaxPoints = 65536;
constexpr int64_t kMaxCells = 4 * kMaxPoints + 16;
constexpr int kBBoxParts = 64;

constexpr size_t align(size_t v) { return (v + 255) / 256 * 256; }

// layout of the scratch array (byte offsets, each 256-byte aligned)
struct Layout {
  static constexpr size_t bbox = 0;                                            // double[4 * parts + 4]
  static constexpr size_t cell_of = align(bbox + sizeof(double) * (4 * kBBoxParts + 4));   // int32[maxP]
  static constexpr size_t cell_count = align(cell_of + sizeof(int32_t) * kMaxPoints);      // int32[maxC]
  static constexpr size_t cell_start = align(cell_count + sizeof(int32_t) * kMaxCells);    // int32[maxC]
  static constexpr size_t cursor = align(cell_start + sizeof(int32_t) * kMaxCells);        // int32[maxC]
  static constexpr size_t perm = align(cursor + sizeof(int32_t) * kMaxCells);              // int64[maxP]
  static constexpr size_t iperm = align(perm + sizeof(int64_t) * kMaxPoints);              // int64[maxP]
  static constexpr size_t xs = align(iperm + sizeof(int64_t) * kMaxPoints);                // double[maxP]
  static constexpr size_t ys = align(xs + sizeof(double) * kMaxPoints);                    // double[maxP]
  static constexpr size_t cnt = align(ys + sizeof(double) * kMaxPoints);                   // int64[maxP + 1]
  static constexpr size_t status = align(cnt + sizeof(int64_t) * (kMaxPoints + 1));        // unsigned
  static constexpr size_t total = align(status + sizeof(unsigned));
};

}  // namespace na

// The scratch.  Host code must not pass `g_noalloc_scratch` itself to a kernel:
// in host code that name is a host-side stand-in, not a device address.
static __device__ __align__(256) unsigned char g_noalloc_scratch[na::Layout::total];

namespace na {

__global__ void k_bbox(const double* __restrict__ pts, int64_t n, double* __restrict__ part, unsigned* err) {
  double mnx = INFINITY, mny = INFINITY, mxx = -INFINITY, mxy = -INFINITY;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double x = pts[2 * i], y = pts[2 * i + 1];
    if (!isfinite(x) || !isfinite(y)) atomicOr(err, kErrNaN);
    mnx = fmin(mnx, x); mxx = fmax(mxx, x);
    mny = fmin(mny, y); mxy = fmax(mxy, y);
  }
  __shared__ double sh[4][256];
  sh[0][threadIdx.x] = mnx; sh[1][threadIdx.x] = mny; sh[2][threadIdx.x] = mxx; sh[3][threadIdx.x] = mxy;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
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

__global__ void k_bbox_final(double* __restrict__ part, int nparts) {
  if (threadIdx.x != 0) return;
  double b[4] = {INFINITY, INFINITY, -INFINITY, -INFINITY};
  for (int p = 0; p < nparts; ++p) {
    b[0] = fmin(b[0], part[4 * p]); b[1] = fmin(b[1], part[4 * p + 1]);
    b[2] = fmax(b[2], part[4 * p + 2]); b[3] = fmax(b[3], part[4 * p + 3]);
  }
  for (int k = 0; k < 4; ++k) part[4 * nparts + k] = b[k];
}

__device__ __forceinline__ int cell_coord(double v, double lo, double h, int nc) {
  int c = (int)floor((v - lo) / h);
  return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

__global__ void k_cells(const double* __restrict__ pts, int64_t n, Grid g, int32_t* __restrict__ cell_of,
                        int32_t* __restrict__ count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int c = cell_coord(pts[2 * i + 1], g.y0, g.hy, g.ncy) * g.ncx + cell_coord(pts[2 * i], g.x0, g.hx, g.ncx);
    cell_of[i] = c;
    atomicAdd(&count[c], 1);
  }
}

// exclusive scan by one block, any length (chunks of 1024 with a running offset)
template <typename T>
__global__ void k_scan1(const T* __restrict__ in, T* __restrict__ out, int64_t len) {
  __shared__ T sh[1024];
  __shared__ T carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < len; base += 1024) {
    int64_t i = base + threadIdx.x;
    T v = i < len ? in[i] : (T)0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      T t = (int)threadIdx.x >= o ? sh[threadIdx.x - o] : (T)0;
      __syncthreads();
      sh[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < len) out[i] = carry + sh[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += sh[1023];
    __syncthreads();
  }
}

__global__ void k_scatter(const int32_t* __restrict__ cell_of, int64_t n, const int32_t* __restrict__ start,
                          int32_t* __restrict__ cursor, int64_t* __restrict__ perm) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int c = cell_of[i];
    perm[start[c] + atomicAdd(&cursor[c], 1)] = i;
  }
}

__global__ void k_cell_sort(const int32_t* __restrict__ start, const int32_t* __restrict__ count, int ncells,
                            int64_t* __restrict__ perm) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) {
    heap_sort_thread(perm + start[c], (int64_t)count[c]);
  }
}

__global__ void k_gather(const double* __restrict__ pts, const int64_t* __restrict__ perm, int64_t n,
                         double* __restrict__ xs, double* __restrict__ ys, int64_t* __restrict__ iperm) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = perm[k];
    xs[k] = pts[2 * i];
    ys[k] = pts[2 * i + 1];
    iperm[i] = k;
  }
}

// count (fill == false) or write (fill == true) the neighbours of ORIGINAL row r
// as original indices; rows are then sorted ascending
template <bool kFill>
__global__ void k_rows(int64_t n, const double* __restrict__ xs, const double* __restrict__ ys,
                       const int64_t* __restrict__ perm, const int64_t* __restrict__ iperm,
                       const int32_t* __restrict__ cstart, const int32_t* __restrict__ ccount, Grid g, double g2,
                       int64_t* __restrict__ cnt, const int64_t* __restrict__ rowptr, int32_t* __restrict__ col) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    int64_t k = iperm[r];
    double xi = xs[k], yi = ys[k];
    int cx = cell_coord(xi, g.x0, g.hx, g.ncx), cy = cell_coord(yi, g.y0, g.hy, g.ncy);
    int64_t w = kFill ? rowptr[r] : 0, c0 = w;
    int64_t num = 0;
    for (int dy = -1; dy <= 1; ++dy) {
      int yy = cy + dy;
      if (yy < 0 || yy >= g.ncy) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        int xx = cx + dx;
        if (xx < 0 || xx >= g.ncx) continue;
        int c = yy * g.ncx + xx;
        for (int j = cstart[c], e = cstart[c] + ccount[c]; j < e; ++j) {
          if (sqdist_rn(xi, yi, xs[j], ys[j]) < g2) {
            if (kFill) {
              col[w++] = (int32_t)perm[j];
            } else {
              ++num;
            }
          }
        }
      }
    }
    if (kFill) heap_sort_thread(col + c0, w - c0);
    else cnt[r] = num;
  }
}

using CtxGetCurrentFn = CUresult (*)(CUcontext*);

static CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<CtxGetCurrentFn>(f);
  }();
  return fn;
}

struct DeviceScratch {
  CUcontext ctx = nullptr;
  unsigned char* base = nullptr;
};

// device address of the scratch array for the current device.  The host name
// of the array is not a device address.  The address is looked up with the
// device current on the first call in a CUDA context and kept for that
// context; a reset of the device (cudaDeviceReset) makes a new context, where
// the module is loaded again and the array may sit elsewhere, so the next
// call looks it up again.
static unsigned char* scratch_for_current_device() {
  static std::mutex mu;
  static DeviceScratch per_dev[64];
  int dev = 0;
  FSA_CUDA(cudaGetDevice(&dev));
  FSA_REQUIRE(dev >= 0 && dev < 64, FSA_ERR_UNSUPPORTED, "device index out of range");
  FSA_CUDA(cudaFree(nullptr));   // makes the device's primary context current (frees nothing)
  CUcontext ctx = nullptr;
  CtxGetCurrentFn get = ctx_get_current();
  if (!get || get(&ctx) != CUDA_SUCCESS) ctx = nullptr;   // context unknown: look up on every call
  std::lock_guard<std::mutex> lk(mu);
  if (!per_dev[dev].base || !ctx || per_dev[dev].ctx != ctx) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      throw Error{FSA_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch) failed: ") + cudaGetErrorString(e)};
    per_dev[dev].base = static_cast<unsigned char*>(p);
    per_dev[dev].ctx = ctx;
  }
  return per_dev[dev].base;
}

}  // namespace na
}  // namespace fsa

using namespace fsa;

extern "C" fsa_status fsa_csr_noalloc(const double* locs_dev, int64_t n, double taper_range, int64_t* rowptr_dev,
                                      int32_t* col_dev, int64_t col_capacity, int64_t* nnz_out,
                                      void* cuda_stream) {
  if (!locs_dev || !rowptr_dev || !nnz_out) {
    set_error("fsa_csr_noalloc: NULL argument");
    return FSA_ERR_ARG;
  }
  if (n < 1 || n > na::kMaxPoints) {
    set_error("fsa_csr_noalloc: n must be in [1, " + std::to_string(na::kMaxPoints) +
              "] (fixed scratch size); use fsa_build for larger problems");
    return FSA_ERR_ARG;
  }
  if (!(taper_range > 0) || !std::isfinite(taper_range)) {
    set_error("fsa_csr_noalloc: taper_range must be > 0");
    return FSA_ERR_ARG;
  }
  try {
    cudaStream_t s = (cudaStream_t)cuda_stream;
    unsigned char* base = na::scratch_for_current_device();
    double* bbox = reinterpret_cast<double*>(base + na::Layout::bbox);
    int32_t* cell_of = reinterpret_cast<int32_t*>(base + na::Layout::cell_of);
    int32_t* ccount = reinterpret_cast<int32_t*>(base + na::Layout::cell_count);
    int32_t* cstart = reinterpret_cast<int32_t*>(base + na::Layout::cell_start);
    int32_t* cursor = reinterpret_cast<int32_t*>(base + na::Layout::cursor);
    int64_t* perm = reinterpret_cast<int64_t*>(base + na::Layout::perm);
    int64_t* iperm = reinterpret_cast<int64_t*>(base + na::Layout::iperm);
    double* xs = reinterpret_cast<double*>(base + na::Layout::xs);
    double* ys = reinterpret_cast<double*>(base + na::Layout::ys);
    int64_t* cnt = reinterpret_cast<int64_t*>(base + na::Layout::cnt);
    unsigned* status_word_dev = reinterpret_cast<unsigned*>(base + na::Layout::status);
    // the scratch keeps the previous call's contents: clear what must start at zero
    FSA_CUDA(cudaMemsetAsync(status_word_dev, 0, sizeof(unsigned), s));
    na::k_bbox<<<na::kBBoxParts, 256, 0, s>>>(locs_dev, n, bbox, status_word_dev);
    FSA_CHECK_LAUNCH();
    na::k_bbox_final<<<1, 32, 0, s>>>(bbox, na::kBBoxParts);
    FSA_CHECK_LAUNCH();
    double hb[4];
    unsigned herr = 0;
    FSA_CUDA(cudaMemcpyAsync(hb, bbox + 4 * na::kBBoxParts, sizeof(hb), cudaMemcpyDeviceToHost, s));
    FSA_CUDA(cudaMemcpyAsync(&herr, status_word_dev, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    FSA_CUDA(cudaStreamSynchronize(s));
    if (herr & kErrNaN) {
      set_error("fsa_csr_noalloc: non-finite location coordinates");
      return FSA_ERR_NAN;
    }
    Grid g = make_grid(hb, taper_range, n);
    const int ncells = g.ncx * g.ncy;
    FSA_REQUIRE(ncells <= na::kMaxCells, FSA_ERR_ARG, "fsa_csr_noalloc: cell grid exceeds the scratch size");
    FSA_CUDA(cudaMemsetAsync(ccount, 0, sizeof(int32_t) * ncells, s));
    FSA_CUDA(cudaMemsetAsync(cursor, 0, sizeof(int32_t) * ncells, s));
    unsigned gb = grid_for(n, 256);
    na::k_cells<<<gb, 256, 0, s>>>(locs_dev, n, g, cell_of, ccount);
    FSA_CHECK_LAUNCH();
    na::k_scan1<int32_t><<<1, 1024, 0, s>>>(ccount, cstart, ncells);
    FSA_CHECK_LAUNCH();
    na::k_scatter<<<gb, 256, 0, s>>>(cell_of, n, cstart, cursor, perm);
    FSA_CHECK_LAUNCH();
    na::k_cell_sort<<<grid_for(ncells, 256), 256, 0, s>>>(cstart, ccount, ncells, perm);
    FSA_CHECK_LAUNCH();
    na::k_gather<<<gb, 256, 0, s>>>(locs_dev, perm, n, xs, ys, iperm);
    FSA_CHECK_LAUNCH();
    const double g2 = taper_range * taper_range;
    FSA_CUDA(cudaMemsetAsync(cnt + n, 0, sizeof(int64_t), s));
    na::k_rows<false><<<gb, 256, 0, s>>>(n, xs, ys, perm, iperm, cstart, ccount, g, g2, cnt, nullptr, nullptr);
    FSA_CHECK_LAUNCH();
    na::k_scan1<int64_t><<<1, 1024, 0, s>>>(cnt, rowptr_dev, n + 1);
    FSA_CHECK_LAUNCH();
    int64_t nnz = 0;
    FSA_CUDA(cudaMemcpyAsync(&nnz, rowptr_dev + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    FSA_CUDA(cudaStreamSynchronize(s));
    *nnz_out = nnz;
    if (!col_dev) return FSA_OK;   // size query
    if (nnz > col_capacity) {
      set_error("fsa_csr_noalloc: col_capacity " + std::to_string(col_capacity) + " < nnz " + std::to_string(nnz));
      return FSA_ERR_ARG;
    }
    na::k_rows<true><<<gb, 256, 0, s>>>(n, xs, ys, perm, iperm, cstart, ccount, g, g2, nullptr, rowptr_dev, col_dev);
    FSA_CHECK_LAUNCH();
    FSA_CUDA(cudaStreamSynchronize(s));
    return FSA_OK;
  } catch (const Error& e) {
    set_error(e.msg);
    return e.code;
  }
}
