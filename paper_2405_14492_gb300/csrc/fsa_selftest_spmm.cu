// Self-test of the FP32 SpMM of the mixed CG loop (declared in
// include/fsa_selftest.h): the shared-memory tile kernel against the row
// kernel on the same handle, operator and seeded block.
#include <cstring>
#include <vector>

#include "fsa_vec.cuh"

namespace fsa {

static __global__ void k_fill_f32(int64_t n, int cols, int ld, uint64_t key, float* __restrict__ out) {
  const int64_t total = n * ld;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t % ld);
    float v = 0.f;
    if (c < cols) v = (float)(rng_at(key, (uint64_t)t) >> 40) * (1.0f / 16777216.0f) * 2.0f - 1.0f;
    out[t] = v;
  }
}

// max |a - b| of non-negative differences, as ordered bit patterns
static __global__ void k_max_abs_diff(int64_t total, const float* __restrict__ a, const float* __restrict__ b,
                                      unsigned long long* __restrict__ out) {
  double mx = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const double d = fabs((double)a[t] - (double)b[t]);
    if (!(d <= mx)) mx = (d != d) ? INFINITY : d;
  }
  atomicMax(out, (unsigned long long)__double_as_longlong(mx));
}

}  // namespace fsa

using namespace fsa;

extern "C" int fsa_selftest_spmm(fsa_handle* hh, const fsa_theta* theta, int ncols, uint64_t seed,
                                 double* max_abs_diff, int* staged_tiles, int* total_tiles) {
  if (!hh || !theta || !max_abs_diff || ncols < 1 || ncols > 127) {
    set_error("fsa_selftest_spmm: bad argument");
    return FSA_ERR_ARG;
  }
  Handle& H = hh->h;
  AllocStreamScope scope(H.stream);
  try {
    cudaStream_t s = H.stream;
    ensure_operator(H, *theta, FSA_MIXED_BF16X2);
    CGLayout lay;
    const int ldc = (ncols + 7) / 8 * 8;
    lay.setup(H.n, ncols, 1, ldc);
    const size_t nc = (size_t)H.n * ldc;
    DevPtr<float> Z(nc), S(nc), V1(nc), H1(nc), V2(nc), H2(nc);
    DevPtr<double> beta(ldc), part((size_t)lay.nblk * ldc);
    DevPtr<unsigned long long> mx(1);
    k_fill_f32<<<grid_for((int64_t)nc, 256), 256, 0, s>>>(H.n, ncols, ldc, rng_key(seed, 11), Z.p);
    k_fill_f32<<<grid_for((int64_t)nc, 256), 256, 0, s>>>(H.n, ncols, ldc, rng_key(seed, 12), S.p);
    FSA_CHECK_LAUNCH();
    FSA_CUDA(cudaMemsetAsync(beta.p, 0, sizeof(double) * ldc, s));
    FSA_CUDA(cudaMemsetAsync(mx.p, 0, sizeof(unsigned long long), s));
    CGScalars none{};
    const StagedLaunch sl = staged_launch(H, ldc);
    launch_spmm_f32(H, lay, sl, s, H.op.vals32.p, Z.p, S.p, V1.p, H1.p, beta.p, part.p, kStepNone, none);
    launch_spmm_fused<float, float>(lay, s, H.rowptr.p, H.col.p, H.op.vals32.p, Z.p, S.p, V2.p, H2.p, beta.p,
                                    part.p, kStepNone, none);
    k_max_abs_diff<<<grid_for((int64_t)nc, 256), 256, 0, s>>>((int64_t)nc, V1.p, V2.p, mx.p);
    k_max_abs_diff<<<grid_for((int64_t)nc, 256), 256, 0, s>>>((int64_t)nc, H1.p, H2.p, mx.p);
    FSA_CHECK_LAUNCH();
    unsigned long long bits = 0;
    FSA_CUDA(cudaMemcpyAsync(&bits, mx.p, sizeof(bits), cudaMemcpyDeviceToHost, s));
    // which tiles fit the staging capacity (the kernel's own test)
    std::vector<int64_t> td((size_t)H.ntiles * 8), rp(H.n + 1);
    std::vector<int32_t> bad(std::max(H.ntiles, 1));
    if (H.ntiles > 0) {
      FSA_CUDA(cudaMemcpyAsync(td.data(), H.tiles.p, sizeof(int64_t) * td.size(), cudaMemcpyDeviceToHost, s));
      FSA_CUDA(cudaMemcpyAsync(bad.data(), H.tile_bad.p, sizeof(int32_t) * H.ntiles, cudaMemcpyDeviceToHost, s));
    }
    FSA_CUDA(cudaMemcpyAsync(rp.data(), H.rowptr.p, sizeof(int64_t) * (H.n + 1), cudaMemcpyDeviceToHost, s));
    FSA_CUDA(cudaStreamSynchronize(s));
    check_err(H);
    int staged = 0;
    for (int k = 0; k < H.ntiles; ++k) {
      const int64_t* d = &td[(size_t)k * 8];
      const int64_t rows = (d[3] - d[2]) + (d[5] - d[4]) + (d[7] - d[6]);
      if (!bad[k] && rows <= sl.cap_rows && rp[d[1]] - rp[d[0]] <= sl.cap_nnz && d[1] - d[0] <= sl.cap_trows) ++staged;
    }
    double d;
    std::memcpy(&d, &bits, sizeof(d));
    *max_abs_diff = d;
    if (staged_tiles) *staged_tiles = staged;
    if (total_tiles) *total_tiles = H.ntiles;
    return FSA_OK;
  } catch (const Error& e) {
    cudaGetLastError();
    set_error(e.msg);
    return e.code;
  }
}
