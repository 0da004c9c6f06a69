// Self-test of the FP32 SpMM of the mixed CG loop (declared in
// include/fsa_selftest.h): the pipelined shared-memory tile kernel against the
// row kernel on the same handle, operator and seeded block, with beta = 0 and
// with a seeded nonzero beta.
#include <cstring>
#include <vector>

#include "fsa_grad.cuh"
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

// beta in (0, 1) for the first cols columns, 0 beyond
static __global__ void k_fill_beta(int cols, int ld, uint64_t key, double* __restrict__ beta) {
  for (int c = threadIdx.x; c < ld; c += blockDim.x)
    beta[c] = c < cols ? ((double)(rng_at(key, (uint64_t)c) >> 11) + 1.0) * 0x1.0p-53 : 0.0;
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
    none.err = H.err;   // bounded waits in the SpMM report a timeout here
    const StagedLaunch sl = staged_launch(H, ldc);
    launch_spmm_f32(H, lay, sl, s, H.op.vals32.p, Z.p, S.p, V1.p, H1.p, beta.p, part.p, kStepNone, none);
    launch_spmm_fused<float, float>(lay, s, H.rowptr.p, H.col.p, H.op.vals32.p, Z.p, S.p, V2.p, H2.p, beta.p,
                                    part.p, kStepNone, none);
    k_max_abs_diff<<<grid_for((int64_t)nc, 256), 256, 0, s>>>((int64_t)nc, V1.p, V2.p, mx.p);
    k_max_abs_diff<<<grid_for((int64_t)nc, 256), 256, 0, s>>>((int64_t)nc, H1.p, H2.p, mx.p);
    FSA_CHECK_LAUNCH();
    // second pass with a nonzero beta (V = Sigma_s~ Z + S + beta V, H = Z + beta H)
    // on seeded V, H: both forms start from the same copies
    k_fill_f32<<<grid_for((int64_t)nc, 256), 256, 0, s>>>(H.n, ncols, ldc, rng_key(seed, 13), V1.p);
    k_fill_f32<<<grid_for((int64_t)nc, 256), 256, 0, s>>>(H.n, ncols, ldc, rng_key(seed, 14), H1.p);
    k_fill_beta<<<1, 128, 0, s>>>(ncols, ldc, rng_key(seed, 15), beta.p);
    FSA_CHECK_LAUNCH();
    FSA_CUDA(cudaMemcpyAsync(V2.p, V1.p, nc * sizeof(float), cudaMemcpyDeviceToDevice, s));
    FSA_CUDA(cudaMemcpyAsync(H2.p, H1.p, nc * sizeof(float), cudaMemcpyDeviceToDevice, s));
    launch_spmm_f32(H, lay, sl, s, H.op.vals32.p, Z.p, S.p, V1.p, H1.p, beta.p, part.p, kStepNone, none);
    launch_spmm_fused<float, float>(lay, s, H.rowptr.p, H.col.p, H.op.vals32.p, Z.p, S.p, V2.p, H2.p, beta.p,
                                    part.p, kStepNone, none);
    k_max_abs_diff<<<grid_for((int64_t)nc, 256), 256, 0, s>>>((int64_t)nc, V1.p, V2.p, mx.p);
    k_max_abs_diff<<<grid_for((int64_t)nc, 256), 256, 0, s>>>((int64_t)nc, H1.p, H2.p, mx.p);
    FSA_CHECK_LAUNCH();
    unsigned long long bits = 0;
    FSA_CUDA(cudaMemcpyAsync(&bits, mx.p, sizeof(bits), cudaMemcpyDeviceToHost, s));
    // which tiles fit the staging capacity (the kernel's own test)
    std::vector<int32_t> pt((size_t)std::max(H.sp_ntiles, 1) * kTileWords);
    if (H.sp_ntiles > 0)
      FSA_CUDA(cudaMemcpyAsync(pt.data(), H.sp_ptile.p, sizeof(int32_t) * (size_t)H.sp_ntiles * kTileWords,
                               cudaMemcpyDeviceToHost, s));
    FSA_CUDA(cudaStreamSynchronize(s));
    check_err(H);
    int staged = 0;
    for (int k = 0; k < H.sp_ntiles; ++k) {
      const int32_t* o = &pt[(size_t)k * kTileWords];
      const int nr = o[1], ng = (nr + kGrpRows - 1) / kGrpRows;
      int ga, gz;
      sp_gofs_range(o[11], ng, ga, gz);
      // with V and H staged (the nonzero-beta pass; the larger layout)
      const SpTileLayout lay = sp_tile_layout(o[3] + o[5] + o[7], nr, o[14], gz - ga, ldc, true);
      if (!o[15] && lay.bytes <= sl.ring.bytes) ++staged;
    }
    double d;
    std::memcpy(&d, &bits, sizeof(d));
    *max_abs_diff = d;
    if (staged_tiles) *staged_tiles = staged;
    if (total_tiles) *total_tiles = H.sp_ntiles;
    return FSA_OK;
  } catch (const Error& e) {
    cudaGetLastError();
    set_error(e.msg);
    return e.code;
  }
}

namespace fsa {

static __global__ void k_fill_bf16(int64_t total, uint64_t key, float scale, __nv_bfloat16* __restrict__ out) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x)
    out[t] = __float2bfloat16_rn(scale * ((float)(rng_at(key, (uint64_t)t) >> 40) * (1.0f / 16777216.0f) * 2.0f - 1.0f));
}

// max |a - b| and max |b| over FP64 arrays (non-negative doubles as ordered bit patterns)
static __global__ void k_max_abs_diff_f64(int64_t total, const double* __restrict__ a, const double* __restrict__ b,
                                          unsigned long long* __restrict__ out) {
  double mx = 0.0, mb = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const double d = fabs(a[t] - b[t]);
    if (!(d <= mx)) mx = (d != d) ? INFINITY : d;
    mb = fmax(mb, fabs(b[t]));
  }
  atomicMax(out, (unsigned long long)__double_as_longlong(mx));
  atomicMax(out + 1, (unsigned long long)__double_as_longlong(mb));
}

// the same over FP32 arrays (stored as FP64 bit patterns)
static __global__ void k_max_abs_diff_f32(int64_t total, const float* __restrict__ a, const float* __restrict__ b,
                                          unsigned long long* __restrict__ out) {
  double mx = 0.0, mb = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const double d = fabs((double)a[t] - (double)b[t]);
    if (!(d <= mx)) mx = (d != d) ? INFINITY : d;
    mb = fmax(mb, fabs((double)b[t]));
  }
  atomicMax(out, (unsigned long long)__double_as_longlong(mx));
  atomicMax(out + 1, (unsigned long long)__double_as_longlong(mb));
}

}  // namespace fsa

extern "C" int fsa_selftest_sddmm(fsa_handle* hh, const fsa_theta* theta, int precision, int cap_rows,
                                  uint64_t seed, double* val_err, double* dval_err) {
  if (!hh || !theta || !val_err || !dval_err || cap_rows < 0 ||
      (precision != FSA_MIXED_BF16 && precision != FSA_MIXED_BF16X2)) {
    set_error("fsa_selftest_sddmm: bad argument");
    return FSA_ERR_ARG;
  }
  Handle& H = hh->h;
  AllocStreamScope scope(H.stream);
  try {
    cudaStream_t s = H.stream;
    ensure_operator(H, *theta, precision);
    Operator& op = H.op;
    const int64_t n = H.n, nnz = H.nnz;
    const int m_pad = op.m_pad;
    const __nv_bfloat16* Alo = op.has_lo ? op.Ab_lo.p : nullptr;
    // residual values and D: tile form (capped staging) against the row form
    FSA_REQUIRE(csr_values_tiles(H, *theta, op.Ab.p, Alo, m_pad, cap_rows), FSA_ERR_UNSUPPORTED,
                "tile form unavailable for this handle");
    DevPtr<double> vt(nnz), Dt(n);
    FSA_CUDA(cudaMemcpyAsync(vt.p, op.vals.p, sizeof(double) * nnz, cudaMemcpyDeviceToDevice, s));
    FSA_CUDA(cudaMemcpyAsync(Dt.p, op.D.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    csr_values_rows(H, *theta, op.Ab.p, Alo, m_pad);
    op.valid = false;   // the operator now holds the row form's values: rebuilt on next use
    DevPtr<unsigned long long> mx(8);
    FSA_CUDA(cudaMemsetAsync(mx.p, 0, 8 * sizeof(unsigned long long), s));
    k_max_abs_diff_f64<<<grid_for(nnz, 256), 256, 0, s>>>(nnz, vt.p, op.vals.p, mx.p);
    k_max_abs_diff_f64<<<grid_for(n, 256), 256, 0, s>>>(n, Dt.p, op.D.p, mx.p + 2);
    FSA_CHECK_LAUNCH();
    // range derivative of the values on seeded BF16 pairs a (zeros if single), b, q
    const size_t nm = (size_t)n * m_pad;
    DevPtr<__nv_bfloat16> zlo, Bh(nm), Bl(nm), Qh(nm), Ql(nm);
    if (!Alo) {
      zlo.alloc(nm);
      FSA_CUDA(cudaMemsetAsync(zlo.p, 0, nm * sizeof(__nv_bfloat16), s));
      Alo = zlo.p;
    }
    k_fill_bf16<<<grid_for((int64_t)nm, 256), 256, 0, s>>>((int64_t)nm, rng_key(seed, 23), 1.0f, Bh.p);
    k_fill_bf16<<<grid_for((int64_t)nm, 256), 256, 0, s>>>((int64_t)nm, rng_key(seed, 24), 1.0f / 256, Bl.p);
    k_fill_bf16<<<grid_for((int64_t)nm, 256), 256, 0, s>>>((int64_t)nm, rng_key(seed, 25), 1.0f, Qh.p);
    k_fill_bf16<<<grid_for((int64_t)nm, 256), 256, 0, s>>>((int64_t)nm, rng_key(seed, 26), 1.0f / 256, Ql.p);
    FSA_CHECK_LAUNCH();
    DevPtr<float> dvt(nnz + 4), dDt(n), dvr(nnz + 4), dDr(n);
    FSA_REQUIRE(dvals_tiles(H, *theta, m_pad, op.Ab.p, Alo, Bh.p, Bl.p, Qh.p, Ql.p, dvt.p, dDt.p, cap_rows),
                FSA_ERR_UNSUPPORTED, "tile form unavailable for this handle");
    dvals_rows(H, *theta, m_pad, op.Ab.p, Alo, Bh.p, Bl.p, Qh.p, Ql.p, dvr.p, dDr.p);
    k_max_abs_diff_f32<<<grid_for(nnz, 256), 256, 0, s>>>(nnz, dvt.p, dvr.p, mx.p + 4);
    k_max_abs_diff_f32<<<grid_for(n, 256), 256, 0, s>>>(n, dDt.p, dDr.p, mx.p + 6);
    FSA_CHECK_LAUNCH();
    unsigned long long bits[8];
    FSA_CUDA(cudaMemcpyAsync(bits, mx.p, sizeof(bits), cudaMemcpyDeviceToHost, s));
    FSA_CUDA(cudaStreamSynchronize(s));
    check_err(H);
    double d[8];
    std::memcpy(d, bits, sizeof(d));
    // max-norm relative differences
    val_err[0] = d[1] > 0 ? d[0] / d[1] : d[0];
    val_err[1] = d[3] > 0 ? d[2] / d[3] : d[2];
    dval_err[0] = d[5] > 0 ? d[4] / d[5] : d[4];
    dval_err[1] = d[7] > 0 ? d[6] / d[7] : d[6];
    return FSA_OK;
  } catch (const Error& e) {
    cudaGetLastError();
    set_error(e.msg);
    return e.code;
  }
}
