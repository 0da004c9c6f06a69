// Self-test of the tcgen05 GEMM against an FP64 reference computed on the
// device from the same BF16 operands (declared in include/fsa_selftest.h).
#include <cstring>

#include "fsa_tc.cuh"

namespace fsa {

__global__ void k_fill_bf16(int64_t rows, int64_t cols, int64_t ld, uint64_t key, float scale,
                            __nv_bfloat16* __restrict__ out) {
  int64_t total = rows * ld;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t c = t % ld;
    float v = 0.f;
    if (c < cols) {
      uint64_t h = rng_at(key, (uint64_t)t);
      v = scale * ((float)(h >> 40) * (1.0f / 16777216.0f) * 2.0f - 1.0f);
    }
    out[t] = __float2bfloat16_rn(v);
  }
}

struct Ops {
  const __nv_bfloat16* a[2];
  const __nv_bfloat16* b[2];
};

// ref and error: one thread per output element
__global__ void k_ref_check(int M, int N, int K, int64_t lda, int64_t ldb, Ops ops, int num_a, int num_b,
                            unsigned pairs, int stack, const float* __restrict__ out, int64_t ldo,
                            int64_t split_stride, int splits, double* __restrict__ err) {
  int ncols = N / stack;
  int64_t total = (int64_t)M * ncols;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(t / ncols), j = (int)(t % ncols);
    double ref = 0.0, mag = 0.0;
    for (int h = 0; h < stack; ++h) {
      int jj = j + h * (N / stack);
      for (int a = 0; a < num_a; ++a)
        for (int b = 0; b < num_b; ++b) {
          if (!(pairs & (1u << (2 * a + b)))) continue;
          for (int k = 0; k < K; ++k) {
            double x = (double)__bfloat162float(ops.a[a][(int64_t)i * lda + k]);
            double y = (double)__bfloat162float(ops.b[b][(int64_t)jj * ldb + k]);
            ref += x * y;
            mag += fabs(x * y);
          }
        }
    }
    double got = 0.0;
    for (int z = 0; z < splits; ++z) got += (double)out[(int64_t)z * split_stride + (int64_t)i * ldo + j];
    double e = fabs(got - ref) / (mag + 1e-30);
    // max via integer compare of non-negative doubles
    atomicMax(reinterpret_cast<unsigned long long*>(err), (unsigned long long)__double_as_longlong(e));
  }
}

}  // namespace fsa

using namespace fsa;

extern "C" int fsa_selftest_tc_gemm(int M, int N, int K, int num_a, int num_b, unsigned pairs, int halves, int splits,
                                    uint64_t seed, double* max_rel_err, int* launched_splits) {
  try {
    cudaStream_t s = nullptr;
    const int stack = halves == 1 ? 2 : (halves >= 2 ? halves : 1);
    int64_t ldk = (K + 63) / 64 * 64;
    DevPtr<__nv_bfloat16> A0((size_t)M * ldk), A1((size_t)M * ldk), B0((size_t)N * ldk), B1((size_t)N * ldk);
    k_fill_bf16<<<256, 256, 0, s>>>(M, K, ldk, rng_key(seed, 11), 1.0f, A0.p);
    k_fill_bf16<<<256, 256, 0, s>>>(M, K, ldk, rng_key(seed, 12), 0.01f, A1.p);
    k_fill_bf16<<<256, 256, 0, s>>>(N, K, ldk, rng_key(seed, 13), 1.0f, B0.p);
    k_fill_bf16<<<256, 256, 0, s>>>(N, K, ldk, rng_key(seed, 14), 0.01f, B1.p);
    FSA_CHECK_LAUNCH();
    TmaMap ma0 = make_tma_bf16(A0.p, M, K, ldk, 128), ma1 = make_tma_bf16(A1.p, M, K, ldk, 128);
    int bn = stack > 1 ? N : std::min(256, (N + 15) / 16 * 16);
    TmaMap mb0 = make_tma_bf16(B0.p, N, K, ldk, bn), mb1 = make_tma_bf16(B1.p, N, K, ldk, bn);
    int ncols = N / stack;
    int kb = (K + 63) / 64;
    int per = (kb + splits - 1) / splits;
    int act = (kb + per - 1) / per;
    DevPtr<float> out((size_t)act * M * ncols);
    DevPtr<unsigned> err(1);
    FSA_CUDA(cudaMemset(err.p, 0, sizeof(unsigned)));
    TcGemm g;
    g.a[0] = &ma0; g.a[1] = &ma1; g.num_a = num_a;
    g.b[0] = &mb0; g.b[1] = &mb1; g.num_b = num_b;
    g.pairs = pairs; g.M = M; g.N = N; g.K = K; g.bn = bn; g.splits = splits; g.stack = stack;
    g.out = out.p; g.ldo = ncols; g.split_stride = (int64_t)M * ncols;
    tc_gemm(g, err.p, s);
    DevPtr<double> e(1);
    FSA_CUDA(cudaMemset(e.p, 0, sizeof(double)));
    Ops ops{{A0.p, A1.p}, {B0.p, B1.p}};
    k_ref_check<<<512, 256, 0, s>>>(M, N, K, ldk, ldk, ops, num_a, num_b, pairs, stack, out.p, ncols,
                                    (int64_t)M * ncols, act, e.p);
    FSA_CHECK_LAUNCH();
    unsigned herr = 0;
    FSA_CUDA(cudaMemcpy(max_rel_err, e.p, sizeof(double), cudaMemcpyDeviceToHost));
    FSA_CUDA(cudaMemcpy(&herr, err.p, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (launched_splits) *launched_splits = act;
    if (herr) return FSA_ERR_TIMEOUT;
    return FSA_OK;
  } catch (const Error& e) {
    set_error(e.msg);
    return e.code;
  }
}

namespace fsa {

// A wait that nothing completes: thread 0 initialises an mbarrier expecting one
// arrival, nobody arrives, and the bounded wait gives up after `polls`
// try_wait polls and records kErrTimeout (the same bounded-wait pattern as the
// tensor-core and SpMM pipelines).  `done` is written afterwards, so the host
// sees that the kernel ran to its end.
__global__ void k_wait_nothing(uint32_t polls, unsigned* __restrict__ err, int* __restrict__ done) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(&bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(1u) : "memory");
    bool ok = false;
    for (uint32_t i = 0; i < polls && !ok; ++i) {
      uint32_t r;
      asm volatile(
          "{\n.reg .pred p;\n"
          "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
          "selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(r)
          : "r"(a), "r"(0u)
          : "memory");
      ok = r != 0;
    }
    if (!ok) atomicOr(err, kErrTimeout);
    *done = 1;
  }
}

__global__ void k_write_one(int* __restrict__ v) { *v = 1; }

}  // namespace fsa

extern "C" int fsa_selftest_wait_timeout(uint32_t polls, int* kernel_finished, int* context_usable) {
  if (!kernel_finished || !context_usable || polls < 1 || polls > (1u << 20)) {
    set_error("fsa_selftest_wait_timeout: bad argument");
    return FSA_ERR_ARG;
  }
  try {
    cudaStream_t s = nullptr;
    DevPtr<unsigned> err(1);
    DevPtr<int> done(2);
    FSA_CUDA(cudaMemset(err.p, 0, sizeof(unsigned)));
    FSA_CUDA(cudaMemset(done.p, 0, 2 * sizeof(int)));
    k_wait_nothing<<<1, 32, 0, s>>>(polls, err.p, done.p);
    FSA_CHECK_LAUNCH();
    FSA_CUDA(cudaDeviceSynchronize());
    // the context is still usable: a second kernel runs and its result comes back
    k_write_one<<<1, 1, 0, s>>>(done.p + 1);
    FSA_CHECK_LAUNCH();
    int h[2] = {0, 0};
    unsigned herr = 0;
    FSA_CUDA(cudaMemcpy(h, done.p, sizeof(h), cudaMemcpyDeviceToHost));
    FSA_CUDA(cudaMemcpy(&herr, err.p, sizeof(herr), cudaMemcpyDeviceToHost));
    *kernel_finished = h[0];
    *context_usable = h[1];
    return (herr & kErrTimeout) ? FSA_ERR_TIMEOUT : FSA_OK;
  } catch (const Error& e) {
    cudaGetLastError();
    set_error(e.msg);
    return e.code;
  }
}
