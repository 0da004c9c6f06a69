// Products of FP64 / FP32 matrices on the tcgen05 tensor cores: each operand
// is split into a BF16 hi + lo pair (about 16 significant bits) and the three
// products hi.hi + hi.lo + lo.hi are accumulated in FP32 (TMEM), over spans of
// the reduction of at most kTcdSpan, whose partial results are added in FP64
// in a fixed order.  Used where an m-column product of the prediction
// (Algorithm 1) would otherwise run on GB300's FP64 units.
#include <algorithm>

#include "fsa_tcd.cuh"

namespace fsa {

constexpr int kTcdSpanBlocks = 64;   // 64-wide K blocks per FP32 span (K <= 4096 per span)
constexpr int kTcdSpansPerLaunch = 16;

// dst (rows x kpad, blocked K-major BF16 hi and lo) from src: element (r, k) is
// src[r * ld + k] (trans = 0) or src[k * ld + r] (trans = 1), zero for k >= K
// or r >= rows.  64 x 64 tiles through shared memory so that both the source
// reads and the blocked writes are coalesced.
template <typename T>
__global__ void k_split_blocked(int64_t rows, int64_t K, int64_t kpad, const T* __restrict__ src, int64_t ld,
                                int trans, __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  __shared__ float tile[64][65];
  const int64_t r0 = (int64_t)blockIdx.x * 64, k0 = (int64_t)blockIdx.y * 64;
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;   // 256 threads: 64 x 4
  for (int yy = ty; yy < 64; yy += 4) {
    float v = 0.f;
    if (!trans) {
      const int64_t r = r0 + yy, k = k0 + tx;
      if (r < rows && k < K) v = (float)src[r * ld + k];
      tile[yy][tx] = v;
    } else {
      const int64_t k = k0 + yy, r = r0 + tx;
      if (r < rows && k < K) v = (float)src[k * ld + r];
      tile[tx][yy] = v;
    }
  }
  __syncthreads();
  for (int yy = ty; yy < 64; yy += 4) {
    const int64_t r = r0 + yy, k = k0 + tx;
    if (r < rows && k < kpad) {
      const int64_t d = blocked_index(r, k, rows);
      split_bf16(tile[yy][tx], hi[d], lo[d]);
    }
  }
}

// FP64 (or precise FP32) values lose bits in the FP32 staging above; for FP64
// sources the pair is formed from the double directly
__global__ void k_split_blocked_f64(int64_t rows, int64_t K, int64_t kpad, const double* __restrict__ src, int64_t ld,
                                    int trans, __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  __shared__ double tile[64][65];
  const int64_t r0 = (int64_t)blockIdx.x * 64, k0 = (int64_t)blockIdx.y * 64;
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
  for (int yy = ty; yy < 64; yy += 4) {
    double v = 0.0;
    if (!trans) {
      const int64_t r = r0 + yy, k = k0 + tx;
      if (r < rows && k < K) v = src[r * ld + k];
      tile[yy][tx] = v;
    } else {
      const int64_t k = k0 + yy, r = r0 + tx;
      if (r < rows && k < K) v = src[k * ld + r];
      tile[tx][yy] = v;
    }
  }
  __syncthreads();
  for (int yy = ty; yy < 64; yy += 4) {
    const int64_t r = r0 + yy, k = k0 + tx;
    if (r < rows && k < kpad) {
      const int64_t d = blocked_index(r, k, rows);
      const double v = tile[yy][tx];
      const __nv_bfloat16 h = __double2bfloat16(v);
      hi[d] = h;
      lo[d] = __double2bfloat16(v - (double)__bfloat162float(h));
    }
  }
}

template <typename T>
static void split_operand(int64_t rows, int64_t K, int64_t kpad, const T* src, int64_t ld, bool trans,
                          __nv_bfloat16* hi, __nv_bfloat16* lo, cudaStream_t s) {
  dim3 grid((unsigned)((rows + 63) / 64), (unsigned)((kpad + 63) / 64));
  if constexpr (std::is_same<T, double>::value)
    k_split_blocked_f64<<<grid, 256, 0, s>>>(rows, K, kpad, src, ld, trans ? 1 : 0, hi, lo);
  else
    k_split_blocked<T><<<grid, 256, 0, s>>>(rows, K, kpad, src, ld, trans ? 1 : 0, hi, lo);
  FSA_CHECK_LAUNCH();
}

// out (FP64, rows x cols, ldo) (+)= sum of the FP32 partials of `spans` spans
__global__ void k_tcd_reduce(int64_t rows, int cols, int spans, const float* __restrict__ part, int64_t ldp,
                             int64_t span_stride, double* __restrict__ out, int64_t ldo, int accumulate) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < rows * cols;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / cols;
    const int c = (int)(t - r * cols);
    double v = accumulate ? out[r * ldo + c] : 0.0;
    for (int z = 0; z < spans; ++z) v += (double)part[(int64_t)z * span_stride + r * ldp + c];
    out[r * ldo + c] = v;
  }
}

template <typename TA, typename TB>
void tc_dgemm(Handle& H, bool ta, bool tb, int M, int N, int K, const TA* A, int64_t lda, const TB* B, int64_t ldb,
              double* C, int64_t ldc, bool accumulate, float* C32, const char* tag) {
  cudaStream_t s = H.stream;
  FSA_REQUIRE(M > 0 && N > 0 && K > 0, FSA_ERR_ARG, "tc_dgemm: empty product");
  const int64_t kpad = ((int64_t)K + 63) / 64 * 64;
  const size_t na = (size_t)M * kpad, nb = (size_t)N * kpad;
  DevPtr<__nv_bfloat16> Ah(na), Al(na), Bh(nb), Bl(nb);
  split_operand<TA>(M, K, kpad, A, lda, ta, Ah.p, Al.p, s);
  split_operand<TB>(N, K, kpad, B, ldb, !tb, Bh.p, Bl.p, s);
  const int bn = std::min(128, (N + 15) / 16 * 16);   // the N tile; B's box has exactly its rows
  TmaMap mAh = make_tma_bf16_blocked(Ah.p, M, kpad, 128), mAl = make_tma_bf16_blocked(Al.p, M, kpad, 128);
  TmaMap mBh = make_tma_bf16_blocked(Bh.p, N, kpad, bn), mBl = make_tma_bf16_blocked(Bl.p, N, kpad, bn);
  TcGemm g;
  g.a[0] = &mAh; g.a[1] = &mAl; g.num_a = 2;
  g.b[0] = &mBh; g.b[1] = &mBl; g.num_b = 2;
  g.pairs = 1u | 2u | 4u;   // hi.hi + hi.lo + lo.hi
  g.M = M; g.N = N; g.bn = bn;
  g.tag = tag;
  const int kb = (int)(kpad / 64);
  if (C32 && kb <= kTcdSpanBlocks) {
    // one span: the FP32 result directly
    g.K = K; g.k0 = 0; g.splits = 1;
    g.out = C32; g.ldo = ldc;
    tc_gemm(g, H.err, s);
    return;
  }
  FSA_REQUIRE(C != nullptr, FSA_ERR_ARG, "tc_dgemm: a reduction longer than one span needs the FP64 output");
  const int spans_total = (kb + kTcdSpanBlocks - 1) / kTcdSpanBlocks;
  const int per_launch = std::min(kTcdSpansPerLaunch, spans_total);
  const int64_t ldp = N;
  DevPtr<float> part((size_t)per_launch * M * ldp);
  g.out = part.p; g.ldo = ldp; g.split_stride = (int64_t)M * ldp;
  for (int b0 = 0, first = 1; b0 < kb; b0 += per_launch * kTcdSpanBlocks, first = 0) {
    const int nbk = std::min(kb - b0, per_launch * kTcdSpanBlocks);
    g.k0 = b0 * 64;
    g.K = std::min<int64_t>((int64_t)nbk * 64, (int64_t)K - g.k0);
    g.splits = (nbk + kTcdSpanBlocks - 1) / kTcdSpanBlocks;
    tc_gemm(g, H.err, s);
    k_tcd_reduce<<<grid_for((int64_t)M * N, 256), 256, 0, s>>>(M, N, g.splits, part.p, ldp, g.split_stride, C, ldc,
                                                                (accumulate || !first) ? 1 : 0);
    FSA_CHECK_LAUNCH();
  }
}

template void tc_dgemm<double, double>(Handle&, bool, bool, int, int, int, const double*, int64_t, const double*,
                                       int64_t, double*, int64_t, bool, float*, const char*);
template void tc_dgemm<float, double>(Handle&, bool, bool, int, int, int, const float*, int64_t, const double*,
                                      int64_t, double*, int64_t, bool, float*, const char*);
template void tc_dgemm<double, float>(Handle&, bool, bool, int, int, int, const double*, int64_t, const float*,
                                      int64_t, double*, int64_t, bool, float*, const char*);
template void tc_dgemm<float, float>(Handle&, bool, bool, int, int, int, const float*, int64_t, const float*,
                                     int64_t, double*, int64_t, bool, float*, const char*);

}  // namespace fsa
