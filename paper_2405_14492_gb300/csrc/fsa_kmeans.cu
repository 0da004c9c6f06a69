// kmeans++ selection of inducing points (paper §4.1, which picks the inducing
// points by kmeans++ seeding; Arthur & Vassilvitskii 2007): the first point
// uniformly, each further point with probability proportional to its squared
// distance to the nearest point chosen so far.
//
// The weights are the integers q_i = floor(d_i^2 2^e) (d^2 = dx*dx + dy*dy with
// every operation rounded on its own), so every sum is exact and the choice
// does not depend on summation order: the GPU picks the same indices as any
// other evaluation of the definition.  Per step: one kernel lowers every q_i
// to the distance to the newest point and sums the weights of each chunk of
// 1024 points; one block then finds the chunk and the point whose inclusive
// prefix sum first exceeds floor(h_k Q / 2^53) (h_k the 53-bit draw k of the
// counter-based SplitMix64 stream 9, Q the total).  No host round trip
// between steps.
#include <cmath>
#include <vector>

#include "fsa_internal.cuh"

namespace fsa {

constexpr int kKppChunk = 1024, kKppThreads = 256;
constexpr uint64_t kStreamKmeanspp = 9;

// floor(h * t / 2^53) for h < 2^53 (exact, 128-bit product)
__device__ __forceinline__ uint64_t kpp_scale(uint64_t h, uint64_t t) {
  const uint64_t hi = __umul64hi(h, t), lo = h * t;
  return (hi << 11) | (lo >> 53);
}

__device__ __forceinline__ uint64_t kpp_weight(double x, double y, double cx, double cy, int e) {
  const double dx = __dsub_rn(x, cx), dy = __dsub_rn(y, cy);
  const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
  return (uint64_t)floor(ldexp(d2, e));
}

// bounding box of the points and the exponent e of the weights:
// e = B - ex with B = 62 - bitlength(n) and diag^2 = f 2^ex, f in [0.5, 1)
__global__ void k_kpp_scale(int64_t n, const double2* __restrict__ p, int* __restrict__ e_out) {
  __shared__ double red[4][kKppChunk];
  double xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double2 v = p[i];
    xmin = fmin(xmin, v.x); xmax = fmax(xmax, v.x);
    ymin = fmin(ymin, v.y); ymax = fmax(ymax, v.y);
  }
  red[0][threadIdx.x] = xmin; red[1][threadIdx.x] = xmax;
  red[2][threadIdx.x] = ymin; red[3][threadIdx.x] = ymax;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int t = 1; t < (int)blockDim.x; ++t) {
      xmin = fmin(xmin, red[0][t]); xmax = fmax(xmax, red[1][t]);
      ymin = fmin(ymin, red[2][t]); ymax = fmax(ymax, red[3][t]);
    }
    const double dx = __dsub_rn(xmax, xmin), dy = __dsub_rn(ymax, ymin);
    const double diag2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    int bits = 0;
    for (uint64_t v = (uint64_t)n; v; v >>= 1) ++bits;
    const int B = 62 - bits;
    int ex = 0;
    if (diag2 > 0.0) frexp(diag2, &ex);
    *e_out = diag2 > 0.0 ? B - ex : B;
  }
}

// the first point: index floor(h_0 n / 2^53)
__global__ void k_kpp_first(int64_t n, uint64_t h0, const double2* __restrict__ p, int64_t* __restrict__ idx,
                            double2* __restrict__ center) {
  const int64_t i = (int64_t)kpp_scale(h0, (uint64_t)n);
  idx[0] = i;
  *center = p[i];
}

// q_i = min(q_i, weight to the newest center) (first: the weight itself);
// bsum[chunk] = sum of the chunk's weights
__global__ void __launch_bounds__(kKppThreads) k_kpp_update(int64_t n, const double2* __restrict__ p,
                                                             const double2* __restrict__ center,
                                                             const int* __restrict__ e_ptr, int first,
                                                             uint64_t* __restrict__ q, uint64_t* __restrict__ bsum) {
  __shared__ uint64_t red[kKppThreads];
  const double2 c = *center;
  const int e = *e_ptr;
  const int64_t b0 = (int64_t)blockIdx.x * kKppChunk;
  uint64_t s = 0;
  for (int j = threadIdx.x; j < kKppChunk; j += kKppThreads) {
    const int64_t i = b0 + j;
    if (i < n) {
      const double2 v = p[i];
      uint64_t w = kpp_weight(v.x, v.y, c.x, c.y, e);
      if (!first) w = min(w, q[i]);
      q[i] = w;
      s += w;
    }
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = kKppThreads / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = red[0];
}

// step k: the first point whose inclusive prefix sum of q exceeds
// floor(h_k Q / 2^53); one block of kKppChunk threads
__global__ void __launch_bounds__(kKppChunk) k_kpp_pick(int64_t n, int nb, const uint64_t* __restrict__ bsum,
                                                         const uint64_t* __restrict__ q, uint64_t h,
                                                         const double2* __restrict__ p, int64_t* __restrict__ idx,
                                                         double2* __restrict__ center, unsigned* __restrict__ err) {
  __shared__ uint64_t sc[kKppChunk];
  __shared__ uint64_t target_sh, base_sh;
  __shared__ int blk_sh;
  __shared__ int64_t pick_sh;
  const int t = threadIdx.x;
  // thread t sums the chunk sums [t * per, (t + 1) * per)
  const int per = (nb + kKppChunk - 1) / kKppChunk;
  uint64_t s = 0;
  for (int b = t * per; b < min(nb, (t + 1) * per); ++b) s += bsum[b];
  sc[t] = s;
  __syncthreads();
  // inclusive scan of the thread sums (Hillis-Steele)
  for (int o = 1; o < kKppChunk; o <<= 1) {
    const uint64_t v = t >= o ? sc[t - o] : 0;
    __syncthreads();
    sc[t] += v;
    __syncthreads();
  }
  if (t == 0) {
    const uint64_t total = sc[kKppChunk - 1];
    target_sh = total ? kpp_scale(h, total) : 0;
    blk_sh = -1;
    pick_sh = -1;
    if (total == 0) atomicOr(err, 1u);
  }
  __syncthreads();
  const uint64_t target = target_sh;
  // the thread whose range holds the target walks its chunk sums
  const uint64_t lo = t ? sc[t - 1] : 0;
  if (sc[kKppChunk - 1] > 0 && lo <= target && target < sc[t]) {
    uint64_t acc = lo;
    for (int b = t * per; b < min(nb, (t + 1) * per); ++b) {
      if (target < acc + bsum[b]) {
        blk_sh = b;
        base_sh = acc;
        break;
      }
      acc += bsum[b];
    }
  }
  __syncthreads();
  const int blk = blk_sh;
  if (blk < 0) return;   // no weight left (reported in err) or the walk found nothing
  // within the chunk: inclusive scan of its weights
  const int64_t i = (int64_t)blk * kKppChunk + t;
  sc[t] = i < n ? q[i] : 0;
  __syncthreads();
  for (int o = 1; o < kKppChunk; o <<= 1) {
    const uint64_t v = t >= o ? sc[t - o] : 0;
    __syncthreads();
    sc[t] += v;
    __syncthreads();
  }
  const uint64_t rel = target - base_sh;
  const uint64_t before = t ? sc[t - 1] : 0;
  if (i < n && before <= rel && rel < sc[t]) pick_sh = i;
  __syncthreads();
  if (t == 0) {
    const int64_t pi = pick_sh;
    if (pi < 0) {
      atomicOr(err, 1u);
      return;
    }
    *idx = pi;
    *center = p[pi];
  }
}

}  // namespace fsa

using namespace fsa;

extern "C" fsa_status fsa_kmeanspp(const double* locs, int64_t n, int32_t m, uint64_t seed, int64_t* idx_out,
                                   void* cuda_stream) {
  if (!locs || !idx_out || n < 1 || m < 1 || m > n || n >= ((int64_t)1 << 31)) {
    set_error("fsa_kmeanspp: bad argument (need 1 <= m <= n < 2^31 and non-NULL pointers)");
    return FSA_ERR_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  AllocStreamScope scope(s);
  TraceRange trace("fsa_kmeanspp");
  try {
    const int nb = (int)((n + kKppChunk - 1) / kKppChunk);
    DevPtr<double2> p(n), center(1);
    DevPtr<uint64_t> q(n), bsum(nb);
    DevPtr<int64_t> idx(m);
    DevPtr<int> e(1);
    DevPtr<unsigned> err(1);
    FSA_CUDA(cudaMemsetAsync(err.p, 0, sizeof(unsigned), s));
    FSA_CUDA(cudaMemcpyAsync(p.p, locs, sizeof(double) * 2 * n, cudaMemcpyHostToDevice, s));
    k_kpp_scale<<<1, kKppChunk, 0, s>>>(n, p.p, e.p);
    FSA_CHECK_LAUNCH();
    const uint64_t key = rng_key(seed, kStreamKmeanspp);
    k_kpp_first<<<1, 1, 0, s>>>(n, rng_at(key, 0) >> 11, p.p, idx.p, center.p);
    FSA_CHECK_LAUNCH();
    for (int k = 1; k < m; ++k) {
      k_kpp_update<<<nb, kKppThreads, 0, s>>>(n, p.p, center.p, e.p, k == 1, q.p, bsum.p);
      FSA_CHECK_LAUNCH();
      k_kpp_pick<<<1, kKppChunk, 0, s>>>(n, nb, bsum.p, q.p, rng_at(key, (uint64_t)k) >> 11, p.p, idx.p + k,
                                         center.p, err.p);
      FSA_CHECK_LAUNCH();
    }
    unsigned herr = 0;
    FSA_CUDA(cudaMemcpyAsync(idx_out, idx.p, sizeof(int64_t) * m, cudaMemcpyDeviceToHost, s));
    FSA_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    FSA_CUDA(cudaStreamSynchronize(s));
    if (herr) {
      set_error("fsa_kmeanspp: fewer than m distinct locations");
      return FSA_ERR_ARG;
    }
    return FSA_OK;
  } catch (const Error& e) {
    cudaGetLastError();
    set_error(e.msg);
    return e.code;
  } catch (const std::exception& e) {
    cudaGetLastError();
    return fail_host_exception("fsa_kmeanspp", e);
  }
}
