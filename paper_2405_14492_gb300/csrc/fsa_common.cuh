// Common device helpers of the FSA library (GB300, sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <cmath>
#include <cstdio>
#include <exception>
#include <new>
#include <string>

#include "../../include/fsa.h"

#if defined(__has_include)
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define FSA_HAVE_NVTX 1
#endif
#endif

namespace fsa {

// Named range around one phase of a call (an NVTX push/pop pair, header-only
// NVTX 3): profilers that record NVTX show the phases on the timeline, and
// `ncu --nvtx --nvtx-include "<name>/"` restricts a capture to the kernels
// of one phase.  Without an attached tool a range costs a few nanoseconds.
struct TraceRange {
  explicit TraceRange(const char* name) {
#ifdef FSA_HAVE_NVTX
    nvtxRangePushA(name);
#else
    (void)name;
#endif
  }
  ~TraceRange() {
#ifdef FSA_HAVE_NVTX
    nvtxRangePop();
#endif
  }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

// ---------------------------------------------------------------------------
// host-side error plumbing
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);

struct Error {
  fsa_status code;
  std::string msg;
};

// Status for a host-side exception other than Error (std::bad_alloc from a host
// container -> FSA_ERR_OOM, anything else, e.g. a thread that could not be
// started -> FSA_ERR_CUDA); records the message like set_error.
fsa_status fail_host_exception(const char* where, const std::exception& e);

#define FSA_CUDA(call)                                                            \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      throw ::fsa::Error{FSA_ERR_CUDA, std::string(#call) + ": " +               \
                                           cudaGetErrorString(e_) + " at " +     \
                                           __FILE__ + ":" + std::to_string(__LINE__)}; \
    }                                                                             \
  } while (0)

void count_launch();

#define FSA_CHECK_LAUNCH()    \
  do {                        \
    ::fsa::count_launch();    \
    FSA_CUDA(cudaGetLastError()); \
  } while (0)

#define FSA_REQUIRE(cond, code, text)                     \
  do {                                                    \
    if (!(cond)) throw ::fsa::Error{(code), (text)};      \
  } while (0)

inline unsigned grid_for(int64_t work, int per_block, int max_blocks = 152 * 32) {
  int64_t b = (work + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (unsigned)b;
}

// ---------------------------------------------------------------------------
// covariance function and taper (paper §2, Assumption 3; §2.1)
// ---------------------------------------------------------------------------
// Squared distance with every operation rounded on its own (no FMA), so the
// taper-support predicate d2 < gamma^2 is reproducible bit for bit.
__device__ __forceinline__ double sqdist_rn(double xi, double yi, double xj, double yj) {
  double dx = __dsub_rn(xi, xj);
  double dy = __dsub_rn(yi, yj);
  return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
}

// Matérn correlation r(d): cov 0 -> exp(-d/rho); cov 1 -> (1+x) exp(-x), x = sqrt(3) d / rho
__device__ __forceinline__ double matern_r(int cov, double d, double rho) {
  if (cov == 0) return exp(-d / rho);
  double x = 1.7320508075688772 * d / rho;
  return (1.0 + x) * exp(-x);
}

// d r / d rho
__device__ __forceinline__ double matern_dr(int cov, double d, double rho) {
  if (cov == 0) return (d / (rho * rho)) * exp(-d / rho);
  double x = 1.7320508075688772 * d / rho;
  return (x * x / rho) * exp(-x);
}

__device__ __forceinline__ float matern_r_f(int cov, float d, float rho) {
  if (cov == 0) return __expf(-d / rho);
  float x = 1.7320508f * d / rho;
  return (1.0f + x) * __expf(-x);
}

// Wendland phi_{3,1} taper (support [0, gamma))
__device__ __forceinline__ double wendland(double d, double gamma) {
  if (!(d < gamma)) return 0.0;
  double t = d / gamma;
  double u = 1.0 - t;
  double u2 = u * u;
  return u2 * u2 * (1.0 + 4.0 * t);
}

// ---------------------------------------------------------------------------
// counter-based SplitMix64 (Steele, Lea & Flood 2014)
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
constexpr uint64_t kGoldenGamma = 0x9E3779B97F4A7C15ull;

// key of a (seed, stream) pair: mix64(seed ^ stream * gamma)
__host__ __device__ __forceinline__ uint64_t rng_key(uint64_t seed, uint64_t stream) {
  return mix64(seed ^ (stream * kGoldenGamma));
}
// output number `ctr` of the SplitMix64 sequence seeded with `key`
__host__ __device__ __forceinline__ uint64_t rng_at(uint64_t key, uint64_t ctr) {
  return mix64(key + (ctr + 1ull) * kGoldenGamma);
}
__device__ __forceinline__ double rademacher_at(uint64_t key, uint64_t ctr) {
  return (rng_at(key, ctr) >> 63) ? -1.0 : 1.0;
}
__device__ __forceinline__ double gaussian_at(uint64_t key, uint64_t ctr) {
  uint64_t h1 = rng_at(key, 2ull * ctr), h2 = rng_at(key, 2ull * ctr + 1ull);
  double u1 = ((double)(h1 >> 11) + 1.0) * 0x1.0p-53;
  double u2 = ((double)(h2 >> 11) + 1.0) * 0x1.0p-53;
  return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}
__device__ __forceinline__ double probe_at(int kind, uint64_t key, uint64_t ctr) {
  return kind == 0 ? rademacher_at(key, ctr) : gaussian_at(key, ctr);
}

constexpr uint64_t kStreamEps2 = 4, kStreamEps1 = 5, kStreamPred = 6;

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// error word shared by kernels: bit flags, written with atomicOr
enum : unsigned {
  kErrNotPD = 1u,
  kErrNaN = 2u,
  kErrTimeout = 4u,
  kErrBounds = 8u,
};

// Checked build (-DFSA_CHECKED; compute-sanitizer is not available here):
// FSA_INDEX_OK(cond, err) tests a data-dependent index before the access it
// guards.  A failed test records kErrBounds in the error word (when the launch
// has one), and the caller skips the access.  In the default build it is the
// constant true, so the guarded code is unchanged.
#ifdef FSA_CHECKED
__device__ __forceinline__ bool fsa_index_ok(bool ok, unsigned* err) {
  if (!ok && err) atomicOr(err, kErrBounds);
  return ok;
}
#define FSA_INDEX_OK(cond, err) ::fsa::fsa_index_ok((cond), (err))
#else
#define FSA_INDEX_OK(cond, err) true
#endif

// in-place ascending heap sort of a[0..len) by one thread: O(len log len)
// steps whatever the input order, so a crowded cell or a long neighbour row
// (a taper range close to the extent of the points) costs seconds at worst,
// not the quadratic time of an insertion sort
template <typename T>
__device__ void heap_sort_thread(T* a, int64_t len) {
  auto sift = [&](int64_t root, int64_t end) {
    T v = a[root];
    for (int64_t ch = 2 * root + 1; ch < end; ch = 2 * root + 1) {
      if (ch + 1 < end && a[ch + 1] > a[ch]) ++ch;
      if (!(a[ch] > v)) break;
      a[root] = a[ch];
      root = ch;
    }
    a[root] = v;
  };
  for (int64_t i = len / 2 - 1; i >= 0; --i) sift(i, len);
  for (int64_t end = len - 1; end > 0; --end) {
    T t = a[0]; a[0] = a[end]; a[end] = t;
    sift(0, end);
  }
}

// an FP32 value as a BF16 hi + lo pair (about 16 significant bits)
__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(v);
  lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

}  // namespace fsa
