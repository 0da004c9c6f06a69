// Bandwidth-oriented block-vector kernels of the CG loop.
//
// Layout: n x ldc row-major.  Element-wise kernels run a flat grid-stride
// loop whose stride (blocks x rows-per-block x ldc) is a multiple of ldc, so
// every thread always touches the same column: loads and stores are fully
// coalesced, and each thread keeps the partial dot product of its column.
// Block partials are reduced over the block's row slots in a fixed order and
// written to part[block][col]; the per-column CG scalars then sum the nblk
// partials in a fixed order, so every dot product is bit-reproducible.
//
// The SpMM (tapered residual Sigma_s~ times the block) runs one warp per row:
// the row's column indices and values are loaded once, coalesced, into the
// lanes and broadcast with shuffles, so the gathers of neighbour rows are
// independent and several stay in flight per lane.
#pragma once
#include <algorithm>
#include <type_traits>

#include "fsa_internal.cuh"
#include "fsa_scalars.cuh"
#include "fsa_solver.cuh"
#include "fsa_tc.cuh"

namespace fsa {

template <typename T> struct VAcc { using type = double; };
template <> struct VAcc<float> { using type = float; };

// block reduction of per-thread column partials -> part[blockIdx.x][col]
__device__ __forceinline__ void vec_block_partials(double acc, int ldc, int rpb, double* __restrict__ red,
                                                   double* __restrict__ part) {
  red[threadIdx.x] = acc;
  __syncthreads();
  if ((int)threadIdx.x < ldc) {
    double s = 0.0;
    for (int r = 0; r < rpb; ++r) s += red[r * ldc + threadIdx.x];
    part[(int64_t)blockIdx.x * ldc + threadIdx.x] = s;
  }
}

#define FSA_VEC_BEGIN                                                          \
  extern __shared__ double red[];                                              \
  const int col = threadIdx.x % ldc;                                           \
  const int64_t row0 = (int64_t)blockIdx.x * rpb + threadIdx.x / ldc;          \
  const int64_t rstride = (int64_t)gridDim.x * rpb;                            \
  double acc = 0.0;                                                            \
  typename VAcc<T>::type sub = 0;                                              \
  int cnt = 0;

#define FSA_VEC_ACC(v)                                              \
  do {                                                              \
    sub += (v);                                                     \
    if (++cnt == 32) { acc += (double)sub; sub = 0; cnt = 0; }      \
  } while (0)

#define FSA_VEC_END                      \
  acc += (double)sub;                    \
  vec_block_partials(acc, ldc, rpb, red, part); \
  finish_scalars(step, part, ldc, c, l, q, red);

// U += a H ; R -= a V ; (X = R Dinv) ; part = ||R||^2
template <typename T>
__global__ void kv_ur_update(int64_t n, int c, int ldc, int rpb, T* __restrict__ U, T* __restrict__ R,
                             const T* __restrict__ H, const T* __restrict__ V, const T* __restrict__ Dinv,
                             T* __restrict__ X, const double* __restrict__ alpha, const int32_t* __restrict__ active,
                             double* __restrict__ part, int step, int l, CGScalars q) {
  FSA_VEC_BEGIN
  const T a = (col < c && active[col]) ? (T)alpha[col] : (T)0;
  for (int64_t i = row0; i < n; i += rstride) {
    const int64_t idx = i * ldc + col;
    if (col < c) {
      T r = R[idx];
      if (a != (T)0) {
        U[idx] = U[idx] + a * H[idx];
        r = r - a * V[idx];
        R[idx] = r;
      }
      if (X) X[idx] = r * Dinv[i];
      FSA_VEC_ACC(r * r);
    } else if (X) {
      X[idx] = (T)0;
    }
  }
  FSA_VEC_END
}

// Z = (R - S) Dinv ; part = r^T z
template <typename T>
__global__ void kv_z_update(int64_t n, int c, int ldc, int rpb, const T* __restrict__ R, const T* __restrict__ S,
                            const T* __restrict__ Dinv, T* __restrict__ Z, double* __restrict__ part, int step,
                            int l, CGScalars q) {
  FSA_VEC_BEGIN
  for (int64_t i = row0; i < n; i += rstride) {
    const int64_t idx = i * ldc + col;
    if (col < c) {
      T r = R[idx];
      T z = (r - S[idx]) * Dinv[i];
      Z[idx] = z;
      FSA_VEC_ACC(r * z);
    } else {
      Z[idx] = (T)0;
    }
  }
  FSA_VEC_END
}

// X = R Dinv
template <typename T>
__global__ void kv_row_scale(int64_t n, int c, int ldc, int rpb, const T* __restrict__ R, const T* __restrict__ Dinv,
                             T* __restrict__ X) {
  const int col = threadIdx.x % ldc;
  const int64_t row0 = (int64_t)blockIdx.x * rpb + threadIdx.x / ldc;
  const int64_t rstride = (int64_t)gridDim.x * rpb;
  for (int64_t i = row0; i < n; i += rstride) {
    const int64_t idx = i * ldc + col;
    X[idx] = col < c ? R[idx] * Dinv[i] : (T)0;
  }
}

#undef FSA_VEC_BEGIN
#undef FSA_VEC_ACC
#undef FSA_VEC_END

// V = Sigma_s~ Z + S + beta V ; H = Z + beta H ; part = h^T v
// NS 32-column slots per lane (ldc <= 32 NS); 8 warps per block.
template <typename T, typename VT, int NS>
__global__ void __launch_bounds__(256) kv_spmm_fused(int64_t n, int c, int ldc, const int64_t* __restrict__ rowptr,
                                                     const int32_t* __restrict__ colidx,
                                                     const VT* __restrict__ vals, const T* __restrict__ Z,
                                                     const T* __restrict__ S, T* __restrict__ V, T* __restrict__ H,
                                                     const double* __restrict__ beta, double* __restrict__ part,
                                                     int step, CGScalars q) {
  __shared__ double red[8][NS * 32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t nwarps = (int64_t)gridDim.x * 8;
  T b[NS];
  double dot[NS];
  typename VAcc<T>::type sub[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    int col = lane + 32 * s;
    b[s] = col < c ? (T)beta[col] : (T)0;
    dot[s] = 0.0;
    sub[s] = 0;
  }
  int cnt = 0;
  for (int64_t i = (int64_t)blockIdx.x * 8 + wib; i < n; i += nwarps) {
    const int64_t rb = rowptr[i], re = rowptr[i + 1];
    T acc[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) acc[s] = 0;
    for (int64_t base = rb; base < re; base += 32) {
      const int m = (int)((re - base) < 32 ? (re - base) : 32);
      int myc = lane < m ? colidx[base + lane] : 0;
      T myv = lane < m ? (T)vals[base + lane] : (T)0;
      if (!FSA_INDEX_OK(myc >= 0 && myc < n, q.err)) { myc = 0; myv = (T)0; }   // checked build
#pragma unroll 4
      for (int t = 0; t < m; ++t) {
        const int j = __shfl_sync(0xffffffffu, myc, t);
        const T v = __shfl_sync(0xffffffffu, myv, t);
        const T* zr = Z + (int64_t)j * ldc;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
          int col = lane + 32 * s;
          if (col < ldc) acc[s] += v * zr[col];
        }
      }
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      int col = lane + 32 * s;
      if (col >= ldc) continue;
      int64_t idx = i * ldc + col;
      if (col < c) {
        T v = acc[s] + S[idx] + (b[s] != (T)0 ? b[s] * V[idx] : (T)0);
        T h = Z[idx] + (b[s] != (T)0 ? b[s] * H[idx] : (T)0);
        V[idx] = v;
        H[idx] = h;
        sub[s] += h * v;
      } else {
        V[idx] = (T)0;
        H[idx] = (T)0;
      }
    }
    if (++cnt == 32) {
#pragma unroll
      for (int s = 0; s < NS; ++s) { dot[s] += (double)sub[s]; sub[s] = 0; }
      cnt = 0;
    }
  }
#pragma unroll
  for (int s = 0; s < NS; ++s) red[wib][lane + 32 * s] = dot[s] + (double)sub[s];
  __syncthreads();
  for (int col = threadIdx.x; col < ldc; col += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w][col];
    part[(int64_t)blockIdx.x * ldc + col] = t;
  }
  finish_scalars(step, part, ldc, c, 0, q, &red[0][0]);
}

// FP32 form: lane L owns columns 4L..4L+3 (ldc <= 128, ldc % 4 == 0), so one
// 16-byte load per active lane gathers a whole neighbour row.
static __global__ void __launch_bounds__(256) kv_spmm_fused_f4(int64_t n, int c, int ldc, const int64_t* __restrict__ rowptr,
                                                        const int32_t* __restrict__ colidx,
                                                        const float* __restrict__ vals, const float* __restrict__ Z,
                                                        const float* __restrict__ S, float* __restrict__ V,
                                                        float* __restrict__ H, const double* __restrict__ beta,
                                                        double* __restrict__ part, int step, CGScalars q) {
  __shared__ double red[8][128];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t nwarps = (int64_t)gridDim.x * 8;
  const int c4 = ldc >> 2;
  const bool act = lane < c4;
  const int col0 = 4 * lane;
  float b[4];
  float sub[4] = {0.f, 0.f, 0.f, 0.f};
  double dot[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int k = 0; k < 4; ++k) b[k] = (act && col0 + k < c) ? (float)beta[col0 + k] : 0.f;
  const bool use_b = (b[0] != 0.f) || (b[1] != 0.f) || (b[2] != 0.f) || (b[3] != 0.f);
  int cnt = 0;
  for (int64_t i = (int64_t)blockIdx.x * 8 + wib; i < n; i += nwarps) {
    const int64_t rb = rowptr[i], re = rowptr[i + 1];
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    // the row's own operands are loaded up front, in flight with the gathers
    const int64_t idx = i * ldc + col0;
    float4 sv = make_float4(0.f, 0.f, 0.f, 0.f), zi = sv, vv = sv, hh = sv;
    if (act) {
      sv = *reinterpret_cast<const float4*>(S + idx);
      zi = *reinterpret_cast<const float4*>(Z + idx);
      if (use_b) {
        vv = *reinterpret_cast<const float4*>(V + idx);
        hh = *reinterpret_cast<const float4*>(H + idx);
      }
    }
    for (int64_t base = rb; base < re; base += 32) {
      const int m = (int)((re - base) < 32 ? (re - base) : 32);
      int myc = lane < m ? colidx[base + lane] : 0;
      float myv = lane < m ? vals[base + lane] : 0.f;
      if (!FSA_INDEX_OK(myc >= 0 && myc < n, q.err)) { myc = 0; myv = 0.f; }   // checked build
#pragma unroll 8
      for (int t = 0; t < m; ++t) {
        const int j = __shfl_sync(0xffffffffu, myc, t);
        const float v = __shfl_sync(0xffffffffu, myv, t);
        if (act) {
          const float4 z = *reinterpret_cast<const float4*>(Z + (int64_t)j * ldc + col0);
          acc.x = fmaf(v, z.x, acc.x);
          acc.y = fmaf(v, z.y, acc.y);
          acc.z = fmaf(v, z.z, acc.z);
          acc.w = fmaf(v, z.w, acc.w);
        }
      }
    }
    if (act) {
      float4 vo = make_float4(acc.x + sv.x, acc.y + sv.y, acc.z + sv.z, acc.w + sv.w);
      float4 ho = zi;
      if (use_b) {
        vo.x += b[0] * vv.x; vo.y += b[1] * vv.y; vo.z += b[2] * vv.z; vo.w += b[3] * vv.w;
        ho.x += b[0] * hh.x; ho.y += b[1] * hh.y; ho.z += b[2] * hh.z; ho.w += b[3] * hh.w;
      }
      // columns >= c hold zeros in Z and S and get zero beta, so they stay zero
      *reinterpret_cast<float4*>(V + idx) = vo;
      *reinterpret_cast<float4*>(H + idx) = ho;
      sub[0] += ho.x * vo.x; sub[1] += ho.y * vo.y; sub[2] += ho.z * vo.z; sub[3] += ho.w * vo.w;
    }
    if (++cnt == 32) {
#pragma unroll
      for (int k = 0; k < 4; ++k) { dot[k] += (double)sub[k]; sub[k] = 0.f; }
      cnt = 0;
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) red[wib][(4 * lane + k) & 127] = act ? dot[k] + (double)sub[k] : 0.0;
  __syncthreads();
  for (int col = threadIdx.x; col < ldc; col += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w][col];
    part[(int64_t)blockIdx.x * ldc + col] = t;
  }
  finish_scalars(step, part, ldc, c, 0, q, &red[0][0]);
}

// asynchronous global -> shared copies (cp.async): the copies of a tile are
// issued without passing through registers and complete as one group
__device__ __forceinline__ void cpa16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cpa8(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cpa4(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// mbarrier and bulk-copy (TMA, non-tensor) primitives of the SpMM pipeline;
// every wait is bounded (kSpSpin polls), after which the caller records
// kErrTimeout and stops
constexpr uint32_t kSpSpin = 1u << 26;
__device__ __forceinline__ uint32_t sp_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void sp_mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sp_smem(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void sp_mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sp_smem(b)) : "memory");
}
__device__ __forceinline__ void sp_mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sp_smem(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool sp_mbar_wait(uint64_t* b, uint32_t parity, const unsigned* gerr) {
  for (uint32_t i = 0; i < kSpSpin; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(sp_smem(b)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (gerr && (i & 4095u) == 4095u && (*(volatile const unsigned*)gerr & kErrTimeout)) return false;
  }
  return false;
}
// records a timed-out wait in the error word (when the launch has one)
__device__ __forceinline__ void sp_flag(unsigned* err) {
  if (err) atomicOr(err, kErrTimeout);
}
// bytes (a multiple of 16) from 16-byte aligned global src to 16-byte aligned shared dst
__device__ __forceinline__ void sp_bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   sp_smem(dst)),
               "l"(src), "r"(bytes), "r"(sp_smem(bar))
               : "memory");
}

// FP32 form over the cell-grid tiles, warp-specialised: one persistent block
// per SM runs its tiles (blockIdx.x, + gridDim.x, ...) through a byte ring of
// shared memory in which consecutive tiles are placed back to back (each at
// its own size).  The producer lane (last warp) gathers the tile records 16
// at a time (cp.async into one of two buffers, completion on an mbarrier),
// places a tile and fills it
// with bulk copies (TMA, completion counted in bytes on the tile slot's full
// barrier): its three neighbour ranges of Z (contiguous runs of rows), its own
// rows of S, V and H (V and H only when some beta is nonzero), the union
// entries of its row groups and the groups' entry offsets (rounded out to
// 16-byte boundaries; the arrays are padded for it).  Before placing a tile
// the producer waits for the release (empty barrier) of the newest earlier
// tile whose bytes it would overwrite, and of the tile that last used the
// slot.  The consumer warps wait on the full barrier, compute the tile from
// shared memory, store V and H, and release the slot on its empty barrier;
// there is no block-wide barrier per tile.
//
// Work unit: a row group (kGrpRows consecutive rows of the tile), taken by the
// consumer warps in turn across tiles.  Lane ch owns the float4 chunk ch of
// every row (ldc <= 128).  Per union entry: one (kGrpRows <= 3) or two
// broadcast 16-byte loads of the entry (staged column, the group's values)
// and one 16-byte load of the staged Z row per lane, then kGrpRows x 4 FMAs;
// each staged Z row is read once per group instead of once per (row, nonzero).  Every row sums its products in
// CSR order (a zero value leaves the sum unchanged), exactly as the row
// kernel.  A tile larger than the ring, or holding a column outside its
// ranges (the cell-grid pattern produces none), gathers from global memory.
constexpr int kSpConsumers = 15, kSpThreads = (kSpConsumers + 1) * 32, kSpSlots = 4;
// true: a tile's own rows of S, V and H are staged in the ring with its Z
// ranges; false: each consumer warp loads its group's rows from global memory
// when it starts the group (the loads complete behind the group's products)
constexpr bool kSpStageOwn = false;
constexpr int kSpRecBatch = 16;   // tile records per bulk copy
constexpr int kSpMeta = 16;   // per slot: p0, nr, n0, r1b, staged, groups and the byte offsets of the parts

// shared-memory bytes of a staged tile and the offsets of its parts from the
// tile's start: Z rows, S, V, H rows, union entries (kEntWords int32 each),
// group offsets (ngo int32, a multiple of 4)
struct SpTileLayout {
  int s, v, h, en, go, bytes;
};
__host__ __device__ __forceinline__ SpTileLayout sp_tile_layout(int zrows, int nr, int64_t nent, int64_t ngo,
                                                                 int ldc, bool use_b) {
  const int64_t rb = (int64_t)ldc * 4;
  SpTileLayout l;
  int64_t off = (int64_t)zrows * rb;
  const int64_t own = kSpStageOwn ? (int64_t)nr * rb : 0;
  l.s = (int)off; off += own;
  l.v = (int)off; if (use_b) off += own;
  l.h = (int)off; if (use_b) off += own;
  l.en = (int)off; off += nent * (kEntWords * 4);
  l.go = (int)off; off += ngo * 4;
  const int64_t bytes = (off + 127) / 128 * 128;
  l.bytes = bytes > (int64_t)1 << 30 ? 1 << 30 : (int)bytes;
  return l;
}

// the int32 range [ga, gz) of gofs holding a tile's ng + 1 group offsets from
// gb, rounded out to 16-byte boundaries
__host__ __device__ __forceinline__ void sp_gofs_range(int gb, int ng, int& ga, int& gz) {
  ga = gb & ~3;
  gz = (gb + ng + 1 + 3) & ~3;
}

struct SpRing {   // the ring's size in bytes
  int bytes;
};

static __global__ void __launch_bounds__(kSpThreads, 1) kv_spmm_tma(
    int ntiles, const int32_t* __restrict__ ptile, SpRing ring, int c, int ldc,
    const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colidx, const int4* __restrict__ gent, const int32_t* __restrict__ gofs, const float* __restrict__ vals,
    const float* __restrict__ Z, const float* __restrict__ S, float* __restrict__ V, float* __restrict__ H,
    const double* __restrict__ beta, double* __restrict__ part, int step, CGScalars q) {
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ __align__(8) uint64_t full_bar[kSpSlots], empty_bar[kSpSlots];
  __shared__ int smeta[kSpSlots][kSpMeta];
  __shared__ __align__(16) float bsh[128];   // beta per column (0 beyond c)
  __shared__ int any_b;
  __shared__ __align__(16) int recs[2][kSpRecBatch][kTileWords];   // tile records, two batches
  __shared__ __align__(8) uint64_t rec_bar[2];
  const int tid = threadIdx.x;
  const int c4 = ldc >> 2;
  const int lane = tid & 31, wib = tid >> 5;
  const float4* Z4 = reinterpret_cast<const float4*>(Z);
  const float4* S4 = reinterpret_cast<const float4*>(S);
  const float4* V4 = reinterpret_cast<const float4*>(V);
  const float4* H4 = reinterpret_cast<const float4*>(H);
  double dacc[4] = {0.0, 0.0, 0.0, 0.0};
  if (tid == 0) {
    any_b = 0;
    for (int s = 0; s < kSpSlots; ++s) {
      sp_mbar_init(&full_bar[s], 1);
      sp_mbar_init(&empty_bar[s], kSpConsumers);
    }
    sp_mbar_init(&rec_bar[0], 1);
    sp_mbar_init(&rec_bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  for (int col = tid; col < 128; col += kSpThreads) {
    const float bv = col < c ? (float)beta[col] : 0.f;
    bsh[col] = bv;
    if (bv != 0.f) any_b = 1;
  }
  __syncthreads();
  const bool use_b = any_b != 0;
  // this block's tiles: k -> blockIdx.x + k * gridDim.x (gridDim.x <= ntiles):
  // the blocks sweep the cell rows together, so the neighbour ranges one block
  // stages are in L2 for the blocks on the adjacent cell rows
  const int nk = (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  if (wib == kSpConsumers) {
    // ---------------- producer ----------------
    if (lane == 0) {
      int issued = 0;
      int head = 0;                    // next free byte of the ring
      int released = -1;               // every tile <= released has been released
      int ra[kSpSlots], rz[kSpSlots];  // byte range [ra, rz) of the tile in each slot (empty: ra = rz)
      for (int s = 0; s < kSpSlots; ++s) ra[s] = rz[s] = 0;
      bool ok = true;
      // wait until tile j (and so every earlier tile) is released
      auto release = [&](int j) {
        if (j <= released) return true;
        if (!sp_mbar_wait(&empty_bar[j % kSpSlots], (uint32_t)(j / kSpSlots) & 1u, q.err)) return false;
        released = j;
        return true;
      };
      // tile records, kSpRecBatch per bulk copy into two alternating buffers:
      // batch bt holds tiles [bt kSpRecBatch, (bt + 1) kSpRecBatch) and uses
      // buffer bt & 1 with barrier phase (bt >> 1) & 1
      int rec_issued = 0, rec_ready = 0;   // batches issued, batches waited for
      auto rec_issue = [&]() {
        const int k0 = rec_issued * kSpRecBatch;
        if (k0 >= nk) return;
        const int cnt = min(kSpRecBatch, nk - k0);
        for (int r = 0; r < cnt; ++r) {
          const int4* src = reinterpret_cast<const int4*>(ptile + ((int64_t)blockIdx.x + (int64_t)(k0 + r) * gridDim.x) *
                                                                      kTileWords);
          int4* dst = reinterpret_cast<int4*>(recs[rec_issued & 1][r]);
#pragma unroll
          for (int w = 0; w < kTileWords / 4; ++w) cpa16(dst + w, src + w);
        }
        // the barrier's one arrival comes when these copies have landed
        asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(sp_smem(&rec_bar[rec_issued & 1]))
                     : "memory");
        ++rec_issued;
      };
      // the record of this block's tile kk (nullptr if a wait ran out)
      auto rec_of = [&](int kk) -> const int* {
        const int bt = kk / kSpRecBatch;
        while (rec_ready <= bt) {
          if (!sp_mbar_wait(&rec_bar[rec_ready & 1], (uint32_t)(rec_ready >> 1) & 1u, q.err)) return nullptr;
          ++rec_ready;
        }
        return recs[bt & 1][kk % kSpRecBatch];
      };
      rec_issue();
      rec_issue();
      for (int k = 0; k < nk && ok; ++k) {
        const int s = k % kSpSlots;
        if (k >= kSpSlots && !release(k - kSpSlots)) { ok = false; break; }
        const int* rec = rec_of(k);
        if (!rec) { ok = false; break; }
        const int p0 = rec[0], nr = rec[1], r0b = rec[2], n0 = rec[3], r1b = rec[4], n1 = rec[5], r2b = rec[6],
                  n2 = rec[7], gb = rec[11], ne = rec[14];
        const int64_t eb = (int64_t)(uint32_t)rec[12] | ((int64_t)rec[13] << 32);
        // the tile's rows and neighbour ranges inside the points (checked build);
        // a record that fails is skipped whole
        const bool rec_ok = FSA_INDEX_OK(p0 >= 0 && nr >= 0 && (int64_t)p0 + nr <= q.nrows && r0b >= 0 && n0 >= 0 &&
                                             (int64_t)r0b + n0 <= q.nrows && r1b >= 0 && n1 >= 0 &&
                                             (int64_t)r1b + n1 <= q.nrows && r2b >= 0 && n2 >= 0 &&
                                             (int64_t)r2b + n2 <= q.nrows && ne >= 0 && eb >= 0,
                                         q.err);
        const int ng = rec_ok ? (nr + kGrpRows - 1) / kGrpRows : 0;
        int ga, gz;
        sp_gofs_range(gb, ng, ga, gz);
        const SpTileLayout lay = sp_tile_layout(n0 + n1 + n2, nr, ne, gz - ga, ldc, use_b);
        const bool staged = rec_ok && !rec[15] && lay.bytes <= ring.bytes;
        int base = 0;
        ra[s] = rz[s] = 0;
        if (staged) {
          if (head + lay.bytes > ring.bytes) head = 0;
          base = head;
          // the newest earlier tile whose bytes overlap [base, base + bytes)
          for (int j = k - 1; j > released && j > k - kSpSlots; --j) {
            const int sj = j % kSpSlots;
            if (ra[sj] < base + lay.bytes && base < rz[sj]) {
              if (!release(j)) ok = false;
              break;
            }
          }
          if (!ok) break;
          head = base + lay.bytes;
          ra[s] = base;
          rz[s] = head;
        }
        int* mt = smeta[s];
        mt[0] = p0; mt[1] = rec_ok ? nr : 0; mt[2] = n0; mt[3] = r1b; mt[4] = staged ? 1 : 0; mt[5] = ng;
        mt[12] = n0 + n1 + n2;   // staged Z rows
        mt[6] = base + lay.go + (gb - ga) * 4;
        mt[7] = base; mt[8] = base + lay.s; mt[9] = base + lay.v; mt[10] = base + lay.h; mt[11] = base + lay.en;
        if (staged) {
          unsigned char* sb = smraw + base;
          const uint32_t rb = (uint32_t)ldc * 4u;
          const uint32_t bz = (uint32_t)(n0 + n1 + n2) * rb, bo = (uint32_t)nr * rb,
                         be = (uint32_t)ne * (uint32_t)(kEntWords * 4),
                         bg = (uint32_t)(gz - ga) * 4u;
          sp_mbar_expect_tx(&full_bar[s], bz + (kSpStageOwn ? (use_b ? 3u : 1u) * bo : 0u) + be + bg);
          if (n0 > 0) sp_bulk_load(sb, Z + (int64_t)r0b * ldc, (uint32_t)n0 * rb, &full_bar[s]);
          if (n1 > 0) sp_bulk_load(sb + (size_t)n0 * rb, Z + (int64_t)r1b * ldc, (uint32_t)n1 * rb, &full_bar[s]);
          if (n2 > 0)
            sp_bulk_load(sb + (size_t)(n0 + n1) * rb, Z + (int64_t)r2b * ldc, (uint32_t)n2 * rb, &full_bar[s]);
          if (kSpStageOwn) sp_bulk_load(sb + lay.s, S + (int64_t)p0 * ldc, bo, &full_bar[s]);
          if (kSpStageOwn && use_b) {
            sp_bulk_load(sb + lay.v, V + (int64_t)p0 * ldc, bo, &full_bar[s]);
            sp_bulk_load(sb + lay.h, H + (int64_t)p0 * ldc, bo, &full_bar[s]);
          }
          if (ne > 0) sp_bulk_load(sb + lay.en, gent + kEntVec * eb, be, &full_bar[s]);
          sp_bulk_load(sb + lay.go, gofs + ga, bg, &full_bar[s]);
        } else {
          sp_mbar_arrive(&full_bar[s]);
        }
        issued = k + 1;
        // the last record of a batch has been read: its buffer takes the
        // batch after next
        if (k % kSpRecBatch == kSpRecBatch - 1) rec_issue();
      }
      if (!ok) sp_flag(q.err);
      // no copy may still be in flight when the block exits: wait (bounded)
      // for the last fill of every slot and for the record batches not yet waited for
      for (int s = 0; s < kSpSlots && s < issued; ++s) {
        const int klast = s + ((issued - 1 - s) / kSpSlots) * kSpSlots;
        if (!sp_mbar_wait(&full_bar[s], (uint32_t)(klast / kSpSlots) & 1u, q.err)) sp_flag(q.err);
      }
      for (; rec_ready < rec_issued; ++rec_ready)
        if (!sp_mbar_wait(&rec_bar[rec_ready & 1], (uint32_t)(rec_ready >> 1) & 1u, q.err)) sp_flag(q.err);
    }
  } else {
    // ---------------- consumers ----------------
    // (dacc: this lane's running h^T v partials of its 4 columns)
    // lanes >= c4 own no columns and only take part in the barrier waits
    const bool lane_on = lane < c4;
    const float4 b4 = lane_on ? make_float4(bsh[4 * lane], bsh[4 * lane + 1], bsh[4 * lane + 2], bsh[4 * lane + 3])
                              : make_float4(0.f, 0.f, 0.f, 0.f);
    float sub[4] = {0.f, 0.f, 0.f, 0.f};
    int rows_since = 0;
    auto flush = [&]() {
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        dacc[kk] += (double)sub[kk];
        sub[kk] = 0.f;
      }
      rows_since = 0;
    };
    // V, H of row i from its product acc, S, Z_i (and V, H for beta != 0)
    auto finish_row = [&](int64_t i, const float4& acc, const float4& sv, const float4& zi, const float4& vv,
                          const float4& hh) {
      float4 vo = make_float4(acc.x + sv.x, acc.y + sv.y, acc.z + sv.z, acc.w + sv.w);
      float4 ho = zi;
      if (use_b) {
        vo.x += b4.x * vv.x; vo.y += b4.y * vv.y; vo.z += b4.z * vv.z; vo.w += b4.w * vv.w;
        ho.x += b4.x * hh.x; ho.y += b4.y * hh.y; ho.z += b4.z * hh.z; ho.w += b4.w * hh.w;
      }
      reinterpret_cast<float4*>(V)[i * c4 + lane] = vo;
      reinterpret_cast<float4*>(H)[i * c4 + lane] = ho;
      sub[0] += ho.x * vo.x; sub[1] += ho.y * vo.y; sub[2] += ho.z * vo.z; sub[3] += ho.w * vo.w;
    };
    int gseq = 0;   // row groups of this block's earlier tiles (the groups are dealt to the warps in turn)
    for (int k = 0; k < nk; ++k) {
      const int s = k % kSpSlots;
      if (!__all_sync(0xffffffffu, sp_mbar_wait(&full_bar[s], (uint32_t)(k / kSpSlots) & 1u, q.err))) {
        if (lane == 0) sp_flag(q.err);
        break;
      }
      const int* mt = smeta[s];
      const int p0 = mt[0], nr = mt[1], n0 = mt[2], r1b = mt[3], ng = mt[5], zrows = mt[12];
      const bool staged = mt[4] != 0;
      const int* gos = reinterpret_cast<const int*>(smraw + mt[6]);
      const float4* zs = reinterpret_cast<const float4*>(smraw + mt[7]);
      const float4* ss = reinterpret_cast<const float4*>(smraw + mt[8]);
      const float4* vs = reinterpret_cast<const float4*>(smraw + mt[9]);
      const float4* hs = reinterpret_cast<const float4*>(smraw + mt[10]);
      const int4* en = reinterpret_cast<const int4*>(smraw + mt[11]);
      int j = (wib - gseq % kSpConsumers + kSpConsumers) % kSpConsumers;
      gseq += ng;
      if (lane_on) {
        for (; j < ng; j += kSpConsumers) {
          const int r0 = j * kGrpRows;
          const int gr = min(kGrpRows, nr - r0);
          float4 acc[kGrpRows];
#pragma unroll
          for (int g = 0; g < kGrpRows; ++g) acc[g] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (staged) {
            const int eb = gos[j], ee = gos[j + 1];
            float4 gs[kGrpRows], gv[kGrpRows], gh[kGrpRows];   // own rows from global memory
            if (!kSpStageOwn) {
#pragma unroll
              for (int g = 0; g < kGrpRows; ++g) {
                gs[g] = gv[g] = gh[g] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (g < gr) {
                  const int64_t x = ((int64_t)p0 + r0 + g) * c4 + lane;
                  gs[g] = S4[x];
                  if (use_b) { gv[g] = V4[x]; gh[g] = H4[x]; }
                }
              }
            }
#pragma unroll 8
            for (int e = eb; e < ee; ++e) {
              const int4 m0 = en[kEntVec * e];
              const int4 m1 = kEntVec == 2 ? en[kEntVec * e + 1] : make_int4(0, 0, 0, 0);
              if (!FSA_INDEX_OK(m0.x >= 0 && m0.x < zrows, q.err)) continue;
              const float4 z = zs[m0.x * c4 + lane];
              const float w[7] = {__int_as_float(m0.y), __int_as_float(m0.z), __int_as_float(m0.w),
                                  __int_as_float(m1.x), __int_as_float(m1.y), __int_as_float(m1.z),
                                  __int_as_float(m1.w)};
#pragma unroll
              for (int g = 0; g < kGrpRows; ++g) {
                acc[g].x = fmaf(w[g], z.x, acc[g].x); acc[g].y = fmaf(w[g], z.y, acc[g].y);
                acc[g].z = fmaf(w[g], z.z, acc[g].z); acc[g].w = fmaf(w[g], z.w, acc[g].w);
              }
            }
#pragma unroll
            for (int g = 0; g < kGrpRows; ++g) {
              if (g < gr) {
                const int r = r0 + g;
                const int64_t i = (int64_t)p0 + r;
                const int zo = n0 + (int)(i - r1b);   // the own row among the staged ones
                if (!FSA_INDEX_OK(zo >= 0 && zo < zrows, q.err)) continue;
                const float4 zi = zs[zo * c4 + lane];
                float4 sv, vv = make_float4(0.f, 0.f, 0.f, 0.f), hh = vv;
                if (kSpStageOwn) {
                  sv = ss[r * c4 + lane];
                  if (use_b) { vv = vs[r * c4 + lane]; hh = hs[r * c4 + lane]; }
                } else {
                  sv = gs[g]; vv = gv[g]; hh = gh[g];
                }
                finish_row(i, acc[g], sv, zi, vv, hh);
              }
            }
          } else {
            // rows gathered from global memory in CSR order
#pragma unroll
            for (int g = 0; g < kGrpRows; ++g) {
              if (g < gr) {
                const int64_t i = (int64_t)p0 + r0 + g;
                const int64_t rb = rowptr[i], re = rowptr[i + 1];
                for (int64_t t = rb; t < re; ++t) {
                  const float v = vals[t];
                  if (!FSA_INDEX_OK(colidx[t] >= 0 && colidx[t] < q.nrows, q.err)) continue;
                  const float4 z = Z4[(int64_t)colidx[t] * c4 + lane];
                  acc[g].x = fmaf(v, z.x, acc[g].x); acc[g].y = fmaf(v, z.y, acc[g].y);
                  acc[g].z = fmaf(v, z.z, acc[g].z); acc[g].w = fmaf(v, z.w, acc[g].w);
                }
                const float4 zi = Z4[i * c4 + lane], sv = S4[i * c4 + lane];
                float4 vv = make_float4(0.f, 0.f, 0.f, 0.f), hh = vv;
                if (use_b) { vv = V4[i * c4 + lane]; hh = H4[i * c4 + lane]; }
                finish_row(i, acc[g], sv, zi, vv, hh);
              }
            }
          }
          rows_since += gr;
          if (rows_since >= 28) flush();
        }
      }
      __syncwarp();
      if (lane == 0) sp_mbar_arrive(&empty_bar[s]);   // this warp is done with stage s
    }
    flush();
  }
  // every copy into the ring has landed (the producer waited for them): the
  // ring holds the consumer warps' column partials now
  __syncthreads();
  double* wdot = reinterpret_cast<double*>(smraw);   // [kSpConsumers][128]
  if (wib < kSpConsumers && lane < c4) {
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) wdot[wib * 128 + 4 * lane + kk] = dacc[kk];
  }
  __syncthreads();
  for (int col = tid; col < ldc; col += kSpThreads) {
    double t = 0.0;
    for (int w = 0; w < kSpConsumers; ++w) t += wdot[w * 128 + col];
    part[(int64_t)blockIdx.x * ldc + col] = t;
  }
  __syncthreads();
  finish_scalars(step, part, ldc, c, 0, q, wdot);
}

// launch shape of kv_spmm_tma: the byte ring takes the shared-memory budget;
// one block per SM.  The cap_* fields describe which tiles fit the ring (for
// the self-test's count): a tile is staged when its layout fits.
struct StagedLaunch {
  int blocks = 0;
  SpRing ring{};
  size_t smem = 0;
};
constexpr size_t kSpSmemMax = 219 * 1024;
// the ring's dynamic shared memory for this translation unit's copy of the
// kernel (every launcher below is static, so it launches the copy whose
// attribute it set); false if the device refuses it (the error is cleared)
static inline bool sp_ring_enabled() {
  static const bool ok = [] {
    const bool r = cudaFuncSetAttribute(kv_spmm_tma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)kSpSmemMax) == cudaSuccess;
    if (!r) cudaGetLastError();
    return r;
  }();
  return ok;
}
static inline StagedLaunch staged_launch(const Handle& Hd, int ldc) {
  (void)ldc;
  StagedLaunch L;
  L.ring.bytes = (int)kSpSmemMax;
  L.smem = kSpSmemMax;
  if (!sp_ring_enabled()) return L;   // blocks = 0: the row kernel runs
  int dev = 0, sms = 152, per = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kv_spmm_tma, kSpThreads, L.smem) != cudaSuccess) {
    cudaGetLastError();
    per = 0;
  }
  L.blocks = per > 0 ? std::min(Hd.sp_ntiles, sms * per) : 0;
  return L;
}

// ---------------------------------------------------------------------------
// FP32 element-wise kernels with 16-byte accesses: thread -> 4 consecutive
// columns (c4 = ldc/4 threads per row, rpb rows per block step), row loop
// unrolled so that several independent loads are in flight per thread.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void vec4_block_partials(const double (&acc)[4], int ldc, int c4, int rpb,
                                                    double* __restrict__ red, double* __restrict__ part) {
#pragma unroll
  for (int k = 0; k < 4; ++k) red[threadIdx.x * 4 + k] = acc[k];
  __syncthreads();
  for (int col = threadIdx.x; col < ldc; col += blockDim.x) {
    double s = 0.0;
    for (int r = 0; r < rpb; ++r) s += red[(r * c4 + col / 4) * 4 + (col & 3)];
    part[(int64_t)blockIdx.x * ldc + col] = s;
  }
}

// U += a H ; R -= a V ; part = ||R||^2.  Two rows per thread per step, their
// loads issued before the arithmetic (as in kv4_z_update).
static __global__ void kv4_ur_update(int64_t n, int c, int ldc, int rpb, float* __restrict__ U, float* __restrict__ R,
                                     const float* __restrict__ H, const float* __restrict__ V,
                                     const double* __restrict__ alpha, const int32_t* __restrict__ active,
                                     double* __restrict__ part, int step, int l, CGScalars q) {
  extern __shared__ double red4[];
  const int c4 = ldc >> 2;
  const int cq = threadIdx.x % c4, col0 = 4 * cq;
  const int64_t row0 = (int64_t)blockIdx.x * rpb + threadIdx.x / c4;
  const int64_t rstride = (int64_t)gridDim.x * rpb;
  float a[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) a[k] = (col0 + k < c && active[col0 + k]) ? (float)alpha[col0 + k] : 0.f;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  float sub[4] = {0.f, 0.f, 0.f, 0.f};
  int cnt = 0;
  auto urow = [&](float4 r, const float4 h, const float4 v, float4 u, const int64_t idx) {
    u.x = fmaf(a[0], h.x, u.x); u.y = fmaf(a[1], h.y, u.y); u.z = fmaf(a[2], h.z, u.z); u.w = fmaf(a[3], h.w, u.w);
    r.x = fmaf(-a[0], v.x, r.x); r.y = fmaf(-a[1], v.y, r.y); r.z = fmaf(-a[2], v.z, r.z); r.w = fmaf(-a[3], v.w, r.w);
    *reinterpret_cast<float4*>(U + idx) = u;
    *reinterpret_cast<float4*>(R + idx) = r;
    sub[0] += r.x * r.x; sub[1] += r.y * r.y; sub[2] += r.z * r.z; sub[3] += r.w * r.w;
  };
  int64_t i = row0;
  for (; i + rstride < n; i += 2 * rstride) {
    const int64_t ia = i * ldc + col0, ib = (i + rstride) * ldc + col0;
    const float4 ra = *reinterpret_cast<const float4*>(R + ia), rb = *reinterpret_cast<const float4*>(R + ib);
    const float4 ha = *reinterpret_cast<const float4*>(H + ia), hb = *reinterpret_cast<const float4*>(H + ib);
    const float4 va = *reinterpret_cast<const float4*>(V + ia), vb = *reinterpret_cast<const float4*>(V + ib);
    const float4 ua = *reinterpret_cast<const float4*>(U + ia), ub = *reinterpret_cast<const float4*>(U + ib);
    urow(ra, ha, va, ua, ia);
    urow(rb, hb, vb, ub, ib);
    if (++cnt == 16) {
#pragma unroll
      for (int k = 0; k < 4; ++k) { acc[k] += (double)sub[k]; sub[k] = 0.f; }
      cnt = 0;
    }
  }
  if (i < n) {
    const int64_t ia = i * ldc + col0;
    urow(*reinterpret_cast<const float4*>(R + ia), *reinterpret_cast<const float4*>(H + ia),
         *reinterpret_cast<const float4*>(V + ia), *reinterpret_cast<const float4*>(U + ia), ia);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) acc[k] += (double)sub[k];
  vec4_block_partials(acc, ldc, c4, rpb, red4, part);
  finish_scalars(step, part, ldc, c, l, q, red4);
}

// Z = (R - S) Dinv ; part = r^T z.  A thread takes two rows per step and
// issues all their loads before the arithmetic: the kernel streams two arrays
// in and one out, and one row in flight per thread left the DRAM half idle.
// at most 51 registers: five blocks of up to 256 threads per SM (the loop is
// latency-bound; more resident warps keep more rows' loads in flight; at six
// blocks the registers spill and it is slower)
static __global__ void __launch_bounds__(256, 5) kv4_z_update(int64_t n, int c, int ldc, int rpb,
                                                            const float* __restrict__ R,
                                    const float* __restrict__ S, const float* __restrict__ Dinv,
                                    float* __restrict__ Z, double* __restrict__ part, int step, int l, CGScalars q) {
  extern __shared__ double red4[];
  const int c4 = ldc >> 2;
  const int cq = threadIdx.x % c4, col0 = 4 * cq;
  const int64_t row0 = (int64_t)blockIdx.x * rpb + threadIdx.x / c4;
  const int64_t rstride = (int64_t)gridDim.x * rpb;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  float sub[4] = {0.f, 0.f, 0.f, 0.f};
  int cnt = 0;
  auto zrow = [&](const float4 r, const float4 sv, const float d, const int64_t idx) {
    // columns >= c hold zeros in R and S, so Z is zero there
    const float4 z = make_float4((r.x - sv.x) * d, (r.y - sv.y) * d, (r.z - sv.z) * d, (r.w - sv.w) * d);
    *reinterpret_cast<float4*>(Z + idx) = z;
    sub[0] += r.x * z.x; sub[1] += r.y * z.y; sub[2] += r.z * z.z; sub[3] += r.w * z.w;
  };
  int64_t i = row0;
#pragma unroll 2
  for (; i + rstride < n; i += 2 * rstride) {
    const int64_t ia = i * ldc + col0, ib = (i + rstride) * ldc + col0;
    const float4 ra = *reinterpret_cast<const float4*>(R + ia);
    const float4 sa = *reinterpret_cast<const float4*>(S + ia);
    const float4 rb = *reinterpret_cast<const float4*>(R + ib);
    const float4 sb = *reinterpret_cast<const float4*>(S + ib);
    const float da = Dinv[i], db = Dinv[i + rstride];
    zrow(ra, sa, da, ia);
    zrow(rb, sb, db, ib);
    if (++cnt == 16) {
#pragma unroll
      for (int k = 0; k < 4; ++k) { acc[k] += (double)sub[k]; sub[k] = 0.f; }
      cnt = 0;
    }
  }
  if (i < n) {
    const int64_t ia = i * ldc + col0;
    zrow(*reinterpret_cast<const float4*>(R + ia), *reinterpret_cast<const float4*>(S + ia), Dinv[i], ia);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) acc[k] += (double)sub[k];
  vec4_block_partials(acc, ldc, c4, rpb, red4, part);
  finish_scalars(step, part, ldc, c, l, q, red4);
}

// Z = (R - S) Dinv ; part = r^T z, streamed through shared memory by bulk
// copies.  A block takes the chunks blockIdx.x, + gridDim.x, ... of kZPer rpb
// rows (R and S rows are contiguous, so a chunk of each is one bulk copy);
// thread 0 keeps kZStages chunks in flight, their completion counted in bytes
// on the slot's mbarrier, and every thread computes its kZPer rows of a landed
// chunk from shared memory (the rows' D^-1 are plain loads issued before the
// wait) and stores Z.  Waits are bounded: a wait that runs out records
// kErrTimeout, the block stops computing, waits (bounded) for its copies in
// flight and still takes part in the scalar step.
constexpr int kZPer = 2, kZStages = 6;
static __global__ void __launch_bounds__(256) kz_bulk(int64_t n, int c, int ldc, int rpb, const float* __restrict__ R,
                                                      const float* __restrict__ S, const float* __restrict__ Dinv,
                                                      float* __restrict__ Z, double* __restrict__ part, int step, int l,
                                                      CGScalars q) {
  extern __shared__ __align__(16) unsigned char zsm[];
  const int c4 = ldc >> 2, crow = kZPer * rpb;   // rows per chunk
  const size_t slot_f = (size_t)crow * ldc;      // floats per array and slot
  float* buf = reinterpret_cast<float*>(zsm);    // [kZStages][R, S][crow * ldc]
  uint64_t* full = reinterpret_cast<uint64_t*>(buf + (size_t)kZStages * 2 * slot_f);
  const int cq = threadIdx.x % c4, rr0 = threadIdx.x / c4;
  const int64_t nchunks = (n + crow - 1) / crow;
  const int64_t mine = nchunks > (int64_t)blockIdx.x ? (nchunks - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kZStages; ++s) sp_mbar_init(&full[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  auto chunk_rows = [&](int64_t k, int64_t& r0) {
    r0 = ((int64_t)blockIdx.x + k * gridDim.x) * crow;
    return (int)min((int64_t)crow, n - r0);
  };
  auto issue = [&](int64_t k) {   // thread 0: chunk k of this block into slot k % kZStages
    int64_t r0;
    const int rows = chunk_rows(k, r0);
    const int s = (int)(k % kZStages);
    const uint32_t bytes = (uint32_t)rows * (uint32_t)ldc * 4u;
    sp_mbar_expect_tx(&full[s], 2u * bytes);
    sp_bulk_load(buf + (size_t)s * 2 * slot_f, R + r0 * ldc, bytes, &full[s]);
    sp_bulk_load(buf + (size_t)s * 2 * slot_f + slot_f, S + r0 * ldc, bytes, &full[s]);
  };
  int64_t issued = 0;
  if (threadIdx.x == 0)
    for (; issued < min((int64_t)kZStages, mine); ++issued) issue(issued);
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  float sub[4] = {0.f, 0.f, 0.f, 0.f};
  int cnt = 0;
  int64_t k = 0;
  for (; k < mine; ++k) {
    int64_t r0;
    const int rows = chunk_rows(k, r0);
    const int s = (int)(k % kZStages);
    float d[kZPer];
#pragma unroll
    for (int j = 0; j < kZPer; ++j) {
      const int rr = rr0 + j * rpb;
      d[j] = rr < rows ? Dinv[r0 + rr] : 0.f;
    }
    const bool ok = sp_mbar_wait(&full[s], (uint32_t)(k / kZStages) & 1u, q.err);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) sp_flag(q.err);
      break;
    }
    const float* bR = buf + (size_t)s * 2 * slot_f;
    const float* bS = bR + slot_f;
#pragma unroll
    for (int j = 0; j < kZPer; ++j) {
      const int rr = rr0 + j * rpb;
      if (rr < rows) {
        const float4 r = *reinterpret_cast<const float4*>(bR + (size_t)rr * ldc + 4 * cq);
        const float4 sv = *reinterpret_cast<const float4*>(bS + (size_t)rr * ldc + 4 * cq);
        // columns >= c hold zeros in R and S, so Z is zero there
        const float4 z = make_float4((r.x - sv.x) * d[j], (r.y - sv.y) * d[j], (r.z - sv.z) * d[j],
                                     (r.w - sv.w) * d[j]);
        *reinterpret_cast<float4*>(Z + (r0 + rr) * ldc + 4 * cq) = z;
        sub[0] += r.x * z.x; sub[1] += r.y * z.y; sub[2] += r.z * z.z; sub[3] += r.w * z.w;
      }
    }
    if (++cnt == 16) {
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) { acc[kk] += (double)sub[kk]; sub[kk] = 0.f; }
      cnt = 0;
    }
    __syncthreads();   // slot s is free
    if (threadIdx.x == 0 && issued < mine) issue(issued++);
  }
  if (threadIdx.x == 0) {
    // after a timed-out wait no copy may still be in flight when the block
    // moves on: wait (bounded) for every chunk issued and not yet consumed
    for (int64_t j = k; j < issued; ++j)
      if (!sp_mbar_wait(&full[j % kZStages], (uint32_t)(j / kZStages) & 1u, nullptr)) sp_flag(q.err);
  }
  __syncthreads();
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) acc[kk] += (double)sub[kk];
  double* red4 = reinterpret_cast<double*>(zsm);   // the stages are idle now
  vec4_block_partials(acc, ldc, c4, rpb, red4, part);
  finish_scalars(step, part, ldc, c, l, q, red4);
}

// launch shape of kz_bulk: rpb x c4 threads, the stages' shared memory, one
// full wave of resident blocks (at most the layout's partial rows); blocks = 0
// where the device refuses the shared memory
struct ZBulkLaunch {
  int blocks = 0, threads = 32, rpb = 1;
  size_t smem = 0;
};
static inline ZBulkLaunch zbulk_launch(const CGLayout& lay) {
  ZBulkLaunch z;
  const int c4 = lay.ldc / 4;
  z.rpb = std::max(1, 256 / c4);
  z.threads = z.rpb * c4;
  const size_t stages = (size_t)kZStages * 2 * kZPer * z.rpb * lay.ldc * sizeof(float) + kZStages * sizeof(uint64_t);
  z.smem = std::max(stages, (size_t)z.threads * 4 * sizeof(double));
  if (cudaFuncSetAttribute(kz_bulk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)z.smem) != cudaSuccess) {
    cudaGetLastError();
    return z;
  }
  int dev = 0, sms = 152, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kz_bulk, z.threads, z.smem) != cudaSuccess) {
    cudaGetLastError();
    per = 0;
  }
  z.blocks = per > 0 ? std::min(lay.nblk, sms * per) : 0;
  return z;
}

// CUDA-event timing of one launch under the profiling hooks (fsa_profile.h):
// records the tag's algorithmic bytes with the launch's device time
struct ProfScope {
  const char* tag;
  double bytes;
  cudaStream_t s;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ProfScope(const char* t, double b, cudaStream_t st, bool want = true) : tag(t), bytes(b), s(st) {
    if (want && profile_on()) {
      e0 = profile_event();
      e1 = profile_event();
      cudaEventRecord(e0, s);
    }
  }
  ~ProfScope() {
    if (e0) {
      cudaEventRecord(e1, s);
      profile_record(tag, e0, e1, bytes);
    }
  }
};

struct Vec4Launch {
  int blocks, threads, rpb;
  size_t smem;
};
// one full wave of the kernel (SM count x its resident blocks, at most the
// layout's partial rows): a second, partly filled wave would leave SMs idle
static inline Vec4Launch vec4_launch(const CGLayout& lay, const void* kernel) {
  Vec4Launch v;
  const int c4 = lay.ldc / 4;
  v.rpb = std::max(1, 256 / c4);
  v.threads = v.rpb * c4;
  v.smem = (size_t)v.threads * 4 * sizeof(double);
  int dev = 0, sms = 152, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, v.threads, v.smem);
  v.blocks = per > 0 ? std::min(lay.nblk, sms * per) : lay.nblk;
  return v;
}

// grid of one full wave: SM count x resident blocks of the kernel
static inline int spmm_f4_blocks() {
  static const int blocks = [] {
    int dev = 0, sms = 152, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kv_spmm_fused_f4, 256, 0);
    return sms * (per > 0 ? per : 1);
  }();
  return blocks;
}

CGScalars make_scalars(Handle& H, const fsa_opts& o, int L);

// the host reads the active-column count after every iteration
inline bool should_poll(int /*it*/) { return true; }

template <typename T, typename VT>
static inline void launch_spmm_fused(const CGLayout& lay, cudaStream_t s, const int64_t* rowptr, const int32_t* col,
                              const VT* vals, const T* Z, const T* S, T* V, T* H, const double* beta,
                              double* part, int step, const CGScalars& q) {
  if constexpr (std::is_same<T, float>::value && std::is_same<VT, float>::value) {
    if (lay.ldc % 4 == 0 && lay.ldc <= 128) {
      const int nb = std::min(lay.nblk, spmm_f4_blocks());
      kv_spmm_fused_f4<<<nb, 256, 0, s>>>(lay.n, lay.c, lay.ldc, rowptr, col, vals, Z, S, V, H, beta, part, step, q);
      FSA_CHECK_LAUNCH();
      return;
    }
  }
  const int ns = (lay.ldc + 31) / 32;
  switch (ns) {
    case 1: kv_spmm_fused<T, VT, 1><<<lay.nblk, 256, 0, s>>>(lay.n, lay.c, lay.ldc, rowptr, col, vals, Z, S, V, H, beta, part, step, q); break;
    case 2: kv_spmm_fused<T, VT, 2><<<lay.nblk, 256, 0, s>>>(lay.n, lay.c, lay.ldc, rowptr, col, vals, Z, S, V, H, beta, part, step, q); break;
    case 3: kv_spmm_fused<T, VT, 3><<<lay.nblk, 256, 0, s>>>(lay.n, lay.c, lay.ldc, rowptr, col, vals, Z, S, V, H, beta, part, step, q); break;
    case 4: kv_spmm_fused<T, VT, 4><<<lay.nblk, 256, 0, s>>>(lay.n, lay.c, lay.ldc, rowptr, col, vals, Z, S, V, H, beta, part, step, q); break;
    default: throw Error{FSA_ERR_UNSUPPORTED, "block of more than 128 columns"};
  }
  FSA_CHECK_LAUNCH();
}

// FP32 SpMM of the CG loop: the staged tile kernel when the handle has tiles,
// the row kernel otherwise
static inline void launch_spmm_f32(const Handle& Hd, const CGLayout& lay, const StagedLaunch& L, cudaStream_t s,
                            const float* vals, const float* Z, const float* S, float* V, float* Hv,
                            const double* beta, double* part, int step, const CGScalars& q) {
  if (Hd.sp_ntiles > 0 && lay.ldc % 4 == 0 && lay.ldc <= 128 && L.blocks > 0 && vals == Hd.op.vals32.p &&
      Hd.op.grp_ent.p && sp_ring_enabled()) {
    // timed under the profiling hooks (tag pcg_spmm); algorithmic bytes: the
    // CSR pattern (column + value per nonzero, row pointers), Z and S read
    // once, V and H read and written once (the union entries the kernel reads
    // instead of the pattern are not counted)
    const bool prof = profile_on() && step != kStepNone;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (prof) {
      e0 = profile_event();
      e1 = profile_event();
      FSA_CUDA(cudaEventRecord(e0, s));
    }
    CGScalars qn = q;
    qn.nrows = Hd.n;   // the bound of the checked build's row checks
    kv_spmm_tma<<<std::min(L.blocks, lay.nblk), kSpThreads, L.smem, s>>>(
        Hd.sp_ntiles, Hd.sp_ptile.p, L.ring, lay.c, lay.ldc, Hd.rowptr.p, Hd.col.p, Hd.op.grp_ent.p, Hd.gofs.p, vals, Z,
        S, V, Hv, beta, part, step, qn);
    FSA_CHECK_LAUNCH();
    if (prof) {
      FSA_CUDA(cudaEventRecord(e1, s));
      const double nb = (double)Hd.n * lay.c * sizeof(float);   // the c columns; not the padding to ldc
      profile_record("pcg_spmm", e0, e1, (double)Hd.nnz * 8.0 + (double)(Hd.n + 1) * 8.0 + 6.0 * nb);
    }
    return;
  }
  launch_spmm_fused<float, float>(lay, s, Hd.rowptr.p, Hd.col.p, vals, Z, S, V, Hv, beta, part, step, q);
}

}  // namespace fsa
