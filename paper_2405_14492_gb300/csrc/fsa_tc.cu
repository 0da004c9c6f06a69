// tcgen05 BF16 GEMM with TMA loads and TMEM accumulators (sm_103a).
// See fsa_tc.cuh for the contract.
//
// Warp roles (192 threads):
//   warp 0 lane 0 : TMA producer (cp.async.bulk.tensor into a ring of stages)
//   warp 1        : TMEM allocator; lane 0 issues tcgen05.mma (M = 128, N = bn,
//                   K = 16 per instruction, 4 per 64-wide K block)
//   warps 2..5    : epilogue (tcgen05.ld of the 128 x bn FP32 accumulator)
// Every mbarrier wait is bounded: on a timeout the kernel sets kErrTimeout,
// stops issuing work, drains the copies it issued, waits for its MMAs and
// frees its TMEM before returning.
#include <cudaTypedefs.h>

#include <atomic>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "fsa_tc.cuh"

namespace fsa {
namespace tc {

constexpr int BM = 128;
constexpr int BK = 64;
constexpr int kThreads = 192;
constexpr int kMaxStages = 8;
constexpr uint32_t kSpinLimit = 1u << 24;

struct Params {
  CUtensorMap ma[2];
  CUtensorMap mb[2];
  int num_a, num_b;
  unsigned pairs;
  int M, bn, kb_base, kblocks, kb_per_split, stages;   // k-blocks [kb_base, kblocks)
  uint32_t blk;                                         // bit a: A_a blocked; bit 2 + b: B_b blocked
  uint32_t a_bytes, b_bytes, stage_bytes, tmem_cols, idesc;
  int stack, n_valid;
  int lower;                                            // 1: only tiles on or below the diagonal
  int vec_store;                                        // 1: rows 16-byte aligned (two 16-byte stores per 8 columns)
  int ntn;                                              // persistent form: N tiles (tile t: M tile t % mtiles, N tile t / mtiles)
  float* out;
  int64_t ldo, split_stride;
  unsigned* err;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait; gives up early when another role of this CTA, or another CTA
// of the grid (global error word), has timed out
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          const unsigned* gerr) {
  for (uint32_t i = 0; i < kSpinLimit; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (abort_flag && *abort_flag) return false;
    if (gerr && (i & 4095u) == 4095u && (*(volatile const unsigned*)gerr & kErrTimeout)) return false;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

// one operand box of K block kb: 64 K columns x the rows from row0
__device__ __forceinline__ void load_operand(void* dst, const CUtensorMap* map, bool blocked, uint64_t* bar, int kb,
                                             int row0) {
  if (blocked)
    tma_load_3d(dst, map, bar, 0, row0, kb);
  else
    tma_load_2d(dst, map, bar, kb * BK, row0);
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms 1024 B apart
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);   // start address
  d |= (uint64_t)1 << 16;                     // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                     // descriptor version (sm_100 family)
  d |= (uint64_t)2 << 61;                     // 128-byte swizzle
  return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 8 consecutive output columns of one row from col: two 16-byte stores when
// the row is 16-byte aligned and all 8 columns are valid, else one by one
__device__ __forceinline__ void store8(float* orow, int col, const float (&v)[8], int n_valid, bool vec) {
  if (vec && col + 8 <= n_valid) {
    *reinterpret_cast<float4*>(orow + col) = make_float4(v[0], v[1], v[2], v[3]);
    *reinterpret_cast<float4*>(orow + col + 4) = make_float4(v[4], v[5], v[6], v[7]);
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (col + j < n_valid) orow[col + j] = v[j];
  }
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__global__ void __launch_bounds__(kThreads, 1) gemm_kernel(const __grid_constant__ Params p) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[kMaxStages];
  __shared__ __align__(8) uint64_t empty_bar[kMaxStages];
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_sh;

  // a symmetric product needs the tiles on and below the diagonal only (the
  // whole CTA leaves before any barrier or TMEM allocation)
  if (p.lower && (int)blockIdx.y * p.bn >= ((int)blockIdx.x + 1) * BM) return;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * BM;
  const int n0 = blockIdx.y * p.bn;
  const int kb0 = p.kb_base + blockIdx.z * p.kb_per_split;
  const int kb1 = min(p.kblocks, kb0 + p.kb_per_split);
  const int nk = kb1 - kb0;
  const int S = p.stages;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&done_bar, 1);
    abort_sh = (*(volatile const unsigned*)p.err & kErrTimeout) ? 1 : 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_base_sh;

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------------------------------------ producer
      int issued = 0;
      for (int i = 0; i < nk && !abort_sh; ++i) {
        int s = i % S;
        uint32_t ph = (uint32_t)(i / S) & 1u;
        if (!mbar_wait(&empty_bar[s], ph ^ 1u, &abort_sh, p.err)) {
          atomicOr(p.err, kErrTimeout);
          abort_sh = 1;
          break;
        }
        uint8_t* st = smem + (size_t)s * p.stage_bytes;
        mbar_expect_tx(&full_bar[s], p.stage_bytes);
        const int kb = kb0 + i;
        for (int a = 0; a < p.num_a; ++a)
          load_operand(st + a * p.a_bytes, &p.ma[a], (p.blk >> a) & 1u, &full_bar[s], kb, m0);
        for (int b = 0; b < p.num_b; ++b)
          load_operand(st + p.num_a * p.a_bytes + b * p.b_bytes, &p.mb[b], (p.blk >> (2 + b)) & 1u, &full_bar[s], kb,
                       n0);
        issued = i + 1;
      }
      // drain: every copy issued by this thread has landed before the CTA exits
      for (int s = 0; s < S && s < issued; ++s) {
        int last = s + ((issued - 1 - s) / S) * S;
        mbar_wait(&full_bar[s], (uint32_t)(last / S) & 1u, nullptr, nullptr);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------------------ MMA issuer
      for (int i = 0; i < nk && !abort_sh; ++i) {
        int s = i % S;
        uint32_t ph = (uint32_t)(i / S) & 1u;
        if (!mbar_wait(&full_bar[s], ph, &abort_sh, p.err)) {
          atomicOr(p.err, kErrTimeout);
          abort_sh = 1;
          break;
        }
        fence_after();
        uint32_t st = smem_u32(smem + (size_t)s * p.stage_bytes);
        int pidx = 0;
        for (int a = 0; a < p.num_a; ++a) {
          for (int b = 0; b < p.num_b; ++b) {
            if (!(p.pairs & (1u << (2 * a + b)))) continue;
            uint64_t da = smem_desc(st + a * p.a_bytes);
            uint64_t db = smem_desc(st + p.num_a * p.a_bytes + b * p.b_bytes);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
              // +32 bytes along K per instruction = +2 in the 16-byte address field
              mma_bf16(tmem, da + 2 * kk, db + 2 * kk, p.idesc, (i > 0 || pidx > 0 || kk > 0) ? 1u : 0u);
            }
            ++pidx;
          }
        }
        mma_commit(&empty_bar[s]);
      }
      mma_commit(&done_bar);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    bool ok = mbar_wait(&done_bar, 0, &abort_sh, p.err);
    if (!ok) {
      atomicOr(p.err, kErrTimeout);
      abort_sh = 1;
    } else {
      fence_after();
      const int q = warp & 3;
      const int row = m0 + q * 32 + lane;
      const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16);
      float* orow = p.out + (int64_t)blockIdx.z * p.split_stride + (int64_t)row * p.ldo;
      const bool in = row < p.M && nk > 0;
      if (p.stack <= 1) {
        for (int c0 = 0; c0 < p.bn; c0 += 8) {
          uint32_t r[8];
          tmem_ld8(taddr + c0, r);
          tmem_wait_ld();
          if (in) {
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
            store8(orow, n0 + c0, v, p.n_valid, p.vec_store != 0);
          }
        }
      } else {
        // split vector operand stacked along N: sum the stack column blocks
        const int h = p.bn / p.stack;
        for (int c0 = 0; c0 < h; c0 += 8) {
          uint32_t r[8], t[8], u[8];
          tmem_ld8(taddr + c0, r);
          tmem_ld8(taddr + h + c0, t);
          if (p.stack == 3) tmem_ld8(taddr + 2 * h + c0, u);
          tmem_wait_ld();
          if (in) {
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              v[j] = __uint_as_float(r[j]) + __uint_as_float(t[j]);
              if (p.stack == 3) v[j] += __uint_as_float(u[j]);
            }
            store8(orow, c0, v, p.n_valid, p.vec_store != 0);
          }
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    // the accumulator is released only after every MMA of this CTA has completed
    mbar_wait(&done_bar, 0, nullptr, nullptr);
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tmem_cols) : "memory");
  }
}

// Persistent form for problems of many output tiles (no split-K): one CTA per
// SM loops over the tiles blockIdx.x, + gridDim.x, ..., tile t being M tile
// t % mtiles of N tile t / mtiles (consecutive CTAs share a B box).  The TMA
// producer runs ahead through the stage ring across tile boundaries; the
// accumulator is double-buffered in TMEM (two column ranges of tmem_cols / 2),
// so the epilogue of tile j (tcgen05.ld + stores) overlaps the MMAs of tile
// j + 1.  Barriers: full/empty per stage (as above), acc_full[b] (MMA commit)
// and acc_empty[b] (one arrival per epilogue warp).  Every wait is bounded.
__global__ void __launch_bounds__(kThreads, 1) gemm_persistent(const __grid_constant__ Params p) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[kMaxStages];
  __shared__ __align__(8) uint64_t empty_bar[kMaxStages];
  __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2], done_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_sh;

  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk = p.kblocks - p.kb_base;
  const int S = p.stages;
  const int mtiles = (p.M + BM - 1) / BM;
  const int ntiles = mtiles * p.ntn;
  const int nt = ntiles > (int)blockIdx.x ? (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
  const uint32_t half = p.tmem_cols / 2;   // columns of one accumulator buffer

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);
    }
    mbar_init(&done_bar, 1);
    abort_sh = (*(volatile const unsigned*)p.err & kErrTimeout) ? 1 : 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_base_sh;

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------------------------------------ producer
      int it = 0;
      for (int j = 0; j < nt && !abort_sh; ++j) {
        const int t = (int)blockIdx.x + j * (int)gridDim.x;
        const int m0 = (t % mtiles) * BM, n0 = (t / mtiles) * p.bn;
        for (int i = 0; i < nk && !abort_sh; ++i, ++it) {
          const int s = it % S;
          const uint32_t ph = (uint32_t)(it / S) & 1u;
          if (!mbar_wait(&empty_bar[s], ph ^ 1u, &abort_sh, p.err)) {
            atomicOr(p.err, kErrTimeout);
            abort_sh = 1;
            break;
          }
          uint8_t* st = smem + (size_t)s * p.stage_bytes;
          mbar_expect_tx(&full_bar[s], p.stage_bytes);
          const int kb = p.kb_base + i;
          for (int a = 0; a < p.num_a; ++a)
            load_operand(st + a * p.a_bytes, &p.ma[a], (p.blk >> a) & 1u, &full_bar[s], kb, m0);
          for (int b = 0; b < p.num_b; ++b)
            load_operand(st + p.num_a * p.a_bytes + b * p.b_bytes, &p.mb[b], (p.blk >> (2 + b)) & 1u, &full_bar[s],
                         kb, n0);
        }
      }
      // drain: every copy issued by this thread has landed before the CTA exits
      for (int s = 0; s < S && s < it; ++s) {
        const int last = s + ((it - 1 - s) / S) * S;
        mbar_wait(&full_bar[s], (uint32_t)(last / S) & 1u, nullptr, nullptr);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ------------------------------------------------------------ MMA issuer
      int it = 0;
      for (int j = 0; j < nt && !abort_sh; ++j) {
        const int b = j & 1;
        // the epilogue has drained this buffer (use j >> 1 of it; fresh buffers pass)
        if (!mbar_wait(&acc_empty[b], ((uint32_t)(j >> 1) & 1u) ^ 1u, &abort_sh, p.err)) {
          atomicOr(p.err, kErrTimeout);
          abort_sh = 1;
          break;
        }
        fence_after();
        const uint32_t acc = tmem + (uint32_t)b * half;
        for (int i = 0; i < nk; ++i, ++it) {
          const int s = it % S;
          const uint32_t ph = (uint32_t)(it / S) & 1u;
          if (!mbar_wait(&full_bar[s], ph, &abort_sh, p.err)) {
            atomicOr(p.err, kErrTimeout);
            abort_sh = 1;
            break;
          }
          fence_after();
          const uint32_t st = smem_u32(smem + (size_t)s * p.stage_bytes);
          int pidx = 0;
          for (int a = 0; a < p.num_a; ++a) {
            for (int bb = 0; bb < p.num_b; ++bb) {
              if (!(p.pairs & (1u << (2 * a + bb)))) continue;
              const uint64_t da = smem_desc(st + a * p.a_bytes);
              const uint64_t db = smem_desc(st + p.num_a * p.a_bytes + bb * p.b_bytes);
#pragma unroll
              for (int kk = 0; kk < BK / 16; ++kk)
                mma_bf16(acc, da + 2 * kk, db + 2 * kk, p.idesc, (i > 0 || pidx > 0 || kk > 0) ? 1u : 0u);
              ++pidx;
            }
          }
          mma_commit(&empty_bar[s]);
        }
        if (abort_sh) break;
        mma_commit(&acc_full[b]);
      }
      mma_commit(&done_bar);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;
    for (int j = 0; j < nt; ++j) {
      const int b = j & 1;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&acc_full[b], (uint32_t)(j >> 1) & 1u, &abort_sh, p.err));
      if (!ok) {
        if (lane == 0) atomicOr(p.err, kErrTimeout);
        abort_sh = 1;
        break;
      }
      fence_after();
      const int t = (int)blockIdx.x + j * (int)gridDim.x;
      const int m0 = (t % mtiles) * BM, n0 = (t / mtiles) * p.bn;
      const int row = m0 + q * 32 + lane;
      const uint32_t taddr = tmem + (uint32_t)b * half + ((uint32_t)(q * 32) << 16);
      float* orow = p.out + (int64_t)row * p.ldo;
      const bool in = row < p.M && nk > 0;
      if (p.stack <= 1) {
        for (int c0 = 0; c0 < p.bn; c0 += 8) {
          uint32_t r[8];
          tmem_ld8(taddr + c0, r);
          tmem_wait_ld();
          if (in) {
            float v[8];
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) v[jj] = __uint_as_float(r[jj]);
            store8(orow, n0 + c0, v, p.n_valid, p.vec_store != 0);
          }
        }
      } else {
        const int h = p.bn / p.stack;
        for (int c0 = 0; c0 < h; c0 += 8) {
          uint32_t r[8], t[8], u[8];
          tmem_ld8(taddr + c0, r);
          tmem_ld8(taddr + h + c0, t);
          if (p.stack == 3) tmem_ld8(taddr + 2 * h + c0, u);
          tmem_wait_ld();
          if (in) {
            float v[8];
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
              v[jj] = __uint_as_float(r[jj]) + __uint_as_float(t[jj]);
              if (p.stack == 3) v[jj] += __uint_as_float(u[jj]);
            }
            store8(orow, c0, v, p.n_valid, p.vec_store != 0);
          }
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[b]);
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    // the accumulators are released only after every MMA of this CTA has completed
    mbar_wait(&done_bar, 0, nullptr, nullptr);
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tmem_cols) : "memory");
  }
}

}  // namespace tc

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void* f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  });
  if (!fn) throw Error{FSA_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled unavailable"};
  return fn;
}

TmaMap make_tma_bf16_blocked(const __nv_bfloat16* ptr, int64_t rows, int64_t kpad, int box_rows) {
  FSA_REQUIRE(((uintptr_t)ptr & 15) == 0, FSA_ERR_ARG, "TMA base not 16-byte aligned");
  FSA_REQUIRE(kpad % 64 == 0 && kpad > 0, FSA_ERR_ARG, "blocked TMA layout needs K a multiple of 64");
  FSA_REQUIRE(box_rows >= 8 && box_rows <= 256, FSA_ERR_ARG, "TMA box rows out of range");
  TmaMap t;
  t.blocked = 1;
  t.box_rows = box_rows;
  cuuint64_t gdim[3] = {64, (cuuint64_t)rows, (cuuint64_t)(kpad / 64)};
  cuuint64_t gstride[2] = {128, (cuuint64_t)rows * 128};
  cuuint32_t box[3] = {64, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = get_encode()(&t.map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16*>(ptr), gdim,
                            gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  FSA_REQUIRE(r == CUDA_SUCCESS, FSA_ERR_CUDA, "cuTensorMapEncodeTiled (blocked) failed: " + std::to_string((int)r));
  return t;
}

TmaMap make_tma_bf16(const __nv_bfloat16* ptr, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
  FSA_REQUIRE(((uintptr_t)ptr & 15) == 0, FSA_ERR_ARG, "TMA base not 16-byte aligned");
  FSA_REQUIRE((ld * 2) % 16 == 0, FSA_ERR_ARG, "TMA row stride not a multiple of 16 bytes");
  FSA_REQUIRE(box_rows >= 8 && box_rows <= 256, FSA_ERR_ARG, "TMA box rows out of range");
  TmaMap t;
  t.box_rows = box_rows;
  cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t gstride[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = get_encode()(&t.map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(ptr), gdim,
                            gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  FSA_REQUIRE(r == CUDA_SUCCESS, FSA_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  return t;
}

int tc_pick_splits(int M, int N, int K, int bn) {
  int tiles = ((M + tc::BM - 1) / tc::BM) * ((N + bn - 1) / bn);
  int kblocks = (K + tc::BK - 1) / tc::BK;
  if (tiles >= 152) return 1;
  // at most two CTAs per SM in one wave: a partly filled second wave costs a whole tile time
  int s = (2 * 152) / tiles;
  int maxs = kblocks / 8;
  if (s > maxs) s = maxs;
  return s < 1 ? 1 : s;
}

int tc_gemm(const TcGemm& g, unsigned* err, cudaStream_t s) {
  FSA_REQUIRE(g.num_a >= 1 && g.num_a <= 2 && g.num_b >= 1 && g.num_b <= 2, FSA_ERR_ARG, "tc_gemm operand count");
  int bn = g.bn > 0 ? g.bn : std::min(256, (g.N + 15) / 16 * 16);
  FSA_REQUIRE(bn % 16 == 0 && bn >= 16 && bn <= 256, FSA_ERR_ARG, "tc_gemm N tile must be a multiple of 16 <= 256");
  const int stack = g.halves ? 2 : std::max(1, g.stack);
  FSA_REQUIRE(stack <= 3, FSA_ERR_ARG, "tc_gemm stack must be 1, 2 or 3");
  FSA_REQUIRE(stack == 1 || (g.N == bn && bn % stack == 0 && (bn / stack) % 8 == 0), FSA_ERR_ARG,
              "tc_gemm stacked epilogue needs N = bn and N/stack a multiple of 8");
  FSA_REQUIRE(g.M > 0 && g.N > 0 && g.K > 0, FSA_ERR_ARG, "tc_gemm empty problem");
  tc::Params p;
  std::memset(&p, 0, sizeof(p));
  // a box fills exactly one operand slot of a stage: BM rows of A, bn rows of
  // B (a larger box would write past its slot and deliver more bytes than the
  // stage's barrier expects)
  for (int a = 0; a < g.num_a; ++a) {
    FSA_REQUIRE(g.a[a]->box_rows == tc::BM, FSA_ERR_ARG, "tc_gemm: A box rows must equal the M tile");
    p.ma[a] = g.a[a]->map;
    if (g.a[a]->blocked) p.blk |= 1u << a;
  }
  for (int b = 0; b < g.num_b; ++b) {
    FSA_REQUIRE(g.b[b]->box_rows == bn, FSA_ERR_ARG, "tc_gemm: B box rows must equal the N tile");
    p.mb[b] = g.b[b]->map;
    if (g.b[b]->blocked) p.blk |= 4u << b;
  }
  p.num_a = g.num_a;
  p.num_b = g.num_b;
  p.pairs = g.pairs;
  p.M = g.M;
  p.bn = bn;
  FSA_REQUIRE(g.k0 >= 0 && g.k0 % tc::BK == 0, FSA_ERR_ARG, "tc_gemm k0 must be a multiple of 64");
  const int count = (g.K + tc::BK - 1) / tc::BK;
  p.kb_base = g.k0 / tc::BK;
  p.kblocks = p.kb_base + count;
  int splits = std::max(1, std::min(g.splits, count));
  p.kb_per_split = (count + splits - 1) / splits;
  splits = (count + p.kb_per_split - 1) / p.kb_per_split;
  p.a_bytes = tc::BM * tc::BK * 2;
  p.b_bytes = (uint32_t)bn * tc::BK * 2;
  p.stage_bytes = p.num_a * p.a_bytes + p.num_b * p.b_bytes;
  const int budget = 113 * 1024 - 1024;
  p.stages = std::max(2, std::min(tc::kMaxStages, budget / (int)p.stage_bytes));
  uint32_t cols = 32;
  while (cols < (uint32_t)bn) cols <<= 1;
  p.tmem_cols = cols;
  // instruction descriptor: D FP32, A BF16, B BF16, both K-major, N >> 3, M >> 4
  p.idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(bn >> 3) << 17) | ((uint32_t)(tc::BM >> 4) << 24);
  p.stack = stack;
  p.lower = g.lower ? 1 : 0;
  p.vec_store = ((uintptr_t)g.out % 16 == 0 && g.ldo % 4 == 0 && g.split_stride % 4 == 0) ? 1 : 0;
  p.n_valid = g.n_valid > 0 ? g.n_valid : (stack > 1 ? bn / stack : g.N);
  p.out = g.out;
  p.ldo = g.ldo;
  p.split_stride = g.split_stride;
  p.err = err;
  size_t smem = (size_t)p.stages * p.stage_bytes + 1024;
  static int sms = 0;
  static std::once_flag attr_once;
  std::call_once(attr_once, [] {
    cudaFuncSetAttribute(tc::gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(tc::gemm_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  });
  FSA_REQUIRE(smem <= 200 * 1024, FSA_ERR_ARG, "tc_gemm stage ring too large");
  dim3 grid((g.M + tc::BM - 1) / tc::BM, (g.N + bn - 1) / bn, splits);
  // many M tiles of one N tile: the persistent form (one CTA per SM, a deeper
  // stage ring, double-buffered accumulators)
  const bool persistent = splits == 1 && (grid.y == 1 || stack == 1) && !g.lower && sms > 0 &&
                          (int)(grid.x * grid.y) >= 2 * sms && 2 * cols <= 512;
  p.ntn = (int)grid.y;
  if (persistent) {
    p.tmem_cols = 2 * cols;
    p.stages = std::max(2, std::min(tc::kMaxStages, (199 * 1024) / (int)p.stage_bytes));
    smem = std::max<size_t>((size_t)p.stages * p.stage_bytes + 1024, 120 * 1024);   // one CTA per SM (TMEM)
    grid = dim3((unsigned)sms, 1, 1);
  }
  const bool prof = g.tag && profile_on();
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (prof) {
    e0 = profile_event();
    e1 = profile_event();
    FSA_CUDA(cudaEventRecord(e0, s));
  }
  if (persistent)
    tc::gemm_persistent<<<grid, tc::kThreads, smem, s>>>(p);
  else
    tc::gemm_kernel<<<grid, tc::kThreads, smem, s>>>(p);
  FSA_CHECK_LAUNCH();
  if (prof) {
    FSA_CUDA(cudaEventRecord(e1, s));
    double bytes = g.alg_bytes;
    if (bytes <= 0) {
      double rows_a = 0, rows_b = 0;
      for (int a = 0; a < g.num_a; ++a) rows_a += g.M;
      for (int b = 0; b < g.num_b; ++b) rows_b += g.N;
      bytes = (rows_a + rows_b) * g.K * 2.0 + (double)g.M * p.n_valid * 4.0 * splits;
    }
    profile_record(g.tag, e0, e1, bytes);
  }
  return 1;
}

// ---------------------------------------------------------------------------
// launch counter and GEMM timing registry
// ---------------------------------------------------------------------------
static std::atomic<uint64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

struct ProfRec {
  std::string tag;
  cudaEvent_t a, b;
  double bytes;
};
static std::mutex g_prof_mu;
static std::atomic<bool> g_prof_on{false};
static std::vector<ProfRec> g_prof;
static std::vector<cudaEvent_t> g_prof_pool;

bool profile_on() { return g_prof_on.load(std::memory_order_relaxed); }

cudaEvent_t profile_event() {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!g_prof_pool.empty()) {
    cudaEvent_t e = g_prof_pool.back();
    g_prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  FSA_CUDA(cudaEventCreate(&e));
  return e;
}

void profile_record(const char* tag, cudaEvent_t a, cudaEvent_t b, double bytes) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof.push_back(ProfRec{tag, a, b, bytes});
}

}  // namespace fsa

extern "C" {

uint64_t fsa_launch_count(void) { return fsa::g_launches.load(); }

void fsa_profile_enable(int on) { fsa::g_prof_on.store(on != 0); }

void fsa_profile_reset(void) {
  std::lock_guard<std::mutex> lk(fsa::g_prof_mu);
  for (auto& r : fsa::g_prof) {
    fsa::g_prof_pool.push_back(r.a);
    fsa::g_prof_pool.push_back(r.b);
  }
  fsa::g_prof.clear();
}

int fsa_profile_collect(const char* tag, int64_t* launches, double* ms, double* bytes) {
  std::lock_guard<std::mutex> lk(fsa::g_prof_mu);
  int64_t n = 0;
  double t = 0, by = 0;
  for (auto& r : fsa::g_prof) {
    if (!tag || r.tag != tag) continue;
    if (cudaEventSynchronize(r.b) != cudaSuccess) return -2;
    float e = 0;
    if (cudaEventElapsedTime(&e, r.a, r.b) != cudaSuccess) return -2;
    ++n;
    t += e;
    by += r.bytes;
  }
  if (launches) *launches = n;
  if (ms) *ms = t;
  if (bytes) *bytes = by;
  return n > 0 ? 0 : -1;
}

}  // extern "C"

namespace fsa {

}  // namespace fsa
