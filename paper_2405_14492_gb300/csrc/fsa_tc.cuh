// tcgen05 (5th-generation tensor core) BF16 GEMM with TMA loads, TMEM
// accumulators and a warp-specialised mbarrier pipeline, for sm_103a.
//
//   D[M x N] (FP32) = sum over operand pairs (a, b) of  A_a[M x K] . B_b[N x K]^T
//
// Both operands are K-major BF16 (row-major with K contiguous), loaded by
// cp.async.bulk.tensor with 128-byte swizzle.  Up to two A and two B tensors
// share one K loop (pairs mask), which gives the hi/lo split products
// (A_hi B_hi + A_hi B_lo + A_lo B_hi) that keep FP32-level accuracy.  With
// `halves`, the epilogue adds output columns j and j + N/2 (B = [x_hi; x_lo]
// stacked along N, so the tensor core sees the split vector operand in one MMA).
#pragma once
#include <cuda.h>

#include "fsa_internal.cuh"

namespace fsa {

struct TmaMap {
  CUtensorMap map;
  int blocked = 0;     // 1: the blocked K-major layout below (3-D map)
  int box_rows = 0;    // rows of one box (one TMA copy fills exactly this many rows)
};

// 2-D K-major BF16 tensor map: rows x cols (cols contiguous, leading dimension
// ld elements, ld * 2 bytes a multiple of 16), box = 64 cols x box_rows rows.
TmaMap make_tma_bf16(const __nv_bfloat16* ptr, int64_t rows, int64_t cols, int64_t ld, int box_rows);

// Blocked K-major layout of a rows x kpad matrix (kpad a multiple of 64): K is
// cut into blocks of 64, and block kb stores columns 64 kb .. 64 kb + 63 of
// all rows, row after row, so that the box of box_rows consecutive rows of one
// K block is one contiguous range of memory (the operands whose K is the
// point index n: a row-major n-long row would put the rows of a box 2n bytes
// apart).  Element (r, k) sits at blocked_index(r, k, rows).  Everything in
// columns k >= K must be stored as zeros (the map does not fill them).
TmaMap make_tma_bf16_blocked(const __nv_bfloat16* ptr, int64_t rows, int64_t kpad, int box_rows);
__host__ __device__ __forceinline__ int64_t blocked_index(int64_t r, int64_t k, int64_t rows) {
  return ((k >> 6) * rows + r) * 64 + (k & 63);
}

struct TcGemm {
  const TmaMap* a[2] = {nullptr, nullptr};
  const TmaMap* b[2] = {nullptr, nullptr};
  int num_a = 1, num_b = 1;
  unsigned pairs = 1;       // bit (2*ia + ib): multiply A_ia with B_ib
  int M = 0;                // rows of D
  int N = 0;                // columns of D (per launch; tiled by bn)
  int K = 0;                // reduction length (from k0)
  int k0 = 0;               // first reduction index (a multiple of 64)
  int bn = 0;               // N tile (multiple of 16, <= 256); 0 = min(N rounded to 16, 256)
  int splits = 1;           // split-K factor (outputs at out + z * split_stride)
  int halves = 0;           // epilogue: out[:, j] = acc[:, j] + acc[:, j + N/2]  (same as stack = 2)
  int stack = 1;            // epilogue: out[:, j] = sum_s acc[:, j + s N/stack], stack in {1, 2, 3}
  float* out = nullptr;
  int64_t ldo = 0;
  int64_t split_stride = 0;
  int n_valid = 0;          // columns of out written (<= N or N/2)
  bool lower = false;       // symmetric result: only the tiles on or below the diagonal are computed
                            // (output tiles strictly above it are left unwritten)
  const char* tag = nullptr;  // profiling tag (fsa_profile.h)
  double alg_bytes = 0;       // algorithmic bytes of this launch (0: from the shapes)
};

// profiling registry (fsa_profile.h)
bool profile_on();
void profile_record(const char* tag, cudaEvent_t a, cudaEvent_t b, double bytes);
cudaEvent_t profile_event();

// Launch; returns the number of kernel launches (1).
int tc_gemm(const TcGemm& g, unsigned* err, cudaStream_t s);

// Largest split-K factor worth using for an (M, N, K) problem on 152 SMs.
int tc_pick_splits(int M, int N, int K, int bn);

}  // namespace fsa
