// Products of FP64 / FP32 matrices on the tensor cores through BF16 hi + lo
// pairs (definitions in fsa_tcd.cu).
#pragma once
#include <type_traits>

#include "fsa_tc.cuh"

namespace fsa {

// C (M x N, row-major, ldc) = op(A) op(B) (+ C when accumulate), op(A) M x K
// (A stored M x K, or K x M when ta), op(B) K x N (B stored K x N, or N x K
// when tb).  Every operand as a BF16 hi + lo pair (~2^-16 relative), three
// products per pair, FP32 accumulation over spans of at most 4096 of K and
// FP64 addition of the spans.  With C32 given and K <= 4096 the FP32 result
// goes to C32 (ldc) instead and C is not used.
template <typename TA, typename TB>
void tc_dgemm(Handle& H, bool ta, bool tb, int M, int N, int K, const TA* A, int64_t lda, const TB* B, int64_t ldb,
              double* C, int64_t ldc, bool accumulate, float* C32, const char* tag);

}  // namespace fsa
