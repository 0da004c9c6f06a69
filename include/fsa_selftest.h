/*
 * fsa_selftest.h — device self-tests of libfsa's building blocks.
 *
 * These entry points exist for the test suite; the paper has no counterpart
 * (they check the tensor-core GEMM that implements the n x m products of
 * paper §3.1 and the Woodbury apply of the appendix "Runtime of the FITC
 * preconditioner").
 */
#ifndef FSA_SELFTEST_H_
#define FSA_SELFTEST_H_

#include <stdint.h>

#include "fsa.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * fsa_selftest_tc_gemm — run the tcgen05/TMA BF16 GEMM on seeded random BF16
 * operands (A_0 ~ U(-1,1), A_1 ~ U(-0.01,0.01), same for B) and compare with an
 * FP64 reference computed on the device from the same BF16 values.
 *   M, N, K      problem size (any M >= 1, N <= 256 multiple of 16 when halves,
 *                K >= 1; ragged edges exercise the TMA zero fill)
 *   num_a, num_b 1 or 2 operand tensors; pairs: bit 2a+b selects A_a B_b^T
 *   halves       0: plain output; 1 or 2: output column j = acc[j] + acc[j + N/2];
 *                3: output column j = acc[j] + acc[j + N/3] + acc[j + 2N/3]
 *   splits       requested split-K factor
 *   max_rel_err  receives max |got - ref| / sum |a b| over the output
 *   launched_splits receives the split count actually used (may be NULL)
 * Returns 0 on success, FSA_ERR_TIMEOUT if a bounded wait in the kernel ran
 * out, another fsa_status on error.  Runs on the current device, legacy stream.
 */
int fsa_selftest_tc_gemm(int M, int N, int K, int num_a, int num_b, unsigned pairs, int halves, int splits,
                         uint64_t seed, double* max_rel_err, int* launched_splits);

/*
 * fsa_selftest_spmm — the FP32 tapered-residual SpMM of the mixed CG loop
 * (V = Sigma_s~ Z + S, H = Z; paper §3.1) in its two forms on the handle's
 * pattern and the FSA_MIXED_BF16X2 operator of theta: the shared-memory tile
 * kernel and the row kernel, on the same seeded block of ncols (1..127)
 * columns.  Both sum each row's products in the same order, so the outputs
 * agree bit for bit.
 *   max_abs_diff  receives max |tile - row| over V and H
 *   staged_tiles  receives the number of tiles that fit the staging capacity
 *                 (the rest run from global memory); may be NULL
 *   total_tiles   receives the number of tiles; may be NULL
 * Returns FSA_OK or an fsa_status.  Runs on the handle's stream.
 */
int fsa_selftest_spmm(fsa_handle* h, const fsa_theta* theta, int ncols, uint64_t seed, double* max_abs_diff,
                      int* staged_tiles, int* total_tiles);

#ifdef __cplusplus
}
#endif

#endif
