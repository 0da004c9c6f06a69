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

#ifdef __cplusplus
}
#endif

#endif
