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
 * (V = Sigma_s~ Z + S + beta V, H = Z + beta H; paper §3.1, Appendix A) in
 * its two forms on the handle's pattern and the FSA_MIXED_BF16X2 operator of
 * theta: the pipelined shared-memory tile kernel and the row kernel, on the
 * same seeded block of ncols (1..127) columns, once with beta = 0 and once
 * with a seeded beta in (0, 1) on seeded V, H.  Both sum each row's products
 * in the same order, so the outputs agree bit for bit.
 *   max_abs_diff  receives max |tile - row| over V and H
 *   staged_tiles  receives the number of tiles that fit the staging capacity
 *                 (the rest run from global memory); may be NULL
 *   total_tiles   receives the number of tiles; may be NULL
 * Returns FSA_OK or an fsa_status.  Runs on the handle's stream.
 */
int fsa_selftest_spmm(fsa_handle* h, const fsa_theta* theta, int ncols, uint64_t seed, double* max_abs_diff,
                      int* staged_tiles, int* total_tiles);

/*
 * fsa_selftest_sddmm — the two sampled dense products of the mixed form in
 * their tile form (m-long rows staged in shared memory per cell-grid tile)
 * against their row form (one warp per row, global gathers), on the handle's
 * pattern:
 *   - the tapered residual values val_ij = (c(s_i,s_j) - a_i.a_j) T(d_ij) and
 *     D_s (paper §2.1, Eq. eqfitcp) of the operator of theta in precision
 *     FSA_MIXED_BF16 or FSA_MIXED_BF16X2;
 *   - their range derivative (paper §2.2), (s1 r'(d) - b_i.a_j - a_i.q_j) T(d)
 *     and its diagonal, with seeded BF16 pairs b and q (n x m_pad).
 *   cap_rows   0: automatic staging capacity; > 0: at most that many staged
 *              rows per tile (larger tiles take the global-memory path)
 *   val_err    receives [max |tile - row| / max |row| over the values,
 *              the same over D_s]
 *   dval_err   the same two figures for the range derivative and its diagonal
 * The operator is rebuilt on the handle's next use.  Returns FSA_OK or an
 * fsa_status.  Runs on the handle's stream.
 */
int fsa_selftest_sddmm(fsa_handle* h, const fsa_theta* theta, int precision, int cap_rows, uint64_t seed,
                       double* val_err, double* dval_err);

/*
 * fsa_selftest_wait_timeout — failure detection without a GPU fault: a kernel
 * waits on an mbarrier that nothing completes, with the bounded wait the
 * library's pipelines use (at most `polls` try_wait polls, 1..2^20), gives up,
 * records the timeout in an error word and returns; a second kernel then runs
 * to show that the context is still usable.  (A self-test; the paper has no
 * counterpart.)
 *   kernel_finished  receives 1 when the waiting kernel ran to its end
 *   context_usable   receives 1 when the kernel launched after it ran
 * Returns FSA_ERR_TIMEOUT when the wait ran out (the expected outcome), FSA_OK
 * if it did not, another fsa_status on error.  Legacy stream, current device.
 */
int fsa_selftest_wait_timeout(uint32_t polls, int* kernel_finished, int* context_usable);

#ifdef __cplusplus
}
#endif

#endif
