/*
 * fsa_profile.h — measurement hooks of libfsa (no counterpart in the paper;
 * they report how the hot path of §3.1 uses the GPU).
 *
 * Launch counting is always on.  Kernel timing, when enabled, brackets every
 * tensor-core GEMM launch with CUDA events recorded on the stream the GEMM is
 * launched on, and attributes the elapsed device time and the GEMM's
 * algorithmic bytes (operands read once, outputs written once) to a tag:
 *   "pcg_AtX"  per-CG-iteration  w = A~^T (D^-1 R)      (split-K)
 *   "pcg_Aq"   per-CG-iteration  s = A~ q
 *   "build"    operator build    A = Sigma_nm L^-T, M = I + A~^T D^-1 A~, probes
 *   "grad"     gradient          B = dK L^-T, F = A~ E, projections
 * and every tiled SpMM of the mixed CG loop:
 *   "pcg_spmm" per-CG-iteration  V = Sigma_s~ Z + S + beta V, H = Z + beta H
 *              (bytes: 8 per nonzero, the row pointers, Z and S read, V and H
 *              read and written)
 * and the element-wise kernels of the mixed CG loop:
 *   "pcg_ur"    U += alpha H, R -= alpha V, |R|^2   (U, R read and written; H, V read)
 *   "pcg_z"     Z = D^-1 (R - S), r^T z             (R, S read, Z written, D^-1 read)
 *   "pcg_split" D^-1 R -> BF16 pieces, transposed   (block read, pieces written)
 * Timing adds one event pair per GEMM launch; it is meant for measurement
 * runs.  Not thread-safe across concurrent callers.
 *
 * Phase ranges (NVTX 3, always on, a few nanoseconds each without a tool):
 *   "fsa_build", "fsa_loglik_grad", "fsa_predict", "fsa_matvec", "fsa_kmeanspp"
 *                       one per C-ABI call
 *   "operator_build"    the theta-dependent build (Sigma_m, A, residual values,
 *                       D_s, Woodbury core), when theta or precision changed
 *   "probes", "pcg", "slq_gradient"
 *                       the phases of a mixed-precision log-likelihood
 *   "loglik_grad_fp64"  the whole FP64-form solve
 *   "serve_loglik_grad", "serve_predict"
 *                       one request of the serving loop
 * `ncu --nvtx --nvtx-include "pcg/"` captures only the CG loop's kernels.
 * A toolkit without the NVTX 3 headers builds the library without ranges.
 */
#ifndef FSA_PROFILE_H_
#define FSA_PROFILE_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Total number of CUDA kernels launched by this library since load. */
uint64_t fsa_launch_count(void);

/* 1: start recording GEMM launch timings; 0: stop (recorded data kept). */
void fsa_profile_enable(int on);

/* Drop recorded timings (and release their events). */
void fsa_profile_reset(void);

/* Synchronise on the recorded events and sum the data of one tag:
 * launches, total device milliseconds and total algorithmic bytes.
 * Returns 0, or a negative value if the tag is unknown or nothing recorded. */
int fsa_profile_collect(const char* tag, int64_t* launches, double* ms, double* bytes);

/* High-water mark, in bytes, of the device memory the library's calls held at
 * once on the current device since the last reset (every library allocation
 * comes from the device's stream-ordered memory pool); reset != 0 restarts it
 * at the current use.  Returns -1 if the pool cannot be queried. */
int64_t fsa_pool_used_high(int reset);

#ifdef __cplusplus
}
#endif

#endif
