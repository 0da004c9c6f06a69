// The mixed-precision form's building blocks shared by its log-likelihood,
// Fisher-information and operator entry points (definitions in fsa_mixed.cu).
#pragma once
#include "fsa_solver.cuh"
#include "fsa_tc.cuh"

namespace fsa {

// tensor-core operand maps of one CG block width (ldc columns)
struct MixedCtx {
  int ldc = 0, c = 0, m_pad = 0;
  int64_t n = 0, n_pad = 0;
  int splits_w = 1;
  TmaMap mAt, mA, mX, mQ;
  TmaMap mAt_lo, mA_lo;     // low halves of A (FSA_MIXED_BF16X2)
  bool lo = false;
  int nsplit = 2;           // BF16 pieces of the vector operands (3: FP32-exact)
  float* wpart = nullptr;   // split-K partials of A^T X (splits_w x m_pad x ldc)
};

// CG block width for c columns with `pieces` BF16 pieces of the vector operands
int mixed_ldc(int c, int pieces);
void mixed_ctx_setup(Handle& H, MixedCtx& C, int64_t n, int c, int ldc);
// w (FP64, m x ldc) = A~^T X, X = rows of src (scaled by rowscale when not NULL)
void mixed_AtX(Handle& H, MixedCtx& C, const float* src, const float* rowscale, double* w, const char* tag);
// S (FP32, n x ldc) = A~ q, q FP64 m x ldc
void mixed_Aq(Handle& H, MixedCtx& C, const double* q, float* S, const char* tag);
// block PCG (Appendix A) on the right-hand sides in H.cg.R32
void pcg_mixed_run(Handle& H, MixedCtx& C, const CGLayout& lay, const fsa_opts& o, int L);

// Operands of the range derivative of the mixed operator (§2.2):
// b = dK L^-T and q = b - A~ E as BF16 hi + lo pairs (blocked K-major layout),
// B^T as a pair, E = L^-1 dSigma_m L^-T (FP64), the derivative of the
// residual values per nonzero and its diagonal dD_s/drho.
struct DerivMixed {
  DevPtr<__nv_bfloat16> Bh, Bl, Qh, Ql, Bth, Btl, zero_lo;
  const __nv_bfloat16* Alo = nullptr;   // A~'s low half (zeros in the single-BF16 form)
  DevPtr<double> E;
  DevPtr<float> dv, dD;
  MixedCtx CBt;   // C with B^T in place of A~^T: B^T X
  MixedCtx CB;    // C with B in place of A~: B q
};
void build_deriv_mixed(Handle& H, const MixedCtx& C, const fsa_theta& th, DerivMixed& Dv);
// out0 = dSigma_dag/dsigma1^2 X = (Sigma_dag X - nugget X) / sigma1^2 and
// out1 = dSigma_dag/drho X = dSigma_s~/drho X + B (A~^T X) + A~ (B^T X - E A~^T X)
// for X (n x C.ldc FP32, zero beyond its columns)
void apply_dsigma_mixed(Handle& H, MixedCtx& C, DerivMixed& Dv, const fsa_theta& th, const float* X, float* out0,
                        float* out1);

}  // namespace fsa
