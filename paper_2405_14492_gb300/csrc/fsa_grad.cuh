// Gradient by columns and the control variate of its trace term
// (definitions in fsa_grad.cu).
#pragma once
#include "fsa_internal.cuh"

namespace fsa {

constexpr int kColTerms = 5;   // per-column sparse terms of k_grad_coldots
constexpr int kCvTerms = 5;    // weighted row sums of the control variate
// slots of Handle::outs written by the gradient (after the log-likelihood's 0..7)
constexpr int kOutGrad = 3, kOutTrace = 8, kOutQuad = 11, kOutTraceP = 14, kOutCvC = 17, kOutCount = 20;

enum GradCv : int { kCvNone = 0, kCvOptPrinted = 1, kCvOne = 2, kCvOptCentred = 3 };

int coldots_blocks();
int cv_blocks();
template <typename T, typename VT, typename DT>
void grad_coldots(Handle& H, int c, int ldc, const VT* vals, const DT* dvals, const T* X, const T* Y, double* part,
                  int nblk);
void grad_lowrank_cols(Handle& H, int m, int c, int ldc, const double* AX, const double* AY, const double* BX,
                       const double* BY, const double* EAY, double* lr);
// tile form (staged per cell-grid tile; false when unavailable, cap_rows_max
// as for csr_values_tiles) and row form of the range derivative of the mixed
// residual values; dvals_mixed takes the tile form where it can
bool dvals_tiles(Handle& H, const fsa_theta& th, int m_pad, const __nv_bfloat16* A, const __nv_bfloat16* Alo,
                 const __nv_bfloat16* B, const __nv_bfloat16* Blo, const __nv_bfloat16* Q, const __nv_bfloat16* Qlo,
                 float* dvals, float* dD, int cap_rows_max);
void dvals_rows(Handle& H, const fsa_theta& th, int m_pad, const __nv_bfloat16* A, const __nv_bfloat16* Alo,
                const __nv_bfloat16* B, const __nv_bfloat16* Blo, const __nv_bfloat16* Q, const __nv_bfloat16* Qlo,
                float* dvals, float* dD);
void dvals_mixed(Handle& H, const fsa_theta& th, int m_pad, const __nv_bfloat16* A, const __nv_bfloat16* Alo,
                 const __nv_bfloat16* B, const __nv_bfloat16* Blo, const __nv_bfloat16* Q, const __nv_bfloat16* Qlo,
                 float* dvals, float* dD);
void dvals_f64(Handle& H, const fsa_theta& th, int m, const double* A, const double* B, const double* F,
               double* dvals, double* dD);

// Operands of the range derivative of the FP64 operator (§2.2): B = dK L^-T
// and F = A E (n x m row-major), E = L^-1 dSigma_m L^-T, the derivative of
// the residual values per nonzero and its diagonal dD_s/drho.
struct DerivF64 {
  DevPtr<double> B, F, E, dv, dD;
};
void build_deriv_f64(Handle& H, const fsa_theta& th, DerivF64& Dv);
// out0 = (Sigma_dag X - nugget X) / sigma1^2, out1 = dSigma_dag/drho X (X n x ldx)
void apply_dsigma_f64(Handle& H, DerivF64& Dv, const fsa_theta& th, const double* X, int k, int ldx, double* out0,
                      double* out1);
void cv_rowdots_mixed(Handle& H, int m_pad, const float* AM, const __nv_bfloat16* A, const __nv_bfloat16* Alo,
                      const __nv_bfloat16* B, const __nv_bfloat16* Blo, const float* D32, const float* dD, double* cv,
                      int nblk);
void cv_rowdots_f64(Handle& H, int m, const double* AM, const double* A, const double* B, const double* D,
                    const double* dD, double* cv, int nblk);
void mspace_traces(Handle& H, int m, const double* E, const double* Minv, double* mtr);
// the gradient, its trace and quadratic parts, the control variate's traces
// and coefficients into H.outs, the per-probe terms into terms (6 l doubles:
// a[3][l] then b[3][l]); cv and mtr are ignored when cv_kind == kCvNone
void grad_final(Handle& H, int c, int ldc, const double* part, int nblk, const double* lr, const double* cv, int ncv,
                const double* mtr, const fsa_theta& th, int cv_kind, double* terms);

}  // namespace fsa
