/*
 * fsa.h — C ABI of the GB300 (sm_103a) implementation of the iterative
 * full-scale approximation (FSA) of Gaussian processes of
 * Gyger, Furrer & Sigrist, "Iterative Methods for Full-Scale Gaussian Process
 * Approximations for Large Spatial Data" (arXiv 2405.14492).
 *
 * Model (paper §2, Eq. NEGLL): y = b + eps, b ~ N(0, Sigma), eps ~ N(0, nugget I),
 * Sigma_ij = sigma1^2 r(|s_i - s_j|; rho) with r the Matérn correlation
 * (nu = 1/2: exp(-d/rho); nu = 3/2: (1 + sqrt(3) d/rho) exp(-sqrt(3) d/rho)).
 * The FSA (§2.1) replaces Sigma + nugget I by
 *     Sigma_dag = Sigma_l + (Sigma - Sigma_l) o T(gamma) + nugget I,
 *     Sigma_l   = Sigma_mn^T Sigma_m^-1 Sigma_mn   (m inducing points),
 *     T(gamma)  = Wendland phi_{3,1} taper, zero for distance >= gamma.
 *
 * Conventions for every call:
 *   - Return value: a status code; nothing throws across the ABI.  The text of
 *     the last error of the calling thread is given by fsa_last_error().
 *   - Ownership: the caller owns every input and output buffer.  Unless a
 *     call says otherwise, buffers are HOST memory; the library copies inputs
 *     into device memory it owns and copies results back before returning.
 *   - Handles are opaque, own all their device memory and are released by
 *     fsa_free().  One handle must not be used from two threads at once.
 *   - Points are row-major (x, y) pairs of double.  Indices in outputs refer
 *     to the caller's original point order.
 *   - Outputs are the log-likelihood l = -L (the paper's L is the NEGATIVE
 *     log-likelihood) and its gradient with respect to the raw parameters
 *     theta = (sigma1^2, rho, nugget).
 *   - The response is taken as centred (y - X beta): no fixed effects.
 */
#ifndef FSA_H_
#define FSA_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FSA_OK = 0,
  FSA_ERR_ARG = 1,             /* invalid argument (size, pointer, parameter) */
  FSA_ERR_OOM = 2,             /* device (or host) memory could not be allocated / admitted */
  FSA_ERR_NOT_PD = 3,          /* a Cholesky pivot <= 0 (Sigma_m or the Woodbury core) */
  FSA_ERR_NO_CONVERGENCE = 4,  /* CG hit its iteration limit; outputs still written */
  FSA_ERR_NAN = 5,             /* a non-finite input or intermediate */
  FSA_ERR_TIMEOUT = 6,         /* a bounded device or host wait ran out */
  FSA_ERR_BUSY = 7,            /* serving: result not ready yet */
  FSA_ERR_CUDA = 8,            /* a CUDA runtime error, or another system error (a thread that could not start) */
  FSA_ERR_UNSUPPORTED = 9,     /* option not available on this device / build */
  FSA_ERR_BOUNDS = 10          /* checked build (FSA_CHECKED) only: a device index check failed, the
                                  access it guarded was skipped; a defect of this library, outputs invalid */
} fsa_status;

typedef enum {
  FSA_EXPONENTIAL = 0,   /* Matérn nu = 1/2 */
  FSA_MATERN_1_5 = 1     /* Matérn nu = 3/2 */
} fsa_cov;

typedef enum {
  FSA_FP64 = 0,          /* every step in FP64 on the CUDA cores */
  FSA_MIXED_BF16 = 1,    /* n x m products on tcgen05 tensor cores: A = Sigma_nm L_m^-T
                            stored once in BF16 (the operator is defined by it, consistently
                            in the operator, preconditioner, probes and log det P);
                            vector operands split hi+lo BF16, FP32 accumulation; vectors
                            FP32; m x m Cholesky / Woodbury core, CG scalars and Lanczos
                            eigen-quadrature in FP64 */
  FSA_MIXED_BF16X2 = 2   /* as FSA_MIXED_BF16, but A is stored as a hi + lo pair of BF16
                            matrices (A = A_hi + A_lo, ~2^-17 relative) and every tensor-core
                            product uses both halves; twice the A traffic, FP32-level operator
                            accuracy (the form that meets 1e-4 relative log-likelihood error
                            at n = 1e6) */
} fsa_precision;

typedef enum {
  FSA_PROBE_RADEMACHER = 0,
  FSA_PROBE_GAUSSIAN = 1
} fsa_probe;

typedef struct {
  double sigma1_sq;      /* marginal variance sigma1^2 > 0 */
  double rho;            /* range rho > 0 */
  double nugget;         /* nugget sigma^2 > 0 */
} fsa_theta;

typedef struct {
  int32_t num_probes;    /* l >= 1 stochastic probes for SLQ / STE (§3.1) */
  double cg_tol;         /* stop a column when ||r||_2 < cg_tol (Appendix A, absolute) */
  int32_t cg_max_iter;   /* iteration limit L (default 1000 when <= 0) */
  int32_t fixed_iters;   /* > 0: run exactly this many CG iterations in every column */
  int32_t precision;     /* fsa_precision */
  int32_t probe;         /* fsa_probe */
  uint64_t seed;         /* probe seed (counter-based SplitMix64, streams 4 and 5) */
  int32_t slq_exact_weight; /* 1: weight z^T P^-1 z instead of the paper's n */
  int32_t want_grad;     /* 0: log-likelihood only */
  int32_t y_on_device;   /* 1: y is a DEVICE pointer (n doubles, caller order) */
  int32_t pred_control_variate; /* fsa_predict: 0 plain D_l of Algorithm 1; 1 D_l with the
                                   diagonal preconditioner D_s as control variate and the
                                   per-point coefficient c_opt; 2 the same with c = 1
                                   (appendix "Preconditioner as control variate") */
  int32_t grad_control_variate; /* fsa_loglik_grad: the FITC preconditioner as control variate
                                   of the gradient's trace estimate (appendix "Preconditioner as
                                   control variate", Eq. Troptc), per parameter
                                     Tr(Sdag^-1 dSdag) ~ (1/l) sum_k (a_k - c b_k) + c Tr(P^-1 dP),
                                   a_k = U_k^T dSdag W_k, b_k = W_k^T dP W_k, W = P^-1 Z:
                                   0 none (the plain STE of §3.3); 1 c = c_opt as printed,
                                   sum_k (a_k - mean a) b_k / sum_k b_k^2; 2 c = 1; 3 the centred
                                   (variance-minimising) slope
                                   sum_k (a_k - mean a)(b_k - mean b) / sum_k (b_k - mean b)^2.
                                   Costs one n x m x m tensor-core product and row dots. */
  int32_t pred_exact_var;       /* fsa_predict, FP64 form: 1 computes D_l = diag(S Sigma_s~^-1 S^T)
                                   exactly, by n_p sparse solves (one per prediction point), in
                                   place of Algorithm 1's simulation: the exact FSA predictive
                                   variances (§2.3), a reference for the simulated ones; cost and
                                   memory grow with n_p (n x n_p right-hand sides). */
  int32_t vec_pieces;           /* mixed forms: BF16 pieces of the vector operands of the
                                   tensor-core products (D^-1 r and q in the CG iteration):
                                   0 or 2: two (about 16 significant bits); 3: three (FP32's 24;
                                   needs 3 x (columns rounded to 16) <= 256, else two are used).
                                   Three cost one more piece of the blocks (not of A~) and
                                   help problems with a long range and a small nugget. */
} fsa_opts;

typedef struct {
  int32_t iters_max;     /* largest CG iteration count over the columns */
  int32_t iters_y;       /* CG iterations of the response column */
  double resid_y;        /* final ||r||_2 of the response column */
  double logdet;         /* SLQ estimate of log det Sigma_dag */
  double logdet_precond; /* log det P_hat (Sylvester, exact) */
  double quad_form;      /* y^T Sigma_dag^-1 y */
  double logdet_se;      /* standard error of the SLQ estimate (sample sd / sqrt(l)) */
  int32_t converged;     /* 1 if every column met cg_tol (or fixed_iters ran) */
  int32_t num_probes;
  int64_t nnz;           /* nonzeros of the tapered residual (diagonal included) */
  double time_ms;        /* device time of the call */
  /* fsa_loglik_grad with want_grad, per parameter (sigma1^2, rho, nugget):
   * the gradient is -1/2 (grad_trace - grad_quad) */
  double grad_trace[3];  /* estimate of Tr(Sigma_dag^-1 dSigma_dag/dtheta) (STE, §3.3; with the
                            control variate when opts.grad_control_variate != 0) */
  double grad_quad[3];   /* u^T dSigma_dag/dtheta u, u = Sigma_dag^-1 y (the CG solution) */
  double trace_precond[3]; /* Tr(P_hat^-1 dP_hat/dtheta), exact (0 without the control variate) */
  double cv_coef[3];     /* the control variate's coefficient c (0 without it) */
  /* mixed forms: 2^-24 |M - I|_inf of the Woodbury core M = I + A~^T D^-1 A~
   * summed on the tensor cores, and whether M was therefore formed in FP64
   * (core_fp64 = 1 when that figure exceeds 1e-3: long ranges with small
   * nuggets, where FP32 sums would lose M's identity part) */
  double core_scale;
  int32_t core_fp64;
  /* mixed forms: 2^-16 sigma1 |L_m^-1|_inf, the relative rounding of A~ =
   * Sigma_nm L_m^-T formed from BF16 pairs on the tensor cores, and whether A~
   * was therefore formed in FP64 before its rounding to the pair (a_fp64 = 1
   * above 1e-4: a badly conditioned Sigma_m, i.e. a long range against the
   * spacing of the inducing points) */
  double a_scale;
  int32_t a_fp64;
} fsa_info;

typedef struct fsa_handle fsa_handle;

/* Defaults: num_probes 50, cg_tol 1e-3, cg_max_iter 1000, fixed_iters 0,
 * FSA_FP64, Rademacher, seed 14492, want_grad 1, pred_control_variate 0. */
void fsa_default_opts(fsa_opts* opts);

/* Human-readable name of a status code (static string). */
const char* fsa_status_string(fsa_status s);

/* Message of the last failed call on this thread (static per thread). */
const char* fsa_last_error(void);

/*
 * fsa_build — theta-free set-up (paper §2.1: taper support; §3.1: sparse +
 * low-rank operator).  Copies the n locations and m inducing points to the
 * device, sorts the points by a cell grid of side >= gamma (internal order),
 * and builds the CSR pattern of {(i,j): |s_i - s_j|^2 < gamma^2} (diagonal
 * included; squared distance without fused multiply-add).
 *   locs      n x 2 row-major host array, n >= 2
 *   inducing  m x 2 row-major host array of distinct points, 1 <= m <= n
 *   taper_range gamma > 0
 *   cov       fsa_cov
 *   cuda_stream a cudaStream_t to run on (NULL: the legacy default stream)
 *   out       receives the handle
 * Errors: FSA_ERR_ARG, FSA_ERR_NAN (non-finite coordinates), FSA_ERR_OOM, FSA_ERR_CUDA.
 */
fsa_status fsa_build(const double* locs, int64_t n, const double* inducing, int32_t m,
                     double taper_range, int32_t cov, void* cuda_stream, fsa_handle** out);

/* Number of nonzeros of the taper pattern (diagonal included). */
int64_t fsa_nnz(const fsa_handle* h);

/*
 * fsa_get_csr — the taper pattern in the caller's point order, columns
 * ascending: rowptr (n+1, int64) and col (nnz, int32) host arrays, both
 * caller-owned and sized by the caller (nnz from fsa_nnz).  Synchronises the
 * handle's stream.
 * Errors: FSA_ERR_ARG (NULL argument), FSA_ERR_OOM, FSA_ERR_CUDA.
 */
fsa_status fsa_get_csr(fsa_handle* h, int64_t* rowptr, int32_t* col);

/*
 * fsa_loglik_grad — log-likelihood and gradient (paper Eq. NEGLLDNEGLLFSA)
 * by block preconditioned CG with the FITC preconditioner (Eq. eqfitcp),
 * stochastic Lanczos quadrature for log det (§3.1, §3.3) and stochastic trace
 * estimation for the gradient (§3.1, §3.3); CG with Lanczos tridiagonals per
 * Appendix A.
 *   y       n values in the caller's point order (host, or device if
 *           opts->y_on_device)
 *   theta   covariance parameters
 *   opts    options (NULL: defaults)
 *   loglik  receives l(theta) = -[n/2 log 2pi + 1/2 log det + 1/2 y^T Sigma_dag^-1 y]
 *   grad    3 doubles, receives dl/d(sigma1^2, rho, nugget) (ignored when
 *           want_grad = 0; may be NULL then)
 *   info    optional diagnostics (may be NULL)
 * Errors: FSA_ERR_ARG, FSA_ERR_NOT_PD, FSA_ERR_NO_CONVERGENCE (outputs
 * written), FSA_ERR_NAN, FSA_ERR_OOM, FSA_ERR_UNSUPPORTED, FSA_ERR_CUDA.
 */
fsa_status fsa_loglik_grad(fsa_handle* h, const double* y, const fsa_theta* theta,
                           const fsa_opts* opts, double* loglik, double* grad,
                           fsa_info* info);

/*
 * fsa_grad_terms — the per-probe terms of the gradient's stochastic trace
 * estimate (§3.3) from the last fsa_loglik_grad on this handle that computed
 * the gradient: a[j][k] = U_k^T dSigma_dag/dtheta_j W_k and, with the control
 * variate, b[j][k] = W_k^T dP_hat/dtheta_j W_k (appendix "Preconditioner as
 * control variate"; zeros without it), j = (sigma1^2, rho, nugget),
 * k = 0 .. l-1 (U = Sigma_dag^-1 Z, W = P_hat^-1 Z).
 *   a, b        caller-owned HOST arrays of 3 * num_probes doubles, row-major [j][k]
 *   num_probes  the l of that call
 * Errors: FSA_ERR_ARG (NULL pointer, no gradient computed yet, or num_probes
 * different from that call's l), FSA_ERR_CUDA.
 */
fsa_status fsa_grad_terms(fsa_handle* h, double* a, double* b, int32_t num_probes);

/*
 * fsa_fisher — Fisher information of theta = (sigma1^2, rho, nugget) by
 * stochastic trace estimation (appendix "Fisher scoring"):
 *   I_kj = 1/2 Tr(Sigma_dag^-1 dSigma_k Sigma_dag^-1 dSigma_j)
 *        ~ 1/2 (1/l) sum_i (dSigma_k Sigma_dag^-1 z_i)^T (Sigma_dag^-1 dSigma_j z_i),
 * z_i Rademacher or Gaussian (opts->probe) from SplitMix64 stream 7, counter
 * i n + point index (caller order).  The 3 l solves (z_i, dSigma_sigma1^2 z_i,
 * dSigma_rho z_i) run as one block of the FITC-preconditioned CG (Appendix A)
 * with opts->cg_tol / fixed_iters; opts->precision selects the FP64 or the
 * mixed form (mixed: l <= 42).
 *   fisher      HOST double[9], row-major: the symmetric part of the estimate
 *   fisher_raw  HOST double[9] or NULL: the estimate as it stands (not
 *               symmetric for finite l)
 *   info        optional: iters_max, converged, num_probes, nnz, time_ms
 * Errors: FSA_ERR_ARG, FSA_ERR_UNSUPPORTED (too many probes for the mixed
 * form), FSA_ERR_NO_CONVERGENCE (outputs written), FSA_ERR_NAN, FSA_ERR_NOT_PD,
 * FSA_ERR_OOM, FSA_ERR_CUDA.  Synchronises the handle's stream.
 */
fsa_status fsa_fisher(fsa_handle* h, const fsa_theta* theta, const fsa_opts* opts, double* fisher,
                      double* fisher_raw, fsa_info* info);

/*
 * fsa_matvec — the FSA operator and its preconditioner on caller vectors
 * (paper §3.1: Sigma_dag v = Sigma_s~ v + Sigma_mn^T Sigma_m^-1 Sigma_mn v;
 * appendix "Runtime of the FITC preconditioner": P_hat^-1 v by Woodbury).
 *   which   0: Sigma_dag v, 1: P_hat^-1 v, 2: Sigma_s~ v (sparse part only)
 *   v, out  n x k row-major host arrays (k >= 1), caller's point order,
 *           caller-owned
 * Uses the operator built for theta with the given precision (built on first
 * use and cached in the handle for an unchanged theta and precision).
 * Synchronises the handle's stream.
 * Errors: FSA_ERR_ARG (NULL pointer, k < 1, which outside 0..2, bad theta or
 * precision), FSA_ERR_NOT_PD, FSA_ERR_NAN, FSA_ERR_OOM, FSA_ERR_CUDA.
 */
fsa_status fsa_matvec(fsa_handle* h, const fsa_theta* theta, int32_t precision, int32_t which,
                      const double* v, int32_t k, double* out);

/*
 * fsa_logdet_precond — log det P_hat by Sylvester's theorem (appendix
 * "Runtime of the FITC preconditioner") for theta at the given precision;
 * *out receives it.  Builds (or reuses) the operator like fsa_matvec.
 * Errors: FSA_ERR_ARG, FSA_ERR_NOT_PD, FSA_ERR_NAN, FSA_ERR_OOM, FSA_ERR_CUDA.
 */
fsa_status fsa_logdet_precond(fsa_handle* h, const fsa_theta* theta, int32_t precision,
                              double* out);

/*
 * fsa_predict — predictive mean (§2.3) and simulation-based predictive
 * variances (Algorithm 1, Proposition 1) at n_p new locations.
 *   pred_locs   n_p x 2 row-major host array
 *   num_var_samples s >= 1 probes for the stochastic diagonal D_l (probe kind
 *               and seed from opts; stream 6, counter = k * n_p + p)
 *   mean, var   n_p doubles each (host); var may be NULL (means only)
 * Linear solves: FITC-PCG for Sigma_dag^-1 y; D_s-preconditioned block CG
 * for Sigma_s~^-1 [Sigma_mn^T, S z_1..z_s]; Sigma_dag^-1 Sigma_mn^T by the exact
 * identity W2 M^-1 Sigma_m with M = Sigma_m + Sigma_mn W2 (Woodbury).
 * Computed in the FP64 form (opts->precision must be FSA_FP64).
 * Errors: FSA_ERR_ARG (NULL pointer, n_p < 1, num_var_samples outside
 * [1, 4096] when var is given, bad theta or options), FSA_ERR_UNSUPPORTED
 * (a mixed precision), FSA_ERR_NOT_PD, FSA_ERR_NO_CONVERGENCE (outputs
 * written), FSA_ERR_NAN (non-finite prediction locations), FSA_ERR_OOM,
 * FSA_ERR_CUDA.
 */
fsa_status fsa_predict(fsa_handle* h, const double* y, const fsa_theta* theta,
                       const fsa_opts* opts, const double* pred_locs, int64_t n_p,
                       int32_t num_var_samples, double* mean, double* var, fsa_info* info);

/* Release a handle and all its device memory. */
void fsa_free(fsa_handle* h);

/*
 * fsa_kmeanspp — kmeans++ selection of m inducing points among the n
 * locations (paper §4.1, which chooses its inducing points this way; seeding
 * of Arthur & Vassilvitskii 2007): the first point uniformly, each further
 * point with probability proportional to its squared distance to the nearest
 * point chosen so far.  The weights are the integers floor(d^2 2^e), d^2 =
 * dx*dx + dy*dy with every operation rounded on its own, e = 62 -
 * bitlength(n) - ex where the squared bounding-box diagonal is f 2^ex, f in
 * [0.5, 1) (so n weights sum below 2^62): sums are exact and the result is
 * reproducible bit for bit.  Draw k is h_k = (SplitMix64 output k of seed,
 * stream 9) >> 11: the first index is floor(h_0 n / 2^53), and step k picks
 * the first index whose inclusive prefix sum of the weights exceeds
 * floor(h_k Q / 2^53), Q their total.
 *   locs       n x 2 row-major HOST array, 1 <= n < 2^31
 *   m          1 <= m <= n
 *   seed       draw seed
 *   idx_out    receives the m chosen indices (caller order), caller-owned host array
 *   cuda_stream a cudaStream_t (NULL: the legacy default stream)
 * Returns FSA_OK; FSA_ERR_ARG for bad arguments or fewer than m distinct
 * locations; FSA_ERR_OOM / FSA_ERR_CUDA on device failures.  Allocates and
 * frees its device memory; synchronises the stream before returning.
 */
fsa_status fsa_kmeanspp(const double* locs, int64_t n, int32_t m, uint64_t seed, int64_t* idx_out,
                        void* cuda_stream);

/*
 * fsa_csr_noalloc — the taper-support pattern of fsa_build + fsa_get_csr
 * (same rows, same ascending columns, caller's point order), computed without
 * allocating any memory.  The paper has no counterpart: this entry point exists
 * for callers that cannot allocate device memory, e.g. a process whose device
 * memory is owned by its own pool or capped allocator, or code running where
 * cudaMalloc must not be called.  All temporaries live in one fixed-size
 * device array compiled into the library (about 6 MB, held on every GPU that
 * loads the library until the process exits); the call makes no cudaMalloc,
 * cudaFree or other allocating call.
 *   locs_dev      n x 2 row-major DEVICE array of locations
 *   n             1 <= n <= 65536 (the size of the fixed array); larger n is
 *                 rejected with FSA_ERR_ARG (use fsa_build instead)
 *   taper_range   gamma > 0
 *   rowptr_dev    DEVICE int64[n + 1]; all n + 1 entries are written by every
 *                 call that gets past the argument checks, including the size
 *                 query and the col_capacity error below, so a caller can keep
 *                 them and skip a second count
 *   col_dev       DEVICE int32[col_capacity], written; NULL: a size query that
 *                 sets *nnz_out and rowptr_dev and writes no columns
 *   col_capacity  capacity of col_dev; if it is below the pattern's nonzeros the
 *                 call returns FSA_ERR_ARG with *nnz_out and rowptr_dev set
 *   nnz_out       HOST int64, receives the number of nonzeros
 *   cuda_stream   stream to run on (NULL: legacy default stream); the call
 *                 synchronises this stream before returning
 * Errors: FSA_ERR_ARG, FSA_ERR_NAN (non-finite coordinates), FSA_ERR_CUDA.
 * The first call on a device looks up the device address of the fixed array
 * (cudaGetSymbolAddress, with that device current) and keeps it for the
 * device's current CUDA context; make that first call before any stream
 * capture.  After a device reset the next call looks the address up again.
 * Each row is sorted in O(deg log deg) steps, so a taper range near the
 * extent of the points (rows of up to n neighbours) stays bounded in time.  Every call shares the same array and its
 * contents persist between calls (the call clears what must start at zero), so
 * calls that overlap on the GPU (from two streams or threads at once) race.
 */
fsa_status fsa_csr_noalloc(const double* locs_dev, int64_t n, double taper_range, int64_t* rowptr_dev,
                           int32_t* col_dev, int64_t col_capacity, int64_t* nnz_out, void* cuda_stream);

/* Estimate of the device bytes one loglik+grad call on a problem of this size
 * holds (structure + operator + CG block), used for admission control. */
int64_t fsa_footprint_bytes(int64_t n, int32_t m, int64_t nnz, int32_t num_probes,
                            int32_t precision);

/* ------------------------------------------------------------------------
 * Serving: a persistent request loop on one GPU with continuous batching.
 * The paper evaluates one problem at a time; the server runs many
 * independent problems (different n, m, theta) at once.  Each request is
 * exactly one fsa_build followed by one fsa_loglik_grad or fsa_predict, and
 * its result is bit-for-bit the one those calls give alone.
 *
 * Scheduling: requests wait in arrival order.  A request is admitted when one
 * of the max_slots slots is idle and its device-memory footprint estimate
 * fits in what the running requests leave of the budget; a later request
 * that fits may go ahead of an earlier one that does not, at most 8 times
 * for the oldest waiting request.  A running request keeps its CSR pattern,
 * Sigma_m Cholesky, operator and CG block resident on the device; the slots
 * run on separate CUDA streams, so the work of all admitted requests overlaps
 * on the GPU.  A request whose estimate exceeds the whole budget is refused
 * at submission with FSA_ERR_OOM.
 * ------------------------------------------------------------------------ */
typedef enum {
  FSA_REQ_LOGLIK_GRAD = 0,   /* fsa_loglik_grad */
  FSA_REQ_PREDICT = 1        /* fsa_predict */
} fsa_request_kind;

typedef struct {
  int32_t device;            /* CUDA device ordinal */
  int32_t max_slots;         /* requests running at once, 1..64 (default 4) */
  int64_t hbm_budget_bytes;  /* admission limit on the summed footprint estimates of the
                                running requests; <= 0: 85 % of the device memory free at
                                creation (default) */
} fsa_server_cfg;

typedef struct {
  int32_t kind;              /* fsa_request_kind */
  const double* locs;        /* n x 2 row-major host array (copied at submission) */
  int64_t n;
  const double* inducing;    /* m x 2 row-major host array (copied) */
  int32_t m;
  double taper_range;
  int32_t cov;               /* fsa_cov */
  const double* y;           /* n host values (copied) */
  fsa_theta theta;
  fsa_opts opts;             /* y_on_device must be 0 */
  const double* pred_locs;   /* FSA_REQ_PREDICT: n_p x 2 host array (copied) */
  int64_t n_p;
  int32_t num_var_samples;
  double* mean;              /* FSA_REQ_PREDICT outputs: caller-owned host arrays of n_p
                                doubles, written before the result becomes ready; they must
                                stay valid until then (var may be NULL: means only) */
  double* var;
} fsa_request;

typedef struct {
  int32_t status;            /* fsa_status of the request's own build and solve */
  int32_t kind;
  double loglik;             /* FSA_REQ_LOGLIK_GRAD: as fsa_loglik_grad */
  double grad[3];
  fsa_info info;
  double queue_ms;           /* submission -> admission */
  double run_ms;             /* admission -> completion (build, solve, release) */
  double latency_ms;         /* submission -> completion */
  int64_t footprint_bytes;   /* admission estimate */
  int32_t slot;
  char message[160];         /* error text of a failed request */
} fsa_result;

typedef struct {
  int64_t submitted, completed, failed, pending;
  int32_t running, peak_running;
  int64_t budget_bytes, in_use_bytes, peak_in_use_bytes;
  double p50_ms, p99_ms, mean_ms;   /* latency percentiles (nearest rank) of completed requests */
  double completed_per_s;           /* completed / (last completion - first submission) */
} fsa_server_stats;

typedef struct fsa_server fsa_server;

/* Defaults: device 0, 4 slots, budget 85 % of free device memory. */
void fsa_default_server_cfg(fsa_server_cfg* cfg);

/* Starts the slot threads and streams.  Errors: FSA_ERR_ARG, FSA_ERR_CUDA. */
fsa_status fsa_server_create(const fsa_server_cfg* cfg, fsa_server** out);

/* Queues a request; *ticket identifies it.  Inputs are copied before the call
 * returns.  Errors: FSA_ERR_ARG, FSA_ERR_OOM (estimate above the whole budget). */
fsa_status fsa_serve_submit(fsa_server* s, const fsa_request* req, uint64_t* ticket);

/* FSA_OK: *out holds the result (its own status in out->status) and the
 * ticket is released; FSA_ERR_BUSY: still waiting or running; FSA_ERR_ARG:
 * unknown or already retrieved ticket. */
fsa_status fsa_serve_poll(fsa_server* s, uint64_t ticket, fsa_result* out);

/* As fsa_serve_poll, but blocks up to timeout_s seconds (< 0: no limit);
 * FSA_ERR_TIMEOUT when the limit passes first. */
fsa_status fsa_serve_wait(fsa_server* s, uint64_t ticket, double timeout_s, fsa_result* out);

/* Counters and latency percentiles over the server's life so far. */
fsa_status fsa_server_get_stats(fsa_server* s, fsa_server_stats* out);

/* Blocks until every submitted request has completed, then stops the slots
 * and frees the server; results not retrieved are discarded. */
void fsa_server_destroy(fsa_server* s);

#ifdef __cplusplus
}
#endif

#endif /* FSA_H_ */
