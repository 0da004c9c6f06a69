// Dense FP64 linear algebra on the CUDA cores: a tiled GEMM with optional
// split-K (deterministic reduction), a blocked right-looking Cholesky and a
// blocked forward triangular solve.  Used for the m x m Cholesky of Sigma_m and
// of the Woodbury core (paper appendix "Runtime of the FITC preconditioner"),
// for the explicit L^-1 that turns the n x m triangular solve into a GEMM, and
// for every product of the plain FP64 form.
#include "fsa_internal.cuh"

namespace fsa {

// ---------------------------------------------------------------------------
// C = alpha * op(A) diag(scale) op(B) + beta * C      (FP64, row-major)
//   op(A)(i,k) = TA ? A[k*lda + i] : A[i*lda + k]
//   op(B)(k,j) = TB ? B[j*ldb + k] : B[k*ldb + j]
// ---------------------------------------------------------------------------
constexpr int GBM = 64, GBN = 64, GBK = 16;

template <int TA, int TB>
__global__ void __launch_bounds__(256) k_dgemm(int M, int N, int K, const double* __restrict__ A, int64_t lda,
                                                    const double* __restrict__ B, int64_t ldb,
                                                    const double* __restrict__ scale, double* __restrict__ C,
                                                    int64_t ldc, double alpha, double beta, int kchunk,
                                                    double* __restrict__ partial, int tri) {
  __shared__ double As[GBK][GBM + 1];
  __shared__ double Bs[GBK][GBN + 1];
  int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  int i0 = blockIdx.x * GBM, j0 = blockIdx.y * GBN;
  int kbeg = blockIdx.z * kchunk;
  int kend = min(K, kbeg + kchunk);
  // the K range where neither operand tile is known to be zero (an empty range
  // leaves acc = 0, which the epilogue writes as usual)
  if (tri & kTriA_KgeI) kbeg = max(kbeg, i0);
  if (tri & kTriA_KleI) kend = min(kend, i0 + GBM);
  if (tri & kTriB_KgeJ) kbeg = max(kbeg, j0);
  if (tri & kTriB_KleJ) kend = min(kend, j0 + GBN);
  if ((tri & kTriSymLower) && j0 >= i0 + GBM) kend = kbeg;   // above the diagonal: mirrored afterwards
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int k0 = kbeg; k0 < kend; k0 += GBK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int t = threadIdx.x + 256 * r;
      int ii, kk;
      if (TA == 0) { ii = t / GBK; kk = t % GBK; } else { kk = t / GBM; ii = t % GBM; }
      int gi = i0 + ii, gk = k0 + kk;
      double v = 0.0;
      if (gi < M && gk < kend) {
        v = TA == 0 ? A[(int64_t)gi * lda + gk] : A[(int64_t)gk * lda + gi];
        if (scale) v *= scale[gk];
      }
      As[kk][ii] = v;
      int jj;
      if (TB == 0) { kk = t / GBN; jj = t % GBN; } else { jj = t / GBK; kk = t % GBK; }
      int gj = j0 + jj;
      gk = k0 + kk;
      double w = 0.0;
      if (gj < N && gk < kend) w = TB == 0 ? B[(int64_t)gk * ldb + gj] : B[(int64_t)gj * ldb + gk];
      Bs[kk][jj] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GBK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { a[q] = As[kk][ty + 16 * q]; b[q] = Bs[kk][tx + 16 * q]; }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    int gi = i0 + ty + 16 * p;
    if (gi >= M) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int gj = j0 + tx + 16 * q;
      if (gj >= N) continue;
      if (partial) {
        partial[((int64_t)blockIdx.z * M + gi) * N + gj] = acc[p][q];
      } else {
        double* c = &C[(int64_t)gi * ldc + gj];
        *c = alpha * acc[p][q] + (beta == 0.0 ? 0.0 : beta * *c);
      }
    }
  }
}

__global__ void splitk_reduce_kernel(int M, int N, int splits, const double* __restrict__ partial,
                                     double* __restrict__ C, int64_t ldc, double alpha, double beta) {
  int64_t total = (int64_t)M * N;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int z = 0; z < splits; ++z) s += partial[(int64_t)z * total + t];
    int64_t i = t / N, j = t % N;
    double* c = &C[i * ldc + j];
    *c = alpha * s + (beta == 0.0 ? 0.0 : beta * *c);
  }
}

// C[i][j] = C[j][i] for j > i (the strictly upper part from the lower)
__global__ void k_mirror_lower(double* __restrict__ C, int64_t ldc, int M) {
  const int64_t total = (int64_t)M * M;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / M), j = (int)(t % M);
    if (j > i) C[(int64_t)i * ldc + j] = C[(int64_t)j * ldc + i];
  }
}

void dgemm(Workspace& ws, cudaStream_t s, bool ta, bool tb, int M, int N, int K, double alpha,
           const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
           int64_t ldc, const double* scale, int tri) {
  if (M <= 0 || N <= 0) return;
  FSA_REQUIRE(!(tri & kTriSymLower) || M == N, FSA_ERR_ARG, "symmetric dgemm result must be square");
  if (K <= 0) {
    // C = beta * C
    dgemm(ws, s, false, false, M, N, 1, 0.0, C, ldc, C, ldc, beta, C, ldc, nullptr);
    return;
  }
  dim3 grid((M + GBM - 1) / GBM, (N + GBN - 1) / GBN, 1);
  int tiles = grid.x * grid.y;
  int splits = 1;
  // split the K loop when the tile grid is far smaller than the machine
  if (tiles < 152 && K > 4 * GBK * 8) {
    splits = (2 * 152 + tiles - 1) / tiles;
    int maxs = (K + 8 * GBK - 1) / (8 * GBK);
    if (splits > maxs) splits = maxs;
    if (splits > 256) splits = 256;
  }
  int kchunk = ((K + splits - 1) / splits + GBK - 1) / GBK * GBK;
  splits = (K + kchunk - 1) / kchunk;
  grid.z = splits;
  double* part = nullptr;
  if (splits > 1) part = ws.scratch_f64((size_t)splits * M * N);
#define LAUNCH_DG(a, b)                                                                               \
  k_dgemm<a, b><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, scale, C, ldc, alpha, beta, kchunk, \
                                          part, tri)
  if (!ta && !tb) LAUNCH_DG(0, 0);
  else if (!ta && tb) LAUNCH_DG(0, 1);
  else if (ta && !tb) LAUNCH_DG(1, 0);
  else LAUNCH_DG(1, 1);
#undef LAUNCH_DG
  FSA_CHECK_LAUNCH();
  if (splits > 1) {
    splitk_reduce_kernel<<<grid_for((int64_t)M * N, 256), 256, 0, s>>>(M, N, splits, part, C, ldc, alpha, beta);
    FSA_CHECK_LAUNCH();
  }
  if (tri & kTriSymLower) {
    k_mirror_lower<<<grid_for((int64_t)M * M, 256), 256, 0, s>>>(C, ldc, M);
    FSA_CHECK_LAUNCH();
  }
}

// ---------------------------------------------------------------------------
// C (M x N, ld ldc) = A (M x K, ld lda) B (K x N, ld ldb), N <= 128 a multiple
// of 8, FP64: the tall-times-narrow product of the preconditioner apply
// (q = M_P^-1 w, N = the CG block width).  A block owns 32 rows and every
// column (thread: one row, columns tx, tx + 8, ...), so no column tile is
// padded; the K loop is split so that the grid fills the GPU several times
// over, and the split partials are summed in a fixed order.
// ---------------------------------------------------------------------------
template <int NJ>
__global__ void __launch_bounds__(256) k_dgemm_tall(int M, int K, const double* __restrict__ A, int64_t lda,
                                                    const double* __restrict__ B, int64_t ldb, int kchunk,
                                                    double* __restrict__ out, int64_t ldo, int64_t zstride) {
  constexpr int N = 8 * NJ;
  __shared__ double As[32][33];
  __shared__ double Bs[32][N];
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
  const int i0 = blockIdx.x * 32;
  const int kbeg = blockIdx.y * kchunk, kend = min(K, kbeg + kchunk);
  double acc[NJ];
#pragma unroll
  for (int j = 0; j < NJ; ++j) acc[j] = 0.0;
  for (int k0 = kbeg; k0 < kend; k0 += 32) {
    for (int t = threadIdx.x; t < 32 * 32; t += 256) {
      const int r = t >> 5, kk = t & 31;
      const int gi = i0 + r, gk = k0 + kk;
      As[r][kk] = (gi < M && gk < kend) ? A[(int64_t)gi * lda + gk] : 0.0;
    }
    for (int t = threadIdx.x; t < 32 * N; t += 256) {
      const int kk = t / N, j = t - kk * N;
      const int gk = k0 + kk;
      Bs[kk][j] = gk < kend ? B[(int64_t)gk * ldb + j] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      const double a = As[ty][kk];
#pragma unroll
      for (int j = 0; j < NJ; ++j) acc[j] = fma(a, Bs[kk][tx + 8 * j], acc[j]);
    }
    __syncthreads();
  }
  const int gi = i0 + ty;
  if (gi < M) {
    double* o = out + (int64_t)blockIdx.y * zstride + (int64_t)gi * ldo;
#pragma unroll
    for (int j = 0; j < NJ; ++j) o[tx + 8 * j] = acc[j];
  }
}

void dgemm_tall(Workspace& ws, cudaStream_t s, int M, int N, int K, const double* A, int64_t lda, const double* B,
                int64_t ldb, double* C, int64_t ldc) {
  if (M <= 0 || N <= 0) return;
  if (N % 8 != 0 || N > 128 || K <= 0) {
    dgemm(ws, s, false, false, M, N, K, 1.0, A, lda, B, ldb, 0.0, C, ldc, nullptr);
    return;
  }
  const int rt = (M + 31) / 32;
  int splits = std::max(1, std::min((4 * 152 + rt - 1) / rt, (K + 31) / 32));
  const int kchunk = ((K + splits - 1) / splits + 31) / 32 * 32;
  splits = (K + kchunk - 1) / kchunk;
  double* out = C;
  int64_t ldo = ldc, zs = 0;
  if (splits > 1) {
    out = ws.scratch_f64((size_t)splits * M * N);
    ldo = N;
    zs = (int64_t)M * N;
  }
  dim3 grid((unsigned)rt, (unsigned)splits);
  switch (N / 8) {
#define DT_CASE(J) case J: k_dgemm_tall<J><<<grid, 256, 0, s>>>(M, K, A, lda, B, ldb, kchunk, out, ldo, zs); break;
    DT_CASE(1) DT_CASE(2) DT_CASE(3) DT_CASE(4) DT_CASE(5) DT_CASE(6) DT_CASE(7) DT_CASE(8)
    DT_CASE(9) DT_CASE(10) DT_CASE(11) DT_CASE(12) DT_CASE(13) DT_CASE(14) DT_CASE(15) DT_CASE(16)
#undef DT_CASE
  }
  FSA_CHECK_LAUNCH();
  if (splits > 1) {
    splitk_reduce_kernel<<<grid_for((int64_t)M * N, 256), 256, 0, s>>>(M, N, splits, out, C, ldc, 1.0, 0.0);
    FSA_CHECK_LAUNCH();
  }
}

// ---------------------------------------------------------------------------
// Cholesky, lower, in place (row-major, ld = lda), blocked right-looking.
// A pivot <= 0 (or NaN) sets kErrNotPD; the factor then continues with a
// unit pivot so that the kernels stay finite.
// ---------------------------------------------------------------------------
constexpr int CNB = 32;

// the diagonal block, by one warp: lane r holds row r of the block in
// registers (every index is a compile-time constant, so nothing goes to local
// memory); the pivot and the column below it move between lanes by shuffles.
// Rows and columns past nb are the identity and leave the factor unchanged.
__global__ void __launch_bounds__(32) potrf_diag_kernel(double* __restrict__ A, int64_t lda, int kb, int nb,
                                                        unsigned* __restrict__ err) {
  const int r = threadIdx.x;
  double a[CNB];
#pragma unroll
  for (int c = 0; c < CNB; ++c)
    a[c] = (r < nb && c < nb) ? A[(int64_t)(kb + r) * lda + kb + c] : (r == c ? 1.0 : 0.0);
#pragma unroll
  for (int j = 0; j < CNB; ++j) {
    double p = __shfl_sync(0xffffffffu, a[j], j);
    if (!(p > 0.0)) {
      if (r == 0) atomicOr(err, kErrNotPD);
      p = 1.0;
    }
    const double d = sqrt(p);
    if (r == j) a[j] = d;
    else if (r > j) a[j] = a[j] / d;
#pragma unroll
    for (int c = j + 1; c < CNB; ++c) {
      const double lcj = __shfl_sync(0xffffffffu, a[j], c);
      if (r >= c) a[c] -= a[j] * lcj;
    }
  }
  if (r < nb) {
#pragma unroll
    for (int c = 0; c < CNB; ++c)
      if (c < nb) A[(int64_t)(kb + r) * lda + kb + c] = (c <= r) ? a[c] : 0.0;
  }
}

// rows below the diagonal block: L[i, kb:kb+nb] = A[i, kb:kb+nb] L_kk^-T
__global__ void potrf_panel_kernel(double* __restrict__ A, int64_t lda, int m, int kb, int nb) {
  __shared__ double Lkk[CNB][CNB + 1];
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
    int r = t / nb, c = t % nb;
    Lkk[r][c] = A[(int64_t)(kb + r) * lda + kb + c];
  }
  __syncthreads();
  int i = kb + nb + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  // the row in registers: loops over the compile-time block size, guarded by nb
  double x[CNB];
  double* row = A + (int64_t)i * lda + kb;
#pragma unroll
  for (int j = 0; j < CNB; ++j) x[j] = j < nb ? row[j] : 0.0;
#pragma unroll
  for (int j = 0; j < CNB; ++j) {
    if (j < nb) {
      double v = x[j];
#pragma unroll
      for (int t = 0; t < j; ++t) v -= x[t] * Lkk[j][t];
      x[j] = v / Lkk[j][j];
    }
  }
#pragma unroll
  for (int j = 0; j < CNB; ++j)
    if (j < nb) row[j] = x[j];
}

// trailing update of the lower triangle: A[i][j] -= sum_t L[i][kb+t] L[j][kb+t]
__global__ void potrf_syrk_kernel(double* __restrict__ A, int64_t lda, int m, int kb, int nb) {
  __shared__ double Li[32][CNB + 1], Lj[32][CNB + 1];
  int j0 = kb + nb + blockIdx.x * 32, i0 = kb + nb + blockIdx.y * 32;
  if (j0 > i0 + 31) return;  // strictly above the diagonal
  for (int t = threadIdx.y * 32 + threadIdx.x; t < 32 * nb; t += 32 * 8) {
    int r = t / nb, c = t % nb;
    Li[r][c] = (i0 + r < m) ? A[(int64_t)(i0 + r) * lda + kb + c] : 0.0;
    Lj[r][c] = (j0 + r < m) ? A[(int64_t)(j0 + r) * lda + kb + c] : 0.0;
  }
  __syncthreads();
  for (int rr = threadIdx.y; rr < 32; rr += 8) {
    int i = i0 + rr, j = j0 + threadIdx.x;
    if (i >= m || j > i) continue;
    double s = 0.0;
    for (int t = 0; t < nb; ++t) s += Li[rr][t] * Lj[threadIdx.x][t];
    A[(int64_t)i * lda + j] -= s;
  }
}

__global__ void zero_upper_kernel(double* __restrict__ A, int64_t lda, int m) {
  int64_t total = (int64_t)m * m;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(t / m), j = (int)(t % m);
    if (j > i) A[(int64_t)i * lda + j] = 0.0;
  }
}

void cholesky(double* A, int64_t lda, int m, unsigned* err, cudaStream_t s) {
  for (int kb = 0; kb < m; kb += CNB) {
    int nb = min(CNB, m - kb);
    potrf_diag_kernel<<<1, 32, 0, s>>>(A, lda, kb, nb, err);
    FSA_CHECK_LAUNCH();
    int rest = m - kb - nb;
    if (rest > 0) {
      potrf_panel_kernel<<<(rest + 127) / 128, 128, 0, s>>>(A, lda, m, kb, nb);
      FSA_CHECK_LAUNCH();
      int tb = (rest + 31) / 32;
      potrf_syrk_kernel<<<dim3(tb, tb), dim3(32, 8), 0, s>>>(A, lda, m, kb, nb);
      FSA_CHECK_LAUNCH();
    }
  }
  zero_upper_kernel<<<grid_for((int64_t)m * m, 256), 256, 0, s>>>(A, lda, m);
  FSA_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// X = L^-1 B (L lower m x m), B is m x r row-major, in place.
// ---------------------------------------------------------------------------
__global__ void trsm_block_kernel(const double* __restrict__ L, int64_t ldl, int rb, int nb,
                                  double* __restrict__ B, int64_t ldb, int r) {
  __shared__ double Lbb[CNB][CNB + 1];
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
    int a = t / nb, c = t % nb;
    Lbb[a][c] = L[(int64_t)(rb + a) * ldl + rb + c];
  }
  __syncthreads();
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= r) return;
  // the column's block rows in registers (compile-time indices, guarded by nb)
  double x[CNB];
#pragma unroll
  for (int a = 0; a < CNB; ++a) x[a] = a < nb ? B[(int64_t)(rb + a) * ldb + j] : 0.0;
#pragma unroll
  for (int a = 0; a < CNB; ++a) {
    if (a < nb) {
      double v = x[a];
#pragma unroll
      for (int t = 0; t < a; ++t) v -= Lbb[a][t] * x[t];
      x[a] = v / Lbb[a][a];
    }
  }
#pragma unroll
  for (int a = 0; a < CNB; ++a)
    if (a < nb) B[(int64_t)(rb + a) * ldb + j] = x[a];
}

void trsm_lower(Workspace& ws, const double* L, int64_t ldl, int m, double* B, int64_t ldb, int r,
                cudaStream_t s) {
  for (int rb = 0; rb < m; rb += CNB) {
    int nb = min(CNB, m - rb);
    if (rb > 0)
      dgemm(ws, s, false, false, nb, r, rb, -1.0, L + (int64_t)rb * ldl, ldl, B, ldb, 1.0,
            B + (int64_t)rb * ldb, ldb, nullptr);
    trsm_block_kernel<<<(r + 127) / 128, 128, 0, s>>>(L, ldl, rb, nb, B, ldb, r);
    FSA_CHECK_LAUNCH();
  }
}

__global__ void set_identity_kernel(double* __restrict__ A, int64_t lda, int m) {
  int64_t total = (int64_t)m * m;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(t / m), j = (int)(t % m);
    A[(int64_t)i * lda + j] = (i == j) ? 1.0 : 0.0;
  }
}

// L^-1 by right-looking block substitution on X = I: block row kb is solved
// with L_kk (its nonzeros lie in the columns < kb + nb), then subtracted from
// every later block row, X[w:, :w] -= L[w:, kb:w] X[kb:w, :w] (w = kb + nb).
// Each update is a wide product of depth nb, so the GPU is filled from the
// first block on; the columns >= w of those rows are still zero and skipped.
void lower_inverse(Workspace& ws, const double* L, int m, double* Li, cudaStream_t s) {
  set_identity_kernel<<<grid_for((int64_t)m * m, 256), 256, 0, s>>>(Li, m, m);
  FSA_CHECK_LAUNCH();
  for (int kb = 0; kb < m; kb += CNB) {
    const int nb = min(CNB, m - kb), w = kb + nb;
    trsm_block_kernel<<<(w + 127) / 128, 128, 0, s>>>(L, m, kb, nb, Li, m, w);
    FSA_CHECK_LAUNCH();
    if (w < m)
      dgemm(ws, s, false, false, m - w, w, nb, -1.0, L + (int64_t)w * m + kb, m, Li + (int64_t)kb * m, m, 1.0,
            Li + (int64_t)w * m, m, nullptr);
  }
}

__global__ void logdiag_sum_kernel(const double* __restrict__ L, int64_t lda, int m, double* __restrict__ out) {
  __shared__ double sh[256];
  double v = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) v += log(L[(int64_t)i * lda + i]);
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = 2.0 * sh[0];
}

void logdet_from_cholesky(const double* L, int m, double* out_dev, cudaStream_t s) {
  logdiag_sum_kernel<<<1, 256, 0, s>>>(L, m, m, out_dev);
  FSA_CHECK_LAUNCH();
}

}  // namespace fsa
