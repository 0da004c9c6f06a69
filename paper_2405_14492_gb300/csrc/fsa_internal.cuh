// Internal declarations of the FSA library: device buffers, the handle, the
// per-theta operator and the CG workspace.
#pragma once
#include <memory>
#include <vector>

#include "fsa_common.cuh"

namespace fsa {

// ---------------------------------------------------------------------------
// device memory
// ---------------------------------------------------------------------------
// Device memory is stream-ordered (cudaMallocAsync / cudaFreeAsync from the
// device's memory pool) on the stream of the call that allocates it: a free
// waits for that stream's earlier work only, never for the whole device, so
// calls on different streams (the serving slots) overlap on the GPU.  The
// stream is a per-thread setting made by the entry points (AllocStreamScope);
// a buffer remembers the stream it was allocated on and is freed on it.
cudaStream_t current_alloc_stream();
struct AllocStreamScope {
  cudaStream_t prev;
  explicit AllocStreamScope(cudaStream_t s);
  ~AllocStreamScope();
};
void release_pool_memory();   // returns unused pool memory of the current device to the driver

template <typename T>
struct DevPtr {
  T* p = nullptr;
  size_t n = 0;
  cudaStream_t s = nullptr;
  DevPtr() = default;
  explicit DevPtr(size_t k) { alloc(k); }
  DevPtr(const DevPtr&) = delete;
  DevPtr& operator=(const DevPtr&) = delete;
  DevPtr(DevPtr&& o) noexcept : p(o.p), n(o.n), s(o.s) { o.p = nullptr; o.n = 0; }
  DevPtr& operator=(DevPtr&& o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; s = o.s; o.p = nullptr; o.n = 0; }
    return *this;
  }
  void alloc(size_t k) {
    release();
    if (k == 0) k = 1;
    s = current_alloc_stream();
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&p), k * sizeof(T), s);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      p = nullptr;
      throw Error{FSA_ERR_OOM, "device allocation of " + std::to_string(k * sizeof(T)) + " bytes failed"};
    }
    n = k;
  }
  void ensure(size_t k) {
    if (k > n || p == nullptr) alloc(k);
  }
  void release() {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
    n = 0;
  }
  ~DevPtr() { release(); }
};

// growable scratch for split-K partials and temporaries (one stream)
struct Workspace {
  DevPtr<double> f64;
  DevPtr<float> f32;
  double* scratch_f64(size_t k) { f64.ensure(k); return f64.p; }
  float* scratch_f32(size_t k) { f32.ensure(k); return f32.p; }
};

struct Grid {
  double x0 = 0, y0 = 0, hx = 1, hy = 1;
  int ncx = 1, ncy = 1;
};

// ---------------------------------------------------------------------------
// theta-dependent operator (paper §2.1, §3.1, Eq. eqfitcp)
// ---------------------------------------------------------------------------
// SpMM tile record (int32 words): p0, rows, (begin, length) of the three
// staged ranges, first nonzero (low, high words), nonzeros, offset of the
// tile's group offsets in gofs, first union entry (low, high words), union
// entries, bad flag (a copy of tile_bad)
constexpr int kTileWords = 16;
constexpr int kGrpRows = 3;   // rows per SpMM row group
static_assert(kGrpRows >= 1 && kGrpRows <= 7, "a union entry holds at most 7 values");
// int32 words of a union entry (staged column + kGrpRows values, padded to 16 or 32 bytes)
constexpr int kEntWords = kGrpRows <= 3 ? 4 : 8;
constexpr int kEntVec = kEntWords / 4;   // int4 per entry

struct Operator {
  bool valid = false;
  fsa_theta theta{};
  int precision = -1;
  // m-space, FP64
  DevPtr<double> Sm;      // Sigma_m, then overwritten by its Cholesky L_m
  DevPtr<double> Lmi;     // L_m^-1
  DevPtr<double> Mp;      // Woodbury core I + A^T D^-1 A, then its Cholesky L_P
  DevPtr<double> Minv;    // M_P^-1
  DevPtr<double> scal;    // [0] logdet M_P, [1] sum log D, [2] logdet P
  // n-space
  DevPtr<double> A;       // FP64 form: A = Sigma_nm L_m^-T (n x m, internal rows)
  DevPtr<double> vals;    // tapered residual values (nnz), FP64
  DevPtr<double> D;       // D_s = diag(Sigma_s~) (n)
  DevPtr<double> Dinv;
  // mixed form (tensor-core operands)
  DevPtr<__nv_bfloat16> Ab;    // A rounded to BF16, n x m_pad (K-major for A q)
  DevPtr<__nv_bfloat16> Atb;   // its transpose, m_pad x n_pad (K-major for A^T x)
  DevPtr<__nv_bfloat16> Ab_lo, Atb_lo;   // low halves (FSA_MIXED_BF16X2): A = Ab + Ab_lo
  bool has_lo = false;
  DevPtr<float> vals32;
  // per union entry of an SpMM row group (kEntWords words): its staged
  // column, then the FP32 values of the group's kGrpRows rows in that column
  // (0 where the column is not a neighbour of the row, and in the padding)
  DevPtr<int4> grp_ent;
  DevPtr<float> D32, Dinv32;
  double core_scale = 0.0;   // 2^-24 |M - I|_inf of the tensor-core Woodbury core
  bool core_fp64 = false;    // the core was formed in FP64 (core_scale too large)
  double a_scale = 0.0;      // 2^-16 sigma1 |L_m^-1|_inf: the tensor-core A's rounding, relative
  bool a_fp64 = false;       // A = Sigma_nm L_m^-T was formed in FP64 (a_scale too large)
  int m_pad = 0;
  int64_t n_pad = 0;
};

// ---------------------------------------------------------------------------
// CG block state
// ---------------------------------------------------------------------------
struct CGState {
  int c = 0, ldc = 0, L = 0;       // columns, leading dim of n x c arrays, iteration cap
  // n x ldc (FP64 form: double; mixed form: float stored in the f32 buffers)
  DevPtr<double> U, R, Z, H, V, S, W0, X;
  DevPtr<float> U32, R32, Z32, H32, V32, S32, W032;
  DevPtr<__nv_bfloat16> Xb;        // (2 c_pad) x n_pad hi/lo split of D^-1 R (K-major)
  DevPtr<__nv_bfloat16> qb;        // (2 c_pad) x m_pad hi/lo split of q (K-major)
  DevPtr<float> gout;              // split-K partial outputs of the tensor-core GEMMs
  // m x ldc
  DevPtr<double> w, q;
  // per column scalars
  DevPtr<double> rho, alpha, beta, alpha_prev, beta_prev, rnorm, rz0;
  DevPtr<int32_t> active, iters, stop;
  DevPtr<double> tdiag, toff;      // c x L Lanczos tridiagonals
  DevPtr<double> part;             // dot partials [nblk][ldc]
  DevPtr<double> quads;            // e1^T log(T) e1 per column
  DevPtr<double> qlwork;           // QL scratch (c x 2L)
  DevPtr<int32_t> num_active;      // device counter
  DevPtr<unsigned> ticket;         // last-block counter of the fused scalar steps (kept at 0 between launches)
  int nblk = 0;
};

struct Handle {
  int64_t n = 0;
  int m = 0;
  double gamma = 0;
  int cov = 0;
  cudaStream_t stream = nullptr;
  Grid grid;
  DevPtr<double> xs, ys, ind_x, ind_y;     // internal-order coordinates; inducing points
  DevPtr<float4> xy32, ixy32;              // the same as FP32 hi/lo pairs (x_hi, x_lo, y_hi, y_lo)
  DevPtr<int64_t> perm, iperm, rowptr;     // perm[internal] = original
  DevPtr<int32_t> col, cell_start, cell_count;
  int64_t nnz = 0;
  // Tiles of the SDDMM kernels: runs of cells of one grid row (about 24
  // points) whose taper neighbours all lie in three contiguous index ranges
  // (the same cells +-1 in the rows above, at and below).  Per tile 8 int64:
  // p0, p1 (its rows), then [begin, end) of the three ranges.
  DevPtr<int64_t> tiles;
  DevPtr<int32_t> ptile;                   // per tile kTileWords int32 (words 0-10; see tile_records)
  DevPtr<int32_t> scol;                    // per nonzero: row of its column in the tile's staged ranges
  DevPtr<int32_t> tile_bad;                // 1: a column of the tile lies outside its ranges
  // The SpMM's own tiling (larger tiles) and the row groups of its tiles
  // (kGrpRows consecutive rows; the last one of a tile may be shorter).  A
  // group's union list holds, in ascending order, every staged row that is a
  // neighbour of at least one of its rows.
  DevPtr<int32_t> sp_ptile;                // per tile kTileWords int32 (see build_spmm_groups)
  int sp_ntiles = 0;
  DevPtr<int32_t> gofs;                    // per tile, at sp_ptile word 11: its groups' list offsets (ng + 1, tile-relative)
  DevPtr<int4> grp_src;                    // per entry (kEntWords): staged column, then per row the tile-relative nonzero or -1
  int64_t grp_entries = 0;
  int ntiles = 0;
  int64_t max_staged = 0;                  // largest sum of the three range lengths
  int64_t max_tile_rows = 0, max_tile_nnz = 0;
  DevPtr<unsigned> err_buf;
  unsigned* err = nullptr;
  Operator op;
  CGState cg;
  Workspace ws;
  DevPtr<double> y;                        // response in internal order
  DevPtr<double> outs;                     // device results [loglik, logdet, quad, g0, g1, g2, se, ...]
  DevPtr<double> gterms;                   // per-probe gradient terms of the last call: a[3][l], b[3][l]
  int gterms_l = 0;                        // l of gterms (0: none yet)
  int vec_pieces = 2;                      // BF16 pieces of the vector operands (mixed forms; per call)
  double* host_pinned = nullptr;           // pinned mirror of small results
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // side stream for work that overlaps the main stream (SLQ beside the gradient)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

// ---------------------------------------------------------------------------
// building blocks
// ---------------------------------------------------------------------------
template <typename T>
void exclusive_scan(const T* in, T* out, int64_t n, cudaStream_t s);
Grid make_grid(const double bb[4], double gamma, int64_t n);
void build_structure(Handle& H, const double* locs_host);
void build_cross_structure(Handle& H, const double* qx, const double* qy, int64_t nq,
                           DevPtr<int64_t>& rowptr, DevPtr<int32_t>& col, int64_t& nnz);
void export_csr(Handle& H, int64_t* rowptr_host, int32_t* col_host);

// known zero triangles of the operands of dgemm (the products skip them; the
// operand must hold exact zeros there) and a symmetric result (only the tiles
// on and below the diagonal are computed, then mirrored; M == N)
enum DgemmTri : int {
  kTriA_KgeI = 1,     // op(A)(i, k) = 0 for k < i  (op(A) upper triangular, e.g. L^T)
  kTriA_KleI = 2,     // op(A)(i, k) = 0 for k > i  (op(A) lower triangular)
  kTriB_KgeJ = 4,     // op(B)(k, j) = 0 for k < j  (op(B) lower triangular)
  kTriB_KleJ = 8,     // op(B)(k, j) = 0 for k > j  (op(B) upper triangular, e.g. L^T)
  kTriSymLower = 16,  // C symmetric
};
void dgemm(Workspace& ws, cudaStream_t s, bool ta, bool tb, int M, int N, int K, double alpha,
           const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
           int64_t ldc, const double* scale, int tri = 0);
// C = A B for a narrow B (N <= 128 columns, a multiple of 8; else the general
// form): every column in one block, K split across the GPU
void dgemm_tall(Workspace& ws, cudaStream_t s, int M, int N, int K, const double* A, int64_t lda, const double* B,
                int64_t ldb, double* C, int64_t ldc);
void cholesky(double* A, int64_t lda, int m, unsigned* err, cudaStream_t s);
void trsm_lower(Workspace& ws, const double* L, int64_t ldl, int m, double* B, int64_t ldb, int r,
                cudaStream_t s);
void lower_inverse(Workspace& ws, const double* L, int m, double* Li, cudaStream_t s);
void logdet_from_cholesky(const double* L, int m, double* out_dev, cudaStream_t s);

unsigned read_err(Handle& H);   // synchronises the stream
void check_err(Handle& H);      // throws on a set error bit

}  // namespace fsa

// the opaque handle of the C ABI
struct fsa_handle {
  fsa::Handle h;
};

