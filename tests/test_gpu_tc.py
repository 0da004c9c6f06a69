"""Tensor-core path: the tcgen05/TMA BF16 GEMM against an FP64 reference of
the same BF16 operands, and the mixed-precision FSA log-likelihood against
the FP64 oracle under identical probes."""
import ctypes
import math

import numpy as np
import pytest

import fsa_inputs as fi
from oracle import fsa_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import paper_2405_14492_gb300 as F
    return F


def _selftest(M, N, K, na, nb, pairs, halves, splits, seed=1):
    from paper_2405_14492_gb300 import _native as N_
    lib = N_.lib()
    lib.fsa_selftest_tc_gemm.restype = ctypes.c_int
    lib.fsa_selftest_tc_gemm.argtypes = [ctypes.c_int] * 5 + [ctypes.c_uint, ctypes.c_int, ctypes.c_int,
                                                              ctypes.c_uint64, ctypes.POINTER(ctypes.c_double),
                                                              ctypes.POINTER(ctypes.c_int)]
    err = ctypes.c_double(-1.0)
    act = ctypes.c_int(0)
    st = lib.fsa_selftest_tc_gemm(M, N, K, na, nb, pairs, halves, splits, seed, ctypes.byref(err),
                                  ctypes.byref(act))
    return st, err.value, act.value


@pytest.mark.parametrize("M,N,K,na,nb,pairs,halves,splits", [
    (128, 16, 64, 1, 1, 1, 0, 1),          # one tile, one K block
    (256, 144, 320, 1, 1, 1, 1, 1),        # hi/lo halves epilogue (N = 2 x 72)
    (300, 80, 1000, 1, 1, 1, 0, 1),        # ragged M and K (TMA zero fill)
    (1000, 256, 512, 2, 2, 7, 0, 1),       # three split products hi.hi + hi.lo + lo.hi
    (520, 128, 2048, 1, 2, 3, 0, 1),       # one A, two B
    (1024, 144, 20000, 1, 1, 1, 1, 38),    # split-K with halves (the A^T X shape)
    (70, 32, 2000, 1, 1, 1, 0, 5),         # split-K, ragged everything
    (4096, 48, 1024, 1, 1, 1, 1, 1),       # many M tiles (the A q shape)
    (1024, 240, 20000, 2, 1, 5, 3, 38),    # A hi/lo with a three-piece stacked vector (the A^T X shape)
    (3000, 240, 1024, 2, 1, 5, 3, 1),      # same for the A q shape, ragged M
    (50000, 144, 1024, 2, 1, 5, 2, 1),     # persistent form (>= 2 tiles per SM): A q with A hi/lo, ragged M
    (40000, 256, 128, 1, 1, 1, 0, 1),      # persistent form, full 256-column tile, two K blocks
    (39001, 48, 64, 1, 1, 1, 1, 1),        # persistent form, one K block per tile
    (40000, 512, 128, 1, 1, 1, 0, 1),      # persistent form over two N tiles
    (20011, 1024, 256, 2, 2, 7, 0, 1),     # persistent form over four N tiles, split products (the A~ build shape)
])
def test_tc_gemm_selftest(F, M, N, K, na, nb, pairs, halves, splits):
    st, err, act = _selftest(M, N, K, na, nb, pairs, halves, splits)
    assert st == 0, f"status {st}"
    tol = 2e-6 * math.sqrt(K) + 1e-6
    assert err < tol, f"max rel err {err} (tol {tol}), splits {act}"


def test_mixed_operator_close_to_fp64(F):
    n, m, nu, gamma = 20011, 200, 0.5, 0.015
    locs = fi.uniform_locations(n, 71)
    ind = locs[fi.inducing_subset(n, m, 71)]
    th = (1.0, 0.05, 0.05)
    V = np.random.default_rng(3).standard_normal((n, 5))
    with F.FSAHandle(locs, ind, gamma, nu) as h:
        ref0 = h.matvec(th, V, 0, F.FSA_FP64)
        ref1 = h.matvec(th, V, 1, F.FSA_FP64)
        got0 = h.matvec(th, V, 0, F.FSA_MIXED_BF16)
        got1 = h.matvec(th, V, 1, F.FSA_MIXED_BF16)
        ld64 = h.logdet_precond(th, F.FSA_FP64)
        ld16 = h.logdet_precond(th, F.FSA_MIXED_BF16)
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    # the BF16-rounded A~ (unit roundoff 2^-9) changes the operator only
    # outside the taper, (1 - T) o (A~A~^T - AA^T): at most ~2 2^-9 of it; the
    # preconditioner moves with D_i = sigma1^2 + sigma^2 - |a_i|^2, by up to
    # 2^-8 |a_i|^2 / D_i (here 1.9e-3 at the median row, 6.3e-3 at the 90th
    # percentile, 7.8e-2 next to an inducing point); norm-wise in between
    assert rel(got0, ref0) < 1e-2
    assert rel(got1, ref1) < 3e-2
    assert abs(ld16 - ld64) < 1e-3 * abs(ld64)


def test_mixed_x2_operator_close_to_fp64(F):
    """With A stored as a BF16 hi + lo pair the operator is FP32-accurate."""
    n, m, nu, gamma = 20011, 200, 0.5, 0.015
    locs = fi.uniform_locations(n, 72)
    ind = locs[fi.inducing_subset(n, m, 72)]
    th = (1.0, 0.05, 0.05)
    V = np.random.default_rng(4).standard_normal((n, 5))
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    with F.FSAHandle(locs, ind, gamma, nu) as h:
        ref0 = h.matvec(th, V, 0, F.FSA_FP64)
        ref1 = h.matvec(th, V, 1, F.FSA_FP64)
        ld64 = h.logdet_precond(th, F.FSA_FP64)
        got0 = h.matvec(th, V, 0, F.FSA_MIXED_BF16X2)
        got1 = h.matvec(th, V, 1, F.FSA_MIXED_BF16X2)
        ld32 = h.logdet_precond(th, F.FSA_MIXED_BF16X2)
    assert rel(got0, ref0) < 1e-5
    assert rel(got1, ref1) < 1e-4
    assert abs(ld32 - ld64) < 1e-6 * abs(ld64)


@pytest.mark.parametrize("n,m,nu,gamma,l,K", [(20011, 200, 0.5, 0.015, 16, 30), (30011, 300, 1.5, 0.012, 12, 25)])
def test_mixed_x2_loglik_within_1e5_of_oracle(F, n, m, nu, gamma, l, K):
    locs = fi.uniform_locations(n, 82)
    ind = locs[fi.inducing_subset(n, m, 82)]
    th = (1.0, 0.05, 0.01) if nu == 0.5 else (1.0, 0.03, 0.02)
    y = fi.random_field(locs, nu, *th, 82)
    ref = O.IterativeFSA(locs, ind, gamma, nu, th).loglik_grad(y, l, 6, 0.0, fixed_iters=K)
    with F.FSAHandle(locs, ind, gamma, nu) as h:
        ll, g, info = h.loglik_grad(y, th, F.make_opts(num_probes=l, fixed_iters=K, seed=6,
                                                       precision=F.FSA_MIXED_BF16X2))
    assert abs(ll - ref["loglik"]) < 1e-5 * abs(ref["loglik"]), (ll, ref["loglik"])
    assert np.linalg.norm(g - ref["grad"]) < 1e-2 * np.linalg.norm(ref["grad"]), (g, ref["grad"])


@pytest.mark.parametrize("n,m,nu,gamma,l,K", [(20011, 200, 0.5, 0.015, 16, 30), (30011, 300, 1.5, 0.012, 12, 25)])
def test_mixed_loglik_within_1e4_of_oracle(F, n, m, nu, gamma, l, K):
    locs = fi.uniform_locations(n, 81)
    ind = locs[fi.inducing_subset(n, m, 81)]
    th = (1.0, 0.05, 0.05) if nu == 0.5 else (1.0, 0.03, 0.05)
    y = fi.random_field(locs, nu, *th, 81)
    ref = O.IterativeFSA(locs, ind, gamma, nu, th).loglik_grad(y, l, 5, 0.0, fixed_iters=K)
    with F.FSAHandle(locs, ind, gamma, nu) as h:
        ll, g, info = h.loglik_grad(y, th, F.make_opts(num_probes=l, fixed_iters=K, seed=5,
                                                       precision=F.FSA_MIXED_BF16))
        ll64, g64, _ = h.loglik_grad(y, th, F.make_opts(num_probes=l, fixed_iters=K, seed=5))
    assert abs(ll64 - ref["loglik"]) < 1e-6 * abs(ref["loglik"])
    assert abs(ll - ref["loglik"]) < 1e-4 * abs(ref["loglik"]), (ll, ref["loglik"])
    assert np.linalg.norm(g - ref["grad"]) < 2e-2 * np.linalg.norm(ref["grad"]), (g, ref["grad"])


def test_mixed_x2_woodbury_core_accurate_at_large_n(F):
    """n = 2e5 with a long range and small nugget: M - I = A~^T D^-1 A~ has
    entries ~1e4 while the small eigenvalues of M = I + A~^T D^-1 A~ sit near
    1, so an FP32 sum over the whole n would lose the identity.  The mixed
    form must stay within 1e-4 of the FP64 form (same probes, same fixed
    iteration count), for the log det of the preconditioner and the
    log-likelihood."""
    n, m, rho, nug = 199_791, 738, 0.081, 0.028
    locs = fi.uniform_locations(n, 8032)
    ind = locs[fi.inducing_subset(n, m, 8032)]
    gamma = fi.taper_range_for(20, n)
    th = (1.0, rho, nug)
    y = fi.random_field(locs, 0.5, *th, 8032, features=64)
    with F.FSAHandle(locs, ind, gamma, 0.5) as h:
        o = dict(num_probes=16, fixed_iters=40, seed=3, want_grad=False)
        ll64, _, i64 = h.loglik_grad(y, th, F.make_opts(**o))
        ll2, _, i2 = h.loglik_grad(y, th, F.make_opts(precision=F.FSA_MIXED_BF16X2, **o))
    assert abs(i2["logdet_precond"] - i64["logdet_precond"]) < 1e-5 * abs(i64["logdet_precond"])
    assert abs(ll2 - ll64) < 1e-4 * abs(ll64), (ll2, ll64)


def test_mixed_x2_loglik_clustered_points(F):
    """Points with a dense cluster (a few hundred in one taper cell) beside a
    uniform background: the SpMM stages most tiles in shared memory and runs
    the overfull ones from global memory; both paths meet the oracle."""
    rng = np.random.default_rng(4321)
    n_bg, n_cl = 12000, 600
    locs = np.vstack([fi.uniform_locations(n_bg, 83), 0.5 + 0.003 * rng.random((n_cl, 2))])
    n = locs.shape[0]
    m, nu, gamma, l, K = 150, 0.5, 0.02, 8, 25
    ind = locs[fi.inducing_subset(n, m, 83)]
    th = (1.0, 0.05, 0.05)
    y = fi.random_field(locs, nu, *th, 83)
    ref = O.IterativeFSA(locs, ind, gamma, nu, th).loglik_grad(y, l, 4, 0.0, fixed_iters=K)
    with F.FSAHandle(locs, ind, gamma, nu) as h:
        diff, staged, total = _spmm_selftest(h, th, 40)
        ll, g, info = h.loglik_grad(y, th, F.make_opts(num_probes=l, fixed_iters=K, seed=4,
                                                       precision=F.FSA_MIXED_BF16X2))
    # the tile kernel (shared-memory and global tiles) equals the row kernel bit for bit
    assert diff == 0.0 and 0 < staged < total, (diff, staged, total)
    # a dense cluster is the ill-conditioned case: the log-likelihood stays within 1e-4
    assert abs(ll - ref["loglik"]) < 1e-4 * abs(ref["loglik"]), (ll, ref["loglik"])
    assert np.linalg.norm(g - ref["grad"]) < 1e-2 * np.linalg.norm(ref["grad"])


def _spmm_selftest(h, th, ncols, seed=1):
    import ctypes
    from paper_2405_14492_gb300 import _native as N
    f = N.lib().fsa_selftest_spmm
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.POINTER(N.FsaTheta), ctypes.c_int, ctypes.c_uint64,
                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    d, st, tot = ctypes.c_double(-1), ctypes.c_int(-1), ctypes.c_int(-1)
    t = N.FsaTheta(*th)
    N.check(f(h._h, ctypes.byref(t), ncols, seed, ctypes.byref(d), ctypes.byref(st), ctypes.byref(tot)))
    return d.value, st.value, tot.value


@pytest.mark.parametrize("n,gamma,ncols", [(20011, 0.015, 65), (50021, 0.0071, 17), (3001, 0.05, 127),
                                           (200003, fi.taper_range_for(20, 200003), 65), (4001, 0.05, 1)])
def test_spmm_tile_kernel_equals_row_kernel(F, n, gamma, ncols):
    """The shared-memory tile SpMM (row groups over the union of their
    neighbour lists) gives the row kernel's result bit for bit (same per-row
    summation order), for block widths from 1 to 127 columns, at the headline's
    density (20 nonzeros per row) among them."""
    locs = fi.uniform_locations(n, 84)
    ind = locs[fi.inducing_subset(n, 60, 84)]
    with F.FSAHandle(locs, ind, gamma, 0.5) as h:
        diff, staged, total = _spmm_selftest(h, (1.0, 0.05, 0.05), ncols)
    assert diff == 0.0
    # at 128 columns the staging capacity holds fewer rows than these tiles span
    assert total > 0 and (staged > 0 or ncols > 100)


def _sddmm_selftest(h, th, precision, cap_rows, seed=3):
    from paper_2405_14492_gb300 import _native as N
    f = N.lib().fsa_selftest_sddmm
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.POINTER(N.FsaTheta), ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    ve, de = (ctypes.c_double * 2)(), (ctypes.c_double * 2)()
    t = N.FsaTheta(*th)
    N.check(f(h._h, ctypes.byref(t), precision, cap_rows, seed, ve, de))
    return np.array(ve[:]), np.array(de[:])


@pytest.mark.parametrize("n,gamma,m,cap_rows", [(30011, 0.012, 200, 0), (30011, 0.012, 200, 60),
                                                (8009, 0.03, 130, 0)])
@pytest.mark.parametrize("x2", [False, True])
def test_sddmm_tile_forms_match_row_forms(F, n, gamma, m, cap_rows, x2):
    """The tile forms of the mixed residual values (and D_s) and of their range
    derivative agree with the row forms (global gathers) up to FP32 summation
    order.  The tile forms stage the m-long rows in shared memory per
    cell-grid tile; cap_rows = 60 sends most tiles down their global-memory
    path.  The bounds are max-norm relative differences.  Each product is a sum
    of FP32 partial sums over 64-column blocks, added in FP64, so two forms may
    differ by a few FP32 roundings of the partial sums (each <= sigma1^2 / 16;
    at most about 1e-6 over the 16 blocks): 2e-6 for the values and D.  A bias
    of the kind a dropped lo.lo product of the BF16 pairs would leave on D
    (2^-18 of |a_i|^2, 3.4e-6 of max D here) fails it.  1e-5 for the
    derivative (FP32 outputs, two products)."""
    locs = fi.uniform_locations(n, 91)
    ind = locs[fi.inducing_subset(n, m, 91)]
    prec = F.FSA_MIXED_BF16X2 if x2 else F.FSA_MIXED_BF16
    with F.FSAHandle(locs, ind, gamma, 0.5) as h:
        ve, de = _sddmm_selftest(h, (1.0, 0.05, 0.05), prec, cap_rows)
    print(f"values {ve}, derivative {de}")
    assert ve[0] < 2e-6 and ve[1] < 2e-6, ve
    assert de[0] < 1e-5 and de[1] < 1e-5, de
