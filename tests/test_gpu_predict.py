"""Predictive mean and simulation-based variances (Algorithm 1) on the GPU
against the FP64 oracle under identical probes, and against the exact FSA
predictive variances within the estimator's standard deviation."""
import numpy as np
import pytest

import fsa_inputs as fi
from oracle import fsa_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import paper_2405_14492_gb300 as F
    return F


def _case(n, m, n_p, seed, gamma):
    locs = fi.uniform_locations(n, seed)
    ind = locs[fi.inducing_subset(n, m, seed)]
    pred = fi.uniform_locations(n_p, seed, stream=fi.STREAM_PRED_LOCATIONS)
    return locs, ind, pred


@pytest.mark.parametrize("nu,probe", [(0.5, "rademacher"), (1.5, "gaussian")])
def test_predict_parity_same_probes(F, nu, probe):
    n, m, n_p, s, gamma = 3001, 60, 517, 40, 0.05
    locs, ind, pred = _case(n, m, n_p, 91, gamma)
    th = (1.0, 0.08, 0.05)
    y = fi.random_field(locs, nu, *th, 91)
    ref = O.IterativeFSA(locs, ind, gamma, nu, th).predict(y, pred, s, 13, 1e-11, probe=probe)
    kind = F.FSA_PROBE_RADEMACHER if probe == "rademacher" else F.FSA_PROBE_GAUSSIAN
    with F.FSAHandle(locs, ind, gamma, nu) as h:
        mean, var, info = h.predict(y, th, pred, s, F.make_opts(cg_tol=1e-11, seed=13, probe=kind))
    assert info["converged"] == 1
    assert np.max(np.abs(mean - ref["mean"])) < 1e-7 * np.max(np.abs(ref["mean"]))
    assert np.max(np.abs(var - ref["var"])) < 1e-7


def test_predict_statistically_matches_exact_variances(F):
    n, m, n_p, s, gamma = 1500, 40, 300, 400, 0.06
    locs, ind, pred = _case(n, m, n_p, 92, gamma)
    th = (1.0, 0.1, 0.1)
    y = fi.random_field(locs, 0.5, *th, 92)
    D = O.DenseFSA(locs, ind, gamma, 0.5, th)
    mu, var_exact = D.predict(y, pred)
    with F.FSAHandle(locs, ind, gamma, 0.5) as h:
        mean, var, _ = h.predict(y, th, pred, s, F.make_opts(cg_tol=1e-10, seed=3))
    assert np.max(np.abs(mean - mu)) < 1e-7
    # Rademacher diagonal estimator: Var[D_l,p] = (1/s) sum_{k != p} A_pk^2
    _, _, Ssnp, _ = D.cross(pred)
    Amat = Ssnp.T @ np.linalg.solve(D.Ss, Ssnp)
    sd = np.sqrt((np.sum(Amat ** 2, 1) - np.diag(Amat) ** 2) / s)
    assert np.all(np.abs(var - var_exact) <= 5 * sd + 1e-9)


def test_predict_mean_only_and_far_points(F):
    n, m, gamma = 2000, 30, 0.05
    locs = fi.uniform_locations(n, 93)
    ind = locs[fi.inducing_subset(n, m, 93)]
    # prediction points outside the data square, some beyond the taper range of every point
    pred = np.array([[-0.01, 0.5], [1.02, 0.3], [3.0, 3.0], [0.5, 0.5], [-1.0, -1.0]])
    th = (1.0, 0.1, 0.1)
    y = fi.random_field(locs, 0.5, *th, 93)
    ref = O.IterativeFSA(locs, ind, gamma, 0.5, th).predict(y, pred, 8, 5, 1e-11)
    with F.FSAHandle(locs, ind, gamma, 0.5) as h:
        mean, var, _ = h.predict(y, th, pred, 8, F.make_opts(cg_tol=1e-11, seed=5))
        mean2, var2, _ = h.predict(y, th, pred, 8, F.make_opts(cg_tol=1e-11, seed=5), want_var=False)
    assert np.allclose(mean, ref["mean"], atol=1e-8)
    assert np.allclose(var, ref["var"], atol=1e-8)
    assert np.array_equal(mean, mean2) and var2 is None
    # far from every data point: no sparse term, variance is the low-rank (FITC) one
    assert var[2] > 0.0 and var[4] > 0.0


@pytest.mark.parametrize("cv,name", [(1, "copt"), (2, "c1")])
def test_predict_control_variate_parity_same_probes(F, cv, name):
    """D_l with the diagonal preconditioner as control variate (appendix
    "Preconditioner as control variate") against the oracle, same probes."""
    n, m, n_p, s, gamma = 3001, 60, 517, 40, 0.05
    locs, ind, pred = _case(n, m, n_p, 94, gamma)
    th = (1.0, 0.08, 0.05)
    y = fi.random_field(locs, 0.5, *th, 94)
    ref = O.IterativeFSA(locs, ind, gamma, 0.5, th).predict(y, pred, s, 17, 1e-11, control_variate=name)
    with F.FSAHandle(locs, ind, gamma, 0.5) as h:
        mean, var, info = h.predict(y, th, pred, s, F.make_opts(cg_tol=1e-11, seed=17, pred_control_variate=cv))
    assert info["converged"] == 1
    assert np.max(np.abs(mean - ref["mean"])) < 1e-7 * np.max(np.abs(ref["mean"]))
    assert np.max(np.abs(var - ref["var"])) < 1e-7


def test_predict_control_variate_reduces_error_to_exact(F):
    """With c = 1 the estimate is unbiased with Var[D_l,p] = (1/s) sum_{k != p}
    (A - B)_pk^2, A = S Sigma_s~^-1 S^T, B = S D_s^-1 S^T; it stays within five
    of those standard deviations of the exact FSA variances.  With the
    coefficient c_opt the error to the exact variances is smaller than the
    plain estimator's on the same probes (here c = 1 alone is not: the
    diagonal preconditioner's term has variance of its own)."""
    n, m, n_p, s, gamma = 1500, 40, 300, 100, 0.06
    locs, ind, pred = _case(n, m, n_p, 95, gamma)
    th = (1.0, 0.1, 0.1)
    y = fi.random_field(locs, 0.5, *th, 95)
    D = O.DenseFSA(locs, ind, gamma, 0.5, th)
    _, var_exact = D.predict(y, pred)
    with F.FSAHandle(locs, ind, gamma, 0.5) as h:
        _, var_cv, _ = h.predict(y, th, pred, s, F.make_opts(cg_tol=1e-10, seed=4, pred_control_variate=2))
        _, var_co, _ = h.predict(y, th, pred, s, F.make_opts(cg_tol=1e-10, seed=4, pred_control_variate=1))
        _, var_pl, _ = h.predict(y, th, pred, s, F.make_opts(cg_tol=1e-10, seed=4))
    _, _, Ssnp, _ = D.cross(pred)
    A = Ssnp.T @ np.linalg.solve(D.Ss, Ssnp)
    B = Ssnp.T @ (Ssnp / np.diag(D.Ss)[:, None])
    E = A - B
    sd = np.sqrt((np.sum(E ** 2, 1) - np.diag(E) ** 2) / s)
    assert np.all(np.abs(var_cv - var_exact) <= 5 * sd + 1e-9)
    assert np.sqrt(np.mean((var_co - var_exact) ** 2)) < 0.8 * np.sqrt(np.mean((var_pl - var_exact) ** 2))


@pytest.mark.parametrize("m,x2", [(200, True), (200, False), (100, True)])
def test_mixed_predict_parity_same_probes(F, m, x2):
    """The mixed form of Algorithm 1 (its m-column products on the tensor
    cores with BF16 pairs, the sparse solves in FP32, the cores in FP64)
    against the FP64 oracle with the same probes.
    Variances: each of D1, 2 D2, D3 and D_l is a sum of products rounded to
    about 2^-16 (a BF16 pair), so the variance of point p is held to
    3e-4 (|D1| + 2 |D2| + |D3| + |D_l|)_p, a tenth of which is measured.
    Mean: a linear functional of u = Sigma_dag^-1 y, where the mixed operator
    (A~ as a pair, FP32 vectors) differs from the FP64 one by about 2^-16 of
    its norm; the solve amplifies that by up to the conditioning of Sigma_dag,
    lambda_max / nugget, about 1e3 here.  It is held to 2e-3 of max |mean|
    (4e-4 measured).  The single-BF16 operator (A~ rounded to 8 bits, 2^-9)
    is held to ten times both bounds.  m = 100 gives the tensor-core products
    an N tile of 112 rows (N < 128), m = 200 a ragged second N tile."""
    n, n_p, s, gamma = 20011, 3001, 24, fi.taper_range_for(25, 20011)
    locs, ind, pred = _case(n, m, n_p, 94, gamma)
    th = (1.0, 0.05, 0.05)
    y = fi.random_field(locs, 0.5, *th, 94)
    tol_cg = 1e-6 * np.linalg.norm(y)
    ref = O.IterativeFSA(locs, ind, gamma, 0.5, th).predict(y, pred, s, 17, tol_cg)
    prec = F.FSA_MIXED_BF16X2 if x2 else F.FSA_MIXED_BF16
    with F.FSAHandle(locs, ind, gamma, 0.5) as h:
        mean, var, info = h.predict(y, th, pred, s, F.make_opts(cg_tol=tol_cg, seed=17, precision=prec))
    assert info["converged"] == 1
    k = 1.0 if x2 else 10.0
    scale_v = np.abs(ref["D1"]) + 2 * np.abs(ref["D2"]) + np.abs(ref["D3"]) + np.abs(ref["Dl"])
    err_m = np.max(np.abs(mean - ref["mean"])) / np.max(np.abs(ref["mean"]))
    err_v = np.max(np.abs(var - ref["var"]) / scale_v)
    print(f"mixed predict ({'bf16x2' if x2 else 'bf16'}): mean err {err_m:.2e} of max|mean|, "
          f"var err {err_v:.2e} of its parts; iterations {info['iters_y']} / {info['iters_max']}")
    assert err_m < k * 2e-3
    assert err_v < k * 3e-4


def test_exact_variances_match_the_dense_definition(F):
    """pred_exact_var: D_l = diag(S Sigma_s~^-1 S^T) by n_p sparse solves makes
    the predictive variance exact (§2.3); it equals the dense FSA predictive
    variance sigma1^2 + nugget - diag(Sigma_dag_np^T Sigma_dag^-1 Sigma_dag_np)."""
    n, m, n_p, gamma = 1500, 40, 300, 0.06
    locs, ind, pred = _case(n, m, n_p, 95, gamma)
    th = (1.0, 0.1, 0.1)
    y = fi.random_field(locs, 0.5, *th, 95)
    D = O.DenseFSA(locs, ind, gamma, 0.5, th)
    mu, var_exact = D.predict(y, pred)
    with F.FSAHandle(locs, ind, gamma, 0.5) as h:
        mean, var, info = h.predict(y, th, pred, 8, F.make_opts(cg_tol=1e-11, seed=3, pred_exact_var=True))
    assert info["converged"] == 1
    assert np.max(np.abs(mean - mu)) < 1e-7
    assert np.max(np.abs(var - var_exact)) < 1e-8, np.max(np.abs(var - var_exact))
