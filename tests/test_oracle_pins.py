"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a textbook
routine, a closed form, an exact identity, a number printed in the paper, or a
brute force.  A plausible mistake in the oracle (a dropped term, a wrong sign,
a transposed operand, a shifted Lanczos index) fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.optimize as so
import scipy.stats as st

import fsa_inputs as fi
from oracle import fsa_oracle as O
from tests.conftest import golden, read_golden_kv


def _problem(n=150, m=20, nu=0.5, theta=(1.3, 0.15, 0.2), gamma=0.12, seed=7):
    locs = fi.uniform_locations(n, seed)
    idx = fi.inducing_subset(n, m, seed)
    return locs, locs[idx].copy(), gamma, nu, theta


# --------------------------------------------------------------------------
# covariance function, taper, random numbers
# --------------------------------------------------------------------------

def test_splitmix64_published_vectors():
    want = [int(l, 16) for l in open(golden("splitmix64_seed0.txt")) if l.startswith("0x")]
    st_ = np.arange(1, 6, dtype=np.uint64) * O.GOLDEN_GAMMA
    got = [int(x) for x in O._mix64(st_)]
    assert got == want


def test_counter_based_splitmix64_equals_the_sequential_generator():
    """Value k of the counter-based form is output k + 1 of the sequential
    SplitMix64 generator (state += golden gamma, then mix) started at the
    stream key, and a Rademacher entry is 1 - 2 * (top bit of that output),
    at counter column * rows + row."""
    M64 = (1 << 64) - 1
    gam = int(O.GOLDEN_GAMMA)

    def mix(z):
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        return z ^ (z >> 31)

    for seed, stream in ((0, 0), (14492, 4), (2**63 + 5, 9)):
        state = mix(seed ^ ((stream * gam) & M64))
        seq = []
        for _ in range(12):
            state = (state + gam) & M64
            seq.append(mix(state))
        got = O.splitmix64(seed, stream, np.arange(12, dtype=np.uint64))
        assert [int(v) for v in got] == seq
    z = O.rademacher(14492, 4, np.arange(3), 3, 4)
    h = O.splitmix64(14492, 4, np.arange(24, dtype=np.uint64))
    for r in range(3):
        for k in range(4):
            assert z[r, k] == 1.0 - 2.0 * float(int(h[k * 3 + r]) >> 63)
    # Gaussian entry (r, k): Box-Muller of the outputs at counters 2c and 2c + 1,
    # c = k * rows + r, with u = ((h >> 11) + 1) 2^-53
    g = O.gaussian(14492, 4, np.arange(3), 3, 4)
    for r in range(3):
        for k in range(4):
            c = k * 3 + r
            u1 = ((int(h[2 * c]) >> 11) + 1) * 2.0 ** -53
            u2 = ((int(h[2 * c + 1]) >> 11) + 1) * 2.0 ** -53
            assert abs(g[r, k] - math.sqrt(-2 * math.log(u1)) * math.cos(2 * math.pi * u2)) < 1e-14


def test_rademacher_balance_and_independence():
    z = O.rademacher(3, O.STREAM_EPS2, np.arange(4000), 4000, 8)
    assert set(np.unique(z)) == {-1.0, 1.0}
    assert abs(z.mean()) < 0.03
    c = np.corrcoef(z.T)
    assert np.max(np.abs(c - np.eye(8))) < 0.06
    g = O.gaussian(3, O.STREAM_PRED, np.arange(20000), 20000, 2)
    assert abs(g.mean()) < 0.03 and abs(g.var() - 1) < 0.04
    assert st.kstest(g[:, 0], "norm").pvalue > 1e-3


def test_matern15_effective_range_factor_matches_paper():
    """§4: effective range ~ 2.7 * rho for nu = 3/2 (with the sqrt(3) scaling;
    without it the factor would be 4.74)."""
    kv = read_golden_kv("paper_constants.txt")
    x = so.brentq(lambda t: O.corr(t, 1.5, 1.0) - 0.05, 0.1, 20.0)
    assert round(x, 1) == kv["effective_range_factor_matern15"][0]
    for eff, rho in zip(kv["effective_ranges"], kv["range_parameters"]):
        assert abs(eff / kv["effective_range_factor_matern15"][0] - rho) < 6e-5
        # the printed rho gives correlation close to 0.05 at the effective range
        assert abs(float(O.corr(eff, 1.5, rho)) - 0.05) < 0.004


def test_matern_closed_forms_and_derivative():
    d = np.linspace(0, 0.6, 31)
    assert np.allclose(O.corr(d, 0.5, 0.2), np.exp(-d / 0.2))
    assert O.corr(0.0, 1.5, 0.2) == 1.0
    for nu in (0.5, 1.5):
        h = 1e-6
        fd = (O.corr(d, nu, 0.2 + h) - O.corr(d, nu, 0.2 - h)) / (2 * h)
        assert np.allclose(O.dcorr_drho(d, nu, 0.2), fd, rtol=1e-6, atol=1e-9)


def test_wendland_taper_properties():
    g = 0.1
    assert O.taper(0.0, g) == 1.0
    assert O.taper(g, g) == 0.0 and O.taper(2 * g, g) == 0.0
    d = np.linspace(0, g, 101)[:-1]
    assert np.all(np.diff(O.taper(d, g)) <= 0)
    # positive definite in R^2: the taper matrix of random points is PSD
    pts = fi.uniform_locations(300, 11)
    T = O.taper(np.sqrt(O.sqdist(pts, pts)), 0.3)
    assert np.linalg.eigvalsh(T).min() > -1e-10


# --------------------------------------------------------------------------
# neighbour structure
# --------------------------------------------------------------------------

def test_neighbour_csr_brute_force_vs_tree_bit_exact():
    pts = fi.uniform_locations(3000, 5)
    g = 0.03
    a = O.neighbour_csr(pts, pts, g, brute_force_limit=10 ** 8)
    b = O.neighbour_csr(pts, pts, g, brute_force_limit=1)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    rowptr, col = a
    rows = np.repeat(np.arange(3000), np.diff(rowptr))
    # self pair present, columns ascending, support exact, symmetric pattern
    assert np.all(np.isin(np.arange(3000), col[rows == col]))
    for i in range(0, 3000, 97):
        c = col[rowptr[i]:rowptr[i + 1]]
        assert np.all(np.diff(c) > 0)
    d2 = O.sqdist_pairs(pts[rows], pts[col])
    assert np.all(d2 < g * g)
    S = set(zip(rows.tolist(), col.tolist()))
    assert all((j, i) in S for (i, j) in S)
    # nothing missed: count pairs inside the radius by brute force
    assert len(S) == int(np.sum(O.sqdist(pts, pts) < g * g))


def test_neighbour_support_is_strict_at_exact_ties():
    """§2.1: the taper is zero for d >= gamma, so pairs at distance exactly
    gamma are not in the support.  On a lattice of spacing gamma = 1/8 (exact
    binary fractions, so d^2 = gamma^2 holds exactly) each point has itself as
    its only neighbour, in both the brute-force and the tree path; at
    gamma * (1 + 2^-20) the four lattice neighbours join."""
    g = 0.125
    xs = np.arange(12) * g
    pts = np.array([(x, y) for y in xs for x in xs])
    for limit in (10 ** 8, 1):
        rowptr, col = O.neighbour_csr(pts, pts, g, brute_force_limit=limit)
        assert np.array_equal(col, np.arange(len(pts)))
        rowptr, col = O.neighbour_csr(pts, pts, g * (1 + 2.0 ** -20), brute_force_limit=limit)
        deg = np.diff(rowptr)
        assert deg.max() == 5 and deg.min() == 3 and int(deg.sum()) == 144 + 2 * 2 * 11 * 12


def test_neighbour_count_matches_paper_taper_choice():
    """Appendix 'Choice of FSA parameters': gamma = 0.016 <-> n_gamma = 80 at n = 1e5."""
    kv = read_golden_kv("paper_constants.txt")
    n = int(kv["n"][0])
    pts = fi.uniform_locations(n, 1)
    rowptr, _ = O.neighbour_csr(pts, pts, kv["taper_range"][0])
    mean = rowptr[-1] / n
    assert abs(mean - kv["nnz_per_row"][0]) < 1.0
    assert abs(fi.expected_neighbours(kv["taper_range"][0], n) - kv["nnz_per_row"][0]) < 0.5


# --------------------------------------------------------------------------
# FSA covariance assembly
# --------------------------------------------------------------------------

def test_m_equals_n_reduces_to_exact_gp():
    """Inducing points = all points: Sigma_l = Sigma, residual 0, so the FSA is
    the exact GP and the log-likelihood is the textbook Gaussian log density."""
    n = 60
    locs = fi.uniform_locations(n, 2)
    theta = (1.1, 0.08, 0.3)
    y = np.random.default_rng(0).standard_normal(n)
    F = O.DenseFSA(locs, locs, 0.05, 0.5, theta)
    Sig = theta[0] * np.exp(-np.sqrt(O.sqdist(locs, locs)) / theta[1]) + theta[2] * np.eye(n)
    assert np.allclose(F.Sdag, Sig, atol=1e-9)
    ll, _, _ = F.loglik(y)
    want = st.multivariate_normal(mean=np.zeros(n), cov=Sig).logpdf(y)
    assert abs(ll - want) < 1e-7 * abs(want)


def test_fsa_spectral_bounds_and_symmetry():
    locs, ind, g, nu, th = _problem()
    F = O.DenseFSA(locs, ind, g, nu, th)
    assert np.allclose(F.Sdag, F.Sdag.T, atol=1e-12)
    # lambda_min >= nugget for Sigma_s~ and Sigma_dag (proof of Lemma 1)
    assert np.linalg.eigvalsh(F.Ss).min() >= th[2] - 1e-10
    assert np.linalg.eigvalsh(F.Sdag).min() >= th[2] - 1e-10
    # taper support respected
    assert np.all(F.Ss[~F.support] == 0.0)


def test_iterative_structures_match_dense_definition():
    locs, ind, g, nu, th = _problem(nu=1.5)
    D = O.DenseFSA(locs, ind, g, nu, th)
    It = O.IterativeFSA(locs, ind, g, nu, th)
    V = np.random.default_rng(1).standard_normal((locs.shape[0], 3))
    assert np.allclose(It.Ss.toarray(), D.Ss, atol=1e-12)
    assert np.allclose(It.apply(V), D.Sdag @ V, rtol=1e-11, atol=1e-11)


# --------------------------------------------------------------------------
# FITC preconditioner: Woodbury, Sylvester, condition bound
# --------------------------------------------------------------------------

def test_fitc_woodbury_sylvester_and_condition_bound():
    locs, ind, g, nu, th = _problem()
    D = O.DenseFSA(locs, ind, g, nu, th)
    It = O.IterativeFSA(locs, ind, g, nu, th)
    V = np.random.default_rng(2).standard_normal((locs.shape[0], 4))
    assert np.allclose(It.apply_Pinv(V), np.linalg.solve(D.Phat, V), rtol=1e-10, atol=1e-10)
    sign, ld = np.linalg.slogdet(D.Phat)
    assert sign > 0 and abs(It.logdet_P - ld) < 1e-9 * abs(ld)
    # Lemma 2 proof: kappa(P^-1 Sdag) <= (1 + ||Ss - diag(Ss)||_2 / nugget)^2
    ev = sla.eigh(D.Sdag, D.Phat, eigvals_only=True)
    E = D.Ss - np.diag(np.diag(D.Ss))
    bound = (1 + np.linalg.norm(E, 2) / th[2]) ** 2
    assert ev.max() / ev.min() <= bound + 1e-9


def test_fitc_sample_covariance_is_phat():
    locs, ind, g, nu, th = _problem(n=40, m=6)
    It = O.IterativeFSA(locs, ind, g, nu, th)
    D = O.DenseFSA(locs, ind, g, nu, th)
    Z = It.probes(20000, 9)
    C = Z @ Z.T / Z.shape[1]
    assert np.max(np.abs(C - D.Phat)) < 0.08 * np.max(np.abs(D.Phat))


# --------------------------------------------------------------------------
# PCG with Lanczos tridiagonals, SLQ, STE
# --------------------------------------------------------------------------

def test_tiny_taper_makes_fsa_equal_fitc_one_step():
    """gamma below every pair distance: Sigma_dag = P_hat, so PCG converges in
    one iteration with alpha_1 = 1 and T = [1] (Theorem 2 remark, gamma -> 0)."""
    locs, ind, _, nu, th = _problem(n=80, m=10)
    It = O.IterativeFSA(locs, ind, 1e-6, nu, th)
    assert It.rowptr[-1] == 80
    b = np.random.default_rng(3).standard_normal((80, 2))
    res = O.pcg_lanczos(It.apply, It.apply_Pinv, b, 1e-10, 50)
    assert np.all(res["iters"] == 1)
    for k in range(2):
        assert abs(res["diag"][k][0] - 1.0) < 1e-10
    out = It.loglik_grad(b[:, 0], 5, 1, 1e-10, want_grad=False)
    assert abs(out["logdet"] - It.logdet_P) < 1e-9 * abs(It.logdet_P)


def test_pcg_solution_and_ritz_values_within_spectrum():
    locs, ind, g, nu, th = _problem()
    D = O.DenseFSA(locs, ind, g, nu, th)
    It = O.IterativeFSA(locs, ind, g, nu, th)
    b = np.random.default_rng(4).standard_normal((150, 3))
    res = O.pcg_lanczos(It.apply, It.apply_Pinv, b, 1e-11, 500)
    assert np.allclose(res["U"], np.linalg.solve(D.Sdag, b), rtol=1e-8, atol=1e-9)
    ev = sla.eigh(D.Sdag, D.Phat, eigvals_only=True)
    for k in range(3):
        T = np.diag(res["diag"][k]) + np.diag(res["off"][k], 1) + np.diag(res["off"][k], -1)
        ritz = np.linalg.eigvalsh(T)
        assert ritz.min() >= ev.min() * (1 - 1e-8) and ritz.max() <= ev.max() * (1 + 1e-8)


def test_fixed_iteration_pcg_tridiagonal_equals_lanczos():
    """The CG-derived T (Appendix A) equals the tridiagonal of k explicit Lanczos
    steps on L^-1 Sdag L^-T started from L^-1 b/|L^-1 b| (P_hat = L L^T)."""
    locs, ind, g, nu, th = _problem(n=90, m=12)
    D = O.DenseFSA(locs, ind, g, nu, th)
    It = O.IterativeFSA(locs, ind, g, nu, th)
    b = np.random.default_rng(5).standard_normal((90, 1))
    k = 6
    res = O.pcg_lanczos(It.apply, It.apply_Pinv, b, 0.0, 100, fixed_iters=k)
    L = np.linalg.cholesky(D.Phat)
    Aop = sla.solve_triangular(L, sla.solve_triangular(L, D.Sdag, lower=True).T, lower=True).T
    q = sla.solve_triangular(L, b[:, 0], lower=True)
    q /= np.linalg.norm(q)
    Q = [q]
    al, be = [], []
    qprev, bprev = np.zeros_like(q), 0.0
    for j in range(k):
        w = Aop @ Q[-1] - bprev * qprev
        a = Q[-1] @ w
        w -= a * Q[-1]
        for qq in Q:                     # full reorthogonalisation
            w -= (qq @ w) * qq
        al.append(a)
        bb = np.linalg.norm(w)
        be.append(bb)
        qprev, bprev = Q[-1], bb
        Q.append(w / bb)
    assert np.allclose(res["diag"][0], al, rtol=1e-8)
    assert np.allclose(res["off"][0], be[:k - 1], rtol=1e-7)


def test_slq_and_ste_with_full_basis_probes_are_exact():
    """With probes z_i = sqrt(n) L e_i (P_hat = L L^T, i = 1..n) and full
    convergence, the SLQ sum is exactly logdet(P^-1/2 Sdag P^-1/2) (start
    vectors e_i) and the STE is exactly tr(Sdag^-1 dSdag) (sum z z^T = n P_hat),
    so the iterative log-likelihood and gradient equal the dense ones."""
    locs, ind, g, nu, th = _problem(n=70, m=9, nu=1.5, theta=(0.9, 0.2, 0.15), gamma=0.15)
    D = O.DenseFSA(locs, ind, g, nu, th)
    It = O.IterativeFSA(locs, ind, g, nu, th)
    y = np.random.default_rng(6).standard_normal(70)
    Z = math.sqrt(70) * np.linalg.cholesky(D.Phat)
    out = It.loglik_grad(y, 70, 0, 1e-13, max_iter=400, Z=Z)
    ll, logdet, _ = D.loglik(y)
    assert abs(out["logdet"] - logdet) < 1e-8 * abs(logdet)
    assert abs(out["loglik"] - ll) < 1e-8 * abs(ll)
    assert np.allclose(out["grad"], D.grad(y), rtol=1e-7, atol=1e-8)


def test_slq_exact_weight_with_an_unequal_norm_tight_frame_is_exact():
    """Probes z_i = L v_i (P_hat = L L^T) whose v_i form a tight frame,
    (1/l) sum v_i v_i^T = I, with unequal norms: at full convergence the
    exact-weight SLQ sum (1/l) sum |v_i|^2 e_1^T log(T_i) e_1 is exactly
    tr log(L^-1 Sdag L^-T), so the log-determinant is exact, while the paper's
    weight n is not (the norms differ)."""
    n, l = 60, 120
    locs, ind, g, nu, th = _problem(n=n, m=8, nu=1.5, theta=(0.9, 0.2, 0.15), gamma=0.15)
    D = O.DenseFSA(locs, ind, g, nu, th)
    It = O.IterativeFSA(locs, ind, g, nu, th)
    V0 = np.random.default_rng(3).standard_normal((n, l))
    w, Q = np.linalg.eigh(V0 @ V0.T)
    V = math.sqrt(l) * (Q / np.sqrt(w)) @ Q.T @ V0
    assert np.allclose(V @ V.T / l, np.eye(n), atol=1e-12)
    Z = np.linalg.cholesky(D.Phat) @ V
    y = np.random.default_rng(6).standard_normal(n)
    _, logdet, _ = D.loglik(y)
    ew = It.loglik_grad(y, l, 0, 1e-13, max_iter=400, Z=Z, exact_weight=True, want_grad=False)
    assert abs(ew["logdet"] - logdet) < 1e-9 * abs(logdet)
    nw = It.loglik_grad(y, l, 0, 1e-13, max_iter=400, Z=Z, want_grad=False)
    assert abs(nw["logdet"] - logdet) > 1e-3


def test_dense_gradient_matches_central_differences():
    locs, ind, g, nu, th = _problem(n=80, m=10, nu=0.5)
    y = np.random.default_rng(7).standard_normal(80)
    gd = O.DenseFSA(locs, ind, g, nu, th).grad(y)
    for k in range(3):
        h = 1e-5 * th[k]
        tp = list(th); tp[k] += h
        tm = list(th); tm[k] -= h
        fd = (O.DenseFSA(locs, ind, g, nu, tp).loglik(y)[0] - O.DenseFSA(locs, ind, g, nu, tm).loglik(y)[0]) / (2 * h)
        assert abs(fd - gd[k]) < 1e-6 * max(1.0, abs(gd[k]))


def test_euler_homogeneity_of_gradient():
    """Sdag(t s1, rho, t nug) = t Sdag: s1 dl/ds1 + nug dl/dnug = -(n - y^T Sdag^-1 y)/2."""
    locs, ind, g, nu, th = _problem(n=90, m=11, nu=1.5)
    y = np.random.default_rng(8).standard_normal(90)
    F = O.DenseFSA(locs, ind, g, nu, th)
    gr = F.grad(y)
    q = float(y @ np.linalg.solve(F.Sdag, y))
    assert abs(th[0] * gr[0] + th[2] * gr[2] + 0.5 * (90 - q)) < 1e-8 * 90


def test_random_probe_estimates_within_standard_error():
    locs, ind, g, nu, th = _problem(n=400, m=25, gamma=0.08)
    D = O.DenseFSA(locs, ind, g, nu, th)
    It = O.IterativeFSA(locs, ind, g, nu, th)
    y = np.linalg.cholesky(D.Sdag) @ np.random.default_rng(9).standard_normal(400)
    out = It.loglik_grad(y, 200, 123, 1e-10)
    ll, logdet, quad = D.loglik(y)
    assert abs(out["quad"] - quad) < 1e-7 * quad
    assert abs(out["logdet"] - logdet) < 4 * out["logdet_se"] + 1e-9
    gd = D.grad(y)
    se = np.std(out["grad_terms"], axis=1, ddof=1) / math.sqrt(200) * 0.5
    assert np.all(np.abs(out["grad"] - gd) < 4 * se + 1e-9)


# --------------------------------------------------------------------------
# predictive distribution
# --------------------------------------------------------------------------

def test_dense_prediction_m_equals_n_is_kriging():
    n = 50
    locs = fi.uniform_locations(n, 12)
    pred = fi.uniform_locations(20, 12, stream=7)
    th = (1.0, 0.1, 0.2)
    y = np.random.default_rng(10).standard_normal(n)
    F = O.DenseFSA(locs, locs, 0.05, 0.5, th)
    mu, var = F.predict(y, pred)
    S = th[0] * np.exp(-np.sqrt(O.sqdist(locs, locs)) / th[1]) + th[2] * np.eye(n)
    Snp = th[0] * np.exp(-np.sqrt(O.sqdist(locs, pred)) / th[1])
    assert np.allclose(mu, Snp.T @ np.linalg.solve(S, y), atol=1e-8)
    assert np.allclose(var, th[0] + th[2] - np.sum(Snp * np.linalg.solve(S, Snp), 0), atol=1e-8)


def test_algorithm1_with_full_basis_probes_is_exact():
    """Algorithm 1 with 'probes' sqrt(s) e_j (s = n_p) gives the exact diagonal,
    so its variances equal the dense exact FSA variances (Proposition 1)."""
    locs, ind, g, nu, th = _problem(n=120, m=15)
    pred = fi.uniform_locations(30, 3, stream=7)
    y = np.random.default_rng(11).standard_normal(120)
    D = O.DenseFSA(locs, ind, g, nu, th)
    It = O.IterativeFSA(locs, ind, g, nu, th)
    mu, var = D.predict(y, pred)
    out = It.predict(y, pred, 30, 0, 1e-12, Zp=math.sqrt(30) * np.eye(30))
    assert np.allclose(out["mean"], mu, atol=1e-8)
    assert np.allclose(out["var"], var, atol=1e-8)


def test_algorithm1_random_probes_unbiased_within_tolerance():
    locs, ind, g, nu, th = _problem(n=200, m=20)
    pred = fi.uniform_locations(60, 4, stream=7)
    y = np.random.default_rng(12).standard_normal(200)
    D = O.DenseFSA(locs, ind, g, nu, th)
    It = O.IterativeFSA(locs, ind, g, nu, th)
    _, var = D.predict(y, pred)
    s = 400
    out = It.predict(y, pred, s, 77, 1e-12)
    # Rademacher diagonal estimator: Var[D_l,j] = (1/s) sum_{k != j} A_jk^2
    C, _, Ssnp, _ = D.cross(pred)
    Amat = Ssnp.T @ np.linalg.solve(D.Ss, Ssnp)
    sd = np.sqrt((np.sum(Amat ** 2, 1) - np.diag(Amat) ** 2) / s)
    assert np.all(np.abs(out["var"] - var) <= 5 * sd + 1e-9)


def test_algorithm1_gaussian_probes_unbiased_with_the_gaussian_variance():
    """Gaussian probes: z_j (A z)_j has mean A_jj and variance
    sum_k A_jk^2 + A_jj^2 (E z^4 = 3), so each point's D_l error stays within 5
    of those standard deviations and their root mean square over the points is
    near 1 (Algorithm 1 with N(0, I) probes)."""
    locs, ind, g, nu, th = _problem(n=200, m=20)
    pred = fi.uniform_locations(60, 4, stream=7)
    y = np.random.default_rng(12).standard_normal(200)
    D = O.DenseFSA(locs, ind, g, nu, th)
    It = O.IterativeFSA(locs, ind, g, nu, th)
    _, var = D.predict(y, pred)
    s = 400
    out = It.predict(y, pred, s, 78, 1e-12, probe="gaussian")
    _, _, Ssnp, _ = D.cross(pred)
    Amat = Ssnp.T @ np.linalg.solve(D.Ss, Ssnp)
    sd = np.sqrt((np.sum(Amat ** 2, 1) + np.diag(Amat) ** 2) / s)
    zsc = (out["var"] - var) / sd
    assert np.all(np.abs(zsc) <= 5)
    assert 0.6 < np.sqrt(np.mean(zsc ** 2)) < 1.5


def test_control_variate_with_full_basis_probes_stays_exact():
    """With probes sqrt(s) e_j the sample mean of b_k = z_k o (S P_s^-1 S^T z_k)
    equals diag(S P_s^-1 S^T) exactly, so the control-variate estimator of D_l
    (appendix "Preconditioner as control variate") stays exact for any c."""
    locs, ind, g, nu, th = _problem(n=120, m=15)
    pred = fi.uniform_locations(30, 3, stream=7)
    y = np.random.default_rng(11).standard_normal(120)
    _, var = O.DenseFSA(locs, ind, g, nu, th).predict(y, pred)
    It = O.IterativeFSA(locs, ind, g, nu, th)
    for cv in ("copt", "c1"):
        out = It.predict(y, pred, 30, 0, 1e-12, Zp=math.sqrt(30) * np.eye(30), control_variate=cv)
        assert np.allclose(out["var"], var, atol=1e-8)


def test_control_variate_c1_unbiased_with_reduced_variance():
    """c = 1: D_l = mean(a - b) + diag(S P_s^-1 S^T) is unbiased, and for
    Rademacher probes Var[D_l,p] = (1/s) sum_{k != p} (A - B)_pk^2 with
    A = S Sigma_s~^-1 S^T and B = S D_s^-1 S^T (built densely here)."""
    locs, ind, g, nu, th = _problem(n=200, m=20)
    pred = fi.uniform_locations(60, 4, stream=7)
    y = np.random.default_rng(12).standard_normal(200)
    D = O.DenseFSA(locs, ind, g, nu, th)
    It = O.IterativeFSA(locs, ind, g, nu, th)
    _, var = D.predict(y, pred)
    s = 400
    out = It.predict(y, pred, s, 77, 1e-12, control_variate="c1")
    _, _, Ssnp, _ = D.cross(pred)
    Amat = Ssnp.T @ np.linalg.solve(D.Ss, Ssnp)
    Bmat = Ssnp.T @ (Ssnp / np.diag(D.Ss)[:, None])
    E = Amat - Bmat
    sd_cv = np.sqrt((np.sum(E ** 2, 1) - np.diag(E) ** 2) / s)
    sd_plain = np.sqrt((np.sum(Amat ** 2, 1) - np.diag(Amat) ** 2) / s)
    assert np.all(np.abs(out["var"] - var) <= 5 * sd_cv + 1e-9)
    assert np.all(out["c"] == 1.0)
    # the diagonal preconditioner captures most of the estimator's variance here
    assert np.mean(sd_cv) < 0.7 * np.mean(sd_plain)


def test_control_variate_copt_is_the_least_squares_coefficient():
    """c_opt of each point is the least-squares slope of (a_k - mean a) on b_k
    through the origin, i.e. the c minimising sum_k (a_k - mean a - c b_k)^2."""
    locs, ind, g, nu, th = _problem(n=150, m=20)
    pred = fi.uniform_locations(25, 5, stream=7)
    y = np.random.default_rng(13).standard_normal(150)
    It = O.IterativeFSA(locs, ind, g, nu, th)
    s = 12
    Zp = O.rademacher(9, O.STREAM_PRED, np.arange(25), 25, s)
    out = It.predict(y, pred, s, 9, 1e-12, Zp=Zp, control_variate="copt")
    plain = It.predict(y, pred, s, 9, 1e-12, Zp=Zp)
    _, St, _ = It.cross_structures(pred)
    X = np.linalg.solve(It.Ss.toarray(), St.T @ Zp)
    a = Zp * (St @ X)
    b = Zp * (St @ ((St.T @ Zp) / It.D[:, None]))
    for p in range(25):
        if np.sum(b[p] ** 2) == 0:
            assert out["c"][p] == 0.0
            continue
        slope = np.linalg.lstsq(b[p][:, None], a[p] - a[p].mean(), rcond=None)[0][0]
        assert abs(out["c"][p] - slope) <= 1e-8 * (1 + abs(slope))
    # the plain estimate is the c = 0 member of the family
    assert np.allclose(plain["Dl"], a.mean(1), atol=1e-10)


def test_iteration_trends_in_m_with_and_without_fitc():
    """§4 (Table 1 and the iteration figure): with the FITC preconditioner CG
    needs far fewer iterations than without, and the count falls as m grows,
    while without a preconditioner it rises (effective range 0.2)."""
    n = 2000
    locs = fi.uniform_locations(n, 11)
    b = np.random.default_rng(1).standard_normal((n, 1))
    fitc, none = [], []
    for m in (10, 40, 160):
        ind = locs[fi.inducing_subset(n, m, 11)].copy()
        It = O.IterativeFSA(locs, ind, 0.05, 0.5, (1.0, 0.2 / 3, 0.05))
        fitc.append(int(O.pcg_lanczos(It.apply, It.apply_Pinv, b, 1e-6, 5000)["iters"][0]))
        none.append(int(O.pcg_lanczos(It.apply, lambda V: V.copy(), b, 1e-6, 5000)["iters"][0]))
    assert fitc[0] > fitc[1] > fitc[2]
    assert none[0] < none[1] < none[2]
    assert all(f < 0.75 * u for f, u in zip(fitc, none))


# --------------------------------------------------------------------------
# preconditioner derivative and the gradient control variate (appendix
# "Preconditioner as control variate", Eq. Troptc)
# --------------------------------------------------------------------------

def test_fitc_derivative_and_trace_match_finite_differences():
    """dP_hat from central differences of the dense P_hat(theta); the O(n m^2)
    Tr(P_hat^-1 dP_hat) from Jacobi's formula d logdet P_hat (central
    differences of a dense slogdet) and from a dense solve."""
    locs, ind, g, nu, th = _problem(n=90, m=11, nu=1.5)
    D = O.DenseFSA(locs, ind, g, nu, th)
    It = O.IterativeFSA(locs, ind, g, nu, th)
    V = np.random.default_rng(14).standard_normal((90, 3))
    for k in range(3):
        h = 1e-5 * th[k]
        tp = list(th); tp[k] += h
        tm = list(th); tm[k] -= h
        Pp, Pm = O.DenseFSA(locs, ind, g, nu, tp).Phat, O.DenseFSA(locs, ind, g, nu, tm).Phat
        dP = D.dPhat(k)
        assert np.max(np.abs((Pp - Pm) / (2 * h) - dP)) < 1e-7 * max(1.0, np.max(np.abs(dP)))
        assert np.allclose(It.dP_apply(k, V), dP @ V, rtol=1e-11, atol=1e-11)
        tr = It.trace_Pinv_dP(k)
        jac = (np.linalg.slogdet(Pp)[1] - np.linalg.slogdet(Pm)[1]) / (2 * h)
        assert abs(tr - jac) < 1e-7 * max(1.0, abs(tr))
        assert abs(tr - np.trace(np.linalg.solve(D.Phat, dP))) < 1e-10 * max(1.0, abs(tr))


def test_gradient_control_variate_with_full_basis_probes_stays_exact():
    """With probes z_i = sqrt(n) L e_i (P_hat = L L^T) the mean of
    b_i = z_i^T P^-1 dP P^-1 z_i is exactly Tr(P_hat^-1 dP_hat), so every
    control-variate coefficient leaves the STE gradient exact."""
    locs, ind, g, nu, th = _problem(n=70, m=9, nu=1.5, theta=(0.9, 0.2, 0.15), gamma=0.15)
    D = O.DenseFSA(locs, ind, g, nu, th)
    It = O.IterativeFSA(locs, ind, g, nu, th)
    y = np.random.default_rng(6).standard_normal(70)
    Z = math.sqrt(70) * np.linalg.cholesky(D.Phat)
    gd = D.grad(y)
    for cv in ("c1", "copt", "copt_centered"):
        out = It.loglik_grad(y, 70, 0, 1e-13, max_iter=400, Z=Z, control_variate=cv)
        assert np.allclose(out["grad"], gd, rtol=1e-7, atol=1e-8)
        assert np.allclose(out["trace_P"], [np.trace(np.linalg.solve(D.Phat, D.dPhat(k))) for k in range(3)],
                           rtol=1e-9)


def test_gradient_control_variate_c1_exact_when_fsa_equals_fitc():
    """gamma below every pair distance: Sigma_dag = P_hat for every theta, so
    a_i = b_i and the c = 1 estimate is Tr(P_hat^-1 dP_hat) = Tr(Sdag^-1 dSdag)
    for any probes; the plain estimate is not."""
    locs, ind, _, nu, th = _problem(n=80, m=10)
    It = O.IterativeFSA(locs, ind, 1e-6, nu, th)
    D = O.DenseFSA(locs, ind, 1e-6, nu, th)
    y = np.random.default_rng(3).standard_normal(80)
    gd = D.grad(y)
    out = It.loglik_grad(y, 5, 1, 1e-12, control_variate="c1")
    assert np.allclose(out["grad"], gd, rtol=1e-9, atol=1e-9)
    plain = It.loglik_grad(y, 5, 1, 1e-12)
    assert np.max(np.abs(plain["grad"] - gd)) > 1e-3


def test_ste_gradient_euler_homogeneity_with_the_same_probes():
    """Sdag and P_hat are homogeneous of degree 1 in (s1, nugget), so
    s1 dSdag_0 + nug dSdag_2 = Sdag and s1 dP_0 + nug dP_2 = P_hat: the plain
    STE gives s1 g_0 + nug g_2 = -1/2 (mean_k z_k^T P^-1 z_k - y^T u), the c = 1
    control variate the exact -1/2 (n - y^T u), and
    s1 Tr(P^-1 dP_0) + nug Tr(P^-1 dP_2) = n."""
    locs, ind, g, nu, th = _problem(n=300, m=20, gamma=0.1)
    It = O.IterativeFSA(locs, ind, g, nu, th)
    D = O.DenseFSA(locs, ind, g, nu, th)
    y = np.random.default_rng(4).standard_normal(300)
    plain = It.loglik_grad(y, 8, 5, 1e-11)
    cv = It.loglik_grad(y, 8, 5, 1e-11, control_variate="c1")
    Z = plain["Z"]
    zPz = float(np.mean(np.einsum("ij,ij->j", Z, np.linalg.solve(D.Phat, Z))))
    lhs = lambda gr: th[0] * gr[0] + th[2] * gr[2]
    assert abs(lhs(plain["grad"]) + 0.5 * (zPz - plain["quad"])) < 1e-8 * 300
    assert abs(lhs(cv["grad"]) + 0.5 * (300 - cv["quad"])) < 1e-8 * 300
    assert abs(lhs(cv["trace_P"]) - 300) < 1e-9 * 300


def test_gradient_control_variate_coefficients_are_least_squares_slopes():
    """Per parameter, with a_i = U_i^T dSdag W_i and b_i = W_i^T dP_hat W_i
    built from dense solves: c_opt as printed is the slope of (a - mean a) on b
    through the origin; the centred coefficient is the ordinary least-squares
    slope of a on b (intercept free)."""
    locs, ind, g, nu, th = _problem(n=150, m=20)
    D = O.DenseFSA(locs, ind, g, nu, th)
    It = O.IterativeFSA(locs, ind, g, nu, th)
    y = np.random.default_rng(15).standard_normal(150)
    l = 12
    Z = It.probes(l, 21)
    U = np.linalg.solve(D.Sdag, Z)
    W = np.linalg.solve(D.Phat, Z)
    o1 = It.loglik_grad(y, l, 21, 1e-12, Z=Z, control_variate="copt")
    o2 = It.loglik_grad(y, l, 21, 1e-12, Z=Z, control_variate="copt_centered")
    for k in range(3):
        a = np.einsum("ij,ij->j", U, D.dSdag(k) @ W)
        b = np.einsum("ij,ij->j", W, D.dPhat(k) @ W)
        c1 = np.linalg.lstsq(b[:, None], a - a.mean(), rcond=None)[0][0]
        c2 = np.polyfit(b, a, 1)[0]
        assert abs(o1["cv_c"][k] - c1) <= 1e-6 * (1 + abs(c1))
        assert abs(o2["cv_c"][k] - c2) <= 1e-6 * (1 + abs(c2))


def test_gradient_control_variate_c1_unbiased_with_reduced_error():
    """Over 40 probe seeds of 10 probes each, the c = 1 gradient stays within
    4 standard errors of the exact gradient, and its error in the range
    derivative is well below that of the plain STE (§4: the FITC control
    variate reduces the variance of the gradient estimate)."""
    locs, ind, g, nu, th = _problem(n=400, m=25, gamma=0.08)
    D = O.DenseFSA(locs, ind, g, nu, th)
    It = O.IterativeFSA(locs, ind, g, nu, th)
    y = np.linalg.cholesky(D.Sdag) @ np.random.default_rng(9).standard_normal(400)
    gd = D.grad(y)
    cv = np.array([It.loglik_grad(y, 10, s, 1e-10, control_variate="c1")["grad"] for s in range(40)])
    plain = np.array([It.loglik_grad(y, 10, s, 1e-10)["grad"] for s in range(40)])
    se = cv.std(axis=0, ddof=1) / math.sqrt(40)
    assert np.all(np.abs(cv.mean(axis=0) - gd) < 4 * se)
    rmse = lambda a: np.sqrt(np.mean((a - gd) ** 2, axis=0))
    assert rmse(cv)[1] < 0.5 * rmse(plain)[1]


# --------------------------------------------------------------------------
# Fisher information by STE (appendix "Fisher scoring")
# --------------------------------------------------------------------------

def test_dense_fisher_is_the_expected_negative_hessian():
    """I = -Hessian of E_y[l(theta; y)] = -1/2 [logdet Sdag(theta) +
    tr(Sdag(theta)^-1 Sdag(theta0))] + const at theta0 (y ~ N(0, Sdag(theta0))),
    by central second differences of dense slogdet / solve; the nugget entry is
    1/2 sum_i 1/lambda_i^2 over the eigenvalues of Sdag."""
    locs, ind, g, nu, th = _problem(n=64, m=8, nu=1.5, theta=(0.9, 0.2, 0.15), gamma=0.15)
    D = O.DenseFSA(locs, ind, g, nu, th)
    F = D.fisher()
    lam = np.linalg.eigvalsh(D.Sdag)
    assert abs(F[2, 2] - 0.5 * np.sum(lam ** -2.0)) < 1e-10 * F[2, 2]

    def f(t):
        S = O.DenseFSA(locs, ind, g, nu, t).Sdag
        return -0.5 * (np.linalg.slogdet(S)[1] + np.trace(np.linalg.solve(S, D.Sdag)))

    for k in range(3):
        for j in range(3):
            hk, hj = 1e-3 * th[k], 1e-3 * th[j]

            def at(a, b):
                t = list(th); t[k] += a; t[j] += b
                return f(t)

            hess = (at(hk, hj) - at(hk, -hj) - at(-hk, hj) + at(-hk, -hj)) / (4 * hk * hj)
            assert abs(-hess - F[k, j]) < 2e-5 * np.max(np.abs(F))


def test_fisher_ste_with_hadamard_probes_is_exact():
    """Sylvester-Hadamard probes (entries +-1, H H^T = n I) make the STE sum
    the exact trace, so the estimate equals the dense Fisher information."""
    locs, ind, g, nu, th = _problem(n=64, m=8, nu=1.5, theta=(0.9, 0.2, 0.15), gamma=0.15)
    F = O.DenseFSA(locs, ind, g, nu, th).fisher()
    It = O.IterativeFSA(locs, ind, g, nu, th)
    out = It.fisher_ste(64, 0, 1e-12, Z=sla.hadamard(64).astype(np.float64))
    assert np.allclose(out["fisher_raw"], F, rtol=1e-9, atol=1e-9)
    assert np.allclose(out["fisher"], F, rtol=1e-9, atol=1e-9)


def test_fisher_ste_random_probes_within_standard_error():
    locs, ind, g, nu, th = _problem(n=400, m=25, gamma=0.08)
    F = O.DenseFSA(locs, ind, g, nu, th).fisher()
    out = O.IterativeFSA(locs, ind, g, nu, th).fisher_ste(100, 3, 1e-10)
    assert set(np.unique(out["Z"])) == {-1.0, 1.0}
    se = out["terms"].std(axis=2, ddof=1) / math.sqrt(100)
    assert np.all(np.abs(out["fisher_raw"] - F) < 4 * se)
    assert np.allclose(out["fisher"], out["fisher"].T)
    assert np.all(np.linalg.eigvalsh(out["fisher"]) > 0)


def test_fisher_scoring_converges_to_the_maximum_likelihood_estimate():
    """Fisher scoring with the dense gradient and Fisher information reaches
    the maximiser of the dense log-likelihood found independently by L-BFGS-B
    (the optimiser of §4), from a start 20-30 % off in every parameter."""
    n, m = 150, 20
    locs = fi.uniform_locations(n, 81)
    ind = locs[fi.inducing_subset(n, m, 81)].copy()
    g, nu, th0 = 0.15, 1.5, (1.0, 0.1, 0.1)
    y = np.linalg.cholesky(O.DenseFSA(locs, ind, g, nu, th0).Sdag) @ np.random.default_rng(81).standard_normal(n)

    def negll(p):
        D = O.DenseFSA(locs, ind, g, nu, tuple(np.exp(p)))
        return -D.loglik(y)[0], -D.grad(y) * np.exp(p)

    r = so.minimize(negll, np.log(th0), jac=True, method="L-BFGS-B",
                    options=dict(ftol=1e-15, gtol=1e-10, maxiter=500))
    mle = np.exp(r.x)
    th = mle * np.array([1.3, 0.8, 1.2])
    for _ in range(15):
        D = O.DenseFSA(locs, ind, g, nu, tuple(th))
        th = O.fisher_scoring_step(th, D.grad(y), D.fisher())
    assert np.max(np.abs(th / mle - 1)) < 1e-6


# --------------------------------------------------------------------------
# the FITC preconditioner for a Vecchia approximation (§5)
# --------------------------------------------------------------------------

def _vecchia(n=200, m=20, m_v=8, theta=(1.0, 0.1, 0.05), seed=3):
    locs = fi.uniform_locations(n, seed)
    ind = locs[fi.inducing_subset(n, m, seed)].copy()
    return locs, ind, O.VecchiaFITC(locs, ind, m_v, 0.5, theta)


def test_vecchia_factor_matches_its_definition():
    """B unit lower triangular with B_{i,N(i)} = -A_i over the min(m_v, i-1)
    nearest earlier points (brute force), Sigma_V = (B^T D^-1 B)^-1 applied by
    the two triangular solves, and log det Sigma_V = sum log D_i (det B = 1)."""
    locs, ind, V = _vecchia()
    n = locs.shape[0]
    B = V.B.toarray()
    assert np.array_equal(np.diag(B), np.ones(n)) and np.all(np.triu(B, 1) == 0)
    for i in (0, 1, 5, 8, 9, 57, 199):
        d2 = np.array([np.sum((locs[i] - locs[j]) ** 2) for j in range(i)])
        want = set(np.argsort(d2, kind="stable")[:min(8, i)].tolist())
        assert set(np.nonzero(B[i, :i])[0].tolist()) <= want and len(V.N[i]) == min(8, i)
        assert set(V.N[i].tolist()) == want
    SV = np.linalg.inv(B.T @ np.diag(1.0 / V.D) @ B)
    x = np.random.default_rng(1).standard_normal((n, 3))
    assert np.allclose(V.apply_SigmaV(x), SV @ x, rtol=1e-10, atol=1e-10)
    assert abs(np.linalg.slogdet(SV)[1] - np.sum(np.log(V.D))) < 1e-10 * n


def test_vecchia_is_exact_where_the_conditioning_loses_nothing():
    """m_v = n - 1 conditions on every earlier point: Sigma_V = Sigma.  The
    exponential covariance on sorted points of a line is a Markov (Ornstein-
    Uhlenbeck) process: m_v = 1 is already exact.  m_v = 0: Sigma_V = diag(Sigma)."""
    th = (1.0, 0.1, 0.05)
    locs = fi.uniform_locations(60, 3)
    full = O.VecchiaFITC(locs, locs[:5], 59, 0.5, th)
    Sig = O.cov_matrix(locs, locs, 0.5, 1.0, 0.1)
    assert np.allclose(full.apply_SigmaV(np.eye(60)), Sig, atol=1e-12)
    xs = np.sort(np.random.default_rng(2).random(80))
    line = np.column_stack([xs, np.full(80, 0.3)])
    ou = O.VecchiaFITC(line, line[:4], 1, 0.5, th)
    assert np.allclose(ou.apply_SigmaV(np.eye(80)), O.cov_matrix(line, line, 0.5, 1.0, 0.1), atol=1e-12)
    none = O.VecchiaFITC(locs, locs[:5], 0, 0.5, th)
    assert np.allclose(none.apply_SigmaV(np.eye(60)), np.eye(60), atol=1e-15)


def test_vecchia_fitc_preconditioner_and_posterior_solve():
    """P_hat = Sigma_l + diag(Sigma - Sigma_l) + nugget I from dense
    definitions; the posterior solve equals (Sigma_V^-1 + W)^-1 v, which the
    printed form W (Sigma_V + W^-1)^-1 Sigma_V^-1 v of Eq. VL_v2 does not."""
    locs, ind, V = _vecchia()
    n, nug = locs.shape[0], 0.05
    K = O.cov_matrix(ind, locs, 0.5, 1.0, 0.1)
    Sl = K.T @ np.linalg.solve(O.cov_matrix(ind, ind, 0.5, 1.0, 0.1), K)
    P = Sl + np.diag(np.diag(O.cov_matrix(locs, locs, 0.5, 1.0, 0.1) - Sl) + nug)
    x = np.random.default_rng(4).standard_normal((n, 2))
    assert np.allclose(V.apply_Pinv(x), np.linalg.solve(P, x), rtol=1e-10, atol=1e-10)
    assert abs(V.logdet_P - np.linalg.slogdet(P)[1]) < 1e-10 * n
    SV = V.apply_SigmaV(np.eye(n))
    want = np.linalg.solve(np.linalg.inv(SV) + np.eye(n) / nug, x)
    got, iters = V.posterior_solve(x, 1e-12)
    assert np.allclose(got, want, rtol=1e-9, atol=1e-10)
    printed = (np.linalg.solve(SV + nug * np.eye(n), np.linalg.solve(SV, x))) / nug
    assert np.max(np.abs(printed - want)) > 1e-2 * np.max(np.abs(want))


def test_vecchia_loglik_by_slq_exact_with_full_basis_probes_and_within_se():
    locs, ind, V = _vecchia()
    n = locs.shape[0]
    C = V.apply_SigmaV(np.eye(n)) + 0.05 * np.eye(n)
    y = np.linalg.cholesky(C) @ np.random.default_rng(5).standard_normal(n)
    ll = -0.5 * (n * O.LOG2PI + np.linalg.slogdet(C)[1] + y @ np.linalg.solve(C, y))
    K = O.cov_matrix(ind, locs, 0.5, 1.0, 0.1)
    Sl = K.T @ np.linalg.solve(O.cov_matrix(ind, ind, 0.5, 1.0, 0.1), K)
    P = Sl + np.diag(np.diag(O.cov_matrix(locs, locs, 0.5, 1.0, 0.1) - Sl) + 0.05)
    out = V.loglik(y, n, 0, 1e-12, Z=math.sqrt(n) * np.linalg.cholesky(P))
    assert abs(out["loglik"] - ll) < 1e-9 * abs(ll)
    Z = V.probes(60, 7)
    r = V.loglik(y, 60, 7, 1e-10, Z=Z)
    terms = []
    for k in range(60):
        rk = O.pcg_lanczos(V.apply, V.apply_Pinv, Z[:, k:k + 1], 1e-10, 5000)
        terms.append(n * O.lanczos_quadrature(rk["diag"][0], rk["off"][0]))
    se = np.std(terms, ddof=1) / math.sqrt(60)
    assert abs(r["logdet"] - np.linalg.slogdet(C)[1]) < 4 * se


def test_vecchia_fitc_iterations_fall_with_m():
    """§5.2: the FITC preconditioner speeds up CG for the Vecchia system; with
    more inducing points it needs fewer iterations (effective range 0.2)."""
    n = 1500
    locs = fi.uniform_locations(n, 13)
    x = np.random.default_rng(2).standard_normal((n, 1))
    fitc, none = [], []
    for m in (10, 50, 200):
        V = O.VecchiaFITC(locs, locs[fi.inducing_subset(n, m, 13)].copy(), 10, 0.5, (1.0, 0.2 / 3, 0.05))
        fitc.append(int(V.posterior_solve(x, 1e-8)[1][0]))
        none.append(int(V.posterior_solve(x, 1e-8, precondition=False)[1][0]))
    assert fitc[0] > fitc[1] > fitc[2]
    assert fitc[2] < 0.6 * none[2] and none[0] == none[1] == none[2]


# --------------------------------------------------------------------------
# kmeans++ selection of inducing points (§4.1)
# --------------------------------------------------------------------------

def test_kmeanspp_distinct_and_first_uniform():
    locs = fi.uniform_locations(500, 21)
    idx = O.kmeanspp(locs, 60, 3)
    assert len(set(idx.tolist())) == 60                 # a chosen point has weight 0 afterwards
    h0 = int(O.splitmix64(3, O.STREAM_KMEANSPP, np.arange(1, dtype=np.uint64))[0]) >> 11
    assert idx[0] == (h0 * 500) >> 53
    with pytest.raises(ValueError):                     # three distinct points cannot give four
        O.kmeanspp(np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 0.0]]), 4, 1)


def test_kmeanspp_second_point_follows_d2_distribution():
    """Over many seeds the second point is drawn with probability proportional
    to its squared distance from the first (chi-square test, brute-force
    expected counts from the definition of D^2 sampling)."""
    locs = np.array([[0.0, 0.0], [0.1, 0.0], [0.3, 0.0], [0.6, 0.0], [1.0, 0.0]])
    counts = np.zeros((5, 5))
    for seed in range(6000):
        a, b = O.kmeanspp(locs, 2, seed)
        counts[a, b] += 1
    for a in range(5):
        d2 = (locs[:, 0] - locs[a, 0]) ** 2
        if counts[a].sum() < 200:
            continue
        exp = counts[a].sum() * d2 / d2.sum()
        keep = exp > 0
        chi2 = np.sum((counts[a, keep] - exp[keep]) ** 2 / exp[keep])
        assert st.chi2.sf(chi2, keep.sum() - 1) > 1e-4, (a, counts[a], exp)
        assert counts[a, a] == 0


def test_kmeanspp_integer_weights_are_exact_scaled_distances():
    """With a power-of-two scale the integer weights are floor(d^2 2^e) exactly;
    e keeps n * (bounding-box diagonal)^2 * 2^e below 2^62."""
    locs = fi.uniform_locations(1000, 22)
    e = O.kmeanspp_scale_exponent(locs)
    dx = locs[:, 0].max() - locs[:, 0].min()
    dy = locs[:, 1].max() - locs[:, 1].min()
    assert 1000 * (dx * dx + dy * dy) * 2.0 ** e <= 2.0 ** 62
    assert 1000 * (dx * dx + dy * dy) * 2.0 ** (e + 2) > 2.0 ** 62   # and is not needlessly small


def test_every_planted_mistake_of_the_sweep_still_applies():
    """The planted-mistake sweep (tests/oracle_mutation_sweep.py) stays in step with
    the oracle: each entry's original text occurs in the source, and its
    planted text differs from it."""
    import importlib.util
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("mutation_sweep", os.path.join(root, "tests", "oracle_mutation_sweep.py"))
    ms = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(ms)
    src = open(os.path.join(root, "oracle", "fsa_oracle.py")).read()
    assert len(ms.MUTATIONS) >= 60
    for label, old, new, _ in ms.MUTATIONS:
        assert old in src, label
        assert old != new, label
