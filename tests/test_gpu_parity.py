"""GPU-vs-oracle parity through the C ABI (FP64 form).

Bars: bit-exact neighbour structure; 1e-10 relative (norm-wise) for FP64
operator products and log det P_hat; 1e-6 relative for log det, log-likelihood
and gradient under identical probes and a fixed CG iteration count.
"""
import math

import numpy as np
import pytest

import fsa_inputs as fi
from oracle import fsa_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fsa():
    import paper_2405_14492_gb300 as F
    return F


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def _setup(n, m, nu, gamma, seed):
    locs = fi.uniform_locations(n, seed)
    idx = fi.inducing_subset(n, m, seed)
    return locs, locs[idx].copy()


# ---------------------------------------------------------------------------
# neighbour structure
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,gamma", [(2, 0.5), (3001, 0.03), (20011, 0.012), (100_003, 0.0045)])
def test_csr_bit_exact(fsa, n, gamma):
    locs = fi.uniform_locations(n, 21)
    with fsa.FSAHandle(locs, locs[:1], gamma) as h:
        rp, col = h.csr()
    rp0, col0 = O.neighbour_csr(locs, locs, gamma)
    assert np.array_equal(rp, rp0)
    assert np.array_equal(col, col0)


def test_csr_degenerate_layouts(fsa):
    # coincident points, a line of points (zero extent in y), taper wider than the domain
    cases = [np.tile([[0.3, 0.7]], (40, 1)),
             np.column_stack([np.linspace(0, 1, 500), np.full(500, 0.25)]),
             fi.uniform_locations(300, 3) * 0.01]
    for locs, g in zip(cases, (0.1, 0.011, 0.5)):
        with fsa.FSAHandle(locs, locs[:1], g) as h:
            rp, col = h.csr()
        rp0, col0 = O.neighbour_csr(locs, locs, g)
        assert np.array_equal(rp, rp0) and np.array_equal(col, col0)


# ---------------------------------------------------------------------------
# operator parity (FP64)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,m,nu,gamma", [(2000, 50, 0.5, 0.05), (9001, 130, 1.5, 0.03)])
def test_operator_parity_fp64(fsa, n, m, nu, gamma):
    locs, ind = _setup(n, m, nu, gamma, 31)
    th = (1.2, 0.08, 0.07)
    It = O.IterativeFSA(locs, ind, gamma, nu, th)
    V = np.random.default_rng(5).standard_normal((n, 3))
    with fsa.FSAHandle(locs, ind, gamma, nu) as h:
        assert _rel(h.matvec(th, V, 0), It.apply(V)) < 1e-10
        assert _rel(h.matvec(th, V, 1), It.apply_Pinv(V)) < 1e-10
        assert _rel(h.matvec(th, V, 2), It.Ss @ V) < 1e-10
        ld = h.logdet_precond(th)
    assert abs(ld - It.logdet_P) < 1e-10 * abs(It.logdet_P)


# ---------------------------------------------------------------------------
# log-likelihood and gradient parity (same probes, fixed iterations)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,m,nu,gamma,l,K", [(2000, 50, 0.5, 0.05, 20, 25), (6007, 97, 1.5, 0.025, 9, 18)])
def test_loglik_grad_parity_fixed_iters(fsa, n, m, nu, gamma, l, K):
    locs, ind = _setup(n, m, nu, gamma, 41)
    th = (1.0, 0.1, 0.1) if nu == 0.5 else (0.8, 0.05, 0.05)
    y = fi.random_field(locs, nu, th[0], th[1], th[2], 41)
    It = O.IterativeFSA(locs, ind, gamma, nu, th)
    ref = It.loglik_grad(y, l, 777, 0.0, fixed_iters=K)
    with fsa.FSAHandle(locs, ind, gamma, nu) as h:
        ll, g, info = h.loglik_grad(y, th, fsa.make_opts(num_probes=l, fixed_iters=K, seed=777))
    assert abs(info["logdet"] - ref["logdet"]) < 1e-6 * abs(ref["logdet"])
    assert abs(ll - ref["loglik"]) < 1e-6 * abs(ref["loglik"])
    assert abs(info["quad_form"] - ref["quad"]) < 1e-6 * abs(ref["quad"])
    assert _rel(g, ref["grad"]) < 1e-6


def test_loglik_grad_parity_tolerance_mode(fsa):
    """Config-1 shape (n = 2000, m = 50, exponential, gamma = 0.05, l = 20, tol 1e-8)."""
    w = fi.SMALL_EXP_N2K
    locs, ind, _, _, _ = w.make(with_response=False)
    th = (w.sigma1_sq, w.rho, w.nugget)
    D = O.DenseFSA(locs, ind, w.gamma, w.nu, th)
    y = np.linalg.cholesky(D.Sdag) @ np.random.default_rng(w.seed).standard_normal(w.n)
    It = O.IterativeFSA(locs, ind, w.gamma, w.nu, th)
    ref = It.loglik_grad(y, w.num_probes, w.seed, w.cg_tol)
    with fsa.FSAHandle(locs, ind, w.gamma, w.nu) as h:
        ll, g, info = h.loglik_grad(y, th, fsa.make_opts(num_probes=w.num_probes, cg_tol=w.cg_tol, seed=w.seed))
    assert info["converged"] == 1
    assert abs(ll - ref["loglik"]) < 1e-6 * abs(ref["loglik"])
    assert _rel(g, ref["grad"]) < 1e-6
    # statistical agreement with the dense Cholesky log-likelihood / gradient
    ll_d, logdet_d, quad_d = D.loglik(y)
    assert abs(info["quad_form"] - quad_d) < 1e-6 * quad_d
    assert abs(info["logdet"] - logdet_d) < 4 * info["logdet_se"]


def test_exact_weight_and_gaussian_probes(fsa):
    locs, ind = _setup(1500, 40, 0.5, 0.06, 51)
    th = (1.0, 0.1, 0.1)
    y = fi.random_field(locs, 0.5, *th, 51)
    It = O.IterativeFSA(locs, ind, 0.06, 0.5, th)
    ref = It.loglik_grad(y, 8, 99, 0.0, fixed_iters=20, probe="gaussian", exact_weight=True)
    with fsa.FSAHandle(locs, ind, 0.06, 0.5) as h:
        ll, g, info = h.loglik_grad(y, th, fsa.make_opts(num_probes=8, fixed_iters=20, seed=99,
                                                         probe=fsa.FSA_PROBE_GAUSSIAN, slq_exact_weight=True))
    assert abs(ll - ref["loglik"]) < 1e-6 * abs(ref["loglik"])
    assert _rel(g, ref["grad"]) < 1e-6


def test_error_paths(fsa):
    locs, ind = _setup(500, 20, 0.5, 0.05, 61)
    y = np.random.default_rng(0).standard_normal(500)
    with fsa.FSAHandle(locs, ind, 0.05) as h:
        with pytest.raises(fsa.FsaError) as e:
            h.loglik_grad(y, (1.0, -0.1, 0.1))
        assert e.value.status == 1
        bad = y.copy()
        bad[3] = np.nan
        with pytest.raises(fsa.FsaError) as e:
            h.loglik_grad(bad, (1.0, 0.1, 0.1))
        assert e.value.status == 5
        # iteration limit: outputs written, status NO_CONVERGENCE
        ll, g, info = h.loglik_grad(y, (1.0, 0.1, 0.1), fsa.make_opts(num_probes=4, cg_tol=1e-30, cg_max_iter=3))
        assert info["status"] == 4 and math.isfinite(ll) and info["iters_max"] == 3
    # a duplicated inducing point: Sigma_m singular (exact zero pivot) -> FSA_ERR_NOT_PD
    ind2 = np.vstack([ind[:1], ind])
    with fsa.FSAHandle(locs, ind2, 0.05) as h:
        with pytest.raises(fsa.FsaError) as e:
            h.loglik_grad(y, (1.0, 0.1, 0.1))
        assert e.value.status == 3


def test_autograd_function_passes_the_kernel_gradient(fsa):
    """FSALogLik with a real handle: forward gives the C-ABI log-likelihood and
    backward its STE gradient (same probes and fixed-order reductions, so the
    same values), which match the oracle's under the same probes."""
    import torch
    locs, ind = _setup(2000, 50, 0.5, 0.05, 41)
    th = (1.0, 0.1, 0.1)
    y = fi.random_field(locs, 0.5, *th, 41)
    opts = fsa.make_opts(num_probes=8, fixed_iters=15, seed=5)
    with fsa.FSAHandle(locs, ind, 0.05, 0.5) as h:
        ll0, g0, _ = h.loglik_grad(y, th, opts)
        theta = torch.tensor(th, dtype=torch.float64, requires_grad=True)
        ll = fsa.FSALogLik.apply(theta, h, y, opts)
        ll.backward()
    assert abs(ll.item() - ll0) <= 1e-12 * abs(ll0)
    assert np.allclose(theta.grad.numpy(), g0, rtol=1e-12, atol=0.0)
    ref = O.IterativeFSA(locs, ind, 0.05, 0.5, th).loglik_grad(y, 8, 5, 0.0, fixed_iters=15)
    assert _rel(theta.grad.numpy(), ref["grad"]) < 1e-6
