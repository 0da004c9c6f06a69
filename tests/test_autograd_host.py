"""Host logic of the ``FSALogLik`` torch.autograd.Function, on the CPU.

The Function only marshals: forward calls ``handle.loglik_grad`` and keeps the
gradient, backward returns grad_output times it.  Here the handle is a stand-in
whose log-likelihood and gradient are the dense oracle's exact ones (Eq.
NEGLLDNEGLLFSA), so the checks below isolate the wrapper: the value and
gradient it passes on, the chain rule through a reparameterisation, and
agreement with central finite differences of step 1e-4.
"""
import numpy as np
import pytest
import torch

import fsa_inputs as fi
import paper_2405_14492_gb300 as F
from oracle import fsa_oracle as O


class DenseHandle:
    """Duck-typed stand-in for FSAHandle backed by the dense oracle."""

    def __init__(self, locs, inducing, gamma, nu):
        self.args = (locs, inducing, gamma, nu)
        self.calls = 0

    def loglik_grad(self, y, theta, opts=None):
        self.calls += 1
        D = O.DenseFSA(*self.args, tuple(float(t) for t in theta))
        return D.loglik(y)[0], D.grad(y), {"status": 0}


@pytest.fixture(scope="module")
def problem():
    n, m = 120, 15
    locs = fi.uniform_locations(n, 71)
    ind = locs[fi.inducing_subset(n, m, 71)].copy()
    y = np.random.default_rng(71).standard_normal(n)
    return DenseHandle(locs, ind, 0.12, 1.5), y, (0.9, 0.15, 0.2)


def test_forward_value_and_backward_gradient(problem):
    h, y, th = problem
    theta = torch.tensor(th, dtype=torch.float64, requires_grad=True)
    ll = F.FSALogLik.apply(theta, h, y)
    assert ll.dtype == torch.float64 and ll.dim() == 0
    D = O.DenseFSA(*h.args, th)
    assert ll.item() == D.loglik(y)[0]
    (2.5 * ll).backward()
    assert np.array_equal(theta.grad.numpy(), 2.5 * D.grad(y))


def test_chain_rule_matches_central_differences_in_log_parameters(problem):
    """An optimiser's view: phi = log theta, loss = -l(exp(phi)) / n; the
    autograd gradient equals central differences of step 1e-4 in phi."""
    h, y, th = problem
    n = y.shape[0]
    phi = torch.tensor(np.log(th), dtype=torch.float64, requires_grad=True)
    loss = -F.FSALogLik.apply(torch.exp(phi), h, y) / n
    loss.backward()

    def f(p):
        return -O.DenseFSA(*h.args, tuple(np.exp(p))).loglik(y)[0] / n

    p0 = np.log(th)
    for k in range(3):
        e = np.zeros(3)
        e[k] = 1e-4
        fd = (f(p0 + e) - f(p0 - e)) / 2e-4
        assert abs(float(phi.grad[k]) - fd) < 1e-6 * max(1.0, abs(fd))


def test_gradcheck_and_one_handle_call_per_forward(problem):
    h, y, th = problem
    theta = torch.tensor(th, dtype=torch.float64, requires_grad=True)
    before = h.calls
    assert torch.autograd.gradcheck(lambda t: F.FSALogLik.apply(t, h, y), (theta,), eps=1e-5, atol=1e-4,
                                    rtol=1e-4)
    # gradcheck's forward evaluations each call the handle exactly once
    assert h.calls > before
    before = h.calls
    ll = F.FSALogLik.apply(theta, h, y)
    ll.backward()
    assert h.calls == before + 1


def test_lbfgs_driver_reaches_the_dense_maximum_likelihood_estimate():
    """``fit_mle`` (L-BFGS in log-parameters on top of FSALogLik), driven by
    the dense stand-in, reaches the maximiser of the dense log-likelihood
    that scipy's L-BFGS-B finds independently, from a start 20-30 % off in
    every parameter; every objective evaluation is one handle call."""
    so = pytest.importorskip("scipy.optimize")
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
    h = DenseHandle(locs, ind, g, nu)
    out = F.fit_mle(h, y, mle * np.array([1.3, 0.8, 1.2]))
    assert out["converged"]
    assert np.max(np.abs(out["theta"] / mle - 1)) < 1e-5
    assert abs(out["loglik"] + r.fun) < 1e-8 * abs(r.fun)
    # one handle call per evaluation, plus the final one for the returned loglik
    assert h.calls == out["evaluations"] + 1


def test_lbfgs_driver_reports_an_unfinished_run(problem):
    """With too few iterations for its gradient tolerance, ``fit_mle`` returns
    its last iterate with ``converged`` false (and a log-likelihood no lower
    than at the start)."""
    h, y, th = problem
    start = np.array(th) * np.array([1.5, 0.6, 1.4])
    out = F.fit_mle(h, y, start, max_iter=2, tol_grad=1e-12)
    assert not out["converged"]
    assert out["iterations"] <= 2
    ll0 = O.DenseFSA(*h.args, tuple(start)).loglik(y)[0]
    assert out["loglik"] >= ll0
