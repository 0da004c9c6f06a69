"""The FITC preconditioner as control variate for the gradient's trace
estimate (appendix "Preconditioner as control variate", Eq. Troptc) on the
GPU, against the oracle's ``loglik_grad(control_variate=...)`` with the same
probes and the same number of CG iterations.

Per parameter the estimate is (1/l) sum_k (a_k - c b_k) + c Tr(P_hat^-1 dP_hat)
with a_k = U_k^T dSigma W_k, b_k = W_k^T dP_hat W_k.  The exact trace
Tr(P_hat^-1 dP_hat) (an O(n m^2) computation on both sides), the per-probe b_k,
the coefficient c and the gradient are compared one by one.  Each per-probe
term is a bilinear form of CG solutions, compared on the Cauchy-Schwarz scale
of parity_helpers; c and the gradient on the error those terms carry into them.
"""
import numpy as np
import pytest

import fsa_inputs as fi
from oracle import fsa_oracle as O
from parity_helpers import bilinear_scales, mixed_traceP_scales, precond_scales

pytestmark = pytest.mark.gpu

# FP64 form: a relative 1e-6 for gradients under the same probes, on
# |x| |M y| + |M x| |y| of each bilinear term (parity_helpers).  Mixed BF16X2
# form: delta = 4 x 2^-17, the bound of the headline-path test; its exact
# traces Tr(P_hat^-1 dP_hat) move with the pair-rounded D_s (parity_helpers).
CASES = [
    # n, m, nu, theta, nnz per row, l, K, precision name, delta
    (3001, 40, 0.5, (1.0, 0.1, 0.1), 16, 12, 25, "fp64", 1e-6),
    (20011, 200, 1.5, (1.0, 0.03, 0.02), 20, 12, 20, "bf16x2", 4 * 2.0 ** -17),
]


def _run(n, m, nu, th, k, l, K, prec, kind, seed):
    import paper_2405_14492_gb300 as F
    locs = fi.uniform_locations(n, seed)
    ind = locs[fi.inducing_subset(n, m, seed)]
    gamma = fi.taper_range_for(k, n)
    y = fi.random_field(locs, nu, *th, seed)
    S = O.IterativeFSA(locs, ind, gamma, nu, th)
    ref = S.loglik_grad(y, l, seed, 0.0, fixed_iters=K, control_variate=kind)
    precision = {"fp64": F.FSA_FP64, "bf16x2": F.FSA_MIXED_BF16X2}[prec]
    with F.FSAHandle(locs, ind, gamma, nu) as h:
        ll, g, info = h.loglik_grad(y, th, F.make_opts(num_probes=l, fixed_iters=K, seed=seed, precision=precision,
                                                       grad_control_variate=kind))
        a, b = h.grad_terms(l)
    return S, ref, g, info, a, b


@pytest.mark.parametrize("kind", ["c1", "copt", "copt_centered"])
@pytest.mark.parametrize("n,m,nu,th,k,l,K,prec,tol", CASES)
def test_gradient_control_variate_matches_oracle(n, m, nu, th, k, l, K, prec, tol, kind):
    S, ref, g, info, a, b = _run(n, m, nu, th, k, l, K, prec, kind, 41)
    sa, sb = bilinear_scales(S, ref), precond_scales(S, ref)
    trP, trP_ref = np.array(info["trace_precond"]), ref["trace_P"]
    cc, cc_ref = np.array(info["cv_coef"]), ref["cv_c"]
    b_ref, a_ref = ref["cv_terms"], ref["grad_terms"]
    # trace bound: FP64 tol relative; mixed: the first-order effect of the pair-rounded D_s
    scale_trP = tol * np.abs(trP_ref) if prec == "fp64" else 3 * mixed_traceP_scales(S)
    err_trP = np.abs(trP - trP_ref) / scale_trP
    r_a = (np.abs(a - a_ref) / sa[:, 1:]).max(axis=1)
    r_b = (np.abs(b - b_ref) / sb).max(axis=1)
    # the estimate (1/l) sum (a_k - c b_k) + c Tr(P^-1 dP): scale of each part
    scale_g = 0.5 * (sa[:, 1:].mean(axis=1) + np.abs(cc_ref) * sb.mean(axis=1) + sa[:, 0])
    err_g = np.abs(g - ref["grad"]) / scale_g
    print(f"{prec} {kind}: trP {err_trP} b {r_b} a {r_a} c {cc} vs {cc_ref} grad {err_g}")
    assert np.all(err_trP < 1.0), (trP, trP_ref, scale_trP)
    assert np.all(r_b < tol), (b, b_ref)
    assert np.all(r_a < tol)
    if kind == "c1":
        assert np.all(cc == 1.0)
    else:
        # c is a ratio of probe sums; its error follows from those of a and b
        sbc = b_ref - (b_ref.mean(axis=1, keepdims=True) if kind == "copt_centered" else 0.0)
        den = np.sum(sbc * sbc, axis=1)
        dc = tol * (np.sum(sa[:, 1:] * np.abs(sbc), axis=1) + 2 * np.abs(cc_ref) * np.sum(sb * np.abs(sbc), axis=1)) / den
        assert np.all(np.abs(cc - cc_ref) < 3 * dc + 1e-12), (cc, cc_ref, dc)
    # the gradient moves with a, b, c and the exact trace
    dcg = 0.0 if kind == "c1" else np.abs(cc - cc_ref) * np.abs(trP_ref - b_ref.mean(axis=1))
    assert np.all(np.abs(g - ref["grad"]) < 3 * (tol * scale_g + 0.5 * dcg + 0.5 * np.abs(cc_ref) * scale_trP)), \
        (g, ref["grad"], err_g)


def test_control_variate_c1_reduces_the_range_derivative_spread():
    """With c = 1 the per-probe terms a_k - b_k of the range derivative spread
    less than the plain a_k (the reason for the control variate)."""
    n, m, nu, th, k, l, K = 20011, 200, 0.5, (1.0, 0.05, 0.05), 20, 24, 30
    S, ref, g, info, a, b = _run(n, m, nu, th, k, l, K, "bf16x2", "c1", 43)
    assert np.std(a[1] - b[1]) < 0.7 * np.std(a[1]), (np.std(a[1] - b[1]), np.std(a[1]))
