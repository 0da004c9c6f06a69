"""The headline kernel path of the mixed BF16X2 form against the FP64 oracle.

At n >= 5e4 the S = A~ q product runs as the persistent tensor-core GEMM (one
CTA per SM looping over at least two M tiles per SM), A~^T X as the many-split
GEMM and the CG block product as the TMA SpMM: the kernels that carry the
n = 1e6 evaluation.  Both sides run the same number of CG iterations with the
same Rademacher probes (Appendix A; §3.3), so the estimates differ only by the
mixed form's roundings.

The gradient is compared component by component, and so are its two parts
per parameter, the trace estimate t_j (the mean of the per-probe terms
U_k^T dSigma_j W_k) and the quadratic term q_j = u^T dSigma_j u (§3.3), and
every per-probe term.  Each is a bilinear form x^T M y of CG solutions with an
indefinite M, so a relative perturbation delta of the solves moves it by at
most delta (|x| |M y| + |M x| |y|); that scale, computed from the oracle's
solves, can exceed |x^T M y| many times where M's sparse and low-rank parts
cancel (the range derivative).
"""
import numpy as np
import pytest

import fsa_inputs as fi
from oracle import fsa_oracle as O
from parity_helpers import bilinear_scales, gradient_scale

pytestmark = pytest.mark.gpu

# The mixed BF16X2 form keeps A~ as a BF16 pair (~2^-17 relative), vectors in
# FP32 and the vector operands of the tensor-core products as two BF16 pieces.
# The log-likelihood and its parts are held to 1e-5 relative (they match to
# about 1e-6).  The solves themselves carry a relative error of about
# 2^-17 times a small amplification (u^T u, which weighs the components where
# the mixed perturbation acts most, is off by 1.8e-5 at n = 6e4), so every
# gradient term x^T M y is held to delta = 4 x 2^-17 of its Cauchy-Schwarz
# scale |x| |M y| + |M x| |y| (parity_helpers).
LOGLIK_TOL = 1e-5
SOLVE_DELTA = 4 * 2.0 ** -17


def _terms(ref):
    """Trace and quadratic parts of the oracle gradient: g = -1/2 (t - q)."""
    t = ref["grad_terms"].mean(axis=1)
    q = t + 2.0 * ref["grad"]
    return t, q


CASES = [
    # n, m, nu, theta, nnz per row, probes, iterations, seed
    (60013, 256, 0.5, (1.0, 0.02, 0.01), 20, 16, 20, 91),
    (80021, 384, 1.5, (1.0, 0.02, 0.05), 20, 12, 16, 92),
]


@pytest.mark.parametrize("n,m,nu,th,k,l,K,seed", CASES)
def test_mixed_x2_headline_path_matches_oracle(n, m, nu, th, k, l, K, seed):
    import paper_2405_14492_gb300 as F
    locs = fi.uniform_locations(n, seed)
    ind = locs[fi.inducing_subset(n, m, seed)]
    gamma = fi.taper_range_for(k, n)
    y = fi.random_field(locs, nu, *th, seed)
    assert n >= 2 * 152 * 128   # the persistent GEMM's launch condition (two M tiles per SM)
    S = O.IterativeFSA(locs, ind, gamma, nu, th)
    ref = S.loglik_grad(y, l, seed, 0.0, fixed_iters=K)
    scales = bilinear_scales(S, ref)
    with F.FSAHandle(locs, ind, gamma, nu) as h:
        ll, g, info = h.loglik_grad(y, th, F.make_opts(num_probes=l, fixed_iters=K, seed=seed,
                                                       precision=F.FSA_MIXED_BF16X2))
        a, _ = h.grad_terms(l)
    t, q = _terms(ref)
    err_ll = abs(ll - ref["loglik"]) / abs(ref["loglik"])
    r_a = np.abs(a - ref["grad_terms"]) / scales[:, 1:]
    r_q = np.abs(np.array(info["grad_quad"]) - q) / scales[:, 0]
    r_t = np.abs(np.array(info["grad_trace"]) - t) / scales[:, 1:].mean(axis=1)
    r_g = np.abs(g - ref["grad"]) / gradient_scale(scales)
    print(f"n={n} m={m}: loglik rel {err_ll:.2e}; quad rel {abs(info['quad_form'] - ref['quad']) / abs(ref['quad']):.2e}; "
          f"logdet rel {abs(info['logdet'] - ref['logdet']) / abs(ref['logdet']):.2e}; error / scale: "
          f"terms {r_a.max(axis=1)}, quadratic {r_q}, trace {r_t}, gradient {r_g}; "
          f"scale / |term| of the quadratic {scales[:, 0] / np.abs(q)}")
    assert err_ll < LOGLIK_TOL, (ll, ref["loglik"])
    assert abs(info["quad_form"] - ref["quad"]) < LOGLIK_TOL * abs(ref["quad"])
    assert abs(info["logdet"] - ref["logdet"]) < LOGLIK_TOL * abs(ref["logdet"])
    assert np.all(r_a < SOLVE_DELTA)
    assert np.all(r_q < SOLVE_DELTA), (info["grad_quad"], q)
    assert np.all(r_t < SOLVE_DELTA), (info["grad_trace"], t)
    assert np.all(r_g < SOLVE_DELTA), (g, ref["grad"])
