"""Central finite differences of the deterministic pieces of the
log-likelihood on the GPU path, through the autograd.Function.

The STE gradient (§3.3) is -1/2 (t - q) per parameter: t estimates
Tr(Sigma_dag^-1 dSigma_dag) and q = u^T dSigma_dag u, u = Sigma_dag^-1 y.
Two pieces are deterministic and checked against central differences of step
1e-4 (relative to each parameter) of values the library computes:
  * q_j = -d(y^T Sigma_dag^-1 y)/dtheta_j, with y^T Sigma_dag^-1 y from CG run
    to a tight tolerance;
  * Tr(P_hat^-1 dP_hat/dtheta_j) = d log det P_hat / dtheta_j (Jacobi's
    formula), with log det P_hat from the Sylvester identity (appendix
    "Runtime of the FITC preconditioner"), computed when the control variate is on.
The workload has the exponential covariance, the range, nugget and
nonzeros per row of the n = 1e6 evaluation, at n = 20011.
"""
import numpy as np
import pytest

import fsa_inputs as fi

pytestmark = pytest.mark.gpu

FD_TOL = 1e-6
STEP = 1e-4


def test_fd_of_deterministic_pieces_through_autograd():
    import torch

    import paper_2405_14492_gb300 as F
    n, m, nu, seed = 20011, 200, 0.5, 51
    th0 = np.array([1.0, 0.02, 0.01])
    locs = fi.uniform_locations(n, seed)
    ind = locs[fi.inducing_subset(n, m, seed)]
    gamma = fi.taper_range_for(20, n)
    y = fi.random_field(locs, nu, *th0, seed)
    tight = dict(num_probes=8, cg_tol=1e-9 * np.linalg.norm(y), cg_max_iter=4000, seed=seed, precision=F.FSA_FP64)
    with F.FSAHandle(locs, ind, gamma, nu) as h:
        theta = torch.tensor(th0, dtype=torch.float64, requires_grad=True)
        ll = F.FSALogLik.apply(theta, h, y, F.make_opts(grad_control_variate="c1", **tight))
        ll.backward()
        info = h.last_info
        assert info["converged"] == 1
        trace, quad = np.array(info["grad_trace"]), np.array(info["grad_quad"])
        trP = np.array(info["trace_precond"])
        # the autograd gradient is the STE gradient assembled from its parts
        assert np.allclose(theta.grad.numpy(), -0.5 * (trace - quad), rtol=1e-12, atol=0.0)
        for j in range(3):
            hj = STEP * th0[j]
            vals = []
            for sgn in (1.0, -1.0):
                tj = th0.copy()
                tj[j] += sgn * hj
                _, _, inf = h.loglik_grad(y, tj, F.make_opts(want_grad=False, **tight))
                vals.append((inf["quad_form"], h.logdet_precond(tj, F.FSA_FP64)))
            fd_quad = (vals[0][0] - vals[1][0]) / (2 * hj)
            fd_ldp = (vals[0][1] - vals[1][1]) / (2 * hj)
            print(f"theta_{j}: q {quad[j]:.10e} fd {-fd_quad:.10e}; trP {trP[j]:.10e} fd {fd_ldp:.10e}")
            assert abs(-fd_quad - quad[j]) < FD_TOL * abs(quad[j]), (j, quad[j], -fd_quad)
            assert abs(fd_ldp - trP[j]) < FD_TOL * abs(trP[j]), (j, trP[j], fd_ldp)
