"""The n = 1e5 Matern-3/2 workload (m = 500 inducing points, 30 nonzeros per
row, 50 probes, CG tolerance 1e-3): the mixed BF16X2 form against the FP64
form on the same probes.  The log-likelihood of the mixed form must be within
1e-4 (relative) of the FP64 form's; each gradient component within 1e-2 of
the scale of its own terms (the STE gradient's trace and quadratic parts,
which the mixed solves carry to about 2^-17 of their size, amplified by the
CG tolerance; the components themselves can be small differences of them)."""
import numpy as np
import pytest

import fsa_inputs as fi

pytestmark = pytest.mark.gpu


def test_matern15_n1e5_mixed_within_1e4_of_fp64():
    import paper_2405_14492_gb300 as F
    w = fi.MATERN15_N1E5
    locs, ind, _, y, _ = w.make()
    th = (w.sigma1_sq, w.rho, w.nugget)
    o = dict(num_probes=w.num_probes, cg_tol=w.cg_tol, cg_max_iter=2000, seed=w.seed)
    with F.FSAHandle(locs, ind, w.taper_range(), w.nu) as h:
        ll64, g64, i64 = h.loglik_grad(y, th, F.make_opts(**o))
        ll2, g2, i2 = h.loglik_grad(y, th, F.make_opts(precision=F.FSA_MIXED_BF16X2, **o))
    assert i64["converged"] == 1 and i2["converged"] == 1
    rel = abs(ll2 - ll64) / abs(ll64)
    terms = 0.5 * (w.n * np.log(2 * np.pi) + abs(i64["logdet"]) + abs(i64["quad_form"]))
    scale = np.abs(np.array(i64["grad_trace"])) + np.abs(np.array(i64["grad_quad"]))
    gerr = np.abs(np.asarray(g2) - np.asarray(g64)) / scale
    print(f"n = 1e5 Matern 3/2: loglik {ll64:.8e} (FP64) {ll2:.8e} (mixed), rel {rel:.2e}, "
          f"vs terms {abs(ll2 - ll64) / terms:.2e}; grad err / term scale {gerr}; "
          f"iterations {i64['iters_max']} / {i2['iters_max']}")
    assert rel < 1e-4, (ll2, ll64)
    assert np.all(gerr < 1e-2), (g2, g64)
