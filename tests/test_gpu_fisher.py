"""Fisher information by stochastic trace estimation (appendix "Fisher
scoring") on the GPU against the oracle's ``fisher_ste`` with the same probes
(SplitMix64 stream 7).  Both sides run the 3 l solves to a tight CG
tolerance, so they differ by rounding only.

I is positive semi-definite, so |I_kj| <= sqrt(I_kk I_jj); that is the scale of
each entry's bound.  FP64 form: 1e-6 of it.  Mixed BF16X2 form: its solves
carry a relative error of about 1e-6 and the derivative applies that of the
BF16 pair (~2^-17), so 1e-4 of it.
"""
import numpy as np
import pytest

import fsa_inputs as fi
from oracle import fsa_oracle as O

pytestmark = pytest.mark.gpu

CASES = [
    # n, m, nu, theta, nnz per row, probes, precision name, tolerance
    (3001, 40, 0.5, (1.0, 0.1, 0.1), 16, 10, "fp64", 1e-6),
    (20011, 200, 1.5, (1.0, 0.03, 0.05), 20, 8, "bf16x2", 1e-4),
]


@pytest.mark.parametrize("n,m,nu,th,k,l,prec,tol", CASES)
def test_fisher_matches_oracle(n, m, nu, th, k, l, prec, tol):
    import paper_2405_14492_gb300 as F
    seed = 61
    locs = fi.uniform_locations(n, seed)
    ind = locs[fi.inducing_subset(n, m, seed)]
    gamma = fi.taper_range_for(k, n)
    cg_tol = 1e-9
    ref = O.IterativeFSA(locs, ind, gamma, nu, th).fisher_ste(l, seed, cg_tol, max_iter=5000)
    precision = {"fp64": F.FSA_FP64, "bf16x2": F.FSA_MIXED_BF16X2}[prec]
    with F.FSAHandle(locs, ind, gamma, nu) as h:
        Fs, Fr, info = h.fisher(th, F.make_opts(num_probes=l, cg_tol=cg_tol if prec == "fp64" else 1e-3,
                                                cg_max_iter=5000, seed=seed, precision=precision),
                                raise_on_noconv=True)
    d = np.sqrt(np.abs(np.diag(ref["fisher"])))
    scale = np.outer(d, d)
    err = np.abs(Fs - ref["fisher"]) / scale
    err_raw = np.abs(Fr - ref["fisher_raw"]) / scale
    print(f"{prec}: fisher err / sqrt(I_kk I_jj) max {err.max():.2e}, raw {err_raw.max():.2e}; "
          f"iterations {info['iters_max']} (oracle {np.max(ref['iters'])})")
    assert info["converged"] == 1
    assert np.all(err < tol), (Fs, ref["fisher"])
    assert np.all(err_raw < tol), (Fr, ref["fisher_raw"])
    assert np.allclose(Fs, Fs.T, rtol=0, atol=0)
    assert np.all(np.linalg.eigvalsh(Fs) > 0)


def test_fisher_rejects_bad_arguments():
    import paper_2405_14492_gb300 as F
    locs = fi.uniform_locations(500, 62)
    with F.FSAHandle(locs, locs[:10], 0.1, 0.5) as h:
        with pytest.raises(F.FsaError):
            h.fisher((1.0, 0.1, 0.1), F.make_opts(num_probes=0))
        with pytest.raises(F.FsaError):   # 3 l columns exceed the mixed form's block
            h.fisher((1.0, 0.1, 0.1), F.make_opts(num_probes=43, precision=F.FSA_MIXED_BF16X2))
