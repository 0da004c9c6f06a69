"""Planted-mistake sweep of the FP64 oracle's pins (test infrastructure).

Each entry below plants one plausible mistake in a temporary copy of
``oracle/fsa_oracle.py`` (a dropped term, a wrong sign, a transposed operand,
a shifted index, a wrong constant) and runs the CPU pins of
``tests/test_oracle_pins.py`` against that copy.  A mistake that changes what
the oracle computes must make at least one pin fail.  Entries marked
``equivalent`` change nothing observable, and the reason is stated with them;
the sweep expects them to pass.

The working tree is never modified: every run happens in its own temporary
directory.

    python tests/oracle_mutation_sweep.py            # all entries (several minutes)
    python tests/oracle_mutation_sweep.py -j 8       # eight copies at once
    python tests/oracle_mutation_sweep.py -k taper   # entries whose label contains "taper"

Exit status 0 when every non-equivalent mistake is caught and every
equivalent one passes.
"""
from __future__ import annotations

import argparse
import os
import shutil
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (label, original text, planted text, None or the reason it is equivalent)
MUTATIONS = [
    ("matern15 drops part of (1 + x)", "return (1.0 + x) * np.exp(-x)", "return (1.0 + 0.9 * x) * np.exp(-x)", None),
    ("matern15 range derivative loses a factor x", "return (x * x / rho) * np.exp(-x)",
     "return (x / rho) * np.exp(-x)", None),
    ("taper exponent 3 instead of 4", "out = (1.0 - t) ** 4 * (1.0 + 4.0 * t)",
     "out = (1.0 - t) ** 3 * (1.0 + 4.0 * t)", None),
    ("taper value kept at d = gamma", "return np.where(d < gamma, out, 0.0)", "return np.where(d <= gamma, out, 0.0)",
     "the Wendland taper is 0 at d = gamma"),
    ("support includes d = gamma (brute force)", "r, c = np.nonzero(d2 < g2)", "r, c = np.nonzero(d2 <= g2)", None),
    ("support includes d = gamma (tree)", "keep = sqdist_pairs(rows_pts[r], cols_pts[c]) < g2",
     "keep = sqdist_pairs(rows_pts[r], cols_pts[c]) <= g2", None),
    ("tree search radius too small", "cand = tree.query_ball_point(rows_pts, r=gamma * (1.0 + 1e-6))",
     "cand = tree.query_ball_point(rows_pts, r=gamma * (1.0 - 1e-3))", None),
    ("CSR sorted by column first", "order = np.lexsort((c, r))", "order = np.lexsort((r, c))", None),
    ("SplitMix64 counter not offset by one", "c = counters.astype(np.uint64) + np.uint64(1)",
     "c = counters.astype(np.uint64)", None),
    ("Rademacher from the low bit", "return 1.0 - 2.0 * (h >> np.uint64(63)).astype(np.float64)",
     "return 1.0 - 2.0 * (h & np.uint64(1)).astype(np.float64)", None),
    ("Box-Muller radius loses the factor 2", "z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)",
     "z = np.sqrt(-np.log(u1)) * np.cos(2.0 * math.pi * u2)", None),
    ("Box-Muller second counter shifted", "h2 = splitmix64(seed, stream, ctr * np.uint64(2) + np.uint64(1))",
     "h2 = splitmix64(seed, stream, ctr * np.uint64(2) + np.uint64(3))", None),
    ("kmeans++ weights use d instead of d^2", "d2 = dx * dx + dy * dy\n        return np.floor",
     "d2 = np.sqrt(dx * dx + dy * dy)\n        return np.floor", None),
    ("kmeans++ picks the first prefix sum >= target",
     'i = int(np.searchsorted(cum, np.uint64(target), side="right"))',
     'i = int(np.searchsorted(cum, np.uint64(target), side="left"))',
     "differs only when a 53-bit draw lands exactly on a prefix sum (probability about 1/Q, Q near 2^60)"),
    ("residual diagonal not clamped (iterative)", "resid[diag_mask] = np.maximum(resid[diag_mask], 0.0)",
     "resid[diag_mask] = resid[diag_mask]", "the clamp only acts on rounding-level negatives at inducing points"),
    ("residual diagonal shifted (dense)", "np.fill_diagonal(resid, np.maximum(np.diag(resid), 0.0))",
     "np.fill_diagonal(resid, np.diag(resid) + 1e-3)", None),
    ("nugget scaled", "vals[diag_mask] += nug", "vals[diag_mask] += 1.01 * nug", None),
    ("low-rank part scaled in the residual", "lowrank = self._rowdots(self.A, self.A, rows, cols)",
     "lowrank = 0.999 * self._rowdots(self.A, self.A, rows, cols)", None),
    ("dense FITC preconditioner scaled", "self.Phat = np.diag(self.D) + self.Sl",
     "self.Phat = np.diag(self.D) + 0.999 * self.Sl", None),
    ("Woodbury core with D^-2", "self.Mp = self.Sm + (self.K / self.D) @ self.K.T",
     "self.Mp = self.Sm + (self.K / self.D ** 2) @ self.K.T", None),
    ("Sylvester log-determinant sign of logdet Sigma_m", "                         - 2.0 * np.sum(np.log(np.diag(self.Lm)))",
     "                         + 2.0 * np.sum(np.log(np.diag(self.Lm)))", None),
    ("Woodbury correction sign", "return DV - (corr_ / self.D[:, None] if V.ndim == 2 else corr_ / self.D)",
     "return DV + (corr_ / self.D[:, None] if V.ndim == 2 else corr_ / self.D)", None),
    ("FITC probe with L^-1 instead of L^-T",
     "return self.K.T @ sla.solve_triangular(self.Lm.T, e1, lower=False) + np.sqrt(self.D)[:, None] * e2",
     "return self.K.T @ sla.solve_triangular(self.Lm, e1, lower=True) + np.sqrt(self.D)[:, None] * e2", None),
    ("CG stop rule loosened", "stop = (rn < tol) if fixed_iters <= 0 else np.zeros(len(cols), dtype=bool)",
     "stop = (rn < 1e3 * tol) if fixed_iters <= 0 else np.zeros(len(cols), dtype=bool)", None),
    ("Lanczos diagonal with the current beta", "diag[k].append(1.0 / alpha[t] + beta_prev[k] / alpha_prev[k])",
     "diag[k].append(1.0 / alpha[t] + beta[t] / alpha[t])", None),
    ("Lanczos off-diagonal with the current alpha", "off[k].append(math.sqrt(beta_prev[k]) / alpha_prev[k])",
     "off[k].append(math.sqrt(beta_prev[k]) / alpha[t])", None),
    ("quadrature from the first eigenvector instead of its first row",
     "return float(np.sum(Q[0, :] ** 2 * np.log(lam)))", "return float(np.sum(Q[:, 0] ** 2 * np.log(lam)))", None),
    ("SLQ terms taken from the y column",
     'quads = np.array([lanczos_quadrature(res["diag"][k], res["off"][k]) for k in range(1, num_probes + 1)])',
     'quads = np.array([lanczos_quadrature(res["diag"][k], res["off"][k]) for k in range(0, num_probes)])', None),
    ("SLQ exact weight ignored", 'weights = res["rz0"][1:] if exact_weight else np.full(num_probes, float(n))',
     "weights = np.full(num_probes, float(n))", None),
    ("logdet P subtracted", "logdet = float(np.mean(terms)) + self.logdet_P",
     "logdet = float(np.mean(terms)) - self.logdet_P", None),
    ("quadratic form with P^-1 y", 'u = res["U"][:, 0]\n        yu = float(y @ u)',
     'u = res["U"][:, 0]\n        yu = float(y @ res["Z0"][:, 0])', None),
    ("gradient quadratic term sign", "g[k] = -0.5 * (tr - qf)", "g[k] = -0.5 * (tr + qf)", None),
    ("sparse derivative: symmetric low-rank terms merged wrongly",
     "dl = (self._rowdots(dK.T, C.T, rows, cols) + self._rowdots(C.T, dK.T, rows, cols)",
     "dl = (2 * self._rowdots(dK.T, C.T, rows, cols)", None),
    ("sparse derivative without the taper", "dvals = (dsig - dl) * self.Tv", "dvals = (dsig - dl)", None),
    ("low-rank derivative drops the dSigma_m term",
     "dSl_V = dK.T @ sla.cho_solve(cho, KV) + C.T @ (dK @ V) - C.T @ (dSm @ sla.cho_solve(cho, KV))",
     "dSl_V = dK.T @ sla.cho_solve(cho, KV) + C.T @ (dK @ V)", None),
    ("dense derivative dSigma_m term sign",
     "dSl = dK.T @ SmK + SmK.T @ dK - SmK.T @ dSm @ SmK\n        return dSl + (dSig - dSl) * self.T",
     "dSl = dK.T @ SmK + SmK.T @ dK + SmK.T @ dSm @ SmK\n        return dSl + (dSig - dSl) * self.T", None),
    ("predictive mean without the sparse part", "mean = Kp.T @ sla.cho_solve(cho_m, self.K @ u) + St @ u",
     "mean = Kp.T @ sla.cho_solve(cho_m, self.K @ u)", None),
    ("cross residual without the taper",
     "vals = (s1 * corr(d, self.nu, rho) - lowrank) * taper(d, self.gamma)",
     "vals = (s1 * corr(d, self.nu, rho) - lowrank)", None),
    ("Algorithm 1: W2 solved with the FSA operator",
     'W2 = pcg_lanczos(lambda V: self.Ss @ V, self.apply_Dinv, self.K.T.copy(), tol, max_iter)["U"]',
     'W2 = pcg_lanczos(self.apply, self.apply_Pinv, self.K.T.copy(), tol, max_iter)["U"]', None),
    ("Algorithm 1: M built from W1", "M = self.Sm + self.K @ W2", "M = self.Sm + self.K @ W1", None),
    ("Algorithm 1: D1 from W2", 'D1 = np.einsum("ij,ij->j", G, (self.K @ W1) @ G)',
     'D1 = np.einsum("ij,ij->j", G, (self.K @ W2) @ G)', None),
    ("Algorithm 1: D2 from W2", 'D2 = np.einsum("ij,ji->i", St @ W1, G)', 'D2 = np.einsum("ij,ji->i", St @ W2, G)',
     None),
    ("Algorithm 1: D2 counted once", "var = s1 + nug - D1 - 2.0 * D2 + D3 - Dl",
     "var = s1 + nug - D1 - 1.0 * D2 + D3 - Dl", None),
    ("Algorithm 1: D3 sign", "var = s1 + nug - D1 - 2.0 * D2 + D3 - Dl", "var = s1 + nug - D1 - 2.0 * D2 - D3 - Dl",
     None),
    ("D_l control variate: exact term with D^-2",
     "exact_b = np.asarray(St.multiply(St) @ (1.0 / self.D)).ravel()",
     "exact_b = np.asarray(St.multiply(St) @ (1.0 / self.D ** 2)).ravel()", None),
    ("D_l control variate: exact term not scaled by c", "Dl = np.mean(a - c[:, None] * b, axis=1) + c * exact_b",
     "Dl = np.mean(a - c[:, None] * b, axis=1) + exact_b", None),
    ("dD_s: low-rank diagonal derivative halved", "dl = 2.0 * np.einsum", "dl = 1.0 * np.einsum", None),
    ("dD_s: variance derivative of Sigma_ii dropped", "dsig0 = 1.0 if which == 0 else 0.0", "dsig0 = 0.0", None),
    ("dM_P: D derivative term sign", "dMp = -(K * (dD / D ** 2)) @ K.T", "dMp = (K * (dD / D ** 2)) @ K.T", None),
    ("dM_P: transpose term duplicated", "dMp += dSm + KdK + KdK.T", "dMp += dSm + 2 * KdK",
     "Tr(M^-1 X) = Tr(M^-1 X^T) for symmetric M"),
    ("dM_P: dSigma_m dropped", "dMp += dSm + KdK + KdK.T", "dMp += KdK + KdK.T", None),
    ("dP apply: dSigma_m term sign",
     "        return out + dK.T @ (C @ V) + C.T @ (dK @ V) - C.T @ (dSm @ (C @ V))",
     "        return out + dK.T @ (C @ V) + C.T @ (dK @ V) + C.T @ (dSm @ (C @ V))", None),
    ("gradient control variate: printed c_opt centred", "den = float(np.sum(b * b))",
     "den = float(np.sum((b - b.mean()) ** 2))", None),
    ("gradient control variate: centred numerator uncentred",
     "c = float(np.sum((per_probe - tr) * bc)) / den", "c = float(np.sum((per_probe - tr) * b)) / den",
     "sum (a - mean a) b = sum (a - mean a)(b - mean b)"),
    ("gradient control variate: trace not scaled by c", "tr = float(np.mean(per_probe - c * b)) + c * trace_P[k]",
     "tr = float(np.mean(per_probe - c * b)) + trace_P[k]", None),
    ("Fisher STE: second solve of the wrong parameter",
     'terms[k, j] = 0.5 * np.einsum("ij,ij->j", dV, X[j])', 'terms[k, j] = 0.5 * np.einsum("ij,ij->j", dV, X[k])',
     None),
    ("Fisher STE: solves of parameters 0 and 1 swapped",
     'X = [res["U"][:, l:2 * l], res["U"][:, 2 * l:], V]', 'X = [res["U"][:, 2 * l:], res["U"][:, l:2 * l], V]',
     None),
    ("Fisher scoring descends instead of ascending",
     "return np.asarray(theta, np.float64) + np.linalg.solve(", "return np.asarray(theta, np.float64) - np.linalg.solve(",
     None),
    ("Vecchia: B gets +A_i", "            vals += (-Ai).tolist()", "            vals += Ai.tolist()", None),
    ("Vecchia: conditional variance without the correction", "            self.D[i] = s1 - float(Ai @ SNi)",
     "            self.D[i] = s1", None),
    ("Vecchia: farthest instead of nearest earlier points",
     'Ni = np.sort(np.argsort(d2, kind="stable")[:k])', 'Ni = np.sort(np.argsort(-d2, kind="stable")[:k])', None),
    ("Vecchia: FITC diagonal without the nugget", "        self.Ds = np.maximum(s1 - np.sum(Al * Al, axis=0), 0.0) + nug",
     "        self.Ds = np.maximum(s1 - np.sum(Al * Al, axis=0), 0.0) + 0.5 * nug", None),
    ("Vecchia: Sigma_V applied with B^-T and B^-1 swapped",
     "        X = sp.linalg.spsolve_triangular(self.BT, V, lower=False)",
     "        X = sp.linalg.spsolve_triangular(self.B, V, lower=True)", None),
    ("Vecchia: posterior solve in the printed order",
     "        return self.apply_SigmaV(res[\"U\"]), res[\"iters\"]",
     "        return res[\"U\"], res[\"iters\"]", None),
    ("dense Fisher without the transpose", "        return np.array([[0.5 * np.sum(X[k] * X[l].T)",
     "        return np.array([[0.5 * np.sum(X[k] * X[l])", None),
]


def _copy_tree(dst):
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"),
                    ignore=shutil.ignore_patterns("__pycache__"))
    os.makedirs(os.path.join(dst, "tests"))
    for f in ("conftest.py", "test_oracle_pins.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(dst, "tests", f))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(dst, "tests", "golden"))
    for f in ("fsa_inputs.py", "pytest.ini"):
        shutil.copy(os.path.join(ROOT, f), os.path.join(dst, f))


def run_one(label, old, new, threads=None):
    """'caught', 'passed' or 'not found' for one planted mistake."""
    env = dict(os.environ)
    if threads:
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            env[v] = str(threads)
    with tempfile.TemporaryDirectory(prefix="oracle_mut_") as tmp:
        _copy_tree(tmp)
        path = os.path.join(tmp, "oracle", "fsa_oracle.py")
        with open(path) as f:
            src = f.read()
        if old not in src:
            return "not found"
        with open(path, "w") as f:
            f.write(src.replace(old, new, 1))
        r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-q", "-x",
                            "-p", "no:cacheprovider"], cwd=tmp, capture_output=True, text=True, env=env)
        return "passed" if r.returncode == 0 else "caught"


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("-k", default="", help="run only entries whose label contains this text")
    ap.add_argument("-j", type=int, default=1, help="copies run at once (BLAS threads are divided among them)")
    args = ap.parse_args()
    todo = [e for e in MUTATIONS if not args.k or args.k in e[0]]
    threads = max(1, (os.cpu_count() or 1) // args.j) if args.j > 1 else None
    with ThreadPoolExecutor(max_workers=max(1, args.j)) as ex:
        results = list(ex.map(lambda e: run_one(e[0], e[1], e[2], threads), todo))
    bad = 0
    for (label, old, new, equivalent), got in zip(todo, results):
        want = "passed" if equivalent else "caught"
        ok = got == want
        bad += not ok
        note = f"  (equivalent: {equivalent})" if equivalent else ""
        print(f"{'ok ' if ok else 'BAD'} {got:9s} {label}{note}", flush=True)
    print(f"{bad} unexpected outcome(s)")
    return 1 if bad else 0


if __name__ == "__main__":
    sys.exit(main())
