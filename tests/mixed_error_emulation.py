"""Numpy emulation of the mixed-precision CG loop's rounding on one request of
the serving stream (analysis script, not collected by pytest).

It replays the algebra of the BF16X2 log-likelihood path in FP64 numpy, with
one switch per rounding, so that each rounding's share of the log-likelihood
difference to the FP64 form can be measured on the CPU:

    a64 / a2   A = Sigma_nm L_m^-T exact, or stored as a BF16 hi + lo pair
    m32        Woodbury core M = I + A^T D^-1 A summed in FP32 over 512-row
               spans, spans added in FP64
    v32        the CG block (R, U, S, Z, V, H) rounded to FP32 after each update
    s2         the vector operands of the two n x m products (D^-1 R and
               q = M^-1 w) split into two BF16 pieces
    w32        A^T X accumulated in FP32 per 4096-row split, splits in FP64
    d32        residual values a_i . a_j summed in FP32 per 64-column block,
               blocks in FP64

The loop has the structure of the GPU's: S = A M^-1 A^T D^-1 R,
Z = D^-1 (R - S), V = Sigma_s Z + S + beta V (the low-rank product taken from
the Woodbury identity), Lanczos tridiagonals from alpha and beta (Appendix
A), SLQ with the weight n (§3.1).  Probes as in the library (SplitMix64
streams 4 and 5, the request's seed).

    python tests/mixed_error_emulation.py 92 50 1e-3 a64,a2,a2_m32_v32_s2_w32

The first configuration is the reference of the printed differences.
"""
import math
import os
import sys
import time

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import fsa_inputs as fi  # noqa: E402
from oracle import fsa_oracle as O  # noqa: E402


def bf16(x):
    """Round to the nearest BF16 (ties to even), returned as float32."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def split2(x):
    """Two BF16 pieces of the FP32 value of x, summed back in FP64."""
    x32 = np.asarray(x, np.float32)
    h = bf16(x32)
    return h.astype(np.float64) + bf16(x32 - h).astype(np.float64)


class Request:
    def __init__(self, index, num_probes):
        req = fi.serving_stream(max(128, index + 1))[index]
        self.req = req
        self.locs, ind, self.y, _ = req.make()
        self.n, self.m, self.l = req.n, req.m, num_probes
        s1, rho, nu = req.sigma1_sq, req.rho, req.nu
        self.gamma = req.taper_range()
        K = O.cov_matrix(ind, self.locs, nu, s1, rho)
        Lm = np.linalg.cholesky(O.cov_matrix(ind, ind, nu, s1, rho))
        self.A64 = sla.solve_triangular(Lm, K, lower=True).T
        self.A2 = split2(self.A64)
        self.rowptr, self.col = O.neighbour_csr(self.locs, self.locs, self.gamma)
        self.rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        self.cols = self.col.astype(np.int64)
        d = np.sqrt(O.sqdist_pairs(self.locs[self.rows], self.locs[self.cols]))
        self.Tv = O.taper(d, self.gamma)
        self.cs = s1 * O.corr(d, nu, rho)
        self.diag = self.rows == self.cols
        self.e1 = O.rademacher(req.seed, O.STREAM_EPS1, np.arange(self.m), self.m, num_probes)
        self.e2 = O.rademacher(req.seed, O.STREAM_EPS2, np.arange(self.n), self.n, num_probes)

    def residual(self, A, d32):
        """Sigma_s~ and D_s for the operator defined by A (§2.1)."""
        low = np.empty(len(self.rows))
        A32 = A.astype(np.float32)
        for s in range(0, len(self.rows), 1 << 16):
            r, c = self.rows[s:s + (1 << 16)], self.cols[s:s + (1 << 16)]
            if d32:
                acc = np.zeros(len(r))
                for b0 in range(0, A.shape[1], 64):
                    acc += np.einsum("ij,ij->i", A32[r, b0:b0 + 64], A32[c, b0:b0 + 64]).astype(np.float64)
                low[s:s + (1 << 16)] = acc
            else:
                low[s:s + (1 << 16)] = np.einsum("ij,ij->i", A[r], A[c])
        res = self.cs - low
        res[self.diag] = np.maximum(res[self.diag], 0.0)
        vals = res * self.Tv
        vals[self.diag] += self.req.nugget
        Ss = sp.csr_matrix((vals, self.col, self.rowptr), shape=(self.n, self.n))
        return Ss, Ss.diagonal().copy()

    def core(self, A, D, m32):
        if not m32:
            return np.eye(self.m) + (A.T / D) @ A
        Mx = np.zeros((self.m, self.m))
        As, Di = A.astype(np.float32), (1.0 / D).astype(np.float32)
        for s0 in range(0, self.n, 512):
            blk = As[s0:s0 + 512]
            Mx += ((blk * Di[s0:s0 + 512, None]).T @ blk).astype(np.float64)
        return np.eye(self.m) + 0.5 * (Mx + Mx.T)

    def loglik(self, name, tol):
        n, m = self.n, self.m
        A = self.A64 if "a64" in name else self.A2
        m32, v32, s2, w32 = ("m32" in name), ("v32" in name), ("s2" in name), ("w32" in name)
        Ss, D = self.residual(A, "d32" in name)
        LM = np.linalg.cholesky(self.core(A, D, m32))
        logdetP = 2 * np.sum(np.log(np.diag(LM))) + np.sum(np.log(D))
        Minv = sla.cho_solve((LM, True), np.eye(m))
        cast = (lambda x: x.astype(np.float32).astype(np.float64)) if v32 else (lambda x: x)
        A32 = A.astype(np.float32)

        def AtX(X):
            if not w32:
                return A.T @ X
            out = np.zeros((m, X.shape[1]))
            X32 = X.astype(np.float32)
            for s0 in range(0, n, 4096):
                out += (A32[s0:s0 + 4096].T @ X32[s0:s0 + 4096]).astype(np.float64)
            return out

        def lowrank(R):
            X = R / D[:, None]
            q = Minv @ AtX(split2(X) if s2 else X)
            return cast(A @ (split2(q) if s2 else q))

        B = np.column_stack([self.y, A @ self.e1 + np.sqrt(D)[:, None] * self.e2])
        c = B.shape[1]
        R = cast(B.copy())
        U = np.zeros_like(R)
        S = lowrank(R)
        Z = cast((R - S) / D[:, None])
        rz = np.einsum("ij,ij->j", R, Z)
        V = cast(Ss @ Z + S)
        H = Z.copy()
        active = np.ones(c, bool)
        alpha_prev, beta_prev = np.ones(c), np.zeros(c)
        dg = [[] for _ in range(c)]
        of = [[] for _ in range(c)]
        it = 0
        for it in range(5000):
            if not active.any():
                break
            cl = np.nonzero(active)[0]
            alpha = rz[cl] / np.einsum("ij,ij->j", H[:, cl], V[:, cl])
            U[:, cl] = cast(U[:, cl] + alpha * H[:, cl])
            R[:, cl] = cast(R[:, cl] - alpha * V[:, cl])
            rn = np.linalg.norm(R[:, cl], axis=0)
            S = lowrank(R[:, cl])
            Zc = cast((R[:, cl] - S) / D[:, None])
            rzn = np.einsum("ij,ij->j", R[:, cl], Zc)
            beta = rzn / rz[cl]
            V[:, cl] = cast(Ss @ Zc + S + beta * V[:, cl])
            H[:, cl] = cast(Zc + beta * H[:, cl])
            for t, k in enumerate(cl):
                dg[k].append(1.0 / alpha[t] + beta_prev[k] / alpha_prev[k])
                if it > 0:
                    of[k].append(math.sqrt(beta_prev[k]) / alpha_prev[k])
            alpha_prev[cl], beta_prev[cl], rz[cl] = alpha, beta, rzn
            active[cl[rn < tol]] = False
        quads = np.array([O.lanczos_quadrature(dg[k], of[k]) for k in range(1, c)])
        logdet = n * quads.mean() + logdetP
        yu = float(self.y @ U[:, 0])
        return -0.5 * (n * O.LOG2PI + logdet + yu), logdet, yu, logdetP, it


def main():
    index, l, tol = int(sys.argv[1]), int(sys.argv[2]), float(sys.argv[3])
    configs = sys.argv[4].split(",")
    P = Request(index, l)
    print(P.req)
    out = {}
    for name in configs:
        t0 = time.time()
        out[name] = P.loglik(name, tol)
        print("%-20s ll %.8f logdet %.5f yu %.5f logdetP %.5f iters %d (%.0f s)"
              % ((name,) + out[name] + (time.time() - t0,)), flush=True)
    ref = out[configs[0]]
    for name, v in out.items():
        print("%-20s rel ll diff %.3e  (shares of |ll|: logdet %.2e, y^T u %.2e, logdet P %.2e)"
              % (name, abs(v[0] - ref[0]) / abs(ref[0]), (v[1] - ref[1]) / abs(ref[0]),
                 (v[2] - ref[2]) / abs(ref[0]), (v[3] - ref[3]) / abs(ref[0])))


if __name__ == "__main__":
    main()
