"""FP64 CPU oracle for the iterative full-scale approximation (FSA).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this module:
only the tests, the smoke check of ``__graft_entry__`` and the CPU-baseline /
reference legs of ``bench.py`` use it.  It shares no code with the CUDA path.

Source: Gyger, Furrer & Sigrist, "Iterative Methods for Full-Scale Gaussian
Process Approximations for Large Spatial Data" (arXiv 2405.14492).  Every
function cites the section / equation / algorithm it follows.

Two modes:
  * ``DenseFSA``     — the plain definition, n <= a few thousand: the FSA
                       covariance built densely (§2.1), dense Cholesky
                       log-likelihood and exact gradient (Eq. NEGLLDNEGLLFSA),
                       exact FSA predictive mean / variances (§2.3, Eq. MuPredFSA).
  * ``IterativeFSA`` — the paper's iterative algorithm step by step: the FITC
                       preconditioner (Eq. eqfitcp) with Woodbury / Sylvester
                       (appendix "Runtime of the FITC preconditioner"), the
                       preconditioned CG with Lanczos tridiagonals (Appendix A),
                       preconditioned SLQ and STE (§3.3), and the simulation
                       based predictive variances (Algorithm 1).

Readings of points where the paper is silent (the same list is kept with the
design notes of the repository):
  * Matérn parameterisation: r(d) = exp(-d/rho) (nu = 1/2) and
    (1 + sqrt(3) d/rho) exp(-sqrt(3) d/rho) (nu = 3/2), Sigma_ij = s1 * r(d_ij).
  * Taper: Wendland phi_{3,1}, T(d) = (1-d/g)^4 (1+4d/g) for d < g, else 0.
  * Support predicate: d^2 = dx*dx + dy*dy evaluated without fused
    multiply-add, pair in the support iff d^2 < g*g (g*g rounded once).
  * Residual diagonal s1 - |a_i|^2 is clamped at 0 (it is exactly 0 at
    inducing points in exact arithmetic).
  * The sampling factor "Sigma_m^{-1/2}" of the FITC sample is read as L^{-T}
    with Sigma_m = L L^T, so that the sample has covariance P_hat.
  * SLQ weight: the paper's n / l (exact weight z^T P^-1 z as an option).
  * CG stop: absolute ||r||_2 < tol on the unpreconditioned residual, u0 = 0.
  * Gradient control variate (appendix "Preconditioner as control variate"):
    P = P_hat; the clamp of the residual diagonal is not differentiated.  The
    printed c_opt (uncentred denominator) and the centred least-squares slope
    are both available, as is c = 1.
  * Fisher information by STE (appendix "Fisher scoring"): probes with
    E[z z^T] = I, no preconditioner in the estimate, symmetric part returned
    beside the raw estimate.
  * Vecchia with the FITC preconditioner (§5): conditioning on the nearest
    earlier points in the given order; Eq. VL_v2 as printed is not an
    identity, and the posterior solve uses
    (Sigma_V^-1 + W)^-1 = Sigma_V (Sigma_V + W^-1)^-1 W^-1 with the same system.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg  # noqa: F401  (sp.linalg.spsolve_triangular)

LOG2PI = math.log(2.0 * math.pi)
GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
STREAM_EPS2 = 4   # probe part on the n data points
STREAM_EPS1 = 5   # probe part on the m inducing points
STREAM_PRED = 6   # prediction-variance probes
STREAM_FISHER = 7   # Fisher-information probes
STREAM_KMEANSPP = 9   # kmeans++ selection of the inducing points


# ----------------------------------------------------------------------------
# Covariance function and taper (§2, Assumption 3; §2.1 taper)
# ----------------------------------------------------------------------------

def corr(d, nu: float, rho: float):
    """Matérn correlation r(d) for nu in {1/2, 3/2} (Assumption 3: r(0) = 1)."""
    d = np.asarray(d, dtype=np.float64)
    if nu == 0.5:
        return np.exp(-d / rho)
    if nu == 1.5:
        x = math.sqrt(3.0) * d / rho
        return (1.0 + x) * np.exp(-x)
    raise ValueError("nu must be 0.5 or 1.5")


def dcorr_drho(d, nu: float, rho: float):
    """Derivative of r(d) with respect to the range rho."""
    d = np.asarray(d, dtype=np.float64)
    if nu == 0.5:
        return (d / (rho * rho)) * np.exp(-d / rho)
    if nu == 1.5:
        x = math.sqrt(3.0) * d / rho
        return (x * x / rho) * np.exp(-x)
    raise ValueError("nu must be 0.5 or 1.5")


def taper(d, gamma: float):
    """Wendland taper phi_{3,1}: compactly supported on [0, gamma) (§2.1)."""
    d = np.asarray(d, dtype=np.float64)
    t = d / gamma
    out = (1.0 - t) ** 4 * (1.0 + 4.0 * t)
    return np.where(d < gamma, out, 0.0)


def sqdist(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Pairwise squared distances dx*dx + dy*dy, each operation rounded
    separately (numpy never fuses multiply and add)."""
    dx = a[:, None, 0] - b[None, :, 0]
    dy = a[:, None, 1] - b[None, :, 1]
    return dx * dx + dy * dy


def sqdist_pairs(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Row-wise squared distances between a[k] and b[k]."""
    dx = a[:, 0] - b[:, 0]
    dy = a[:, 1] - b[:, 1]
    return dx * dx + dy * dy


def cov_matrix(a: np.ndarray, b: np.ndarray, nu: float, sigma1_sq: float, rho: float):
    """Sigma_ab = sigma1^2 r(|a_i - b_j|) (§2)."""
    return sigma1_sq * corr(np.sqrt(sqdist(a, b)), nu, rho)


def dcov_matrix(a, b, nu, sigma1_sq, rho, which: int):
    """Derivative of sigma1^2 r(|a_i - b_j|) with respect to theta[which],
    theta = (sigma1^2, rho, nugget)."""
    d = np.sqrt(sqdist(a, b))
    if which == 0:
        return corr(d, nu, rho)
    if which == 1:
        return sigma1_sq * dcorr_drho(d, nu, rho)
    return np.zeros_like(d)


# ----------------------------------------------------------------------------
# Taper support: the neighbour structure (§2.1)
# ----------------------------------------------------------------------------

def neighbour_csr(rows_pts: np.ndarray, cols_pts: np.ndarray, gamma: float,
                  brute_force_limit: int = 4_000_000):
    """CSR structure of {(i, j) : |r_i - c_j|^2 < gamma^2} with columns in
    ascending order (self pairs included when rows_pts is cols_pts).

    Small problems: brute force over all pairs.  Larger ones: candidate pairs
    from a k-d tree with a slightly larger radius, then the exact predicate.
    """
    g2 = gamma * gamma
    nr, nc = rows_pts.shape[0], cols_pts.shape[0]
    rows_out, cols_out = [], []
    if nr * nc <= brute_force_limit:
        step = max(1, brute_force_limit // max(nc, 1))
        for s in range(0, nr, step):
            d2 = sqdist(rows_pts[s:s + step], cols_pts)
            r, c = np.nonzero(d2 < g2)
            rows_out.append(r + s)
            cols_out.append(c)
    else:
        from scipy.spatial import cKDTree
        tree = cKDTree(cols_pts)
        cand = tree.query_ball_point(rows_pts, r=gamma * (1.0 + 1e-6))
        lens = np.fromiter((len(x) for x in cand), dtype=np.int64, count=nr)
        r = np.repeat(np.arange(nr, dtype=np.int64), lens)
        c = np.fromiter((j for lst in cand for j in lst), dtype=np.int64, count=int(lens.sum()))
        keep = sqdist_pairs(rows_pts[r], cols_pts[c]) < g2
        rows_out.append(r[keep])
        cols_out.append(c[keep])
    r = np.concatenate(rows_out) if rows_out else np.zeros(0, np.int64)
    c = np.concatenate(cols_out) if cols_out else np.zeros(0, np.int64)
    order = np.lexsort((c, r))
    r, c = r[order], c[order]
    rowptr = np.zeros(nr + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr)
    return rowptr, c.astype(np.int32)


# ----------------------------------------------------------------------------
# Counter-based SplitMix64 (Steele, Lea & Flood, OOPSLA 2014)
# ----------------------------------------------------------------------------

def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (mix64 variant with shifts 30, 27, 31)."""
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= np.uint64(0xBF58476D1CE4E5B9)
        z ^= z >> np.uint64(27)
        z *= np.uint64(0x94D049BB133111EB)
        z ^= z >> np.uint64(31)
    return z


def splitmix64(seed: int, stream: int, counters: np.ndarray) -> np.ndarray:
    """Output number `counter` of a SplitMix64 generator whose state is
    seeded with key = mix64(seed XOR stream*gamma): mix64(key + (counter+1)*gamma)."""
    with np.errstate(over="ignore"):
        key = _mix64(np.array([np.uint64(seed) ^ (np.uint64(stream) * GOLDEN_GAMMA)], dtype=np.uint64))[0]
        c = counters.astype(np.uint64) + np.uint64(1)
        state = key + c * GOLDEN_GAMMA
    return _mix64(state)


# ----------------------------------------------------------------------------
# kmeans++ selection of inducing points (§4.1; Arthur & Vassilvitskii 2007)
# ----------------------------------------------------------------------------

def kmeanspp_scale_exponent(locs: np.ndarray) -> int:
    """Exponent e of the integer D^2 weights floor(d^2 * 2^e): the squared
    bounding-box diagonal times 2^e stays <= 2^B with B = 62 - bitlength(n),
    so that n weights sum to less than 2^62."""
    n = locs.shape[0]
    dx = float(locs[:, 0].max() - locs[:, 0].min())
    dy = float(locs[:, 1].max() - locs[:, 1].min())
    diag2 = dx * dx + dy * dy
    B = 62 - int(n).bit_length()
    if diag2 == 0.0:
        return B
    _, ex = math.frexp(diag2)          # diag2 = f * 2^ex, f in [0.5, 1)
    return B - ex


def kmeanspp(locs: np.ndarray, m: int, seed: int) -> np.ndarray:
    """Indices of m inducing points chosen by kmeans++ seeding (D^2 sampling):
    the first point uniformly, each further point i with probability
    proportional to its squared distance to the nearest point chosen so far.
    Weights are the integers q_i = floor(d_i^2 2^e) (d^2 = dx*dx + dy*dy, each
    operation rounded on its own; e from ``kmeanspp_scale_exponent``), so
    sums are exact.  Draw k uses h_k = SplitMix64(seed, stream 9, counter k)
    >> 11 (53 bits): the first index is floor(h_0 n / 2^53); step k picks the
    first i whose inclusive prefix sum of q exceeds floor(h_k Q / 2^53), Q the
    total.  Raises ValueError when fewer than m distinct locations exist."""
    n = locs.shape[0]
    if not (1 <= m <= n):
        raise ValueError("need 1 <= m <= n")
    e = kmeanspp_scale_exponent(locs)
    h = splitmix64(seed, STREAM_KMEANSPP, np.arange(m, dtype=np.uint64)) >> np.uint64(11)
    first = (int(h[0]) * n) >> 53
    idx = [first]

    def weights(c):
        dx = locs[:, 0] - locs[c, 0]
        dy = locs[:, 1] - locs[c, 1]
        d2 = dx * dx + dy * dy
        return np.floor(np.ldexp(d2, e)).astype(np.uint64)

    q = weights(first)
    for k in range(1, m):
        cum = np.cumsum(q, dtype=np.uint64)
        total = int(cum[-1])
        if total == 0:
            raise ValueError("fewer than m distinct locations")
        target = (int(h[k]) * total) >> 53
        i = int(np.searchsorted(cum, np.uint64(target), side="right"))
        idx.append(i)
        q = np.minimum(q, weights(i))
    return np.array(idx, dtype=np.int64)


def rademacher(seed: int, stream: int, rows: np.ndarray, nrows: int, ncols: int) -> np.ndarray:
    """(len(rows), ncols) matrix of +-1 with entry (r, k) drawn at counter
    k * nrows + rows[r] (rows are ORIGINAL indices, so the draw does not
    depend on any internal reordering)."""
    rows = np.asarray(rows, dtype=np.uint64)
    cols = np.arange(ncols, dtype=np.uint64)
    ctr = cols[None, :] * np.uint64(nrows) + rows[:, None]
    h = splitmix64(seed, stream, ctr.ravel()).reshape(ctr.shape)
    return 1.0 - 2.0 * (h >> np.uint64(63)).astype(np.float64)


def gaussian(seed: int, stream: int, rows: np.ndarray, nrows: int, ncols: int) -> np.ndarray:
    """Standard normals by Box-Muller from the counter pair (2c, 2c+1),
    c = k * nrows + row, u = ((h >> 11) + 1) * 2^-53 in (0, 1]."""
    rows = np.asarray(rows, dtype=np.uint64)
    cols = np.arange(ncols, dtype=np.uint64)
    ctr = (cols[None, :] * np.uint64(nrows) + rows[:, None]).ravel()
    h1 = splitmix64(seed, stream, ctr * np.uint64(2))
    h2 = splitmix64(seed, stream, ctr * np.uint64(2) + np.uint64(1))
    u1 = ((h1 >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = ((h2 >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)
    return z.reshape(len(rows), ncols)


# ----------------------------------------------------------------------------
# Dense-exact mode (plain definitions; n up to a few thousand)
# ----------------------------------------------------------------------------

class DenseFSA:
    """The FSA covariance built densely from its definition (§2.1):
    Sigma_l = Sigma_mn^T Sigma_m^-1 Sigma_mn,
    Sigma_s = (Sigma - Sigma_l) o T(gamma),
    Sigma_dag = Sigma_l + Sigma_s + nugget I."""

    def __init__(self, locs, inducing, gamma, nu, theta):
        self.locs = np.asarray(locs, np.float64)
        self.inducing = np.asarray(inducing, np.float64)
        self.gamma, self.nu = float(gamma), float(nu)
        self.theta = tuple(float(t) for t in theta)
        s1, rho, nug = self.theta
        n = self.locs.shape[0]
        d2 = sqdist(self.locs, self.locs)
        self.support = d2 < gamma * gamma
        d = np.sqrt(d2)
        self.T = np.where(self.support, taper(d, gamma), 0.0)
        self.Sigma = s1 * corr(d, nu, rho)
        self.K = cov_matrix(self.inducing, self.locs, nu, s1, rho)          # m x n
        self.Sm = cov_matrix(self.inducing, self.inducing, nu, s1, rho)     # m x m
        self.Sl = self.K.T @ np.linalg.solve(self.Sm, self.K)
        self.Sl = 0.5 * (self.Sl + self.Sl.T)
        resid = self.Sigma - self.Sl
        # residual diagonal clamped at 0 (a reading; exact 0 at inducing points)
        np.fill_diagonal(resid, np.maximum(np.diag(resid), 0.0))
        self.Ss = resid * self.T + nug * np.eye(n)
        self.Sdag = self.Sl + self.Ss
        self.D = np.diag(self.Ss).copy()
        self.Phat = np.diag(self.D) + self.Sl           # Eq. (eqfitcp)

    # -- log-likelihood and exact gradient (Eq. NEGLLDNEGLLFSA) --------------
    def loglik(self, y):
        """l(theta) = -[n/2 log 2pi + 1/2 logdet Sigma_dag + 1/2 y^T Sigma_dag^-1 y]."""
        c, low = sla.cho_factor(self.Sdag, lower=True)
        logdet = 2.0 * np.sum(np.log(np.diag(c)))
        u = sla.cho_solve((c, low), y)
        n = y.shape[0]
        return -0.5 * (n * LOG2PI + logdet + float(y @ u)), logdet, float(y @ u)

    def dSdag(self, which: int) -> np.ndarray:
        """dSigma_dag/dtheta (§2.2): dSigma_l + (dSigma - dSigma_l) o T + dnugget I,
        with dSigma_l = dK^T Sm^-1 K + K^T Sm^-1 dK - K^T Sm^-1 dSm Sm^-1 K."""
        s1, rho, nug = self.theta
        n = self.locs.shape[0]
        if which == 2:
            return np.eye(n)
        dK = dcov_matrix(self.inducing, self.locs, self.nu, s1, rho, which)
        dSm = dcov_matrix(self.inducing, self.inducing, self.nu, s1, rho, which)
        dSig = dcov_matrix(self.locs, self.locs, self.nu, s1, rho, which)
        SmK = np.linalg.solve(self.Sm, self.K)
        dSl = dK.T @ SmK + SmK.T @ dK - SmK.T @ dSm @ SmK
        return dSl + (dSig - dSl) * self.T

    def grad(self, y):
        """Exact d l / d theta = -1/2 [tr(Sdag^-1 dSdag) - u^T dSdag u] (Eq. NEGLLDNEGLLFSA)."""
        Sinv = np.linalg.inv(self.Sdag)
        u = Sinv @ y
        g = np.zeros(3)
        for k in range(3):
            dS = self.dSdag(k)
            g[k] = -0.5 * (np.sum(Sinv * dS.T) - u @ dS @ u)
        return g

    def dPhat(self, which: int) -> np.ndarray:
        """dP_hat/dtheta for P_hat = D_s + Sigma_l (Eq. eqfitcp): the low-rank
        derivative dSigma_l off the diagonal, d(Sigma_ii) on it (the taper is 1
        there, so dD_s,i = dSigma_ii - dSigma_l,ii); the identity for the nugget."""
        s1, rho, nug = self.theta
        n = self.locs.shape[0]
        if which == 2:
            return np.eye(n)
        dK = dcov_matrix(self.inducing, self.locs, self.nu, s1, rho, which)
        dSm = dcov_matrix(self.inducing, self.inducing, self.nu, s1, rho, which)
        dSig_diag = np.diag(dcov_matrix(self.locs, self.locs, self.nu, s1, rho, which))
        SmK = np.linalg.solve(self.Sm, self.K)
        dSl = dK.T @ SmK + SmK.T @ dK - SmK.T @ dSm @ SmK
        return dSl + np.diag(dSig_diag - np.diag(dSl))

    def fisher(self) -> np.ndarray:
        """Exact Fisher information (appendix "Fisher scoring"):
        I_kl = 1/2 tr(Sdag^-1 dSdag_k Sdag^-1 dSdag_l)."""
        X = [np.linalg.solve(self.Sdag, self.dSdag(k)) for k in range(3)]
        return np.array([[0.5 * np.sum(X[k] * X[l].T) for l in range(3)] for k in range(3)])

    # -- exact FSA predictive distribution (§2.3, Eq. MuPredFSA) -------------
    def cross(self, pred):
        """Sigma^dag_{n,np} = Sigma^l_{n,np} + (Sigma_{n,np} - Sigma^l_{n,np}) o T_{n,np}."""
        s1, rho, nug = self.theta
        Kp = cov_matrix(self.inducing, pred, self.nu, s1, rho)
        Snp = cov_matrix(self.locs, pred, self.nu, s1, rho)
        Sl_np = self.K.T @ np.linalg.solve(self.Sm, Kp)
        d2 = sqdist(self.locs, pred)
        Tnp = np.where(d2 < self.gamma * self.gamma, taper(np.sqrt(d2), self.gamma), 0.0)
        Ss_np = (Snp - Sl_np) * Tnp
        return Sl_np + Ss_np, Sl_np, Ss_np, Kp

    def predict(self, y, pred):
        """mu^p = (Sigma^dag_{n,np})^T Sigma_dag^-1 y and
        var^p = sigma1^2 + nugget - diag((Sigma^dag_{n,np})^T Sigma_dag^-1 Sigma^dag_{n,np})."""
        s1, rho, nug = self.theta
        C, _, _, _ = self.cross(pred)
        c = sla.cho_factor(self.Sdag, lower=True)
        mu = C.T @ sla.cho_solve(c, y)
        var = s1 + nug - np.sum(C * sla.cho_solve(c, C), axis=0)
        return mu, var


class VecchiaFITC:
    """A Vecchia approximation of the latent GP with a Gaussian likelihood,
    solved by CG under the FITC preconditioner (§5, "The FITC preconditioner
    for Vecchia approximations").

    Vecchia: in the given order, N(i) holds the min(m_v, i - 1) nearest of the
    earlier points (squared distances as in ``sqdist``, ties to the lower
    index), A_i = Sigma_{N(i),i}^T Sigma_{N(i)}^-1, D_i = Sigma_ii -
    A_i Sigma_{N(i),i}; B is unit lower triangular with B_{i,N(i)} = -A_i, and
    Sigma_V^-1 = B^T D^-1 B.  With the Gaussian likelihood W = I / nugget, the
    response has covariance Sigma_V + W^-1.  FITC: P_hat = Sigma_mn^T
    Sigma_m^-1 Sigma_mn + D_s with D_s = diag(Sigma - Sigma_mn^T Sigma_m^-1
    Sigma_mn) + W^-1 (the residual diagonal clamped at 0), applied by Woodbury
    with the core M_P = Sigma_m + Sigma_mn D_s^-1 Sigma_nm."""

    def __init__(self, locs, inducing, m_v, nu, theta):
        self.locs = np.asarray(locs, np.float64)
        self.inducing = np.asarray(inducing, np.float64)
        self.nu, self.m_v = float(nu), int(m_v)
        self.theta = tuple(float(t) for t in theta)
        s1, rho, nug = self.theta
        n = self.n = self.locs.shape[0]
        rows, cols, vals = list(range(n)), list(range(n)), [1.0] * n
        self.D = np.empty(n)
        self.N = []
        for i in range(n):
            k = min(self.m_v, i)
            if k == 0:
                Ni = np.zeros(0, dtype=np.int64)
            else:
                d2 = sqdist(self.locs[i:i + 1], self.locs[:i])[0]
                Ni = np.sort(np.argsort(d2, kind="stable")[:k])
            self.N.append(Ni)
            if k == 0:
                self.D[i] = s1
                continue
            SNN = cov_matrix(self.locs[Ni], self.locs[Ni], nu, s1, rho)
            SNi = cov_matrix(self.locs[Ni], self.locs[i:i + 1], nu, s1, rho)[:, 0]
            Ai = np.linalg.solve(SNN, SNi)
            self.D[i] = s1 - float(Ai @ SNi)
            rows += [i] * k
            cols += Ni.tolist()
            vals += (-Ai).tolist()
        self.B = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
        self.BT = self.B.T.tocsr()
        # FITC preconditioner (the same construction as Eq. eqfitcp, nugget as W^-1)
        self.K = cov_matrix(self.inducing, self.locs, nu, s1, rho)
        self.Lm = np.linalg.cholesky(cov_matrix(self.inducing, self.inducing, nu, s1, rho))
        Al = sla.solve_triangular(self.Lm, self.K, lower=True)              # m x n
        self.Ds = np.maximum(s1 - np.sum(Al * Al, axis=0), 0.0) + nug
        self.Lp = np.linalg.cholesky(self.Lm @ self.Lm.T + (self.K / self.Ds) @ self.K.T)
        self.logdet_P = (2.0 * np.sum(np.log(np.diag(self.Lp))) - 2.0 * np.sum(np.log(np.diag(self.Lm)))
                         + float(np.sum(np.log(self.Ds))))

    def apply_SigmaV(self, V):
        """Sigma_V V = B^-1 D B^-T V (two sparse triangular solves)."""
        X = sp.linalg.spsolve_triangular(self.BT, V, lower=False)
        X = X * (self.D[:, None] if X.ndim == 2 else self.D)
        return sp.linalg.spsolve_triangular(self.B, X, lower=True)

    def apply(self, V):
        """(Sigma_V + W^-1) V, the response covariance."""
        return self.apply_SigmaV(V) + self.theta[2] * V

    def apply_Pinv(self, V):
        """P_hat^-1 V by Woodbury."""
        V = np.asarray(V)
        Ds = self.Ds[:, None] if V.ndim == 2 else self.Ds
        DV = V / Ds
        return DV - (self.K.T @ sla.cho_solve((self.Lp, True), self.K @ DV)) / Ds

    def probes(self, num_probes, seed):
        """z = Sigma_mn^T L_m^-T eps1 + D_s^1/2 eps2 ~ (0, P_hat), Rademacher eps
        (streams 5 and 4)."""
        e1 = rademacher(seed, STREAM_EPS1, np.arange(self.inducing.shape[0]), self.inducing.shape[0], num_probes)
        e2 = rademacher(seed, STREAM_EPS2, np.arange(self.n), self.n, num_probes)
        return self.K.T @ sla.solve_triangular(self.Lm.T, e1, lower=False) + np.sqrt(self.Ds)[:, None] * e2

    def loglik(self, y, num_probes, seed, tol, max_iter=5000, Z=None):
        """-1/2 [n log 2 pi + logdet(Sigma_V + W^-1) + y^T (Sigma_V + W^-1)^-1 y]
        with the log-determinant by preconditioned SLQ (weight n / l, §3.3)."""
        if Z is None:
            Z = self.probes(num_probes, seed)
        res = pcg_lanczos(self.apply, self.apply_Pinv, np.column_stack([y, Z]), tol, max_iter)
        quads = np.array([lanczos_quadrature(res["diag"][k], res["off"][k]) for k in range(1, Z.shape[1] + 1)])
        logdet = self.n * float(np.mean(quads)) + self.logdet_P
        yu = float(y @ res["U"][:, 0])
        return dict(loglik=-0.5 * (self.n * LOG2PI + logdet + yu), logdet=logdet, quad=yu, iters=res["iters"])

    def posterior_solve(self, v, tol, max_iter=5000, precondition=True):
        """(Sigma_V^-1 + W)^-1 v through the system of Eq. VL_v2, whose matrix
        Sigma_V + W^-1 is solved by CG under the FITC preconditioner (or none).
        As printed, W (Sigma_V + W^-1)^-1 Sigma_V^-1 v is not equal to
        (Sigma_V^-1 + W)^-1 v (for scalars it is w^2 / s^2 times it); the
        identity with the same system is
            (Sigma_V^-1 + W)^-1 = Sigma_V (Sigma_V + W^-1)^-1 W^-1,
        which is what is computed: solve with W^-1 v, then apply Sigma_V."""
        rhs = self.theta[2] * np.asarray(v, np.float64).reshape(self.n, -1)      # W^-1 v
        pinv = self.apply_Pinv if precondition else (lambda V: V.copy())
        res = pcg_lanczos(self.apply, pinv, rhs, tol, max_iter)
        return self.apply_SigmaV(res["U"]), res["iters"]


def fisher_scoring_step(theta, grad, fisher):
    """One Fisher-scoring update (appendix "Fisher scoring"):
    theta + I^-1 dl/dtheta, with l the log-likelihood (so the step ascends l)."""
    return np.asarray(theta, np.float64) + np.linalg.solve(np.asarray(fisher, np.float64),
                                                          np.asarray(grad, np.float64))


# ----------------------------------------------------------------------------
# Iterative mode (the paper's algorithms, step by step)
# ----------------------------------------------------------------------------

def pcg_lanczos(apply_A, apply_Pinv, B, tol, max_iter, fixed_iters=0):
    """Preconditioned CG with Lanczos tridiagonals (Appendix A), for every
    column of B independently (each column stops at its own first iteration
    with ||r||_2 < tol; fixed_iters > 0 runs exactly that many iterations).

    Returns U (solutions), Z0 = P^-1 B, and per column the diagonal and
    off-diagonal of T_tilde, the number of iterations and ||r||."""
    n, c = B.shape
    U = np.zeros_like(B)
    R = B.copy()
    Z = apply_Pinv(R)
    Z0 = Z.copy()
    H = Z.copy()
    rz = np.einsum("ij,ij->j", R, Z)
    rz0 = rz.copy()
    alpha_prev = np.ones(c)
    beta_prev = np.zeros(c)
    active = np.ones(c, dtype=bool)
    diag = [[] for _ in range(c)]
    off = [[] for _ in range(c)]
    iters = np.zeros(c, dtype=np.int64)
    rnorm = np.linalg.norm(R, axis=0)
    n_iter = fixed_iters if fixed_iters > 0 else max_iter
    for l in range(n_iter):
        if not active.any():
            break
        cols = np.nonzero(active)[0]
        V = apply_A(H[:, cols])
        alpha = rz[cols] / np.einsum("ij,ij->j", H[:, cols], V)
        U[:, cols] += alpha * H[:, cols]
        R[:, cols] -= alpha * V
        rn = np.linalg.norm(R[:, cols], axis=0)
        stop = (rn < tol) if fixed_iters <= 0 else np.zeros(len(cols), dtype=bool)
        Zc = apply_Pinv(R[:, cols])
        rz_new = np.einsum("ij,ij->j", R[:, cols], Zc)
        beta = rz_new / rz[cols]
        H[:, cols] = Zc + beta * H[:, cols]
        for t, k in enumerate(cols):
            diag[k].append(1.0 / alpha[t] + beta_prev[k] / alpha_prev[k])
            if l > 0:
                off[k].append(math.sqrt(beta_prev[k]) / alpha_prev[k])
            iters[k] = l + 1
            rnorm[k] = rn[t]
        alpha_prev[cols] = alpha
        beta_prev[cols] = beta
        rz[cols] = rz_new
        active[cols[stop]] = False
    return dict(U=U, Z0=Z0, diag=diag, off=off, iters=iters, rnorm=rnorm, rz0=rz0,
                R=R, converged=not active.any() or fixed_iters > 0)


def lanczos_quadrature(diag, off) -> float:
    """e_1^T log(T) e_1 = sum_j q_1j^2 log(lambda_j) for the tridiagonal T
    (stochastic Lanczos quadrature, §3.1)."""
    d = np.asarray(diag, np.float64)
    e = np.asarray(off, np.float64)
    if d.size == 1:
        return float(math.log(d[0]))
    lam, Q = sla.eigh_tridiagonal(d, e)
    return float(np.sum(Q[0, :] ** 2 * np.log(lam)))


class IterativeFSA:
    """The iterative FSA computations with sparse structures (§3)."""

    def __init__(self, locs, inducing, gamma, nu, theta, csr=None):
        self.locs = np.asarray(locs, np.float64)
        self.inducing = np.asarray(inducing, np.float64)
        self.gamma, self.nu = float(gamma), float(nu)
        self.theta = tuple(float(t) for t in theta)
        s1, rho, nug = self.theta
        self.n, self.m = self.locs.shape[0], self.inducing.shape[0]
        # low-rank part (§2.1): K = Sigma_mn, Sm = Sigma_m, A = K^T L^-T
        self.K = cov_matrix(self.inducing, self.locs, nu, s1, rho)
        self.Sm = cov_matrix(self.inducing, self.inducing, nu, s1, rho)
        try:
            self.Lm = np.linalg.cholesky(self.Sm)
        except np.linalg.LinAlgError as exc:
            raise ValueError("Sigma_m is not positive definite") from exc
        self.A = sla.solve_triangular(self.Lm, self.K, lower=True).T      # n x m
        # tapered residual (§2.1) on the taper support
        if csr is None:
            csr = neighbour_csr(self.locs, self.locs, gamma)
        self.rowptr, self.col = csr
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        cols = self.col.astype(np.int64)
        self.rows = rows
        d = np.sqrt(sqdist_pairs(self.locs[rows], self.locs[cols]))
        self.d = d
        Tv = taper(d, gamma)
        lowrank = self._rowdots(self.A, self.A, rows, cols)
        resid = s1 * corr(d, nu, rho) - lowrank
        diag_mask = rows == cols
        resid[diag_mask] = np.maximum(resid[diag_mask], 0.0)
        vals = resid * Tv
        vals[diag_mask] += nug
        self.vals = vals
        self.Tv = Tv
        self.Ss = sp.csr_matrix((vals, self.col, self.rowptr), shape=(self.n, self.n))
        self.D = self.Ss.diagonal().copy()                    # D_s = diag(Sigma_s tilde)
        # FITC preconditioner (Eq. eqfitcp) via Sylvester / Woodbury with the
        # paper's core M_P = Sigma_m + Sigma_mn D^-1 Sigma_nm
        self.Mp = self.Sm + (self.K / self.D) @ self.K.T
        self.Lp = np.linalg.cholesky(self.Mp)
        self.logdet_P = (2.0 * np.sum(np.log(np.diag(self.Lp)))
                         - 2.0 * np.sum(np.log(np.diag(self.Lm)))
                         + float(np.sum(np.log(self.D))))

    @staticmethod
    def _rowdots(X, Y, rows, cols, chunk=1 << 18):
        out = np.empty(rows.shape[0])
        for s in range(0, rows.shape[0], chunk):
            out[s:s + chunk] = np.einsum("ij,ij->i", X[rows[s:s + chunk]], Y[cols[s:s + chunk]])
        return out

    # -- operators -----------------------------------------------------------
    def apply_Sl(self, V):
        """Sigma_mn^T Sigma_m^-1 Sigma_mn V (§3.1)."""
        return self.K.T @ sla.cho_solve((self.Lm, True), self.K @ V)

    def apply(self, V):
        """Sigma_dag V = Sigma_s~ V + Sigma_mn^T Sigma_m^-1 Sigma_mn V (§3.1)."""
        return self.Ss @ V + self.apply_Sl(V)

    def apply_Pinv(self, V):
        """P^-1 V = D^-1 V - D^-1 K^T M_P^-1 K D^-1 V (Woodbury, appendix
        'Runtime of the FITC preconditioner')."""
        V = np.asarray(V)
        DV = V / self.D[:, None] if V.ndim == 2 else V / self.D
        t = sla.cho_solve((self.Lp, True), self.K @ DV)
        corr_ = self.K.T @ t
        return DV - (corr_ / self.D[:, None] if V.ndim == 2 else corr_ / self.D)

    def apply_Dinv(self, V):
        return V / self.D[:, None] if V.ndim == 2 else V / self.D

    # -- probes (§3.3, appendix 'Runtime of the FITC preconditioner') --------
    def probes(self, num_probes, seed, kind="rademacher"):
        """z = Sigma_mn^T L^-T eps1 + D^1/2 eps2 ~ (0, P_hat); eps1 (m x l) on
        stream 5, eps2 (n x l) on stream 4."""
        draw = rademacher if kind == "rademacher" else gaussian
        e1 = draw(seed, STREAM_EPS1, np.arange(self.m), self.m, num_probes)
        e2 = draw(seed, STREAM_EPS2, np.arange(self.n), self.n, num_probes)
        return self.K.T @ sla.solve_triangular(self.Lm.T, e1, lower=False) + np.sqrt(self.D)[:, None] * e2

    # -- log-likelihood and STE gradient -------------------------------------
    def dS_apply(self, which, V):
        """dSigma_dag/dtheta V (§2.2) with the sparse part evaluated per nonzero."""
        s1, rho, nug = self.theta
        if which == 2:
            return V.copy()
        dK = dcov_matrix(self.inducing, self.locs, self.nu, s1, rho, which)
        dSm = dcov_matrix(self.inducing, self.inducing, self.nu, s1, rho, which)
        cho = (self.Lm, True)
        C = sla.cho_solve(cho, self.K)                     # Sm^-1 K  (m x n)
        # low-rank part applied through m-space products
        KV = self.K @ V
        dSl_V = dK.T @ sla.cho_solve(cho, KV) + C.T @ (dK @ V) - C.T @ (dSm @ sla.cho_solve(cho, KV))
        # sparse part: per nonzero (dSigma_ij - dSigma_l,ij) T_ij
        rows, cols = self.rows, self.col.astype(np.int64)
        if which == 0:
            dsig = corr(self.d, self.nu, rho)
        else:
            dsig = s1 * dcorr_drho(self.d, self.nu, rho)
        dl = (self._rowdots(dK.T, C.T, rows, cols) + self._rowdots(C.T, dK.T, rows, cols)
              - self._rowdots(C.T, (dSm @ C).T, rows, cols))
        dvals = (dsig - dl) * self.Tv
        dSs = sp.csr_matrix((dvals, self.col, self.rowptr), shape=(self.n, self.n))
        return dSs @ V + dSl_V

    def _dlowrank(self, which):
        """dSigma_mn, dSigma_m and C = Sigma_m^-1 Sigma_mn for theta[which] < 2."""
        s1, rho, nug = self.theta
        dK = dcov_matrix(self.inducing, self.locs, self.nu, s1, rho, which)
        dSm = dcov_matrix(self.inducing, self.inducing, self.nu, s1, rho, which)
        C = sla.cho_solve((self.Lm, True), self.K)
        return dK, dSm, C

    def dD(self, which):
        """dD_s/dtheta: dSigma_ii - dSigma_l,ii per point (the taper is 1 on the
        diagonal), 1 for the nugget; dSigma_l,ii = 2 dk_i.c_i - c_i.(dSigma_m c_i)."""
        if which == 2:
            return np.ones(self.n)
        s1, rho, nug = self.theta
        dK, dSm, C = self._dlowrank(which)
        dsig0 = 1.0 if which == 0 else 0.0          # d(s1 r(0)) with r(0) = 1
        dl = 2.0 * np.einsum("ij,ij->j", dK, C) - np.einsum("ij,ij->j", C, dSm @ C)
        return dsig0 - dl

    def dP_apply(self, which, V):
        """dP_hat/dtheta V = dD_s V + dSigma_l V (Eq. eqfitcp differentiated),
        dSigma_l = dK^T Sm^-1 K + K^T Sm^-1 dK - K^T Sm^-1 dSm Sm^-1 K."""
        V = np.asarray(V, np.float64)
        dD = self.dD(which)
        out = dD[:, None] * V if V.ndim == 2 else dD * V
        if which == 2:
            return out
        dK, dSm, C = self._dlowrank(which)
        return out + dK.T @ (C @ V) + C.T @ (dK @ V) - C.T @ (dSm @ (C @ V))

    def trace_Pinv_dP(self, which):
        """Tr(P_hat^-1 dP_hat/dtheta) in O(n m^2) (appendix "Runtime of the FITC
        preconditioner": like the log-determinant): Jacobi's formula applied to
        the Sylvester identity logdet P_hat = logdet M_P - logdet Sigma_m + logdet D_s,
            Tr(M_P^-1 dM_P) - Tr(Sigma_m^-1 dSigma_m) + sum_i dD_i / D_i,
        dM_P = dSigma_m + dK D^-1 K^T + K D^-1 dK^T - K diag(dD / D^2) K^T."""
        dD = self.dD(which)
        K, D = self.K, self.D
        dMp = -(K * (dD / D ** 2)) @ K.T
        tr_m = 0.0
        if which < 2:
            dK, dSm, _ = self._dlowrank(which)
            KdK = (K / D) @ dK.T
            dMp += dSm + KdK + KdK.T
            tr_m = float(np.trace(sla.cho_solve((self.Lm, True), dSm)))
        return float(np.trace(sla.cho_solve((self.Lp, True), dMp))) - tr_m + float(np.sum(dD / D))

    def loglik_grad(self, y, num_probes, seed, tol, max_iter=1000, fixed_iters=0,
                    probe="rademacher", exact_weight=False, want_grad=True, Z=None,
                    control_variate=None):
        """Log-likelihood by preconditioned SLQ (§3.3) and gradient by STE (§3.3).
        ``Z`` replaces the random probes (used by deterministic checks).

        ``control_variate`` ("copt" or "c1") uses the preconditioner as control
        variate in the trace estimate (appendix "Preconditioner as control
        variate", Eq. Troptc): per parameter, with a_k = U_k^T dSdag W_k (the
        plain STE term) and b_k = W_k^T dP_hat W_k (W = P_hat^-1 Z),
            Tr(Sdag^-1 dSdag) ~ (1/l) sum_k (a_k - c b_k) + c Tr(P_hat^-1 dP_hat),
        c = c_opt = sum_k (a_k - mean a) b_k / sum_k b_k^2 (as printed; 0 where
        sum_k b_k^2 = 0), c = 1 ("c1"), or ("copt_centered") the variance-
        minimising slope sum_k (a_k - mean a)(b_k - mean b) / sum_k (b_k - mean b)^2
        (0 where the denominator vanishes).  The printed denominator is not
        centred: where mean b dominates the spread of b, as it does here
        (mean b estimates Tr(P_hat^-1 dP_hat)), the printed c_opt is near 0 and
        the estimate is close to the plain one."""
        if control_variate not in (None, "copt", "copt_centered", "c1"):
            raise ValueError("control_variate must be None, 'copt', 'copt_centered' or 'c1'")
        n = self.n
        if Z is None:
            Z = self.probes(num_probes, seed, probe)
        num_probes = Z.shape[1]
        B = np.column_stack([y, Z])
        res = pcg_lanczos(self.apply, self.apply_Pinv, B, tol, max_iter, fixed_iters)
        quads = np.array([lanczos_quadrature(res["diag"][k], res["off"][k]) for k in range(1, num_probes + 1)])
        weights = res["rz0"][1:] if exact_weight else np.full(num_probes, float(n))
        terms = weights * quads
        logdet = float(np.mean(terms)) + self.logdet_P
        u = res["U"][:, 0]
        yu = float(y @ u)
        ll = -0.5 * (n * LOG2PI + logdet + yu)
        out = dict(loglik=ll, logdet=logdet, quad=yu, logdet_P=self.logdet_P,
                   logdet_se=float(np.std(terms, ddof=1) / math.sqrt(num_probes)) if num_probes > 1 else 0.0,
                   iters=res["iters"], rnorm=res["rnorm"], Z=Z, res=res, quads=quads)
        if want_grad:
            U = res["U"][:, 1:]
            W = res["Z0"][:, 1:]                # P^-1 z
            g = np.zeros(3)
            g_terms = np.zeros((3, num_probes))
            cv_c, cv_terms, trace_P = np.zeros(3), np.zeros((3, num_probes)), np.zeros(3)
            for k in range(3):
                dW = self.dS_apply(k, np.column_stack([W, u]))
                per_probe = np.einsum("ij,ij->j", U, dW[:, :num_probes])
                tr = float(np.mean(per_probe))
                if control_variate is not None:
                    b = np.einsum("ij,ij->j", W, self.dP_apply(k, W))
                    trace_P[k] = self.trace_Pinv_dP(k)
                    if control_variate == "c1":
                        c = 1.0
                    elif control_variate == "copt":
                        den = float(np.sum(b * b))
                        c = float(np.sum((per_probe - tr) * b)) / den if den > 0 else 0.0
                    else:
                        bc = b - np.mean(b)
                        den = float(np.sum(bc * bc))
                        c = float(np.sum((per_probe - tr) * bc)) / den if den > 0 else 0.0
                    tr = float(np.mean(per_probe - c * b)) + c * trace_P[k]
                    cv_c[k], cv_terms[k] = c, b
                qf = float(u @ dW[:, num_probes])
                g[k] = -0.5 * (tr - qf)
                g_terms[k] = per_probe
            out["grad"] = g
            out["grad_terms"] = g_terms
            if control_variate is not None:
                out["cv_c"], out["cv_terms"], out["trace_P"] = cv_c, cv_terms, trace_P
        return out

    # -- Fisher information by STE (appendix "Fisher scoring") ---------------
    def fisher_ste(self, num_probes, seed, tol, max_iter=1000, probe="rademacher", Z=None):
        """I_kl = 1/2 Tr(Sdag^-1 dSdag_k Sdag^-1 dSdag_l) estimated by STE:
            1/2 (1/l) sum_i (z_i^T Sdag^-1 dSdag_k)(Sdag^-1 dSdag_l z_i),
        z_i with E[z z^T] = I (Rademacher or Gaussian, stream 7; ``Z`` replaces
        them).  The solves Sdag^-1 z_i and Sdag^-1 dSdag_l z_i run as one block of
        FITC-preconditioned CG (Appendix A); z_i^T Sdag^-1 dSdag_k is
        (dSdag_k Sdag^-1 z_i)^T.  Returns the estimate as printed ("fisher_raw",
        not symmetric for finite l) and its symmetric part ("fisher")."""
        n = self.n
        if Z is None:
            draw = rademacher if probe == "rademacher" else gaussian
            Z = draw(seed, STREAM_FISHER, np.arange(n), n, num_probes)
        l = Z.shape[1]
        # right-hand sides z_i, dSdag_0 z_i, dSdag_1 z_i (dSdag_2 = I: no solve)
        B = np.column_stack([Z, self.dS_apply(0, Z), self.dS_apply(1, Z)])
        res = pcg_lanczos(self.apply, self.apply_Pinv, B, tol, max_iter)
        V = res["U"][:, :l]
        X = [res["U"][:, l:2 * l], res["U"][:, 2 * l:], V]
        terms = np.empty((3, 3, l))
        for k in range(3):
            dV = self.dS_apply(k, V)
            for j in range(3):
                terms[k, j] = 0.5 * np.einsum("ij,ij->j", dV, X[j])
        F = terms.mean(axis=2)
        return dict(fisher=0.5 * (F + F.T), fisher_raw=F, terms=terms, iters=res["iters"],
                    converged=res["converged"], Z=Z)

    # -- predictive distribution (§2.3 and Algorithm 1) ----------------------
    def cross_structures(self, pred):
        """Sigma_{m,np}, and the sparse S = Sigma^s_{n,np} as an (n_p x n) CSR
        (rows: prediction points) with values
        (Sigma_{n,np} - Sigma^l_{n,np}) o T_{n,np}."""
        s1, rho, nug = self.theta
        Kp = cov_matrix(self.inducing, pred, self.nu, s1, rho)
        Ap = sla.solve_triangular(self.Lm, Kp, lower=True).T            # n_p x m
        rowptr, col = neighbour_csr(pred, self.locs, self.gamma)
        rows = np.repeat(np.arange(pred.shape[0]), np.diff(rowptr))
        cols = col.astype(np.int64)
        d = np.sqrt(sqdist_pairs(pred[rows], self.locs[cols]))
        lowrank = self._rowdots(Ap, self.A, rows, cols)
        vals = (s1 * corr(d, self.nu, rho) - lowrank) * taper(d, self.gamma)
        St = sp.csr_matrix((vals, col, rowptr), shape=(pred.shape[0], self.n))
        return Kp, St, (rowptr, col)

    def predict(self, y, pred, num_samples, seed, tol, max_iter=1000, probe="rademacher",
                u=None, Zp=None, control_variate=None):
        """Predictive mean (§2.3) and simulation-based variances (Algorithm 1).
        ``Zp`` replaces the random probes (used by deterministic checks).
        ``control_variate`` ("copt" or "c1") estimates the diagonal D_l with the
        diagonal preconditioner P_s = D_s as control variate (appendix
        "Preconditioner as control variate"): per point p, with
        a_k = z_k o (S Sigma_s~^-1 S^T z_k) and b_k = z_k o (S P_s^-1 S^T z_k),
            D_l = (1/l) sum_k (a_k - c b_k) + c diag(S P_s^-1 S^T),
        c = c_opt = sum_k (a_k - mean_k a_k) b_k / sum_k b_k^2 (the appendix's
        formula as printed, elementwise per point; 0 where sum_k b_k^2 = 0), or
        c = 1 ("c1")."""
        s1, rho, nug = self.theta
        n_p = pred.shape[0]
        Kp, St, _ = self.cross_structures(pred)
        cho_m = (self.Lm, True)
        if u is None:
            u = pcg_lanczos(self.apply, self.apply_Pinv, y[:, None], tol, max_iter)["U"][:, 0]
        mean = Kp.T @ sla.cho_solve(cho_m, self.K @ u) + St @ u
        # deterministic diagonals D1, D2, D3 with PCG solves (Algorithm 1)
        W1 = pcg_lanczos(self.apply, self.apply_Pinv, self.K.T.copy(), tol, max_iter)["U"]
        W2 = pcg_lanczos(lambda V: self.Ss @ V, self.apply_Dinv, self.K.T.copy(), tol, max_iter)["U"]
        M = self.Sm + self.K @ W2
        G = sla.cho_solve(cho_m, Kp)                                  # Sm^-1 Sigma_{m,np}
        D1 = np.einsum("ij,ij->j", G, (self.K @ W1) @ G)
        D2 = np.einsum("ij,ji->i", St @ W1, G)
        V = St @ W2
        D3 = np.einsum("ij,ji->i", V, np.linalg.solve(M, V.T))
        # stochastic diagonal D_l (lines 4-8 of Algorithm 1)
        if Zp is None:
            draw = rademacher if probe == "rademacher" else gaussian
            Zp = draw(seed, STREAM_PRED, np.arange(n_p), n_p, num_samples)
        StZ = St.T @ Zp
        X = pcg_lanczos(lambda V_: self.Ss @ V_, self.apply_Dinv, StZ, tol, max_iter)["U"]
        a = Zp * (St @ X)
        Dl = np.mean(a, axis=1)
        c = None
        if control_variate is not None:
            b = Zp * (St @ (StZ / self.D[:, None]))            # z o S P_s^-1 S^T z
            exact_b = np.asarray(St.multiply(St) @ (1.0 / self.D)).ravel()   # diag(S P_s^-1 S^T)
            if control_variate == "c1":
                c = np.ones(n_p)
            else:
                den = np.sum(b * b, axis=1)
                num = np.sum((a - Dl[:, None]) * b, axis=1)
                c = np.divide(num, den, out=np.zeros(n_p), where=den > 0)
            Dl = np.mean(a - c[:, None] * b, axis=1) + c * exact_b
        var = s1 + nug - D1 - 2.0 * D2 + D3 - Dl
        return dict(mean=mean, var=var, D1=D1, D2=D2, D3=D3, Dl=Dl, u=u, Zp=Zp, c=c)

