"""Error scales for comparing bilinear forms of CG solutions.

A term e = x^T M y, with x and y solutions of CG and M a derivative of the
operator (an indefinite matrix), moves by at most
    |delta e| <= delta (|x| |M y| + |M x| |y|)
when x and y carry relative errors up to delta (Cauchy-Schwarz).  Where the
mixed-precision form perturbs the solves, its per-probe gradient terms are
compared on that scale rather than on |e|, which can be far smaller than the
two norms' product when M's sparse and low-rank parts cancel.
"""
import numpy as np


def column_blocks(ref):
    """X = U with u in column 0 and Y = W with u in column 0, from an oracle
    ``loglik_grad`` result (the blocks whose columns the gradient pairs)."""
    res = ref["res"]
    U = res["U"]
    W = res["Z0"].copy()
    W[:, 0] = U[:, 0]
    return U, W


def bilinear_scales(S, ref):
    """scale[j, k] = |X_k| |dSigma_j Y_k| + |dSigma_j X_k| |Y_k| for the three
    parameters j and every column k (k = 0: the quadratic term u^T dSigma_j u)."""
    X, Y = column_blocks(ref)
    c = X.shape[1]
    nx, ny = np.linalg.norm(X, axis=0), np.linalg.norm(Y, axis=0)
    out = np.empty((3, c))
    for j in range(3):
        MV = S.dS_apply(j, np.column_stack([X, Y]))
        out[j] = nx * np.linalg.norm(MV[:, c:], axis=0) + np.linalg.norm(MV[:, :c], axis=0) * ny
    return out


def gradient_scale(scales):
    """Scale of dl/dtheta_j = -1/2 (mean_k e_jk - e_j0) from the per-term scales."""
    return 0.5 * (scales[:, 1:].mean(axis=1) + scales[:, 0])


def precond_scales(S, ref):
    """scale[j, k] = 2 |W_k| |dP_hat_j W_k| for the control variate's terms
    b_jk = W_k^T dP_hat_j W_k (probe columns only)."""
    W = ref["res"]["Z0"][:, 1:]
    nw = np.linalg.norm(W, axis=0)
    return np.array([2.0 * nw * np.linalg.norm(S.dP_apply(j, W), axis=0) for j in range(3)])


# relative rounding of an inner product of two BF16 hi + lo pairs (each ~2^-17)
PAIR_EPS = 2.0 ** -16


def mixed_traceP_scales(S):
    """First-order bounds on Tr(P_hat^-1 dP_hat_j) of the mixed form, whose
    D_s,i = sigma1^2 - |a_i|^2 + nugget is formed from A~ rounded to a BF16
    pair: |delta D_i| <= PAIR_EPS |a_i|^2 (a cancellation where |a_i|^2 is
    close to sigma1^2), and the range derivative dD_i = -(2 b_i.a_i - a_i.f_i)
    from pairs likewise.  With Tr(P^-1) ~ sum 1/D_i and
    Tr(P^-1 dP_rho) ~ sum dD_i / D_i (the low-rank corrections are O(m/n)):
        nugget:    PAIR_EPS sum |a_i|^2 / D_i^2
        rho:       PAIR_EPS sum (2 |b_i||a_i| + |a_i||f_i|) / D_i
                   + PAIR_EPS sum |dD_i| |a_i|^2 / D_i^2
        sigma1^2:  nugget / sigma1^2 times the nugget bound."""
    import scipy.linalg as sla
    s1, rho, nug = S.theta
    A, D = S.A, S.D
    a2 = np.sum(A * A, axis=1)
    dK, dSm, _ = S._dlowrank(1)
    B = sla.solve_triangular(S.Lm, dK, lower=True).T
    Li = sla.solve_triangular(S.Lm, np.eye(S.m), lower=True)
    F = A @ (Li @ dSm @ Li.T)
    dD = S.dD(1)
    na, nb, nf = np.sqrt(a2), np.linalg.norm(B, axis=1), np.linalg.norm(F, axis=1)
    s_nug = PAIR_EPS * np.sum(a2 / D ** 2)
    s_rho = PAIR_EPS * (np.sum((2 * nb * na + na * nf) / D) + np.sum(np.abs(dD) * a2 / D ** 2))
    return np.array([nug / s1 * s_nug, s_rho, s_nug])
