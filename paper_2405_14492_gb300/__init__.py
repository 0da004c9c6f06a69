"""GB300-native iterative full-scale approximation (FSA) for Gaussian processes.

Python front end of libfsa.so (C ABI in include/fsa.h): argument marshalling
only; every step of the computation runs in the library's CUDA kernels.
PyTorch is used for device memory and streams (``FSALogLik`` wraps the
log-likelihood as a ``torch.autograd.Function``).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _native as N
from ._native import (FSA_EXPONENTIAL, FSA_FP64, FSA_MATERN_1_5, FSA_MIXED_BF16, FSA_MIXED_BF16X2,
                      FSA_PROBE_GAUSSIAN, FSA_PROBE_RADEMACHER, FsaError, FsaInfo, FsaOpts, FsaTheta)

__all__ = ["FSAHandle", "FSAServer", "FSALogLik", "FsaError", "FSA_EXPONENTIAL", "FSA_MATERN_1_5", "FSA_FP64",
           "FSA_MIXED_BF16", "FSA_MIXED_BF16X2", "FSA_PROBE_RADEMACHER", "FSA_PROBE_GAUSSIAN", "make_opts",
           "cov_code", "fit_mle"]


def cov_code(nu: float) -> int:
    if nu == 0.5:
        return FSA_EXPONENTIAL
    if nu == 1.5:
        return FSA_MATERN_1_5
    raise ValueError("nu must be 0.5 or 1.5")


FSA_PRED_CV_NONE, FSA_PRED_CV_COPT, FSA_PRED_CV_C1 = 0, 1, 2
# control variate of the gradient's trace estimate: none, c_opt as printed, c = 1, centred c_opt
FSA_GRAD_CV = {None: 0, "copt": 1, "c1": 2, "copt_centered": 3}


def make_opts(num_probes=50, cg_tol=1e-3, cg_max_iter=1000, fixed_iters=0, precision=FSA_FP64,
              probe=FSA_PROBE_RADEMACHER, seed=14492, slq_exact_weight=False, want_grad=True,
              y_on_device=False, pred_control_variate=FSA_PRED_CV_NONE, grad_control_variate=None,
              pred_exact_var=False, vec_pieces=2) -> FsaOpts:
    o = N.default_opts()
    o.num_probes, o.cg_tol, o.cg_max_iter, o.fixed_iters = num_probes, cg_tol, cg_max_iter, fixed_iters
    o.precision, o.probe, o.seed = precision, probe, seed
    o.slq_exact_weight, o.want_grad, o.y_on_device = int(slq_exact_weight), int(want_grad), int(y_on_device)
    o.pred_control_variate = int(pred_control_variate)
    o.grad_control_variate = FSA_GRAD_CV[grad_control_variate]
    o.pred_exact_var = int(pred_exact_var)
    o.vec_pieces = int(vec_pieces)
    return o


def _theta(theta) -> FsaTheta:
    s1, rho, nug = (float(t) for t in theta)
    return FsaTheta(s1, rho, nug)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def kmeanspp(locs, m: int, seed: int = 14492, stream=None) -> np.ndarray:
    """Indices of m inducing points chosen among the locations by kmeans++
    seeding on the GPU (``fsa_kmeanspp``; paper §4.1)."""
    locs = _f64(locs).reshape(-1, 2)
    n = locs.shape[0]
    out = np.empty(int(m), dtype=np.int64)
    N.check(N.lib().fsa_kmeanspp(locs.ctypes.data, n, int(m), int(seed), out.ctypes.data, stream))
    return out


class FSAHandle:
    """A built FSA problem: locations, inducing points, taper range, covariance
    family (``fsa_build``).  Owns its device memory; ``close()`` frees it."""

    def __init__(self, locs, inducing, taper_range: float, nu: float = 0.5, stream: int = 0):
        self._locs = _f64(locs)
        self._ind = _f64(inducing)
        self.n, self.m = self._locs.shape[0], self._ind.shape[0]
        self.nu = nu
        h = C.c_void_p()
        N.check(N.lib().fsa_build(N.ptr(self._locs), self.n, N.ptr(self._ind), self.m, float(taper_range),
                                  cov_code(nu), C.c_void_p(stream), C.byref(h)))
        self._h = h

    @property
    def nnz(self) -> int:
        return int(N.lib().fsa_nnz(self._h))

    def csr(self):
        """Taper pattern in the caller's point order (``fsa_get_csr``)."""
        rowptr = np.empty(self.n + 1, np.int64)
        col = np.empty(self.nnz, np.int32)
        N.check(N.lib().fsa_get_csr(self._h, N.ptr(rowptr), N.ptr(col)))
        return rowptr, col

    def loglik_grad(self, y, theta, opts: FsaOpts | None = None, raise_on_noconv: bool = False):
        """(loglik, grad[3], info dict) via ``fsa_loglik_grad``.  ``y`` is a
        host array, or a CUDA torch tensor when opts.y_on_device is set."""
        opts = opts or make_opts()
        th = _theta(theta)
        ll = C.c_double()
        g = np.zeros(3)
        info = FsaInfo()
        if opts.y_on_device:
            yp = C.c_void_p(int(y.data_ptr()))
        else:
            yh = _f64(y)
            yp = N.ptr(yh)
        st = N.lib().fsa_loglik_grad(self._h, yp, C.byref(th), C.byref(opts), C.byref(ll),
                                     g.ctypes.data_as(N.DP), C.byref(info))
        if st != N.FSA_OK and (st != 4 or raise_on_noconv):
            N.check(st)
        d = info.as_dict()
        d["status"] = st
        self.last_info = d
        return ll.value, g, d

    def grad_terms(self, num_probes: int):
        """Per-probe terms (a, b), each 3 x l, of the last gradient (``fsa_grad_terms``)."""
        a = np.empty((3, num_probes))
        b = np.empty((3, num_probes))
        N.check(N.lib().fsa_grad_terms(self._h, N.ptr(a), N.ptr(b), int(num_probes)))
        return a, b

    def fisher(self, theta, opts: FsaOpts | None = None, raise_on_noconv: bool = False):
        """(symmetric Fisher information 3 x 3, the raw estimate, info) by
        stochastic trace estimation (``fsa_fisher``)."""
        opts = opts or make_opts()
        th = _theta(theta)
        F = np.empty((3, 3))
        Fr = np.empty((3, 3))
        info = FsaInfo()
        st = N.lib().fsa_fisher(self._h, C.byref(th), C.byref(opts), N.ptr(F), N.ptr(Fr), C.byref(info))
        if st != N.FSA_OK and (st != 4 or raise_on_noconv):
            N.check(st)
        d = info.as_dict()
        d["status"] = st
        return F, Fr, d

    def matvec(self, theta, v, which=0, precision=FSA_FP64):
        """Sigma_dag v (0), P_hat^-1 v (1) or Sigma_s~ v (2) (``fsa_matvec``)."""
        v = _f64(v)
        vv = v.reshape(self.n, -1)
        out = np.empty_like(vv)
        th = _theta(theta)
        N.check(N.lib().fsa_matvec(self._h, C.byref(th), precision, which, N.ptr(vv), vv.shape[1], N.ptr(out)))
        return out.reshape(v.shape)

    def logdet_precond(self, theta, precision=FSA_FP64) -> float:
        th = _theta(theta)
        out = C.c_double()
        N.check(N.lib().fsa_logdet_precond(self._h, C.byref(th), precision, C.byref(out)))
        return out.value

    def predict(self, y, theta, pred_locs, num_var_samples=50, opts: FsaOpts | None = None, want_var=True):
        """Predictive mean and simulation-based variances (``fsa_predict``)."""
        opts = opts or make_opts()
        th = _theta(theta)
        yh = _f64(y)
        pl = _f64(pred_locs)
        n_p = pl.shape[0]
        mean = np.empty(n_p)
        var = np.empty(n_p) if want_var else None
        info = FsaInfo()
        st = N.lib().fsa_predict(self._h, N.ptr(yh), C.byref(th), C.byref(opts), N.ptr(pl), n_p,
                                 int(num_var_samples), N.ptr(mean), N.ptr(var) if want_var else None,
                                 C.byref(info))
        if st not in (N.FSA_OK, 4):
            N.check(st)
        return mean, var, info.as_dict()

    def close(self):
        if getattr(self, "_h", None):
            N.lib().fsa_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class FSAServer:
    """Persistent serving loop on one GPU with continuous batching
    (``fsa_server_create`` / ``fsa_serve_submit`` / ``fsa_serve_poll`` /
    ``fsa_serve_wait``).  Each request is one build plus one likelihood or
    prediction call; the server admits requests by slot and device-memory
    footprint and runs the admitted ones concurrently on its slot streams."""

    def __init__(self, max_slots: int = 4, hbm_budget_bytes: int = 0, device: int = 0):
        cfg = N.FsaServerCfg()
        N.lib().fsa_default_server_cfg(C.byref(cfg))
        cfg.device, cfg.max_slots, cfg.hbm_budget_bytes = device, max_slots, int(hbm_budget_bytes)
        s = C.c_void_p()
        N.check(N.lib().fsa_server_create(C.byref(cfg), C.byref(s)))
        self._s = s
        self._outs = {}   # ticket -> prediction output arrays (kept alive until retrieved)

    def _submit(self, kind, locs, inducing, taper_range, nu, y, theta, opts, pred_locs=None,
                num_var_samples=0, want_var=True):
        locs, inducing, y = _f64(locs), _f64(inducing), _f64(y)
        q = N.FsaRequest()
        q.kind = kind
        q.locs, q.n = locs.ctypes.data, locs.shape[0]
        q.inducing, q.m = inducing.ctypes.data, inducing.shape[0]
        q.taper_range, q.cov = float(taper_range), cov_code(nu)
        q.y = y.ctypes.data
        q.theta = _theta(theta)
        q.opts = opts or make_opts()
        outs = None
        if kind == N.FSA_REQ_PREDICT:
            pl = _f64(pred_locs)
            mean = np.empty(pl.shape[0])
            var = np.empty(pl.shape[0]) if want_var else None
            q.pred_locs, q.n_p, q.num_var_samples = pl.ctypes.data, pl.shape[0], int(num_var_samples)
            q.mean = mean.ctypes.data
            q.var = var.ctypes.data if want_var else None
            outs = (mean, var)
        t = C.c_uint64()
        N.check(N.lib().fsa_serve_submit(self._s, C.byref(q), C.byref(t)))
        if outs is not None:
            self._outs[t.value] = outs
        return t.value

    def submit_loglik(self, locs, inducing, taper_range, nu, y, theta, opts: FsaOpts | None = None) -> int:
        return self._submit(N.FSA_REQ_LOGLIK_GRAD, locs, inducing, taper_range, nu, y, theta, opts)

    def submit_predict(self, locs, inducing, taper_range, nu, y, theta, pred_locs, num_var_samples=50,
                       opts: FsaOpts | None = None, want_var=True) -> int:
        return self._submit(N.FSA_REQ_PREDICT, locs, inducing, taper_range, nu, y, theta, opts, pred_locs,
                            num_var_samples, want_var)

    def _result(self, ticket, r: "N.FsaResult"):
        d = {"status": r.status, "kind": r.kind, "loglik": r.loglik, "grad": np.array(list(r.grad)),
             "info": r.info.as_dict(), "queue_ms": r.queue_ms, "run_ms": r.run_ms, "latency_ms": r.latency_ms,
             "footprint_bytes": r.footprint_bytes, "slot": r.slot, "message": r.message.decode()}
        if ticket in self._outs:
            d["mean"], d["var"] = self._outs.pop(ticket)
        return d

    def poll(self, ticket):
        """The result dict, or None while the request waits or runs."""
        r = N.FsaResult()
        st = N.lib().fsa_serve_poll(self._s, ticket, C.byref(r))
        if st == 7:
            return None
        N.check(st)
        return self._result(ticket, r)

    def wait(self, ticket, timeout_s: float = -1.0):
        r = N.FsaResult()
        N.check(N.lib().fsa_serve_wait(self._s, ticket, float(timeout_s), C.byref(r)))
        return self._result(ticket, r)

    def stats(self) -> dict:
        st = N.FsaServerStats()
        N.check(N.lib().fsa_server_get_stats(self._s, C.byref(st)))
        return st.as_dict()

    def close(self):
        if getattr(self, "_s", None):
            N.lib().fsa_server_destroy(self._s)
            self._s = None
            self._outs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _autograd_function():
    import torch

    class FSALogLik(torch.autograd.Function):
        """l(theta) as a differentiable torch scalar: forward calls
        ``fsa_loglik_grad`` (the hand-written adjoint kernels give the STE
        gradient), backward returns grad_output * dl/dtheta."""

        @staticmethod
        def forward(ctx, theta, handle, y, opts=None):
            th = theta.detach().double().cpu().numpy()
            ll, g, _ = handle.loglik_grad(y, th, opts)
            ctx.save_for_backward(torch.as_tensor(g, dtype=theta.dtype, device=theta.device))
            return torch.as_tensor(ll, dtype=theta.dtype, device=theta.device)

        @staticmethod
        def backward(ctx, grad_out):
            (g,) = ctx.saved_tensors
            return grad_out * g, None, None, None

    return FSALogLik


class _Lazy:
    def __init__(self):
        self._f = None

    def __getattr__(self, k):
        if self._f is None:
            self._f = _autograd_function()
        return getattr(self._f, k)


FSALogLik = _Lazy()


def fit_mle(handle, y, theta0, opts=None, max_iter: int = 100, tol_grad: float = 1e-9, history_size: int = 10):
    """Maximum-likelihood estimate of theta = (sigma1^2, rho, nugget) by L-BFGS
    on top of ``FSALogLik`` (the paper estimates its parameters this way, §4).

    The optimiser works on phi = log theta, so every iterate stays positive,
    and minimises -l(exp(phi)) / n with torch's L-BFGS and a strong-Wolfe line
    search.  Every objective evaluation is one ``handle.loglik_grad`` call
    (one ``fsa_loglik_grad`` on a GPU handle).  ``opts`` fixes the probes
    (its seed) for every call, so the objective is one deterministic function
    of theta, as the line search needs.  Stops when the gradient in phi falls
    below ``tol_grad`` (scaled by 1/n) or after ``max_iter`` iterations.

    Returns a dict: theta (np.ndarray), loglik at theta, iterations,
    evaluations (handle calls) and converged (gradient criterion met)."""
    import torch

    y_np = np.asarray(y, dtype=np.float64)
    n = y_np.shape[0]
    phi = torch.tensor(np.log(np.asarray(theta0, dtype=np.float64)), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.LBFGS([phi], lr=1.0, max_iter=max_iter, tolerance_grad=tol_grad, tolerance_change=0.0,
                            history_size=history_size, line_search_fn="strong_wolfe")
    evals = [0]

    def closure():
        opt.zero_grad()
        loss = -FSALogLik.apply(torch.exp(phi), handle, y_np, opts) / n
        loss.backward()
        evals[0] += 1
        return loss

    opt.step(closure)
    state = opt.state[opt._params[0]]
    th = np.exp(phi.detach().numpy())
    ll, g, _ = handle.loglik_grad(y_np, th, opts)
    gphi = np.max(np.abs(-np.asarray(g) * th / n))
    return {"theta": th, "loglik": float(ll), "iterations": int(state.get("n_iter", 0)),
            "evaluations": evals[0], "converged": bool(gphi <= tol_grad)}
