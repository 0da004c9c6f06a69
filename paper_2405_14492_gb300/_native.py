"""ctypes binding of libfsa.so — argument marshalling only.

Every function here has the name of the C entry point in include/fsa.h and
forwards to it; no step of the computation runs in Python.  Loading fails
loudly if the library has not been built (there is no fallback).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# FSA_CHECKED=1 in the environment loads the checked build (device index
# checks that report FSA_ERR_BOUNDS; build.py --checked) in place of the default
CHECKED = os.environ.get("FSA_CHECKED", "") not in ("", "0")
LIB_PATH = os.path.join(_HERE, "libfsa_checked.so" if CHECKED else "libfsa.so")

FSA_OK = 0
STATUS = {0: "FSA_OK", 1: "FSA_ERR_ARG", 2: "FSA_ERR_OOM", 3: "FSA_ERR_NOT_PD", 4: "FSA_ERR_NO_CONVERGENCE",
          5: "FSA_ERR_NAN", 6: "FSA_ERR_TIMEOUT", 7: "FSA_ERR_BUSY", 8: "FSA_ERR_CUDA", 9: "FSA_ERR_UNSUPPORTED",
          10: "FSA_ERR_BOUNDS"}
FSA_EXPONENTIAL, FSA_MATERN_1_5 = 0, 1
FSA_FP64, FSA_MIXED_BF16, FSA_MIXED_BF16X2 = 0, 1, 2
FSA_PROBE_RADEMACHER, FSA_PROBE_GAUSSIAN = 0, 1


class FsaTheta(C.Structure):
    _fields_ = [("sigma1_sq", C.c_double), ("rho", C.c_double), ("nugget", C.c_double)]


class FsaOpts(C.Structure):
    _fields_ = [("num_probes", C.c_int32), ("cg_tol", C.c_double), ("cg_max_iter", C.c_int32),
                ("fixed_iters", C.c_int32), ("precision", C.c_int32), ("probe", C.c_int32),
                ("seed", C.c_uint64), ("slq_exact_weight", C.c_int32), ("want_grad", C.c_int32),
                ("y_on_device", C.c_int32), ("pred_control_variate", C.c_int32),
                ("grad_control_variate", C.c_int32), ("pred_exact_var", C.c_int32),
                ("vec_pieces", C.c_int32)]


class FsaInfo(C.Structure):
    _fields_ = [("iters_max", C.c_int32), ("iters_y", C.c_int32), ("resid_y", C.c_double),
                ("logdet", C.c_double), ("logdet_precond", C.c_double), ("quad_form", C.c_double),
                ("logdet_se", C.c_double), ("converged", C.c_int32), ("num_probes", C.c_int32),
                ("nnz", C.c_int64), ("time_ms", C.c_double), ("grad_trace", C.c_double * 3),
                ("grad_quad", C.c_double * 3), ("trace_precond", C.c_double * 3), ("cv_coef", C.c_double * 3),
                ("core_scale", C.c_double), ("core_fp64", C.c_int32), ("a_scale", C.c_double),
                ("a_fp64", C.c_int32)]

    def as_dict(self):
        d = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            d[k] = list(v) if isinstance(v, C.Array) else v
        return d


FSA_REQ_LOGLIK_GRAD, FSA_REQ_PREDICT = 0, 1


class FsaServerCfg(C.Structure):
    _fields_ = [("device", C.c_int32), ("max_slots", C.c_int32), ("hbm_budget_bytes", C.c_int64)]


class FsaRequest(C.Structure):
    _fields_ = [("kind", C.c_int32), ("locs", C.c_void_p), ("n", C.c_int64), ("inducing", C.c_void_p),
                ("m", C.c_int32), ("taper_range", C.c_double), ("cov", C.c_int32), ("y", C.c_void_p),
                ("theta", FsaTheta), ("opts", FsaOpts), ("pred_locs", C.c_void_p), ("n_p", C.c_int64),
                ("num_var_samples", C.c_int32), ("mean", C.c_void_p), ("var", C.c_void_p)]


class FsaResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("kind", C.c_int32), ("loglik", C.c_double), ("grad", C.c_double * 3),
                ("info", FsaInfo), ("queue_ms", C.c_double), ("run_ms", C.c_double), ("latency_ms", C.c_double),
                ("footprint_bytes", C.c_int64), ("slot", C.c_int32), ("message", C.c_char * 160)]


class FsaServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64), ("pending", C.c_int64),
                ("running", C.c_int32), ("peak_running", C.c_int32), ("budget_bytes", C.c_int64),
                ("in_use_bytes", C.c_int64), ("peak_in_use_bytes", C.c_int64), ("p50_ms", C.c_double),
                ("p99_ms", C.c_double), ("mean_ms", C.c_double), ("completed_per_s", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class FsaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None

P = C.c_void_p
DP = C.POINTER(C.c_double)


def _declare(lib):
    sig = {
        "fsa_default_opts": (None, [C.POINTER(FsaOpts)]),
        "fsa_status_string": (C.c_char_p, [C.c_int]),
        "fsa_last_error": (C.c_char_p, []),
        "fsa_build": (C.c_int, [P, C.c_int64, P, C.c_int32, C.c_double, C.c_int32, P, C.POINTER(P)]),
        "fsa_nnz": (C.c_int64, [P]),
        "fsa_get_csr": (C.c_int, [P, P, P]),
        "fsa_loglik_grad": (C.c_int, [P, P, C.POINTER(FsaTheta), C.POINTER(FsaOpts), DP, DP,
                                      C.POINTER(FsaInfo)]),
        "fsa_grad_terms": (C.c_int, [P, P, P, C.c_int32]),
        "fsa_fisher": (C.c_int, [P, C.POINTER(FsaTheta), C.POINTER(FsaOpts), P, P, C.POINTER(FsaInfo)]),
        "fsa_matvec": (C.c_int, [P, C.POINTER(FsaTheta), C.c_int32, C.c_int32, P, C.c_int32, P]),
        "fsa_logdet_precond": (C.c_int, [P, C.POINTER(FsaTheta), C.c_int32, DP]),
        "fsa_predict": (C.c_int, [P, P, C.POINTER(FsaTheta), C.POINTER(FsaOpts), P, C.c_int64, C.c_int32,
                                  P, P, C.POINTER(FsaInfo)]),
        "fsa_free": (None, [P]),
        "fsa_footprint_bytes": (C.c_int64, [C.c_int64, C.c_int32, C.c_int64, C.c_int32, C.c_int32]),
        "fsa_default_server_cfg": (None, [C.POINTER(FsaServerCfg)]),
        "fsa_server_create": (C.c_int, [C.POINTER(FsaServerCfg), C.POINTER(P)]),
        "fsa_serve_submit": (C.c_int, [P, C.POINTER(FsaRequest), C.POINTER(C.c_uint64)]),
        "fsa_serve_poll": (C.c_int, [P, C.c_uint64, C.POINTER(FsaResult)]),
        "fsa_serve_wait": (C.c_int, [P, C.c_uint64, C.c_double, C.POINTER(FsaResult)]),
        "fsa_server_get_stats": (C.c_int, [P, C.POINTER(FsaServerStats)]),
        "fsa_server_destroy": (None, [P]),
        "fsa_pool_used_high": (C.c_int64, [C.c_int]),
        "fsa_kmeanspp": (C.c_int, [P, C.c_int64, C.c_int32, C.c_uint64, P, P]),
    }
    for name, (res, args) in sig.items():
        if not hasattr(lib, name):
            continue
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args


def lib():
    """The loaded libfsa.so, or libfsa_checked.so under FSA_CHECKED=1 (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError(f"{LIB_PATH} not found: build it first (python -c 'import __graft_entry__ as g; g.build()')")
        _lib = C.CDLL(LIB_PATH)
        _declare(_lib)
    return _lib


def check(status: int):
    if status != FSA_OK:
        msg = lib().fsa_last_error().decode()
        raise FsaError(status, msg)


def default_opts() -> FsaOpts:
    o = FsaOpts()
    lib().fsa_default_opts(C.byref(o))
    return o


def ptr(a: np.ndarray):
    return C.c_void_p(a.ctypes.data)
