#!/usr/bin/env python
"""Benchmark: FSA log-likelihood + gradient evaluations per second on GB300.

One step = one call of ``fsa_loglik_grad`` (the whole theta-dependent hot
path: covariance and A~ build, residual values, Woodbury core, probes, block
PCG with Lanczos tridiagonals, SLQ log det, STE gradient) on the workload
n = 1e6 uniform locations, m = 1000 inducing points, exponential covariance
(sigma1^2 = 1, rho = 0.02, nugget = 0.01), taper for ~20 nonzeros per row,
l = 64 Rademacher probes, CG tolerance 1e-3, mixed BF16 / FP32 / FP64 form.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead, on a bounded window of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import fsa_inputs as fi  # noqa: E402

METRIC = "FSA loglik+grad evals/s at n=1e6,m=1000 (mixed vs FP64); serving p50/p99 ms"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.rows = []
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for k, v in zip(names, r[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(k)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _source_hash(name):
    h = hashlib.sha256()
    with open(os.path.join(ROOT, "paper_2405_14492_gb300", "csrc", name), "rb") as f:
        h.update(f.read())
    return h.hexdigest()[:16]


def _traffic_for(kernel_tag):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    from the current source of that kernel (else None)."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    e = d.get(kernel_tag)
    if not e or e.get("source_sha") != _source_hash(e.get("source", "fsa_tc.cu")):
        return None
    return e.get("dram_bytes_per_launch_full")


def make_workload(name, with_response=True, features=256):
    w = fi.WORKLOADS[name]
    locs = fi.uniform_locations(w.n, w.seed)
    idx = fi.inducing_subset(w.n, w.m, w.seed)
    y = fi.random_field(locs, w.nu, w.sigma1_sq, w.rho, w.nugget, w.seed, features=features) if with_response else None
    return w, locs, locs[idx].copy(), y


def window_sample(locs, y, n_target):
    """Points of the workload inside a lower-left square window holding about
    n_target points (same density, same taper, same inducing points)."""
    side = math.sqrt(n_target / locs.shape[0])
    sel = np.nonzero((locs[:, 0] < side) & (locs[:, 1] < side))[0]
    return locs[sel], y[sel], side


# ----------------------------------------------------------------------------
# CPU oracle arm (reference arm of this benchmark and the cpu_baseline field)
# ----------------------------------------------------------------------------
def oracle_sample_eval(w, locs, ind, y, n_sample):
    """Time one oracle log-likelihood + gradient on a window sample; return
    (seconds, n_s, evals/s scaled to the full n by n_s / n)."""
    from oracle import fsa_oracle as O
    ls, ys, side = window_sample(locs, y, n_sample)
    th = (w.sigma1_sq, w.rho, w.nugget)
    t0 = time.perf_counter()
    it = O.IterativeFSA(ls, ind, w.taper_range(), w.nu, th)
    out = it.loglik_grad(ys, w.num_probes, w.seed, w.cg_tol, max_iter=1000)
    dt = time.perf_counter() - t0
    return dt, ls.shape[0], (1.0 / dt) * (ls.shape[0] / w.n), int(np.max(out["iters"]))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w, locs, ind, y = make_workload(args.workload)
    n_s = args.ref_sample
    for _ in range(args.warmup):
        oracle_sample_eval(w, locs, ind, y, n_s)
    vals, secs = [], []
    for _ in range(args.steps):
        dt, ns, v, iters = oracle_sample_eval(w, locs, ind, y, n_s)
        vals.append(v)
        secs.append(dt)
    value = float(np.median(vals))
    cores = os.cpu_count()
    sample = (f"window of {ns} of the {w.n} points (same density, taper, {w.m} inducing points, "
              f"l={w.num_probes}, tol {w.cg_tol}); evals/s scaled by n_s/n (per-eval cost is O(n) at fixed m)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * float(np.median(secs)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name, "n": w.n, "m": w.m, "num_probes": w.num_probes},
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def combine_ranks(elapsed_ms, steps, world, dist=None, device="cpu"):
    """Whole-job timing of a replicas run: the timed region's length is the
    maximum over the ranks (every rank evaluates its own problem, the job ends
    with the slowest), and the throughput counts the evaluations of all ranks.
    Returns (max elapsed ms, evaluations per second of the job)."""
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([float(elapsed_ms)], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    return elapsed_ms, world * steps / (elapsed_ms / 1000.0)


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def run_gpu(args):
    import ctypes

    import torch

    import paper_2405_14492_gb300 as F
    from paper_2405_14492_gb300 import _native as N

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    lib = N.lib()
    lib.fsa_launch_count.restype = ctypes.c_uint64
    lib.fsa_profile_collect.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    w, locs, ind, y = make_workload(args.workload)
    if world > 1:   # replicas: each rank evaluates its own problem
        y = y + 1e-3 * rank
    th = (w.sigma1_sq, w.rho, w.nugget)
    # consecutive evaluations alternate between theta and theta with sigma1^2
    # scaled by 1 + 1e-12, so that every timed evaluation rebuilds the
    # theta-dependent operator (Sigma_m and its Cholesky, A, the residual
    # values, D, the Woodbury core) as an optimiser's evaluations would
    th_alt = (w.sigma1_sq * (1.0 + 1e-12), w.rho, w.nugget)

    calls = [0]

    def next_theta():   # the theta of the next evaluation (never the previous one's)
        calls[0] += 1
        return th if calls[0] % 2 == 0 else th_alt
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    h = F.FSAHandle(locs, ind, w.taper_range(), w.nu, stream=stream.cuda_stream)
    build_s = time.perf_counter() - t0
    y_dev = torch.tensor(y, device="cuda", dtype=torch.float64)
    prec = {"bf16x2": F.FSA_MIXED_BF16X2, "bf16": F.FSA_MIXED_BF16, "fp64": F.FSA_FP64}[args.precision]
    opts = F.make_opts(num_probes=w.num_probes, cg_tol=w.cg_tol, precision=prec, seed=w.seed,
                       y_on_device=True, vec_pieces=args.vec_pieces)
    infos = []
    for k in range(args.warmup):
        ll, g, info = h.loglik_grad(y_dev, next_theta(), opts)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    lib.fsa_profile_reset()
    lib.fsa_profile_enable(1)
    l0 = lib.fsa_launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        ll, g, info = h.loglik_grad(y_dev, next_theta(), opts)
        infos.append(info)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = int(lib.fsa_launch_count() - l0)
    lib.fsa_profile_enable(0)
    clk = clocks.stop()
    if dist:
        dist.barrier()
    elapsed_ms, value = combine_ranks(e0.elapsed_time(e1), args.steps, world, dist, "cuda")
    ms_per_step = elapsed_ms / args.steps
    # dominant kernel: the per-iteration tensor-core GEMMs
    prof = {}
    for tag in ("pcg_Aq", "pcg_AtX", "pcg_spmm", "pcg_ur", "pcg_z", "pcg_split", "pcg_q", "pcg_reduce", "build",
                "grad", "phase_build", "phase_probes", "phase_pcg", "phase_grad"):
        nl, ms, by = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
        if lib.fsa_profile_collect(tag.encode(), ctypes.byref(nl), ctypes.byref(ms), ctypes.byref(by)) == 0:
            prof[tag] = {"launches": nl.value, "ms": ms.value, "bytes": by.value}
    peaks, peak_src = _peaks()
    dom = max(("pcg_Aq", "pcg_AtX"), key=lambda k: prof.get(k, {}).get("ms", 0.0))
    roof = None
    if dom in prof:
        d = prof[dom]
        per_launch_ms = d["ms"] / d["launches"]
        per_launch_bytes = d["bytes"] / d["launches"]
        achieved = per_launch_bytes / (per_launch_ms / 1000.0) / 1e9
        roof = {"bound": "hbm", "kernel": f"tc_gemm[{dom}]", "achieved": round(achieved, 1),
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4),
                "traffic": _traffic_for(dom), "alg_bytes_per_launch": per_launch_bytes,
                "avg_launch_ms": per_launch_ms, "peak_source": f"{peak_src} (copy bandwidth)",
                "launches": d["launches"], "share_of_step": round(d["ms"] / elapsed_ms, 4)}
        if "pcg_spmm" in prof:
            d2 = prof["pcg_spmm"]
            ach = d2["bytes"] / d2["launches"] / (d2["ms"] / d2["launches"] / 1000.0) / 1e9
            roof["spmm"] = {"kernel": "kv_spmm_tma", "bound": "hbm", "achieved": round(ach, 1),
                            "traffic": _traffic_for("pcg_spmm"),
                            "frac": round(ach / peaks["hbm_gbs"], 4), "alg_bytes_per_launch": d2["bytes"] / d2["launches"],
                            "avg_launch_ms": d2["ms"] / d2["launches"], "launches": d2["launches"],
                            "share_of_step": round(d2["ms"] / elapsed_ms, 4)}
        other = "pcg_AtX" if dom == "pcg_Aq" else "pcg_Aq"
        if other in prof:
            o = prof[other]
            roof["other_gemm"] = {"kernel": f"tc_gemm[{other}]",
                                  "achieved": round(o["bytes"] / o["launches"] / (o["ms"] / o["launches"] / 1000) / 1e9, 1),
                                  "share_of_step": round(o["ms"] / elapsed_ms, 4)}
    # where a step's time goes: the four phases (CUDA events on the call's
    # stream) and, inside the CG loop, its per-iteration kernels
    per = lambda tag: prof.get(tag, {}).get("ms", 0.0) / args.steps
    phases = {k: round(per("phase_" + k), 3) for k in ("build", "probes", "pcg", "grad")}
    loop_tags = ("pcg_AtX", "pcg_reduce", "pcg_q", "pcg_Aq", "pcg_z", "pcg_spmm", "pcg_ur", "pcg_split")
    loop_kernels = sum(per(t) for t in loop_tags)
    breakdown = {"ms_per_step": round(ms_per_step, 3), "phases_ms": phases,
                 "outside_phases_ms": round(ms_per_step - sum(phases.values()), 3),
                 "pcg_kernels_ms": {t: round(per(t), 3) for t in loop_tags},
                 "pcg_outside_kernels_ms": round(phases["pcg"] - loop_kernels, 3),
                 "unattributed_frac": round((ms_per_step - sum(phases.values()) + phases["pcg"] - loop_kernels)
                                            / ms_per_step, 4)}
    result = {"metric": METRIC, "value": round(value, 4), "unit": "evals/s", "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": True,
              "scaling": "weak", "vs_baseline": None, "dtype": "bf16+f32+f64", "data": "synthetic",
              "config": {"workload": w.name, "n": w.n, "m": w.m, "nu": w.nu, "theta": list(th),
                         "taper_range": w.taper_range(), "nnz_per_row": h.nnz / w.n, "num_probes": w.num_probes,
                         "cg_tol": w.cg_tol, "precision": args.precision, "parallelism": f"replicas{world}",
                         "l2": "inputs larger than L2 (A~ alone is 2 GB BF16)",
                         "cg_iters_max": int(infos[-1]["iters_max"]), "cg_iters_y": int(infos[-1]["iters_y"]),
                         "build_s_theta_free": round(build_s, 3),
                         "theta_dependent_build": "in every timed evaluation (theta alternates by 1e-12)"},
              "gpu_launches": launches, "clocks": clk, "roofline": roof, "kernel_times": prof,
              "step_breakdown": breakdown,
              "loglik": ll, "grad": list(map(float, g)), "logdet_se": infos[-1]["logdet_se"]}
    # end to end through the C ABI with a host (pinned) response
    if not args.no_e2e:
        y_pin = torch.empty(w.n, dtype=torch.float64, pin_memory=True)
        y_pin.numpy()[:] = y
        opts_h = F.make_opts(num_probes=w.num_probes, cg_tol=w.cg_tol, precision=prec, seed=w.seed)
        h.loglik_grad(y_pin.numpy(), next_theta(), opts_h)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.steps):
            h.loglik_grad(y_pin.numpy(), next_theta(), opts_h)
        e2e_s = (time.perf_counter() - t0) / args.steps
        result["e2e"] = {"value": round(world / e2e_s, 4), "unit": "evals/s", "h2d_bytes_per_step": 8 * w.n,
                         "d2h_bytes_per_step": 8 * 4, "timing": "host wall clock around the C-ABI call"}
    # kmeans++ selection of the workload's inducing points on the GPU (paper
    # §4.1's choice; theta-free preprocessing, not part of the metric)
    if rank == 0:
        try:
            F.kmeanspp(locs[:2048], 16, 1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sel = F.kmeanspp(locs, w.m, w.seed)
            dt = time.perf_counter() - t0
            result["kmeanspp"] = {"n": w.n, "m": w.m, "seconds": round(dt, 4), "distinct": len(set(sel.tolist())) == w.m,
                                  "timing": "host wall clock around fsa_kmeanspp (copy of the locations included)"}
        except Exception as exc:   # reported in the line, the measurement above stands
            result["kmeanspp"] = {"error": str(exc)[:200]}
    # the faster single-BF16 operator form (lower accuracy) on the same workload and probes
    if args.precision != "bf16" and not args.no_fp64 and rank == 0:
        opts1 = F.make_opts(num_probes=w.num_probes, cg_tol=w.cg_tol, precision=F.FSA_MIXED_BF16, seed=w.seed,
                            y_on_device=True)
        h.loglik_grad(y_dev, th, opts1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(3):
            ll1, g1, _ = h.loglik_grad(y_dev, next_theta(), opts1)
        torch.cuda.synchronize()
        result["bf16_single_form"] = {"evals_per_s": round(3.0 / (time.perf_counter() - t0), 4), "loglik": ll1}
    # the plain FP64 GPU form on the same workload and probes
    if not args.no_fp64 and rank == 0:
        opts64 = F.make_opts(num_probes=w.num_probes, cg_tol=w.cg_tol, precision=F.FSA_FP64, seed=w.seed,
                             y_on_device=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ll64, g64, info64 = h.loglik_grad(y_dev, th, opts64)
        torch.cuda.synchronize()
        t64 = time.perf_counter() - t0
        result["fp64_form"] = {"evals_per_s": round(1.0 / t64, 5), "seconds_per_eval": round(t64, 3),
                               "loglik": ll64, "grad": list(map(float, g64)), "cg_iters_max": int(info64["iters_max"]),
                               "mixed_loglik_rel_err": abs(ll - ll64) / abs(ll64),
                               "mixed_loglik_err_vs_terms": abs(ll - ll64) / (0.5 * (w.n * math.log(2 * math.pi) +
                                                                                     abs(info64["logdet"]) +
                                                                                     abs(info64["quad_form"]))),
                               "mixed_speedup": round(value / world * t64, 2)}
        if "bf16_single_form" in result:
            result["bf16_single_form"]["loglik_rel_err_vs_fp64"] = abs(result["bf16_single_form"]["loglik"] - ll64) / abs(ll64)
    h.close()
    if rank == 0 and args.predict_steps > 0:
        result["predict"] = run_predict_leg(args, F, lib)
    if rank == 0 and args.serve_requests > 0:
        result["serving"] = run_serving(args, F)
    if rank == 0 and world == 1 and not args.no_cpu:
        dt, ns, v, iters = oracle_sample_eval(w, locs, ind, y, args.cpu_sample)
        # scaling check: a window twice as large should take about twice as long
        dt2, ns2, v2, iters2 = oracle_sample_eval(w, locs, ind, y, 2 * args.cpu_sample)
        result["cpu_baseline"] = {"value": v, "unit": "evals/s", "cores": os.cpu_count(), "kind": "oracle",
                                  "sample": f"one oracle loglik+grad on a window of {ns} of the {w.n} points "
                                            f"(same density, taper, all {w.m} inducing points), {dt:.1f} s, "
                                            f"scaled by n_s/n",
                                  "window_cg_iters": iters, "full_cg_iters": int(infos[-1]["iters_max"]),
                                  "double_window": {"n_s": ns2, "seconds": round(dt2, 2), "cg_iters": iters2,
                                                    "evals_per_s_scaled": v2,
                                                    "time_ratio_vs_window": round(dt2 / dt, 3)}}
    if rank == 0 and args.cpu_full:
        # the oracle on the whole workload, one evaluation (minutes, tens of GB of host memory)
        from oracle import fsa_oracle as O
        t0 = time.perf_counter()
        it = O.IterativeFSA(locs, ind, w.taper_range(), w.nu, th)
        out = it.loglik_grad(y, w.num_probes, w.seed, w.cg_tol, max_iter=1000)
        dtf = time.perf_counter() - t0
        result["cpu_full"] = {"seconds": round(dtf, 1), "evals_per_s": 1.0 / dtf, "cores": os.cpu_count(),
                              "cg_iters": int(np.max(out["iters"])), "loglik": out["loglik"],
                              "kind": "oracle", "sample": f"the whole workload, n = {w.n}, one evaluation"}
    if rank == 0:
        print(json.dumps(result), flush=True)
    if dist:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------
# prediction leg: n = 2e5 training, n_p = 1e5 prediction points, m = 800, s = 100
# ----------------------------------------------------------------------------
def run_predict_leg(args, F, lib):
    """Algorithm 1 at the predictive-distribution workload: the mixed form timed
    (CUDA events on the handle's stream), the plain FP64 form once with the
    same probes, and both against the exact FSA predictive variances of the
    first 2000 prediction points (D_l by sparse solves, pred_exact_var)."""
    import ctypes

    import torch
    w = fi.WORKLOADS["pred-n2e5-np1e5-m800"]
    locs = fi.uniform_locations(w.n, w.seed)
    ind = locs[fi.inducing_subset(w.n, w.m, w.seed)]
    y = fi.random_field(locs, w.nu, w.sigma1_sq, w.rho, w.nugget, w.seed, features=256)
    pred = fi.uniform_locations(w.n_pred, w.seed, stream=fi.STREAM_PRED_LOCATIONS)
    th = (w.sigma1_sq, w.rho, w.nugget)
    th_alt = (w.sigma1_sq * (1.0 + 1e-12), w.rho, w.nugget)
    s = w.num_var_samples
    stream = torch.cuda.Stream()
    out = {"workload": w.name, "n": w.n, "n_pred": w.n_pred, "m": w.m, "num_var_samples": s, "probe": "gaussian",
           "cg_tol": w.cg_tol}
    with F.FSAHandle(locs, ind, w.taper_range(), w.nu, stream=stream.cuda_stream) as h:
        mk = lambda prec, **kw: F.make_opts(cg_tol=w.cg_tol, seed=w.seed, precision=prec,
                                            probe=F.FSA_PROBE_GAUSSIAN, **kw)
        h.predict(y, th_alt, pred, s, mk(F.FSA_MIXED_BF16X2))   # warm-up
        torch.cuda.synchronize()
        lib.fsa_profile_reset()
        lib.fsa_profile_enable(1)
        times = []
        for k in range(args.predict_steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            mean_x, var_x, info_x = h.predict(y, th if k % 2 == 0 else th_alt, pred, s, mk(F.FSA_MIXED_BF16X2))
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        lib.fsa_profile_enable(0)
        nl, ms, by = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
        gemm_ms = ms.value if lib.fsa_profile_collect(b"predict", ctypes.byref(nl), ctypes.byref(ms),
                                                      ctypes.byref(by)) == 0 else 0.0
        t_mixed = statistics.median(times) / 1000.0
        out["mixed"] = {"seconds_per_eval": round(t_mixed, 4), "evals_per_s": round(1.0 / t_mixed, 4),
                        "iters_u": int(info_x["iters_y"]), "iters_sparse": int(info_x["iters_max"]),
                        "tensor_gemm_share": round(gemm_ms / args.predict_steps / (t_mixed * 1000.0), 4),
                        "tensor_gemm_launches_per_eval": int(nl.value) // max(1, args.predict_steps)}
        if not args.no_predict_fp64:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            mean_64, var_64, info_64 = h.predict(y, th, pred, s, mk(F.FSA_FP64))
            t64 = time.perf_counter() - t0
            out["fp64"] = {"seconds_per_eval": round(t64, 3), "iters_u": int(info_64["iters_y"]),
                           "iters_sparse": int(info_64["iters_max"])}
            out["mixed_speedup_vs_fp64"] = round(t64 / t_mixed, 2)
            # the same point set, probes and theta: the mixed form's rounding alone
            if k % 2 == 1:   # the last timed evaluation ran at theta_alt
                mean_x, var_x, _ = h.predict(y, th, pred, s, mk(F.FSA_MIXED_BF16X2))
            out["mixed_vs_fp64"] = {"mean_max_abs": float(np.max(np.abs(mean_x - mean_64))),
                                    "var_max_abs": float(np.max(np.abs(var_x - var_64))),
                                    "var_rms": float(np.sqrt(np.mean((var_x - var_64) ** 2)))}
            # exact FSA predictive variances of the first 2000 prediction points
            ns = min(2000, w.n_pred)
            t0 = time.perf_counter()
            _, var_ex, _ = h.predict(y, th, pred[:ns], s, mk(F.FSA_FP64, pred_exact_var=True))
            out["exact_subset"] = {"points": ns, "seconds": round(time.perf_counter() - t0, 3),
                                   "rmse_mixed": float(np.sqrt(np.mean((var_x[:ns] - var_ex) ** 2))),
                                   "rmse_fp64": float(np.sqrt(np.mean((var_64[:ns] - var_ex) ** 2))),
                                   "paper_context": "RMSE 5.0e-4 at l = 50 and 1.2e-4 at l = 500, n = n_p = 1e5, "
                                                    "64-core EPYC (Table 2)"}
    return out


# ----------------------------------------------------------------------------
# serving leg: the Poisson request stream through the persistent server
# ----------------------------------------------------------------------------
def _make_request_inputs(args):
    num, idx = args
    return fi.serving_stream(num)[idx].make()


def _serving_opts(F, req, precision):
    return F.make_opts(num_probes=req.num_probes, cg_tol=1e-3, precision=precision, seed=req.seed)


def _submit_request(F, srv, req, data, precision):
    locs, ind, y, pred = data
    th = (req.sigma1_sq, req.rho, req.nugget)
    opts = _serving_opts(F, req, precision)
    if req.kind == "loglik":
        return srv.submit_loglik(locs, ind, req.taper_range(), req.nu, y, th, opts)
    return srv.submit_predict(locs, ind, req.taper_range(), req.nu, y, th, pred, req.num_var_samples, opts)


def _run_alone(F, req, data, precision):
    """One request on its own (build + solve), as the one-at-a-time path runs
    it; returns (seconds, loglik or None, (mean, var) or None)."""
    import torch
    locs, ind, y, pred = data
    th = (req.sigma1_sq, req.rho, req.nugget)
    opts = _serving_opts(F, req, precision)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with F.FSAHandle(locs, ind, req.taper_range(), req.nu) as h:
        if req.kind == "loglik":
            ll, _, info = h.loglik_grad(y, th, opts)
            out = ((ll, info["logdet"], info["quad_form"], req.n), None)
        else:
            mean, var, _ = h.predict(y, th, pred, req.num_var_samples, opts)
            out = (None, (mean, var))
    torch.cuda.synchronize()
    return time.perf_counter() - t0, out[0], out[1]


def run_serving(args, F):
    """Replays the request stream (Poisson arrivals) against one server in the
    mixed form; reports latency (arrival to completion) and service time
    percentiles and completed evaluations per second.  On the same requests it
    times the one-request-at-a-time paths, FP64 and mixed, and compares every
    result with the FP64 one."""
    import multiprocessing as mp

    reqs = fi.serving_stream(512)[: args.serve_requests]
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(16, os.cpu_count() or 4)) as pool:
        data = pool.map(_make_request_inputs, [(512, k) for k in range(len(reqs))], chunksize=4)
    prec = F.FSA_MIXED_BF16X2
    with F.FSAServer(max_slots=args.serve_slots) as srv:
        # warm-up: one request of each kind, not counted
        warm = [next(r for r in reqs if r.kind == k) for k in ("loglik", "predict")]
        for r in warm:
            srv.wait(_submit_request(F, srv, r, data[r.index], prec), 600.0)
        base = srv.stats()
        tickets = []
        t0 = time.perf_counter()
        for r in reqs:
            dt = t0 + r.arrival_s - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            tickets.append(_submit_request(F, srv, r, data[r.index], prec))
        res = [srv.wait(t, 3600.0) for t in tickets]
        wall = time.perf_counter() - t0
        st = srv.stats()
    lat = np.array([r["latency_ms"] for r in res])
    run = np.array([r["run_ms"] for r in res])
    ok = [r for r in res if r["status"] in (0, 4)]
    pct = lambda a, q: float(np.percentile(a, q, method="inverted_cdf"))
    served = {"requests": len(reqs), "arrival_rate_per_s": 200.0, "slots": args.serve_slots,
              "completed": len(ok), "failed": len(res) - len(ok),
              "latency_p50_ms": pct(lat, 50), "latency_p99_ms": pct(lat, 99),
              "service_p50_ms": pct(run, 50), "service_p99_ms": pct(run, 99),
              "evals_per_s": round(len(ok) / wall, 3), "wall_s": round(wall, 2), "precision": "bf16x2",
              "peak_running": st["peak_running"], "peak_footprint_gb": round(st["peak_in_use_bytes"] / 1e9, 2),
              "budget_gb": round(st["budget_bytes"] / 1e9, 1), "warmup_requests": base["completed"]}
    # the same requests one at a time: FP64 and mixed
    t64, tmx = 0.0, 0.0
    lerr, terr, merr, verr = [], [], [], []
    for r, sr in zip(reqs, res):
        d64, ll64, mv64 = _run_alone(F, r, data[r.index], F.FSA_FP64)
        dmx, _, _ = _run_alone(F, r, data[r.index], prec)
        t64 += d64
        tmx += dmx
        if r.kind == "loglik" and ll64:
            ll64v, logdet64, quad64, n = ll64
            lerr.append(abs(sr["loglik"] - ll64v) / abs(ll64v))
            # against the magnitude of the terms ll is the difference of
            terms = 0.5 * (n * math.log(2 * math.pi) + abs(logdet64) + abs(quad64))
            terr.append(abs(sr["loglik"] - ll64v) / terms)
        elif mv64 is not None and "mean" in sr:
            merr.append(float(np.max(np.abs(sr["mean"] - mv64[0])) / max(1e-300, np.max(np.abs(mv64[0])))))
            verr.append(float(np.max(np.abs(sr["var"] - mv64[1]))))
    served["fp64_one_at_a_time"] = {"requests": len(reqs), "evals_per_s": round(len(reqs) / t64, 3),
                                    "seconds": round(t64, 2), "same_requests": True}
    served["mixed_one_at_a_time"] = {"requests": len(reqs), "evals_per_s": round(len(reqs) / tmx, 3),
                                     "seconds": round(tmx, 2)}
    served["speedup_vs_fp64_one_at_a_time"] = round(served["evals_per_s"] / (len(reqs) / t64), 2)
    served["overlap_gain_vs_mixed_one_at_a_time"] = round(served["evals_per_s"] / (len(reqs) / tmx), 2)
    served["loglik_rel_err_vs_fp64_max"] = float(max(lerr)) if lerr else None
    served["loglik_err_vs_terms_max"] = float(max(terr)) if terr else None
    served["loglik_requests_over_1e-4"] = {"relative": int(sum(e > 1e-4 for e in lerr)),
                                           "against_terms": int(sum(e > 1e-4 for e in terr)),
                                           "of": len(lerr)}
    served["predict_mean_rel_err_vs_fp64_max"] = float(max(merr)) if merr else None
    served["predict_var_abs_err_vs_fp64_max"] = float(max(verr)) if verr else None
    return served


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="exp-n1e6-m1000", choices=sorted(fi.WORKLOADS))
    ap.add_argument("--precision", default="bf16x2", choices=["bf16x2", "bf16", "fp64"])
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=4000)
    ap.add_argument("--cpu-full", action="store_true")
    ap.add_argument("--ref-sample", type=int, default=2500)
    ap.add_argument("--predict-steps", type=int, default=3)
    ap.add_argument("--no-predict-fp64", action="store_true")
    ap.add_argument("--vec-pieces", type=int, default=2, choices=[2, 3])
    ap.add_argument("--serve-requests", type=int, default=48)
    ap.add_argument("--serve-slots", type=int, default=8)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
