"""Seeded synthetic inputs for the FSA Gaussian-process workloads.

This module is shared by the CPU oracle, the tests and the benchmark.  It holds
no arithmetic of the FSA method itself (no full-scale approximation, no solver,
no estimator): only input generation in the shape of the paper's simulation
design (§4: locations uniform on the unit square, inducing points drawn as a
random subset of the locations, a stationary Gaussian random field as response).

Random numbers that the *method* draws (the Rademacher / Gaussian probes of the
stochastic estimators) are NOT generated here: each side implements the same
counter-based SplitMix64 generator from its published definition.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 14492

# stream ids of the input generators
STREAM_LOCATIONS = 1
STREAM_INDUCING = 2
STREAM_RESPONSE = 3
STREAM_PRED_LOCATIONS = 7


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(stream)])


def uniform_locations(n: int, seed: int, stream: int = STREAM_LOCATIONS) -> np.ndarray:
    """n points uniform on [0,1]^2, row-major (n, 2) float64."""
    return _rng(seed, stream).random((n, 2))


def inducing_subset(n: int, m: int, seed: int) -> np.ndarray:
    """Indices of m distinct locations drawn uniformly without replacement
    (the paper's Assumption 2), in the order drawn."""
    if m > n:
        raise ValueError("m > n")
    return _rng(seed, STREAM_INDUCING).choice(n, size=m, replace=False).astype(np.int64)


def expected_neighbours(gamma: float, n: int) -> float:
    """Expected number of points (self included) within distance gamma of a
    uniform point of the unit square, for n uniform points: 1 + (n-1)*area,
    with area = pi g^2 - 8 g^3 / 3 + g^4 / 2 the mean area of a disc of radius
    g clipped to the square (valid for g <= 1)."""
    g = float(gamma)
    return 1.0 + (n - 1) * (math.pi * g * g - 8.0 * g ** 3 / 3.0 + g ** 4 / 2.0)


def taper_range_for(nnz_per_row: float, n: int) -> float:
    """Taper range gamma giving about `nnz_per_row` nonzeros per row (diagonal
    included) for n uniform points on the unit square (bisection)."""
    lo, hi = 0.0, 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if expected_neighbours(mid, n) < nnz_per_row:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def random_field(locs: np.ndarray, nu: float, sigma1_sq: float, rho: float,
                 nugget: float, seed: int, features: int = 2048) -> np.ndarray:
    """A stationary Matérn-type Gaussian random field plus white noise at the
    given locations, by random Fourier features (Rahimi & Recht 2007).

    Frequencies follow the Matérn spectral density, proportional to
    (2 nu / rho^2 + |omega|^2)^-(nu + 1): a bivariate Student-t with 2 nu
    degrees of freedom and scale 1/rho, for the parameterisation
    r(d) = exp(-d/rho) (nu = 1/2) and (1 + sqrt(3) d/rho) exp(-sqrt(3) d/rho)
    (nu = 3/2); i.e. omega = g * sqrt(2 nu / chi2_{2 nu}) / rho, g ~ N(0, I).
    The field is an approximate draw from the true (un-approximated) GP,
    like the paper's simulated data; the result is used as the response y.
    """
    rng = _rng(seed, STREAM_RESPONSE)
    n = locs.shape[0]
    scale = 1.0 / rho
    g = rng.standard_normal((features, 2))
    chi = rng.chisquare(2.0 * nu, size=(features, 1))
    omega = scale * g * np.sqrt(2.0 * nu / chi)
    phase = rng.random(features) * 2.0 * math.pi
    y = np.zeros(n)
    chunk = 1 << 15
    for s in range(0, n, chunk):
        arg = locs[s:s + chunk] @ omega.T + phase
        y[s:s + chunk] = np.cos(arg).sum(axis=1)
    y *= math.sqrt(2.0 * sigma1_sq / features)
    y += math.sqrt(nugget) * rng.standard_normal(n)
    return y


@dataclass
class Workload:
    """One synthetic workload of the paper's shape."""
    name: str
    n: int
    m: int
    nu: float               # 0.5 (exponential) or 1.5
    sigma1_sq: float
    rho: float
    nugget: float
    nnz_per_row: float | None = None   # taper chosen for this many nonzeros/row
    gamma: float | None = None         # or given directly
    num_probes: int = 50
    cg_tol: float = 1e-3
    seed: int = BASE_SEED
    n_pred: int = 0
    num_var_samples: int = 0
    extra: dict = field(default_factory=dict)

    def taper_range(self) -> float:
        if self.gamma is not None:
            return float(self.gamma)
        return taper_range_for(self.nnz_per_row, self.n)

    def make(self, with_response: bool = True):
        locs = uniform_locations(self.n, self.seed)
        idx = inducing_subset(self.n, self.m, self.seed)
        inducing = locs[idx].copy()
        y = None
        if with_response:
            y = random_field(locs, self.nu, self.sigma1_sq, self.rho, self.nugget, self.seed)
        pred = None
        if self.n_pred:
            pred = uniform_locations(self.n_pred, self.seed, STREAM_PRED_LOCATIONS)
        return locs, inducing, idx, y, pred


# The five workloads (sizes, covariance and approximation parameters).
SMALL_EXP_N2K = Workload("small-exp-n2000-m50", n=2000, m=50, nu=0.5, sigma1_sq=1.0, rho=0.1,
                         nugget=0.1, gamma=0.05, num_probes=20, cg_tol=1e-8, seed=BASE_SEED + 1)
MATERN15_N1E5 = Workload("matern15-n1e5-m500", n=100_000, m=500, nu=1.5, sigma1_sq=1.0, rho=0.05,
                         nugget=0.05, nnz_per_row=30, num_probes=50, cg_tol=1e-3, seed=BASE_SEED + 2)
EXP_N1E6 = Workload("exp-n1e6-m1000", n=1_000_000, m=1000, nu=0.5, sigma1_sq=1.0, rho=0.02,
                    nugget=0.01, nnz_per_row=20, num_probes=64, cg_tol=1e-3, seed=BASE_SEED + 3)
PRED_N2E5 = Workload("pred-n2e5-np1e5-m800", n=200_000, m=800, nu=0.5, sigma1_sq=1.0, rho=0.05,
                     nugget=0.05, nnz_per_row=25, num_probes=50, cg_tol=1e-3, seed=BASE_SEED + 4,
                     n_pred=100_000, num_var_samples=100)

# The headline's points, taper and probes with few inducing points: the same
# SpMM and element-wise CG kernels on a device footprint of a few GB (the
# profiling case of those kernels).
EXP_N1E6_M128 = Workload("exp-n1e6-m128", n=1_000_000, m=128, nu=0.5, sigma1_sq=1.0, rho=0.02,
                         nugget=0.01, nnz_per_row=20, num_probes=64, cg_tol=1e-3, seed=BASE_SEED + 3)

WORKLOADS = {w.name: w for w in (SMALL_EXP_N2K, MATERN15_N1E5, EXP_N1E6, PRED_N2E5, EXP_N1E6_M128)}


# ----------------------------------------------------------------------------
# Serving stream: independent problems of mixed size arriving as a Poisson process
# ----------------------------------------------------------------------------
STREAM_SERVING = 8
SERVING_SEED = BASE_SEED + 5


@dataclass
class ServingRequest:
    index: int
    arrival_s: float        # arrival time after the stream starts
    kind: str               # "loglik" (likelihood + gradient) or "predict"
    n: int
    m: int
    rho: float
    nugget: float
    sigma1_sq: float = 1.0
    nu: float = 0.5
    nnz_per_row: float = 20.0
    num_probes: int = 50
    n_pred: int = 0
    num_var_samples: int = 0

    @property
    def seed(self) -> int:
        return SERVING_SEED * 1000 + self.index

    def taper_range(self) -> float:
        return taper_range_for(self.nnz_per_row, self.n)

    def make(self, features: int = 64):
        """Locations, inducing points, response (and prediction locations)."""
        locs = uniform_locations(self.n, self.seed)
        ind = locs[inducing_subset(self.n, self.m, self.seed)].copy()
        y = random_field(locs, self.nu, self.sigma1_sq, self.rho, self.nugget, self.seed, features=features)
        pred = uniform_locations(self.n_pred, self.seed, STREAM_PRED_LOCATIONS) if self.n_pred else None
        return locs, ind, y, pred


def serving_stream(num_requests: int = 512, rate_per_s: float = 200.0, seed: int = SERVING_SEED):
    """Requests with Poisson arrivals at ``rate_per_s``; n log-uniform in
    [5e3, 2e5], m uniform in {100, ..., 1000}, range log-uniform in
    [0.01, 0.2], nugget log-uniform in [0.01, 0.5], unit marginal variance,
    exponential covariance, taper for about 20 nonzeros per row, 50 probes;
    an even mix of likelihood+gradient and prediction calls, the latter with
    n/2 prediction locations and 50 variance samples."""
    rng = _rng(seed, STREAM_SERVING)
    gaps = rng.exponential(1.0 / rate_per_s, num_requests)
    arrivals = np.cumsum(gaps) - gaps[0]
    n = np.exp(rng.uniform(math.log(5e3), math.log(2e5), num_requests)).astype(np.int64)
    m = rng.integers(100, 1001, num_requests)
    rho = np.exp(rng.uniform(math.log(0.01), math.log(0.2), num_requests))
    nug = np.exp(rng.uniform(math.log(0.01), math.log(0.5), num_requests))
    kinds = np.array(["loglik", "predict"] * ((num_requests + 1) // 2))[:num_requests]
    kinds = kinds[rng.permutation(num_requests)]
    out = []
    for k in range(num_requests):
        pred = kinds[k] == "predict"
        out.append(ServingRequest(index=k, arrival_s=float(arrivals[k]), kind=str(kinds[k]), n=int(n[k]),
                                  m=int(min(m[k], n[k])), rho=float(rho[k]), nugget=float(nug[k]),
                                  n_pred=int(n[k] // 2) if pred else 0, num_var_samples=50 if pred else 0))
    return out
