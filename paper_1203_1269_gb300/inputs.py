"""Seeded synthetic inputs for the GP likelihood / kriging workloads.

This module is the one piece shared by the CUDA path's tests and benchmark
and by the CPU oracle's tests: it only draws designs, responses and theta
candidates.  It holds none of the method's arithmetic (no correlation, no
factorisation, no likelihood).

The paper's experiments use maximin Latin-hypercube designs on the
Goldstein-Price and Hartman-6 test functions (Section 4).  Those functions and
the maximin criterion are not used here: seeded random designs and the smooth
synthetic responses below stand in for them, with the paper's shapes
(n ~ 4000, d = 6, p = 1.95, a theta population per optimiser generation).

Every generator uses numpy.random.Generator(PCG64(seed)).
"""
from dataclasses import dataclass, field
import math

import numpy as np

BASE_SEED = 1269


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_design(g: np.random.Generator, n: int, d: int) -> np.ndarray:
    """n points i.i.d. uniform on [0,1]^d."""
    return g.random((n, d))


def random_lhd(g: np.random.Generator, n: int, d: int) -> np.ndarray:
    """Random Latin hypercube on [0,1]^d: x_ik = (pi_k(i) + U_ik) / n with an
    independent permutation pi_k per dimension."""
    x = np.empty((n, d))
    for k in range(d):
        perm = g.permutation(n)
        x[:, k] = (perm + g.random(n)) / n
    return x


def log_uniform_thetas(g: np.random.Generator, T: int, d: int, lo=-2.0, hi=1.0) -> np.ndarray:
    """T candidate theta vectors with log10 theta_k ~ U[lo, hi] i.i.d."""
    return 10.0 ** g.uniform(lo, hi, size=(T, d))


def grid_thetas(d: int, m: int, lo=-2.0, hi=1.0) -> np.ndarray:
    """Full tensor grid of 10^linspace(lo, hi, m) per dimension (m^d rows)."""
    axis = 10.0 ** np.linspace(lo, hi, m)
    mesh = np.meshgrid(*([axis] * d), indexing="ij")
    return np.stack([a.reshape(-1) for a in mesh], axis=1)


# --- synthetic responses (stand-ins for the paper's test functions) -------

def y_trig2(x):
    """y = sin(2 pi x1) + 0.5 cos(3 pi x2) + x1 x2."""
    return np.sin(2 * np.pi * x[:, 0]) + 0.5 * np.cos(3 * np.pi * x[:, 1]) + x[:, 0] * x[:, 1]


def y_sinsum(x):
    """y = sum_k sin(2 pi x_k) / k + 0.1 sum_k x_k^2."""
    k = np.arange(1, x.shape[1] + 1)
    return (np.sin(2 * np.pi * x) / k).sum(axis=1) + 0.1 * (x ** 2).sum(axis=1)


def y_bump(x):
    """y = exp(-||x - 0.5||^2) + 0.05 sum_k x_k."""
    return np.exp(-((x - 0.5) ** 2).sum(axis=1)) + 0.05 * x.sum(axis=1)


def y_wave(x):
    """y = sum_k (x_k - 0.5) sin(4 x_k) + x1 x2 x3."""
    return ((x - 0.5) * np.sin(4 * x)).sum(axis=1) + x[:, 0] * x[:, 1] * x[:, 2]


@dataclass
class Workload:
    name: str
    x: np.ndarray          # n x d design
    y: np.ndarray          # n responses
    thetas: np.ndarray     # T x d candidates
    p: float
    delta: float
    xs: np.ndarray = field(default=None)  # N x d prediction points (or None)

    @property
    def n(self):
        return self.x.shape[0]

    @property
    def d(self):
        return self.x.shape[1]

    @property
    def T(self):
        return self.thetas.shape[0]


def small_grid_fit(n=200, N=1000, seed=BASE_SEED + 0) -> Workload:
    """n=200, d=2, x ~ U[0,1]^2, y_trig2, p=2, delta=1e-8; theta on an 8 x 8
    grid of 10^linspace(-2,1,8); N=1000 uniform prediction points."""
    g = rng(seed)
    x = uniform_design(g, n, 2)
    y = y_trig2(x)
    xs = uniform_design(g, N, 2)
    return Workload("n200_d2_grid64", x, y, grid_thetas(2, 8), 2.0, 1e-8, xs)


def hartman_shape(n=4000, d=6, T=256, seed=BASE_SEED + 1) -> Workload:
    """n=4000, d=6, random LHD, y_sinsum, p=1.95, delta=1e-7; T=256 thetas
    log10-uniform in [-2,1]^6 (a multi-start population)."""
    g = rng(seed)
    x = random_lhd(g, n, d)
    y = y_sinsum(x)
    th = log_uniform_thetas(g, T, d)
    return Workload(f"n{n}_d{d}_T{T}", x, y, th, 1.95, 1e-7)


def batched_split(n=2048, d=8, T=1024, seed=BASE_SEED + 2) -> Workload:
    """n=2048, d=8, x ~ U[0,1]^8, y_bump, p=2, delta=1e-6; T=1024 thetas."""
    g = rng(seed)
    x = uniform_design(g, n, d)
    y = y_bump(x)
    th = log_uniform_thetas(g, T, d)
    return Workload(f"n{n}_d{d}_T{T}", x, y, th, 2.0, 1e-6)


def large_instance(n=16384, d=10, T=32, N=100000, seed=BASE_SEED + 3) -> Workload:
    """n=16384, d=10, random LHD, y_wave, p=1.9, delta=1e-6; T=32 thetas;
    N=1e5 uniform prediction points."""
    g = rng(seed)
    x = random_lhd(g, n, d)
    y = y_wave(x)
    th = log_uniform_thetas(g, T, d)
    xs = uniform_design(g, N, d) if N else None
    return Workload(f"n{n}_d{d}_T{T}", x, y, th, 1.9, 1e-6, xs)


@dataclass
class Request:
    rid: int
    arrival_s: float
    kind: str              # "fit" or "predict"
    n: int
    d: int
    p: float
    delta: float
    seed: int
    target: int = -1       # for predict: rid of a fit request


def serving_stream(count=2000, rate=200.0, seed=BASE_SEED + 4, fit_frac=0.5,
                   n_lo=256, n_hi=8192):
    """Poisson arrivals at `rate` req/s; n log-uniform in [n_lo, n_hi];
    d uniform in {2..12}; p in {1.5, 1.95, 2}; delta in {1e-8, 1e-6}.
    A predict names an earlier fit request as its target (the first request
    is always a fit)."""
    g = rng(seed)
    t = 0.0
    reqs = []
    fits = []
    for i in range(count):
        t += g.exponential(1.0 / rate)
        kind = "fit" if (not fits or g.random() < fit_frac) else "predict"
        n = int(round(math.exp(g.uniform(math.log(n_lo), math.log(n_hi)))))
        d = int(g.integers(2, 13))
        p = float(g.choice([1.5, 1.95, 2.0]))
        delta = float(g.choice([1e-8, 1e-6]))
        r = Request(i, t, kind, n, d, p, delta, int(g.integers(0, 2**31 - 1)))
        if kind == "predict":
            r.target = int(fits[int(g.integers(0, len(fits)))])
        else:
            fits.append(i)
        reqs.append(r)
    return reqs


def request_data(req: Request, N=1000):
    """Design, response, thetas (32 for a fit) and prediction points of one
    serving request, drawn from its own seed.  y as in hartman_shape."""
    g = rng(req.seed)
    x = random_lhd(g, req.n, req.d)
    y = y_sinsum(x)
    th = log_uniform_thetas(g, 32, req.d)
    xs = uniform_design(g, N, req.d)
    return x, y, th, xs
