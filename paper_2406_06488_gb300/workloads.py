"""Seeded synthetic two-sample inputs shaped like the paper's Gaussian experiments.

This module only draws input data; it holds none of the test's arithmetic, and it
is the one piece of code that both the CUDA path's callers and the CPU oracle's
callers use.  All draws come from numpy's PCG64 generator (``default_rng``) keyed
by (seed, stream) so that X and Y are independent streams and every workload is
reproducible.

Workloads (the paper draws X ~ N_p(0, I) and Y ~ N_p(mu, I), Section 5.2):

* ``small``      ED, nx = ny = 100, p = 10, Y mean 0.2 on every coordinate
* ``tiny``       ED, nx = ny = 4, p = 3 (exhaustive check of all 70 relabelings)
* ``highdim``    ED, nx = 2000, ny = 3000, p = 1000, Y mean 0.05 on the first 50
                 coordinates
* ``mmd``        Gaussian MMD, nx = ny = 10000, p = 100, Y ~ N(0, 1.1 I),
                 bandwidth sigma = sqrt(p)
* ``mmd_laplace`` the same shape with the Laplacian kernel exp(-d / sigma), sigma = sqrt(p)
* ``mmd_median`` the same shape, Gaussian kernel, bandwidth from the median heuristic
* ``batched``    512 independent ED tests, nx, ny uniform on {50..2000}, p uniform on
                 {20..500}, half null, half with Y mean 0.1 on every coordinate
* ``serving``    Poisson request stream (see ``serving_requests``)
* ``null_specs`` / ``power_specs``  the paper's statistical experiments (Section 5):
                 null replications (X, Y ~ N_p(0, I), nx = ny = 200, p = 100 or 1000) and
                 the three power settings (Y mean eps on the first j coordinates)
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class TwoSampleSpec:
    nx: int
    ny: int
    p: int
    stat: str = "ed"          # "ed" or "mmd"
    sigma: float = 1.0        # kernel bandwidth (MMD only)
    y_mean: float = 0.0       # mean of Y on the shifted coordinates
    y_mean_coords: int = -1   # number of shifted leading coordinates (-1 = all)
    y_var: float = 1.0        # variance of every coordinate of Y
    B: int = 1000
    seed: int = 0             # permutation-stream seed
    data_seed: int = 0        # data seed


def gaussian_pair(spec: TwoSampleSpec):
    """X ~ N_p(0, I) (nx rows), Y ~ N_p(mu, y_var I) (ny rows), both float32 row-major."""
    rx = np.random.default_rng([spec.data_seed, 0])
    ry = np.random.default_rng([spec.data_seed, 1])
    X = rx.standard_normal((spec.nx, spec.p), dtype=np.float32)
    Y = ry.standard_normal((spec.ny, spec.p), dtype=np.float32)
    if spec.y_var != 1.0:
        Y *= np.float32(math.sqrt(spec.y_var))
    if spec.y_mean != 0.0:
        k = spec.p if spec.y_mean_coords < 0 else min(spec.y_mean_coords, spec.p)
        Y[:, :k] += np.float32(spec.y_mean)
    return np.ascontiguousarray(X), np.ascontiguousarray(Y)


SMALL = TwoSampleSpec(nx=100, ny=100, p=10, y_mean=0.2, B=1000, seed=0, data_seed=0)
TINY = TwoSampleSpec(nx=4, ny=4, p=3, y_mean=0.2, B=70, seed=0, data_seed=0)
HIGHDIM = TwoSampleSpec(nx=2000, ny=3000, p=1000, y_mean=0.05, y_mean_coords=50, B=10000,
                        seed=0, data_seed=0)
MMD = TwoSampleSpec(nx=10000, ny=10000, p=100, stat="mmd", sigma=10.0, y_var=1.1, B=10000,
                    seed=0, data_seed=0)

# the MMD shape with the Laplacian kernel exp(-d / sigma), and with the Gaussian kernel
# whose bandwidth comes from the median heuristic (sigma = -1 selects it)
MMD_LAPLACE = TwoSampleSpec(nx=10000, ny=10000, p=100, stat="mmd_laplace", sigma=10.0, y_var=1.1, B=10000,
                            seed=0, data_seed=0)
MMD_MEDIAN = TwoSampleSpec(nx=10000, ny=10000, p=100, stat="mmd", sigma=-1.0, y_var=1.1, B=10000,
                           seed=0, data_seed=0)

# a test beyond device memory: n = 400,000 pooled rows, whose packed upper blocks
# (about 2 n^2 = 320 GB) exceed the GPU's memory; it runs in the streaming mode
STREAM = TwoSampleSpec(nx=200000, ny=200000, p=64, y_mean=0.01, B=10000, seed=0, data_seed=0)

NAMED = {"small": SMALL, "tiny": TINY, "highdim": HIGHDIM, "mmd": MMD, "mmd_laplace": MMD_LAPLACE,
         "mmd_median": MMD_MEDIAN, "stream": STREAM}


def batched_specs(n_tests: int = 512, B: int = 5000, master_seed: int = 0):
    """Uneven independent ED tests: nx, ny ~ U{50..2000}, p ~ U{20..500};
    even test ids are null, odd ones have Y mean 0.1 on every coordinate.
    The permutation seed of test t is t."""
    r = np.random.default_rng([master_seed, 2])
    nx = r.integers(50, 2001, size=n_tests)
    ny = r.integers(50, 2001, size=n_tests)
    p = r.integers(20, 501, size=n_tests)
    out = []
    for t in range(n_tests):
        out.append(TwoSampleSpec(nx=int(nx[t]), ny=int(ny[t]), p=int(p[t]), stat="ed",
                                 y_mean=0.0 if t % 2 == 0 else 0.1, B=B, seed=t,
                                 data_seed=master_seed * 1_000_003 + t + 1))
    return out


def serving_requests(rate_per_s: float, n_requests: int, master_seed: int = 0,
                     n_range=(100, 20000), p_range=(10, 2000), B_choices=(1000, 5000, 20000)):
    """Poisson arrivals at rate_per_s; nx, ny log-uniform on n_range, p log-uniform on
    p_range, B uniform on B_choices, ED / Gaussian MMD (sigma = sqrt(p)) half each.
    Returns a list of (arrival_time_s, TwoSampleSpec)."""
    r = np.random.default_rng([master_seed, 3])
    t = np.cumsum(r.exponential(1.0 / rate_per_s, size=n_requests))
    lo, hi = math.log(n_range[0]), math.log(n_range[1])
    nx = np.exp(r.uniform(lo, hi, size=n_requests)).astype(np.int64)
    ny = np.exp(r.uniform(lo, hi, size=n_requests)).astype(np.int64)
    plo, phi = math.log(p_range[0]), math.log(p_range[1])
    p = np.exp(r.uniform(plo, phi, size=n_requests)).astype(np.int64)
    Bs = r.choice(np.asarray(B_choices), size=n_requests)
    kinds = r.integers(0, 2, size=n_requests)
    out = []
    for k in range(n_requests):
        stat = "ed" if kinds[k] == 0 else "mmd"
        out.append((float(t[k]), TwoSampleSpec(nx=int(nx[k]), ny=int(ny[k]), p=int(p[k]), stat=stat,
                                               sigma=math.sqrt(float(p[k])), B=int(Bs[k]), seed=k,
                                               data_seed=master_seed * 7_000_003 + k + 1)))
    return out


def null_specs(reps: int = 2000, n: int = 200, p: int = 100, B: int = 200, stat: str = "ed",
               master_seed: int = 0):
    """Null replications of Section 5: X and Y both N_p(0, I), nx = ny = n (the paper's
    "n = 200" read as the size of each sample), B permutations; replication r has
    permutation seed r and its own data seed."""
    return [TwoSampleSpec(nx=n, ny=n, p=p, stat=stat, sigma=math.sqrt(p), B=B, seed=r,
                          data_seed=master_seed * 10_000_019 + 7 * p + 100_003 * r + 1)
            for r in range(reps)]


def power_specs(setting: int, reps: int = 500, B: int = 200, points=None, master_seed: int = 0):
    """The power experiments of Section 5 (Y ~ N_p(mu, I), mu = eps on the first j
    coordinates, B = 200 permutations, 500 replications per point):
    setting 1: nx = ny in 60..360 step 20, p = 50, j = 5, eps = 0.25;
    setting 2: nx = ny = 200, p in 200..2000 step 100, j = 50, eps = 0.1;
    setting 3: as setting 2 with j = p / 10.
    Returns [(x value of the point, [TwoSampleSpec] * reps)]; `points` restricts the
    x values."""
    if setting == 1:
        xs = list(range(60, 361, 20))
        make = lambda x: dict(nx=x, ny=x, p=50, y_mean=0.25, y_mean_coords=5)
    elif setting in (2, 3):
        xs = list(range(200, 2001, 100))
        make = lambda x: dict(nx=200, ny=200, p=x, y_mean=0.1,
                              y_mean_coords=50 if setting == 2 else x // 10)
    else:
        raise ValueError("setting must be 1, 2 or 3")
    if points is not None:
        xs = [x for x in xs if x in set(points)]
    out = []
    for x in xs:
        kw = make(x)
        out.append((x, [TwoSampleSpec(B=B, seed=r, data_seed=master_seed * 10_000_019 + 1_000_003 * setting
                                      + 1009 * x + 100_003 * r + 2, **kw) for r in range(reps)]))
    return out
