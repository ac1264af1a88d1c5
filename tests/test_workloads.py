"""The input recipe (paper_2406_06488_gb300/workloads.py) as stated for the workloads:
Gaussian samples shaped like the paper's experiments (Section 5), with the mean shift
and variance where the recipe puts them (checked within CLT bounds), reproducible
draws from independent X and Y streams, and the batched, serving and statistical
experiment specifications with their stated ranges."""
import math

import numpy as np

from paper_2406_06488_gb300 import workloads as wl


def test_highdim_shapes_mean_shift_and_unit_variance():
    spec = wl.HIGHDIM
    X, Y = wl.gaussian_pair(spec)
    assert X.shape == (2000, 1000) and Y.shape == (3000, 1000)
    assert X.dtype == np.float32 and Y.dtype == np.float32
    assert X.flags["C_CONTIGUOUS"] and Y.flags["C_CONTIGUOUS"]
    my = Y.mean(axis=0, dtype=np.float64)
    # mean 0.05 on the first 50 coordinates only (sd of a 50-coordinate average of
    # 3000-row means: 1 / sqrt(150000) = 0.0026)
    assert abs(my[:50].mean() - 0.05) < 0.012
    assert abs(my[50:].mean()) < 0.004
    assert abs(X.mean(dtype=np.float64)) < 0.003
    assert abs(X.var(dtype=np.float64) - 1.0) < 0.005 and abs(Y[:, 50:].var(dtype=np.float64) - 1.0) < 0.005


def test_mmd_variance_of_y():
    X, Y = wl.gaussian_pair(wl.MMD)
    assert X.shape == (10000, 100) and Y.shape == (10000, 100)
    assert abs(Y.var(dtype=np.float64) - 1.1) < 0.01
    assert abs(X.var(dtype=np.float64) - 1.0) < 0.01
    assert abs(Y.mean(dtype=np.float64)) < 0.003
    assert wl.MMD.sigma == math.sqrt(wl.MMD.p) and wl.MMD.B == 10000
    assert wl.MMD_LAPLACE.stat == "mmd_laplace" and wl.MMD_MEDIAN.sigma < 0


def test_draws_are_reproducible_and_streams_independent():
    a = wl.gaussian_pair(wl.SMALL)
    b = wl.gaussian_pair(wl.SMALL)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    other = wl.gaussian_pair(wl.TwoSampleSpec(nx=100, ny=100, p=10, y_mean=0.2, data_seed=1))
    assert not np.array_equal(a[0], other[0])
    # X does not depend on anything about Y; Y's shift is added to the same draws
    null = wl.gaussian_pair(wl.TwoSampleSpec(nx=100, ny=100, p=10, data_seed=0))
    assert np.array_equal(a[0], null[0])
    assert np.allclose(a[1] - null[1], np.float32(0.2), atol=1e-6)


def test_named_workloads():
    assert (wl.SMALL.nx, wl.SMALL.ny, wl.SMALL.p, wl.SMALL.y_mean, wl.SMALL.B) == (100, 100, 10, 0.2, 1000)
    assert (wl.TINY.nx, wl.TINY.ny, wl.TINY.p) == (4, 4, 3)
    assert (wl.STREAM.nx + wl.STREAM.ny, wl.STREAM.p, wl.STREAM.B) == (400000, 64, 10000)
    assert set(wl.NAMED) >= {"small", "tiny", "highdim", "mmd", "mmd_laplace", "mmd_median", "stream"}


def test_batched_specs():
    specs = wl.batched_specs(512, B=5000)
    assert len(specs) == 512
    nx = np.array([s.nx for s in specs])
    ny = np.array([s.ny for s in specs])
    p = np.array([s.p for s in specs])
    assert nx.min() >= 50 and nx.max() <= 2000 and ny.min() >= 50 and ny.max() <= 2000
    assert p.min() >= 20 and p.max() <= 500
    assert 900 < nx.mean() < 1150 and 230 < p.mean() < 290          # uniform means 1025 and 260
    assert all(s.y_mean == (0.0 if t % 2 == 0 else 0.1) and s.seed == t and s.B == 5000 and s.stat == "ed"
               for t, s in enumerate(specs))
    assert len({s.data_seed for s in specs}) == 512


def test_serving_requests():
    reqs = wl.serving_requests(300.0, 2000)
    t = np.array([r[0] for r in reqs])
    assert np.all(np.diff(t) > 0)
    assert abs(t[-1] / 2000 - 1 / 300.0) < 0.1 / 300.0               # Poisson arrivals at the rate
    specs = [r[1] for r in reqs]
    assert all(100 <= s.nx <= 20000 and 100 <= s.ny <= 20000 and 10 <= s.p <= 2000 for s in specs)
    assert {s.B for s in specs} <= {1000, 5000, 20000}
    mmd = [s for s in specs if s.stat == "mmd"]
    assert 0.45 < len(mmd) / len(specs) < 0.55
    assert all(s.sigma == math.sqrt(s.p) for s in mmd)
    # log-uniform: the median of nx near sqrt(100 * 20000)
    assert 1000 < np.median([s.nx for s in specs]) < 2000


def test_statistical_experiment_specs():
    null = wl.null_specs(reps=10, p=100)
    assert all(s.nx == s.ny == 200 and s.p == 100 and s.y_mean == 0.0 and s.B == 200 for s in null)
    assert len({s.data_seed for s in null}) == 10
    pts1 = wl.power_specs(1, reps=3)
    assert [x for x, _ in pts1] == list(range(60, 361, 20))
    assert all(s.nx == s.ny == x and s.p == 50 and s.y_mean_coords == 5 and s.y_mean == 0.25
               for x, ss in pts1 for s in ss)
    pts2 = wl.power_specs(2, reps=2, points=[200, 2000])
    assert [x for x, _ in pts2] == [200, 2000] and all(s.y_mean_coords == 50 for _, ss in pts2 for s in ss)
    pts3 = wl.power_specs(3, reps=2, points=[1000])
    assert pts3[0][1][0].y_mean_coords == 100
