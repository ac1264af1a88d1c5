"""The Laplacian-kernel MMD and the median-heuristic bandwidth on the GPU against the
FP64 oracle (statistics within 1e-5 relative; the selected bandwidth within the
rounding of the FP32 distances it is chosen from)."""
import numpy as np
import pytest

import oracle
from paper_2406_06488_gb300 import workloads

pytestmark = pytest.mark.gpu

REL_TOL = 1e-5
PRECS = ["split_bf16", "plain_fp32"]


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_06488_gb300 import ept
    c = ept.Context(0)
    yield c
    c.close()


def _pair(nx, ny, p, seed, shift=0.3):
    return workloads.gaussian_pair(workloads.TwoSampleSpec(nx=nx, ny=ny, p=p, y_mean=shift, data_seed=seed))


def _check(res, ref, B):
    assert abs(res.observed - ref["observed"]) <= REL_TOL * abs(ref["observed"])
    if B > 0:
        got = np.asarray(res.stats)
        rel = np.abs(got - ref["stats"]) / np.abs(ref["stats"])
        assert rel.max() <= REL_TOL, rel.max()
        near = np.abs(ref["stats"] - ref["observed"]) <= 1e-5 * abs(ref["observed"])
        assert abs(res.n_ge - ref["n_ge"]) <= int(near.sum())


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("nx,ny,p", [(100, 100, 10), (37, 290, 7), (300, 5, 40)])
def test_laplace_fixed_bandwidth(ctx, prec, nx, ny, p):
    X, Y = _pair(nx, ny, p, seed=nx + ny)
    sigma = float(np.sqrt(p))
    res = ctx.test(X, Y, B=400, seed=3, stat="mmd_laplace", sigma=sigma, prec=prec)
    ref = oracle.permutation_test(X, Y, B=400, seed=3, stat="mmd_laplace", sigma=sigma)
    _check(res, ref, 400)
    assert res.sigma == sigma


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("stat", ["mmd", "mmd_laplace"])
@pytest.mark.parametrize("nx,ny,p", [(100, 100, 10), (61, 200, 3), (257, 300, 30)])
def test_median_bandwidth(ctx, prec, stat, nx, ny, p):
    X, Y = _pair(nx, ny, p, seed=7 * nx + ny)
    res = ctx.test(X, Y, B=300, seed=5, stat=stat, sigma="median", prec=prec)
    want = oracle.median_pairs(X, Y)
    # the k-th smallest of values known to ~1e-6 relative is known to the same accuracy
    assert abs(res.sigma - want) <= 2e-6 * want, (res.sigma, want)
    # statistics: the oracle with the bandwidth the GPU selected
    ref = oracle.permutation_test(X, Y, B=300, seed=5, stat=stat, sigma=res.sigma)
    _check(res, ref, 300)


def test_median_bandwidth_of_coinciding_rows_is_rejected(ctx):
    from paper_2406_06488_gb300 import ept
    X = np.zeros((6, 3), dtype=np.float32)
    Y = np.zeros((5, 3), dtype=np.float32)
    with pytest.raises(ept.EptError) as e:
        ctx.test(X, Y, B=10, stat="mmd", sigma="median")
    assert e.value.status == 1
    with pytest.raises(ept.EptError):
        ctx.test(X, Y, B=10, stat="mmd", sigma=0.0)


@pytest.mark.parametrize("prec", PRECS)
def test_blocks_with_median_bandwidth(ctx, prec):
    X, Y = _pair(70, 90, 6, seed=11)
    K = ctx.build_blocks(X, Y, stat="mmd_laplace", sigma="median", prec=prec)
    res = ctx.test(X, Y, B=0, stat="mmd_laplace", sigma="median", prec=prec)
    W = np.concatenate([X, Y])
    ref = oracle.block_matrix(W, W, "mmd_laplace", res.sigma)
    assert np.max(np.abs(K - ref)) <= 2e-6


def test_mixed_batch(ctx):
    tests = []
    kinds = [("ed", 1.0), ("mmd", 2.0), ("mmd_laplace", 2.0), ("mmd", "median"), ("mmd_laplace", "median")]
    for k, (stat, sigma) in enumerate(kinds * 2):
        X, Y = _pair(40 + 30 * k, 150 - 10 * k, 3 + k, seed=100 + k)
        tests.append(dict(X=X, Y=Y, B=200 + 10 * k, seed=k, stat=stat, sigma=sigma))
    got = ctx.test_batch(tests)
    for t, r in zip(tests, got):
        alone = ctx.test(t["X"], t["Y"], B=t["B"], seed=t["seed"], stat=t["stat"], sigma=t["sigma"])
        assert r.sigma == alone.sigma
        assert abs(r.observed - alone.observed) <= REL_TOL * abs(alone.observed)
        assert np.max(np.abs(np.asarray(r.stats) - np.asarray(alone.stats)) / np.abs(np.asarray(alone.stats))) <= REL_TOL


def test_full_size_mmd_median_sampled(ctx):
    # the MMD shape (nx = ny = 10000, p = 100) with the median-heuristic bandwidth:
    # sampled draws against the oracle at the bandwidth the GPU selected, and the
    # bandwidth against the median of a random sample of pooled pairs
    spec = workloads.MMD_MEDIAN
    X, Y = workloads.gaussian_pair(spec)
    res = ctx.test(X, Y, B=2000, seed=spec.seed, stat=spec.stat, sigma="median")
    st = np.asarray(res.stats)
    obs = oracle.stat_select(X, Y, oracle.perm_select(spec.seed, spec.nx, spec.ny, 0, 1)[0], spec.stat, res.sigma)
    assert abs(res.observed - obs) <= REL_TOL * abs(obs)
    for b in list(range(1, 16)) + [2000]:
        sel = oracle.perm_select(spec.seed, spec.nx, spec.ny, b, 1)[0]
        v = oracle.stat_select(X, Y, sel, spec.stat, res.sigma)
        assert abs(st[b - 1] - v) <= REL_TOL * abs(v), (b, st[b - 1], v)
    W = np.concatenate([X, Y]).astype(np.float64)
    r = np.random.default_rng(0)
    i, j = r.integers(0, W.shape[0], 200000), r.integers(0, W.shape[0], 200000)
    keep = i != j
    d = np.sqrt(((W[i[keep]] - W[j[keep]]) ** 2).sum(axis=1))
    # the sample median of 2e5 pairs is within a few 1e-3 of the population median
    assert abs(np.median(d) - res.sigma) <= 0.01 * res.sigma
