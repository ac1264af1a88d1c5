"""Seeded random parity sweep: shapes, statistics, bandwidths, permutation counts and
every way of running a test (tensor-core and plain paths, batches, the streaming mode,
the pre-computation baseline, stream ranges, caller relabelings) against the FP64
oracle on the same inputs.

Tolerances as in test_gpu_parity.py: relative error <= 1e-5 on every statistic, the
count #{stat* >= observed} equal except through near-ties."""
import numpy as np
import pytest

import oracle
from paper_2406_06488_gb300 import workloads

pytestmark = pytest.mark.gpu

REL_TOL = 1e-5
N_CASES = 24


@pytest.fixture(scope="module")
def ept_mod():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_06488_gb300 import ept
    return ept


@pytest.fixture(scope="module")
def ctxs(ept_mod):
    plain = ept_mod.Context(0)
    stream = ept_mod.Context(0)
    stream.set_option("stream_blocks", 40)
    yield plain, stream
    plain.close()
    stream.close()


def _case(k):
    r = np.random.default_rng([2406, k])
    nx = int(r.choice([1, 2, 7, 31, 64, 129, 255, 256, 300, 511, 700]))
    ny = int(r.choice([1, 3, 33, 100, 257, 400, 640, 900]))
    p = int(r.choice([1, 2, 5, 17, 64, 65, 130]))
    B = int(r.choice([0, 1, 63, 256, 257, 700]))
    stat = str(r.choice(["ed", "mmd", "mmd_laplace"]))
    sigma = float(r.uniform(0.5, 3.0)) * np.sqrt(p)
    spec = workloads.TwoSampleSpec(nx=nx, ny=ny, p=p, y_mean=float(r.choice([0.0, 0.1, 0.5])),
                                   y_var=float(r.choice([1.0, 1.3])), data_seed=1000 + k)
    X, Y = workloads.gaussian_pair(spec)
    return X, Y, B, int(r.integers(0, 2**40)), stat, sigma


def _check(res_stats, res_obs, res_nge, ref, B, lo=0, hi=None):
    ref_stats, ref_obs = ref["stats"][lo:hi], ref["observed"]
    assert abs(res_obs - ref_obs) <= REL_TOL * abs(ref_obs), (res_obs, ref_obs)
    if len(ref_stats):
        got = np.asarray(res_stats)
        rel = np.abs(got - ref_stats) / np.abs(ref_stats)
        assert rel.max() <= REL_TOL, "max relative error %.3g at b=%d" % (rel.max(), int(rel.argmax()) + 1)
        near = np.abs(ref_stats - ref_obs) <= 1e-5 * abs(ref_obs)
        ref_nge = int(np.count_nonzero(ref_stats >= ref_obs))
        assert abs(res_nge - ref_nge) <= int(near.sum()), (res_nge, ref_nge)


@pytest.mark.parametrize("k", range(N_CASES))
def test_random_case_every_mode(ctxs, k):
    plain_ctx, stream_ctx = ctxs
    X, Y, B, seed, stat, sigma = _case(k)
    ref = oracle.permutation_test(X, Y, B=B, seed=seed, stat=stat, sigma=sigma)
    for prec in ("split_bf16", "plain_fp32", "pooled_fp32"):
        r = plain_ctx.test(X, Y, B=B, seed=seed, stat=stat, sigma=sigma, prec=prec)
        _check(r.stats if B else [], r.observed, r.n_ge, ref, B)
        assert r.p_value == (1.0 + r.n_ge) / (1.0 + B)
    r = stream_ctx.test(X, Y, B=B, seed=seed, stat=stat, sigma=sigma)
    assert r.n_windows >= 1
    _check(r.stats if B else [], r.observed, r.n_ge, ref, B)
    if B >= 2:
        lo = B // 3
        r = plain_ctx.test_range(X, Y, b_first=lo + 1, count=B - lo, seed=seed, stat=stat, sigma=sigma)
        _check(r.stats, r.observed, r.n_ge, ref, B, lo=lo)
        masks = oracle.pack_masks(oracle.perm_select(seed, X.shape[0], Y.shape[0], 1, B))
        r = plain_ctx.test_masks(X, Y, masks, stat=stat, sigma=sigma)
        _check(r.stats, r.observed, r.n_ge, ref, B)


def test_random_cases_as_one_batch(ctxs):
    plain_ctx, _ = ctxs
    cases = [_case(k) for k in range(N_CASES)]
    tests = [dict(X=X, Y=Y, B=B, seed=seed, stat=stat, sigma=sigma) for X, Y, B, seed, stat, sigma in cases]
    res = plain_ctx.test_batch(tests)
    for (X, Y, B, seed, stat, sigma), r in zip(cases, res):
        ref = oracle.permutation_test(X, Y, B=B, seed=seed, stat=stat, sigma=sigma)
        _check(r.stats if B else [], r.observed, r.n_ge, ref, B)
