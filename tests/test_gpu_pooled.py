"""GPU parity of the pre-computation baseline (Algorithm 5: the full pooled matrix
computed once, each relabeling's three sub-matrices extracted by index and summed)
against the FP64 oracle and the efficient path.

Tolerances as in test_gpu_parity.py: relative error <= 1e-5 on every statistic, the
count #{stat* >= observed} equal except through near-ties."""
import numpy as np
import pytest

import oracle
from paper_2406_06488_gb300 import workloads

pytestmark = pytest.mark.gpu

REL_TOL = 1e-5


@pytest.fixture(scope="module")
def ept_mod():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_06488_gb300 import ept
    return ept


@pytest.fixture(scope="module")
def ctx(ept_mod):
    c = ept_mod.Context(0)
    yield c
    c.close()


def _pair(nx, ny, p, seed=0, shift=0.2):
    return workloads.gaussian_pair(workloads.TwoSampleSpec(nx=nx, ny=ny, p=p, y_mean=shift, data_seed=seed))


def _check(res, ref_stats, ref_obs, B, tol=REL_TOL):
    assert abs(res.observed - ref_obs) <= tol * abs(ref_obs), (res.observed, ref_obs)
    if B > 0:
        got = np.asarray(res.stats)
        rel = np.abs(got - ref_stats) / np.abs(ref_stats)
        assert rel.max() <= tol, "max relative error %.3g at b=%d" % (rel.max(), int(rel.argmax()) + 1)
        near = np.abs(ref_stats - ref_obs) <= 1e-5 * abs(ref_obs)
        ref_nge = int(np.count_nonzero(ref_stats >= ref_obs))
        assert abs(res.n_ge - ref_nge) <= int(near.sum()), (res.n_ge, ref_nge, int(near.sum()))
    assert res.p_value == (1.0 + res.n_ge) / (1.0 + B)


@pytest.mark.parametrize("nx,ny,p,B,stat", [
    (1, 1, 1, 10, "ed"), (9, 1, 4, 50, "mmd"), (255, 2, 5, 300, "mmd_laplace"), (256, 256, 3, 257, "ed"),
    (257, 300, 20, 1023, "mmd"), (3, 600, 2, 129, "ed"), (700, 900, 37, 300, "ed"), (900, 300, 40, 200, "ed"),
    (200, 200, 2000, 200, "ed"), (1000, 1000, 500, 200, "ed")])
def test_pooled_matches_oracle(ctx, nx, ny, p, B, stat):
    X, Y = _pair(nx, ny, p, seed=nx * 5 + ny, shift=0.1)
    sigma = 1.9 if p < 100 else float(np.sqrt(p))
    ref = oracle.permutation_test(X, Y, B=B, seed=nx + 1, stat=stat, sigma=sigma)
    res = ctx.test(X, Y, B=B, seed=nx + 1, stat=stat, sigma=sigma, prec="pooled_fp32")
    _check(res, ref["stats"], ref["observed"], B)


def test_pooled_matches_efficient_path(ctx):
    # the paper's first timing experiment's largest shape (nx = ny = 1000, p = 500, B = 200)
    X, Y = _pair(1000, 1000, 500, seed=2, shift=0.02)
    a = ctx.test(X, Y, B=200, seed=7, prec="pooled_fp32")
    b = ctx.test(X, Y, B=200, seed=7, prec="split_bf16")
    sa, sb = np.asarray(a.stats), np.asarray(b.stats)
    assert np.max(np.abs(sa - sb) / np.abs(sb)) <= 2 * REL_TOL
    assert a.n_ge == b.n_ge or abs(a.n_ge - b.n_ge) <= b.n_near_tie + a.n_near_tie


def test_pooled_masks_range_device(ctx):
    torch = pytest.importorskip("torch")
    X, Y = _pair(4, 4, 3, seed=21, shift=0.6)
    sel, ref_stats = oracle.exhaustive(X, Y, "ed", 1.0)
    res = ctx.test_masks(X, Y, oracle.pack_masks(sel), stat="ed", prec="pooled_fp32")
    assert np.max(np.abs(np.asarray(res.stats) - ref_stats) / np.abs(ref_stats)) <= REL_TOL
    X, Y = _pair(300, 500, 12, seed=4)
    ref = oracle.permutation_test(X, Y, B=400, seed=9, stat="ed")
    r = ctx.test_range(X, Y, b_first=101, count=200, seed=9, stat="ed", prec="pooled_fp32")
    got = np.asarray(r.stats)
    assert np.max(np.abs(got - ref["stats"][100:300]) / np.abs(ref["stats"][100:300])) <= REL_TOL
    rd = ctx.test(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), B=400, seed=9, prec="pooled_fp32")
    assert rd.stats.is_cuda
    rd.stats = rd.stats.cpu().numpy()
    _check(rd, ref["stats"], ref["observed"], 400)


def test_pooled_unsupported(ctx, ept_mod):
    X, Y = _pair(50, 60, 5)
    with pytest.raises(ept_mod.EptError) as e:
        ctx.test_batch([{"X": X, "Y": Y, "B": 10}], prec="pooled_fp32")
    assert e.value.status == 8   # EPT_EUNSUPPORTED
    with pytest.raises(ept_mod.EptError) as e:
        ctx.test(X, Y, B=10, stat="mmd", sigma="median", prec="pooled_fp32")
    assert e.value.status == 8
    ref = oracle.permutation_test(X, Y, B=10, seed=0, stat="ed")
    _check(ctx.test(X, Y, B=10, prec="pooled_fp32"), ref["stats"], ref["observed"], 10)


def test_pooled_zero_permutations(ctx):
    X, Y = _pair(300, 200, 6, seed=14)
    res = ctx.test(X, Y, B=0, seed=0, prec="pooled_fp32")
    assert res.p_value == 1.0 and res.n_ge == 0
    ref = oracle.stat_direct(X, Y, "ed")
    assert abs(res.observed - ref) <= REL_TOL * ref
