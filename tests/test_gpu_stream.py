"""GPU parity of the streaming mode (windows of row panels for tests whose packed
blocks do not fit in device memory) against the FP64 oracle and the resident path.

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
    c.set_option("stream_blocks", 1)   # every window one row panel
    yield c
    c.close()


def _pair(nx, ny, p, seed=0, shift=0.2):
    return workloads.gaussian_pair(workloads.TwoSampleSpec(nx=nx, ny=ny, p=p, y_mean=shift, data_seed=seed))


def _panels(n):
    return (n + 255) // 256


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
    (600, 700, 65, 500, "mmd_laplace")])
def test_stream_one_panel_windows(ctx, nx, ny, p, B, stat):
    X, Y = _pair(nx, ny, p, seed=nx * 5 + ny, shift=0.1)
    sigma = 1.9
    ref = oracle.permutation_test(X, Y, B=B, seed=nx + 1, stat=stat, sigma=sigma)
    res = ctx.test(X, Y, B=B, seed=nx + 1, stat=stat, sigma=sigma)
    assert res.n_windows == _panels(nx + ny)
    _check(res, ref["stats"], ref["observed"], B)


@pytest.mark.parametrize("blocks", [60, 200, 10 ** 9])
def test_stream_window_sizes(ept_mod, blocks):
    # n = 3000: 12 panels of 47 .. 4 stored blocks; windows of several panels
    X, Y = _pair(1400, 1600, 24, seed=3, shift=0.05)
    ref = oracle.permutation_test(X, Y, B=700, seed=5, stat="ed")
    with ept_mod.Context(0) as c:
        c.set_option("stream_blocks", blocks)
        res = c.test(X, Y, B=700, seed=5, stat="ed")
    assert 1 <= res.n_windows <= 12
    if blocks >= 10 ** 9:
        assert res.n_windows == 1
    _check(res, ref["stats"], ref["observed"], 700)


def test_stream_matches_resident(ept_mod):
    # the same test resident and streamed, with the same contraction chunks: the same
    # blocks, partials and scale; the FP64 row sums and partial sums are added in
    # another order (which can move the FP32 rounding of a centring constant), so
    # the statistics agree to far below the parity tolerance, not bitwise.  The
    # resident run's FP64 recomputation of flagged statistics is off here (the
    # streaming mode has none), so that the two compute the same thing.
    X, Y = _pair(9000, 11000, 50, seed=8, shift=0.02)
    with ept_mod.Context(0) as c:
        c.set_option("autotune", 0)
        c.set_option("refine", 0)
        c.set_option("stream_blocks", -1)
        a = c.test(X, Y, B=2000, seed=3, stat="mmd", sigma=9.0)
        c.set_option("stream_blocks", 3000)
        b = c.test(X, Y, B=2000, seed=3, stat="mmd", sigma=9.0)
    assert a.n_windows == 0 and b.n_windows > 1
    sa, sb = np.asarray(a.stats), np.asarray(b.stats)
    assert np.max(np.abs(sa - sb) / np.abs(sa)) <= REL_TOL / 5
    assert abs(a.observed - b.observed) <= REL_TOL / 5 * abs(a.observed)
    assert a.n_ge == b.n_ge


def test_stream_masks_and_range(ctx):
    X, Y = _pair(4, 4, 3, seed=21, shift=0.6)
    sel, ref_stats = oracle.exhaustive(X, Y, "ed", 1.0)
    res = ctx.test_masks(X, Y, oracle.pack_masks(sel), stat="ed")
    assert res.n_windows == 1
    assert np.max(np.abs(np.asarray(res.stats) - ref_stats) / np.abs(ref_stats)) <= REL_TOL
    X, Y = _pair(300, 500, 12, seed=4)
    ref = oracle.permutation_test(X, Y, B=400, seed=9, stat="ed")
    r = ctx.test_range(X, Y, b_first=101, count=200, seed=9, stat="ed")
    assert r.n_windows == 4
    got = np.asarray(r.stats)
    assert np.max(np.abs(got - ref["stats"][100:300]) / np.abs(ref["stats"][100:300])) <= REL_TOL


def test_stream_device_inputs(ctx):
    torch = pytest.importorskip("torch")
    X, Y = _pair(500, 450, 30, seed=6)
    ref = oracle.permutation_test(X, Y, B=333, seed=2, stat="mmd", sigma=6.0)
    res = ctx.test(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), B=333, seed=2, stat="mmd", sigma=6.0)
    assert res.n_windows == 4
    assert res.stats.is_cuda
    res.stats = res.stats.cpu().numpy()
    _check(res, ref["stats"], ref["observed"], 333)


def test_stream_automatic_under_budget(ept_mod):
    # a context budget below the resident scratch: the test streams by itself
    X, Y = _pair(6000, 6000, 16, seed=10, shift=0.03)
    need = ept_mod.estimate_bytes(6000, 6000, 16, 500)
    ref = oracle.permutation_test(X, Y, B=500, seed=1, stat="ed")
    with ept_mod.Context(0, budget_bytes=need // 3) as c:
        res = c.test(X, Y, B=500, seed=1, stat="ed")
    assert res.n_windows > 1
    _check(res, ref["stats"], ref["observed"], 500)


def test_stream_unsupported(ctx, ept_mod):
    X, Y = _pair(50, 60, 5)
    with pytest.raises(ept_mod.EptError) as e:
        ctx.test(X, Y, B=10, prec="plain_fp32")
    assert e.value.status == 8   # EPT_EUNSUPPORTED
    with pytest.raises(ept_mod.EptError) as e:
        ctx.test(X, Y, B=10, stat="mmd", sigma="median")
    assert e.value.status == 8   # EPT_EUNSUPPORTED
    # the context keeps working
    ref = oracle.permutation_test(X, Y, B=10, seed=0, stat="ed")
    _check(ctx.test(X, Y, B=10), ref["stats"], ref["observed"], 10)


def test_stream_stall_hook(ept_mod):
    # the failure path in the streaming mode: the first window's contraction waits
    # out its limit, the call returns EPT_ETIMEOUT and the next call is correct
    X, Y = _pair(400, 300, 9, seed=2)
    with ept_mod.Context(0) as c:
        c.set_option("stream_blocks", 1)
        c.set_option("fault_inject_stall", 1)
        with pytest.raises(ept_mod.EptError) as e:
            c.test(X, Y, B=100, seed=4)
        assert e.value.status == 5   # EPT_ETIMEOUT
        ref = oracle.permutation_test(X, Y, B=100, seed=4, stat="ed")
        _check(c.test(X, Y, B=100, seed=4), ref["stats"], ref["observed"], 100)


def test_stream_large_n_sampled(ept_mod):
    # n = 60000 in windows of at most 8000 blocks (about 0.5 GB): sampled draws against
    # the oracle, the closed-form permutation mean, and the resident run
    spec = workloads.TwoSampleSpec(nx=30000, ny=30000, p=8, y_mean=0.02, B=400, seed=6, data_seed=12)
    X, Y = workloads.gaussian_pair(spec)
    with ept_mod.Context(0) as c:
        c.set_option("stream_blocks", 8000)
        res = c.test(X, Y, B=spec.B, seed=spec.seed)
        c.set_option("stream_blocks", -1)
        resident = c.test(X, Y, B=spec.B, seed=spec.seed)
    assert res.n_windows > 4
    st = np.asarray(res.stats)
    assert np.max(np.abs(st - np.asarray(resident.stats)) / np.abs(st)) <= REL_TOL
    obs = oracle.stat_select(X, Y, oracle.perm_select(spec.seed, spec.nx, spec.ny, 0, 1)[0], "ed", 1.0)
    assert abs(res.observed - obs) <= REL_TOL * abs(obs)
    for b in (1, 400):
        v = oracle.stat_select(X, Y, oracle.perm_select(spec.seed, spec.nx, spec.ny, b, 1)[0], "ed", 1.0)
        assert abs(st[b - 1] - v) <= REL_TOL * abs(v), (b, st[b - 1], v)
    S, tr = oracle.pooled_moments(X, Y, "ed", 1.0)
    mean_ref = oracle.permutation_mean(S, tr, spec.nx, spec.ny, "ed")
    assert abs(st.mean() - mean_ref) <= 5 * st.std() / np.sqrt(spec.B)


def test_stream_zero_permutations(ctx):
    X, Y = _pair(300, 200, 6, seed=14)
    res = ctx.test(X, Y, B=0, seed=0)
    assert res.p_value == 1.0 and res.n_ge == 0 and res.n_windows == 2
    ref = oracle.stat_direct(X, Y, "ed")
    assert abs(res.observed - ref) <= REL_TOL * ref
