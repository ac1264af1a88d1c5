"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on the
same seeded inputs.

Tolerances: relative error <= 1e-5 on every statistic; relabeling masks bit-exact;
the count #{stat* >= observed} equal except through near-ties (permutations whose
oracle statistic lies within 1e-5 |observed| of the observed one)."""
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


def _pair(nx, ny, p, seed=0, shift=0.2, var=1.0, coords=-1):
    return workloads.gaussian_pair(workloads.TwoSampleSpec(nx=nx, ny=ny, p=p, y_mean=shift, y_var=var,
                                                           y_mean_coords=coords, data_seed=seed))


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


# ------------------------------------------------------------ permutation stream
@pytest.mark.parametrize("nx,ny,seed,b0,count", [
    (1, 1, 0, 0, 5), (4, 4, 0, 0, 70), (5, 4, 3, 1, 100), (37, 64, 7, 1, 300), (100, 100, 0, 0, 1001),
    (3, 300, 1, 0, 64), (255, 1, 9, 1000, 50), (2000, 3000, 0, 0, 200), (10000, 10000, 0, 9990, 11)])
def test_masks_bit_exact(ctx, nx, ny, seed, b0, count):
    gpu = ctx.perm_masks(seed, nx, ny, b0, count)
    ref = oracle.pack_masks(oracle.perm_select(seed, nx, ny, b0, count))
    assert gpu.shape == ref.shape
    assert np.array_equal(gpu, ref)


# ------------------------------------------------------------------ block build
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("stat", ["ed", "mmd"])
@pytest.mark.parametrize("nx,ny,p", [(1, 1, 1), (5, 4, 3), (100, 100, 10), (37, 300, 17), (129, 130, 64),
                                     (300, 257, 1000), (600, 700, 65)])
def test_blocks_match_oracle(ctx, prec, stat, nx, ny, p):
    # split_bf16 builds the Gram term on the tensor cores (hi/lo split), plain_fp32 with FP32 FMA
    X, Y = _pair(nx, ny, p, seed=nx + ny + p)
    sigma = float(np.sqrt(p))
    D = ctx.build_blocks(X, Y, stat, sigma, prec=prec)
    Z = np.vstack([X, Y])
    ref = oracle.block_matrix(Z, Z, stat, sigma)
    diag = np.diag(D)
    assert np.all(diag == (0.0 if stat == "ed" else 1.0))
    err = np.abs(D.astype(np.float64) - ref)
    scale = ref.mean() if stat == "ed" else 1.0
    assert err.max() <= 2e-6 * scale + 2e-6 * np.abs(ref).max(), err.max()
    assert np.abs(D - D.T).max() <= 2e-6 * max(scale, 1e-30) + 2e-6 * np.abs(ref).max()


# --------------------------------------------------------------- whole test
@pytest.mark.parametrize("prec", PRECS)
def test_small_config_ed(ctx, prec):
    # ED, nx = ny = 100, p = 10, Y mean 0.2, B = 1000, seed 0
    spec = workloads.SMALL
    X, Y = workloads.gaussian_pair(spec)
    ref = oracle.permutation_test(X, Y, B=spec.B, seed=spec.seed, stat="ed")
    res = ctx.test(X, Y, B=spec.B, seed=spec.seed, stat="ed", prec=prec)
    _check(res, ref["stats"], ref["observed"], spec.B)


@pytest.mark.parametrize("prec", PRECS)
def test_small_mmd(ctx, prec):
    X, Y = _pair(80, 120, 7, seed=4, shift=0.0, var=1.3)
    ref = oracle.permutation_test(X, Y, B=500, seed=11, stat="mmd", sigma=2.5)
    res = ctx.test(X, Y, B=500, seed=11, stat="mmd", sigma=2.5, prec=prec)
    _check(res, ref["stats"], ref["observed"], 500)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("nx,ny,p,B,stat", [
    (1, 1, 1, 10, "ed"), (1, 7, 3, 50, "mmd"), (9, 1, 4, 50, "ed"), (255, 2, 5, 300, "mmd"),
    (256, 256, 3, 257, "ed"), (257, 300, 20, 1023, "mmd"), (3, 600, 2, 129, "ed"), (700, 650, 33, 700, "ed")])
def test_ragged_shapes(ctx, prec, nx, ny, p, B, stat):
    X, Y = _pair(nx, ny, p, seed=nx * 7 + ny, shift=0.1)
    sigma = 1.7
    ref = oracle.permutation_test(X, Y, B=B, seed=nx + 3, stat=stat, sigma=sigma)
    res = ctx.test(X, Y, B=B, seed=nx + 3, stat=stat, sigma=sigma, prec=prec)
    _check(res, ref["stats"], ref["observed"], B)


@pytest.mark.parametrize("prec", PRECS)
def test_zero_permutations(ctx, prec):
    X, Y = _pair(20, 30, 4)
    res = ctx.test(X, Y, B=0, seed=0, prec=prec)
    assert res.p_value == 1.0 and res.n_ge == 0
    ref = oracle.stat_direct(X, Y, "ed")
    assert abs(res.observed - ref) <= REL_TOL * ref


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("stat", ["ed", "mmd"])
@pytest.mark.parametrize("shift", [0.0, 0.8])
def test_exhaustive_70(ctx, prec, stat, shift):
    X, Y = _pair(4, 4, 3, seed=21, shift=shift)
    sel, ref_stats = oracle.exhaustive(X, Y, stat, 1.5)
    masks = oracle.pack_masks(sel)
    res = ctx.test_masks(X, Y, masks, stat=stat, sigma=1.5, prec=prec)
    got = np.asarray(res.stats)
    rel = np.abs(got - ref_stats) / np.abs(ref_stats)
    assert rel.max() <= REL_TOL
    obs = ref_stats[0]
    p_exact = np.count_nonzero(ref_stats >= obs) / 70.0
    near = np.abs(ref_stats - obs) <= 1e-5 * abs(obs)
    assert abs(res.n_ge / 70.0 - p_exact) <= near.sum() / 70.0


def test_identity_column_ties_observed_bitwise(ctx):
    X, Y = _pair(50, 60, 5, seed=2)
    ident = oracle.pack_masks(oracle.perm_select(0, 50, 60, 0, 1))
    for prec in PRECS:
        res = ctx.test_masks(X, Y, np.repeat(ident, 3, axis=0), prec=prec)
        assert np.all(np.asarray(res.stats) == res.observed)
        assert res.n_ge == 3


def test_bad_masks_rejected(ctx):
    from paper_2406_06488_gb300 import ept
    X, Y = _pair(10, 12, 3)
    sel = oracle.perm_select(1, 10, 12, 1, 4)
    m = oracle.pack_masks(sel)
    m[2, 0] ^= 1 << (int(np.flatnonzero(~sel[2])[0]))  # one member too many
    with pytest.raises(ept.EptError) as e:
        ctx.test_masks(X, Y, m)
    assert e.value.status == 1
    m = oracle.pack_masks(sel)
    m[1, 0] |= 1 << 30  # bit beyond n = 22
    with pytest.raises(ept.EptError):
        ctx.test_masks(X, Y, m)


def test_nonfinite_and_bad_args_rejected(ctx):
    from paper_2406_06488_gb300 import ept
    X, Y = _pair(10, 12, 3)
    Xb = X.copy()
    Xb[3, 1] = np.nan
    with pytest.raises(ept.EptError):
        ctx.test(Xb, Y, B=10)
    with pytest.raises(ept.EptError):
        ctx.test(X, Y, B=10, stat="mmd", sigma=0.0)
    with pytest.raises(ept.EptError):
        ctx.test(X[:0], Y, B=10)
    # the context still works after rejected calls
    res = ctx.test(X, Y, B=10)
    assert np.isfinite(res.observed)


@pytest.mark.parametrize("prec", PRECS)
def test_near_duplicates_recomputed(ctx, prec):
    X, Y = _pair(60, 70, 50, seed=8, shift=0.0)
    rng = np.random.default_rng(0)
    X[10] = X[3] + 1e-4 * rng.standard_normal(50).astype(np.float32)
    Y[5] = X[7] + 1e-4 * rng.standard_normal(50).astype(np.float32)
    Y[6] = Y[9]
    ref = oracle.permutation_test(X, Y, B=300, seed=3, stat="ed")
    res = ctx.test(X, Y, B=300, seed=3, prec=prec)
    assert res.n_fixup >= 3
    _check(res, ref["stats"], ref["observed"], 300)


def test_device_inputs_match_host_inputs(ctx):
    import torch
    X, Y = _pair(300, 200, 16, seed=5)
    for prec in PRECS:
        a = ctx.test(X, Y, B=400, seed=2, prec=prec)
        b = ctx.test(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), B=400, seed=2, prec=prec)
        torch.cuda.synchronize()
        assert a.observed == b.observed and a.n_ge == b.n_ge
        assert np.array_equal(np.asarray(a.stats), b.stats.cpu().numpy())


def test_deterministic(ctx):
    X, Y = _pair(500, 400, 30, seed=6)
    for prec in PRECS:
        a = ctx.test(X, Y, B=600, seed=4, prec=prec)
        b = ctx.test(X, Y, B=600, seed=4, prec=prec)
        assert np.array_equal(np.asarray(a.stats), np.asarray(b.stats)) and a.observed == b.observed


# ------------------------------------------------ full-size configurations, sampled
def _full_size_check(ctx, spec, sample_draws):
    X, Y = workloads.gaussian_pair(spec)
    nx, ny = spec.nx, spec.ny
    S, tr = oracle.pooled_moments(X, Y, spec.stat, spec.sigma)
    mean_ref = oracle.permutation_mean(S, tr, nx, ny, spec.stat)
    obs_ref = oracle.stat_select(X, Y, oracle.perm_select(spec.seed, nx, ny, 0, 1)[0], spec.stat, spec.sigma)
    sampled = {}
    for b in sample_draws:
        sel = oracle.perm_select(spec.seed, nx, ny, b, 1)[0]
        sampled[b] = oracle.stat_select(X, Y, sel, spec.stat, spec.sigma)
    for prec in PRECS:
        res = ctx.test(X, Y, B=spec.B, seed=spec.seed, stat=spec.stat, sigma=spec.sigma, prec=prec)
        st = np.asarray(res.stats)
        worst = abs(res.observed - obs_ref) / abs(obs_ref)
        for b, v in sampled.items():
            worst = max(worst, abs(st[b - 1] - v) / abs(v))
        print("%s %s: largest relative error over the observed and %d sampled statistics %.3g"
              % (spec.stat, prec, len(sampled), worst))
        assert abs(res.observed - obs_ref) <= REL_TOL * abs(obs_ref), (prec, res.observed, obs_ref)
        for b, v in sampled.items():
            assert abs(st[b - 1] - v) <= REL_TOL * abs(v), (prec, b, st[b - 1], v)
        # property at any size: the mean of the B statistics is the permutation mean
        assert abs(st.mean() - mean_ref) <= 5 * st.std() / np.sqrt(spec.B), (prec, st.mean(), mean_ref)
        assert res.p_value == (1.0 + res.n_ge) / (1.0 + spec.B)


def test_full_size_highdim_ed(ctx):
    # ED, nx = 2000, ny = 3000, p = 1000, Y mean 0.05 on the first 50 coordinates, B = 10000
    _full_size_check(ctx, workloads.HIGHDIM, [1, 2, 4999, 10000])


def test_full_size_highdim_every_statistic(ctx):
    # the same configuration against the oracle's FP64 Algorithm 1 (three blocks built
    # once, each relabeling assembled by the block swaps; pinned against the direct
    # recomputation on the CPU): all 10,000 permuted statistics and the count
    spec = workloads.HIGHDIM
    X, Y = workloads.gaussian_pair(spec)
    ref = oracle.permutation_test(X, Y, B=spec.B, seed=spec.seed, stat="ed", method="blocks")
    for prec in PRECS:
        res = ctx.test(X, Y, B=spec.B, seed=spec.seed, prec=prec)
        _check(res, ref["stats"], ref["observed"], spec.B)


def test_full_size_mmd(ctx):
    # Gaussian MMD, nx = ny = 10000, p = 100, Y ~ N(0, 1.1 I), sigma = 10, B = 10000:
    # the observed statistic and draws 1..64 against the direct recomputation, plus
    # the last draw, on both precisions
    _full_size_check(ctx, workloads.MMD, list(range(1, 65)) + [10000])


@pytest.mark.parametrize("prec", PRECS)
def test_stream_ranges_combine(ctx, prec):
    # a test split into ranges of the counter-based stream (checkpoint / resume, or
    # one range per GPU) gives the same statistics and count as the whole test
    X, Y = _pair(150, 170, 9, seed=31)
    full = ctx.test(X, Y, B=1000, seed=4, prec=prec)
    a = ctx.test_range(X, Y, b_first=1, count=400, seed=4, prec=prec)
    b = ctx.test_range(X, Y, b_first=401, count=600, seed=4, prec=prec)
    got = np.concatenate([np.asarray(a.stats), np.asarray(b.stats)])
    want = np.asarray(full.stats)
    assert np.max(np.abs(got - want) / np.abs(want)) <= 1e-9
    assert a.observed == full.observed == b.observed
    assert abs((a.n_ge + b.n_ge) - full.n_ge) <= full.n_near_tie
    assert a.p_value == (1.0 + a.n_ge) / 401.0
    # and the range really is draws 401..1000 of the oracle's stream
    ref = oracle.permutation_test(X, Y, B=1000, seed=4, stat="ed")
    rel = np.abs(np.asarray(b.stats) - ref["stats"][400:]) / np.abs(ref["stats"][400:])
    assert rel.max() <= REL_TOL


def test_expired_device_wait_returns_timeout_and_context_recovers(ctx):
    # failure path of the tcgen05 contraction, driven without a fault: the MMA issuer
    # waits on a device flag that nothing sets; the bounded wait expires (2 s), the
    # kernel aborts cleanly and the call reports EPT_ETIMEOUT
    from paper_2406_06488_gb300 import ept
    X, Y = _pair(200, 230, 8, seed=41)
    ctx.set_option("fault_inject_stall", 1)
    with pytest.raises(ept.EptError) as e:
        ctx.test(X, Y, B=500, seed=2, prec="split_bf16")
    assert e.value.status == 5
    # one-shot, and the context (tensor memory, streams, graphs) still works
    res = ctx.test(X, Y, B=500, seed=2, prec="split_bf16")
    ref = oracle.permutation_test(X, Y, B=500, seed=2, stat="ed")
    _check(res, ref["stats"], ref["observed"], 500)


def test_wait_limit_option(ctx):
    # the limit of the bounded waits is a context option: with 100 ms the stalled
    # contraction gives up well before the 2 s default; out-of-range limits are refused
    import time
    from paper_2406_06488_gb300 import ept
    X, Y = _pair(150, 170, 6, seed=43)
    with pytest.raises(ept.EptError):
        ctx.set_option("wait_limit_ms", 5)
    try:
        ctx.set_option("wait_limit_ms", 100)
        ctx.test(X, Y, B=200, seed=3)   # a normal run with the short limit
        ctx.set_option("fault_inject_stall", 1)
        t0 = time.perf_counter()
        with pytest.raises(ept.EptError) as e:
            ctx.test(X, Y, B=200, seed=3)
        assert e.value.status == 5
        assert time.perf_counter() - t0 < 1.5
    finally:
        ctx.set_option("wait_limit_ms", 2000)
    ref = oracle.permutation_test(X, Y, B=200, seed=3, stat="ed")
    _check(ctx.test(X, Y, B=200, seed=3), ref["stats"], ref["observed"], 200)


def test_large_n_sampled(ctx):
    # n = 60000 pooled rows (7.2 GB of packed blocks): sampled draws against the
    # oracle's direct recomputation, and the closed-form permutation mean
    spec = workloads.TwoSampleSpec(nx=30000, ny=30000, p=8, y_mean=0.02, B=400, seed=6, data_seed=12)
    X, Y = workloads.gaussian_pair(spec)
    res = ctx.test(X, Y, B=spec.B, seed=spec.seed)
    st = np.asarray(res.stats)
    obs = oracle.stat_select(X, Y, oracle.perm_select(spec.seed, spec.nx, spec.ny, 0, 1)[0], "ed", 1.0)
    assert abs(res.observed - obs) <= REL_TOL * abs(obs)
    for b in (1, 400):
        v = oracle.stat_select(X, Y, oracle.perm_select(spec.seed, spec.nx, spec.ny, b, 1)[0], "ed", 1.0)
        assert abs(st[b - 1] - v) <= REL_TOL * abs(v), (b, st[b - 1], v)
    S, tr = oracle.pooled_moments(X, Y, "ed", 1.0)
    mean_ref = oracle.permutation_mean(S, tr, spec.nx, spec.ny, "ed")
    assert abs(st.mean() - mean_ref) <= 5 * st.std() / np.sqrt(spec.B)
