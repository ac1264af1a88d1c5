"""Pins for the FP64 CPU oracle: each test checks the oracle against something other
than itself -- values printed in the paper, published known answers, closed forms,
library routines, invariances and brute force on tiny inputs."""
import json
import math
import os
from itertools import combinations

import numpy as np
import pytest
from scipy.spatial.distance import cdist
from scipy.stats import chisquare

import oracle
from paper_2406_06488_gb300 import workloads

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _rand_pair(nx, ny, p, seed, shift=0.0):
    spec = workloads.TwoSampleSpec(nx=nx, ny=ny, p=p, y_mean=shift, data_seed=seed)
    return workloads.gaussian_pair(spec)


# --------------------------------------------------------------------------- Philox
def test_philox_known_answers():
    kat = _load("philox4x32_10_kat.json")
    for v in kat["vectors"]:
        ctr = [int(h, 16) for h in v["counter"]]
        key = [int(h, 16) for h in v["key"]]
        want = [int(h, 16) for h in v["out"]]
        got = oracle.philox4x32_10(ctr, key)
        assert [int(g) for g in got] == want


# --------------------------------------------------------------- permutation stream
def test_stream_draw0_is_identity():
    for nx, ny in [(1, 1), (5, 4), (100, 37)]:
        s = oracle.perm_select(123, nx, ny, 0, 1)[0]
        assert s[:nx].all() and not s[nx:].any()


@pytest.mark.parametrize("nx,ny", [(1, 1), (1, 9), (9, 1), (4, 4), (37, 64), (300, 5)])
def test_stream_exact_count(nx, ny):
    sel = oracle.perm_select(7, nx, ny, 1, 500)
    assert (sel.sum(axis=1) == nx).all()


def test_stream_uniform_over_subsets():
    # nx = 2, ny = 3: every one of the C(5, 2) = 10 subsets has probability 1/10.
    nx, ny, draws = 2, 3, 40000
    sel = oracle.perm_select(2024, nx, ny, 1, draws)
    idx = {c: k for k, c in enumerate(combinations(range(5), 2))}
    counts = np.zeros(len(idx))
    for row in sel:
        counts[idx[tuple(np.flatnonzero(row))]] += 1
    assert chisquare(counts).pvalue > 1e-4


def test_stream_inclusion_and_pair_frequency():
    # E[s_i] = nx/n and E[s_i s_j] = nx(nx-1)/(n(n-1)) for a uniform nx-subset.
    nx, ny, draws = 13, 19, 20000
    n = nx + ny
    sel = oracle.perm_select(99, nx, ny, 1, draws).astype(np.float64)
    p1 = nx / n
    se1 = math.sqrt(p1 * (1 - p1) / draws)
    assert np.abs(sel.mean(axis=0) - p1).max() < 5 * se1
    p2 = nx * (nx - 1) / (n * (n - 1))
    pair = (sel.T @ sel) / draws
    off = pair[~np.eye(n, dtype=bool)]
    se2 = math.sqrt(p2 * (1 - p2) / draws)
    assert np.abs(off - p2).max() < 6 * se2


def test_stream_depends_on_seed_and_draw():
    a = oracle.perm_select(1, 50, 50, 1, 3)
    b = oracle.perm_select(2, 50, 50, 1, 3)
    assert not (a == b).all()
    assert not (a[0] == a[1]).all()
    # counter-based: draw b does not depend on where the batch starts
    c = oracle.perm_select(1, 50, 50, 2, 2)
    assert (c == a[1:]).all()


# ---------------------------------------------------------- Algorithm 2 / swapping
def test_alg2_worked_example():
    g = _load("alg2_worked_example.json")
    got = oracle.alg2_indices(g["nx"], g["ny"], g["idx_p1"])
    for key in ["i1", "i2", "i1s", "i2s", "j1", "j2", "j1s", "j2s"]:
        assert got[key] == g[key], key


def _rows(names, X, Y):
    out = []
    for nm in names:
        src = X if nm[0] == "x" else Y
        out.append(src[int(nm[1:]) - 1])
    return np.stack(out)


@pytest.mark.parametrize("stat", ["ed", "mmd"])
def test_block_swap_equals_recomputation_on_worked_example(stat):
    # Section 4.1: the statistic assembled from the three blocks (Algorithm 1) for the
    # relabeling of the toy example equals the statistic recomputed on
    # x* = (y2, x4, x5, y1, x2), y* = (x1, x3, y3, y4).
    g = _load("alg2_worked_example.json")
    X, Y = _rand_pair(5, 4, 3, seed=11)
    sel = np.zeros((1, 9), dtype=bool)
    sel[0, np.asarray(g["idx_p1"]) - 1] = True
    via_blocks = oracle.test_blocks(X, Y, sel, stat, 1.7)[0]
    xs = _rows(g["x_star"], X, Y).astype(np.float64)
    ys = _rows(g["y_star"], X, Y).astype(np.float64)
    direct = oracle.stat_direct(xs, ys, stat, 1.7)
    assert abs(via_blocks - direct) <= 1e-13 * max(1.0, abs(direct))


@pytest.mark.parametrize("stat", ["ed", "mmd"])
@pytest.mark.parametrize("nx,ny,p", [(7, 11, 3), (40, 25, 6), (120, 180, 2), (1, 5, 4), (5, 1, 4)])
def test_three_implementations_agree(stat, nx, ny, p):
    # Algorithm 4 (recompute), Algorithm 5 (pooled matrix) and Algorithm 1
    # (block swapping) give the same statistics on the same relabelings.
    X, Y = _rand_pair(nx, ny, p, seed=nx * 1000 + ny, shift=0.3)
    sel = oracle.perm_select(5, nx, ny, 0, 40)
    a = oracle.test_direct(X, Y, sel, stat, 2.0)
    b = oracle.test_pooled(X, Y, sel, stat, 2.0)
    c = oracle.test_blocks(X, Y, sel, stat, 2.0)
    scale = np.abs(a).max() + 1e-300
    assert np.abs(a - b).max() <= 1e-12 * scale
    assert np.abs(a - c).max() <= 1e-12 * scale


# ------------------------------------------------------------------ statistic pins
def test_distances_match_library_routine():
    X, Y = _rand_pair(30, 20, 7, seed=3)
    ref = cdist(X.astype(np.float64), Y.astype(np.float64))
    assert np.allclose(oracle.block_matrix(X, Y, "ed"), ref, rtol=1e-13, atol=0)
    sig = 2.5
    kref = np.exp(-ref ** 2 / (2 * sig * sig))
    assert np.allclose(oracle.block_matrix(X, Y, "mmd", sig), kref, rtol=1e-12, atol=0)


def _ed_1d_closed_form(x, y):
    # For scalars, sum_{k,l} |z_k - z_l| = 2 * sum_k (2k - m - 1) z_(k) over the sorted
    # sample z_(1) <= ... <= z_(m); the cross sum follows from the pooled sum.
    def all_pairs(z):
        z = np.sort(z)
        m = z.size
        k = np.arange(1, m + 1, dtype=np.float64)
        return 2.0 * np.sum((2 * k - m - 1) * z)
    sxx, syy = all_pairs(x), all_pairs(y)
    sww = all_pairs(np.concatenate([x, y]))
    sxy = 0.5 * (sww - sxx - syy)
    nx, ny = x.size, y.size
    return 2 * sxy / (nx * ny) - sxx / nx ** 2 - syy / ny ** 2


@pytest.mark.parametrize("nx,ny", [(300, 200), (1, 50), (64, 64)])
def test_ed_p1_closed_form(nx, ny):
    X, Y = _rand_pair(nx, ny, 1, seed=nx + 7 * ny, shift=0.4)
    want = _ed_1d_closed_form(X[:, 0].astype(np.float64), Y[:, 0].astype(np.float64))
    got = oracle.stat_direct(X, Y, "ed")
    assert abs(got - want) <= 1e-11 * abs(want)


def test_ed_and_mmd_nonnegative_and_symmetric():
    for seed in range(5):
        X, Y = _rand_pair(17 + seed, 9 + 3 * seed, 4, seed=seed, shift=0.1 * seed)
        ed = oracle.stat_direct(X, Y, "ed")
        mmd = oracle.stat_direct(X, Y, "mmd", 1.3)
        assert ed >= 0 and mmd >= 0
        assert abs(ed - oracle.stat_direct(Y, X, "ed")) <= 1e-13 * ed
        assert abs(mmd - oracle.stat_direct(Y, X, "mmd", 1.3)) <= 1e-12 * mmd


def test_invariances():
    X, Y = _rand_pair(25, 31, 5, seed=8, shift=0.5)
    X64, Y64 = X.astype(np.float64), Y.astype(np.float64)
    ed = oracle.stat_direct(X64, Y64, "ed")
    mmd = oracle.stat_direct(X64, Y64, "mmd", 2.0)
    c = np.arange(5, dtype=np.float64) - 2.0
    assert abs(oracle.stat_direct(X64 + c, Y64 + c, "ed") - ed) <= 1e-11 * ed
    q, _ = np.linalg.qr(np.random.default_rng(1).standard_normal((5, 5)))
    assert abs(oracle.stat_direct(X64 @ q, Y64 @ q, "ed") - ed) <= 1e-11 * ed
    assert abs(oracle.stat_direct(X64 @ q, Y64 @ q, "mmd", 2.0) - mmd) <= 1e-11 * mmd
    assert abs(oracle.stat_direct(3 * X64, 3 * Y64, "ed") - 3 * ed) <= 1e-12 * ed
    assert abs(oracle.stat_direct(3 * X64, 3 * Y64, "mmd", 6.0) - mmd) <= 1e-12 * mmd


def test_identical_samples_give_zero():
    X, _ = _rand_pair(30, 30, 4, seed=4)
    D = cdist(X.astype(np.float64), X.astype(np.float64))
    assert abs(oracle.stat_direct(X, X, "ed")) <= 1e-13 * D.mean()
    assert abs(oracle.stat_direct(X, X, "mmd", 1.0)) <= 1e-13


def test_pvalue_definition():
    # Section 3.1: (1 + #{stat* >= stat_o}) / (1 + b)
    p, nge = oracle.pvalue([1.0, 2.0, 3.0, 0.5], 2.0)
    assert nge == 2 and p == pytest.approx(3.0 / 5.0, abs=0)
    p, nge = oracle.pvalue([], 1.0)
    assert nge == 0 and p == 1.0


def test_identity_draw_reproduces_observed():
    X, Y = _rand_pair(20, 30, 5, seed=6, shift=0.2)
    res = oracle.permutation_test(X, Y, B=10, seed=3, stat="ed")
    assert res["observed"] == oracle.stat_direct(X, Y, "ed")


# ------------------------------------------------------------- exhaustive checks
@pytest.mark.parametrize("stat", ["ed", "mmd"])
@pytest.mark.parametrize("shift", [0.0, 0.8])
def test_exhaustive_70(stat, shift):
    X, Y = _rand_pair(4, 4, 3, seed=21, shift=shift)
    sel, stats = oracle.exhaustive(X, Y, stat, 1.5)
    assert sel.shape == (70, 8) and (sel.sum(axis=1) == 4).all()
    # all 70 distinct, lexicographic, first one the identity
    assert len({tuple(r) for r in sel}) == 70
    assert sel[0, :4].all()
    # each value equals direct recomputation
    direct = oracle.test_direct(X, Y, sel, stat, 1.5)
    assert np.abs(direct - stats).max() <= 1e-13 * np.abs(stats).max()
    # complements are bitwise equal (canonical evaluation, nx == ny)
    key = {tuple(r): s for r, s in zip(sel, stats)}
    for r, s in zip(sel, stats):
        assert key[tuple(~r)] == s
    observed = stats[0]
    p_exact = np.count_nonzero(stats >= observed) / 70.0
    assert p_exact >= 2 / 70  # identity and its complement
    # The Monte-Carlo estimator on draws of the stream approaches p_exact.
    B = 100000
    draws = oracle.perm_select(77, 4, 4, 1, B)
    mc = np.fromiter((key[tuple(r)] for r in draws), dtype=np.float64, count=B)
    p_mc = (1 + np.count_nonzero(mc >= observed)) / (B + 1)
    se = math.sqrt(p_exact * (1 - p_exact) / B) + 1e-12
    assert abs(p_mc - p_exact) <= 4 * se + 2.0 / B


def _brute_stat(Z, sel, stat, sigma):
    """Eq. 1 / Eq. 2 of one relabeling by scipy's distances (independent of the oracle)."""
    xs, ys = Z[sel].astype(np.float64), Z[~sel].astype(np.float64)

    def blk(a, b):
        d = cdist(a, b)
        if stat == "ed":
            return d
        if stat == "mmd":
            return np.exp(-d ** 2 / (2 * sigma * sigma))
        return np.exp(-d / sigma)
    nx, ny = len(xs), len(ys)
    ed = 2 * blk(xs, ys).sum() / (nx * ny) - blk(xs, xs).sum() / nx ** 2 - blk(ys, ys).sum() / ny ** 2
    return ed if stat == "ed" else -ed


@pytest.mark.parametrize("stat", ["ed", "mmd", "mmd_laplace"])
@pytest.mark.parametrize("nx,ny,p", [(1, 1, 1), (1, 9, 1), (9, 1, 3), (7, 11, 1), (33, 20, 5), (3, 64, 2)])
def test_stat_select_matches_recomputation(stat, nx, ny, p):
    # the threaded single-relabeling statistic (the checker of every full-size sampled
    # test) against scipy's distances and against the pinned Algorithm 4 routine
    X, Y = _rand_pair(nx, ny, p, seed=31 * nx + ny, shift=0.4)
    Z = np.vstack([X, Y])
    sel = oracle.perm_select(17, nx, ny, 0, 6)
    direct = oracle.test_direct(X, Y, sel, stat, 1.3)
    for k, s in enumerate(sel):
        got = oracle.stat_select(X, Y, s, stat, 1.3)
        want = _brute_stat(Z, s, stat, 1.3)
        tol = 1e-13 * max(abs(want), 1e-300) + 1e-15
        assert abs(got - want) <= max(tol, 1e-12 * abs(want)), (k, got, want)
        assert abs(got - direct[k]) <= 1e-13 * max(abs(direct[k]), 1e-300) + 1e-16, (k, got, direct[k])


@pytest.mark.parametrize("stat", ["ed", "mmd", "mmd_laplace"])
def test_pooled_moments_match_library_routine(stat):
    X, Y = _rand_pair(23, 31, 4, seed=41, shift=0.3)
    Z = np.vstack([X, Y]).astype(np.float64)
    D = cdist(Z, Z)
    W = D if stat == "ed" else (np.exp(-D ** 2 / (2 * 1.7 ** 2)) if stat == "mmd" else np.exp(-D / 1.7))
    S, tr = oracle.pooled_moments(X, Y, stat, 1.7)
    assert abs(S - W.sum()) <= 1e-13 * abs(W.sum())
    assert abs(tr - np.trace(W)) <= 1e-13 * max(1.0, abs(np.trace(W)))
    # distances vanish on the diagonal, kernels are 1 there
    assert tr == (0.0 if stat == "ed" else float(len(Z)))


@pytest.mark.parametrize("stat", ["ed", "mmd"])
def test_permutation_mean_equals_exhaustive_mean(stat):
    # the closed form E[stat*] over a uniform nx-subset equals the plain average over
    # all C(n, nx) subsets (brute force, exact up to rounding)
    nx, ny, p = 5, 7, 3
    X, Y = _rand_pair(nx, ny, p, seed=43, shift=0.5)
    Z = np.vstack([X, Y])
    vals = []
    for c in combinations(range(nx + ny), nx):
        s = np.zeros(nx + ny, dtype=bool)
        s[list(c)] = True
        vals.append(_brute_stat(Z, s, stat, 1.9))
    want = float(np.mean(vals))
    S, tr = oracle.pooled_moments(X, Y, stat, 1.9)
    got = oracle.permutation_mean(S, tr, nx, ny, stat)
    assert abs(got - want) <= 1e-12 * abs(want)


@pytest.mark.parametrize("stat", ["ed", "mmd"])
def test_permutation_mean_matches_the_stream(stat):
    # at a size beyond enumeration: the sample mean of B draws of the stream (the
    # statistics by Algorithm 1) lies within a CLT bound of the closed form
    nx, ny, p = 30, 45, 6
    X, Y = _rand_pair(nx, ny, p, seed=13, shift=0.3)
    S, tr = oracle.pooled_moments(X, Y, stat, 2.2)
    want = oracle.permutation_mean(S, tr, nx, ny, stat)
    B = 4000
    st = oracle.permutation_test(X, Y, B=B, seed=9, stat=stat, sigma=2.2, method="blocks")["stats"]
    assert abs(st.mean() - want) <= 5 * st.std() / math.sqrt(B)


@pytest.mark.parametrize("nx,ny", [(4, 4), (3, 5), (5, 2), (1, 4), (4, 1), (2, 2)])
def test_exhaustive_order_is_lexicographic(nx, ny):
    X, Y = _rand_pair(nx, ny, 2, seed=nx * 10 + ny)
    sel, stats = oracle.exhaustive(X, Y, "ed")
    got = [tuple(int(t) for t in np.flatnonzero(r)) for r in sel]
    assert got == list(combinations(range(nx + ny), nx))
    assert stats.shape == (len(got),)


# ------------------------------------------- Laplacian kernel and median bandwidth
def test_laplace_kernel_matches_library_routine():
    # exp(-||x - y|| / sigma) against scipy's distances
    X, Y = _rand_pair(30, 20, 7, seed=13)
    ref = cdist(X.astype(np.float64), Y.astype(np.float64))
    sig = 1.7
    assert np.allclose(oracle.block_matrix(X, Y, "mmd_laplace", sig), np.exp(-ref / sig), rtol=1e-12, atol=0)


@pytest.mark.parametrize("nx,ny,p", [(7, 11, 3), (40, 25, 6), (1, 5, 4)])
def test_laplace_three_implementations_agree(nx, ny, p):
    X, Y = _rand_pair(nx, ny, p, seed=nx * 100 + ny, shift=0.3)
    sel = oracle.perm_select(9, nx, ny, 0, 30)
    a = oracle.test_direct(X, Y, sel, "mmd_laplace", 1.5)
    b = oracle.test_pooled(X, Y, sel, "mmd_laplace", 1.5)
    c = oracle.test_blocks(X, Y, sel, "mmd_laplace", 1.5)
    scale = np.abs(a).max() + 1e-300
    assert np.abs(a - b).max() <= 1e-12 * scale and np.abs(a - c).max() <= 1e-12 * scale


def test_laplace_mmd_properties():
    # the Laplacian kernel is positive definite: MMD^2 >= 0, symmetric, zero for
    # identical samples; invariant to translations and rotations; (cX, cY, c sigma)
    # gives the same value
    X, Y = _rand_pair(25, 31, 5, seed=18, shift=0.5)
    X64, Y64 = X.astype(np.float64), Y.astype(np.float64)
    m = oracle.stat_direct(X64, Y64, "mmd_laplace", 2.0)
    assert m > 0
    assert abs(oracle.stat_direct(Y64, X64, "mmd_laplace", 2.0) - m) <= 1e-12 * m
    assert abs(oracle.stat_direct(X64, X64, "mmd_laplace", 2.0)) <= 1e-13
    q, _ = np.linalg.qr(np.random.default_rng(2).standard_normal((5, 5)))
    assert abs(oracle.stat_direct(X64 @ q + 1.0, Y64 @ q + 1.0, "mmd_laplace", 2.0) - m) <= 1e-11 * m
    assert abs(oracle.stat_direct(3 * X64, 3 * Y64, "mmd_laplace", 6.0) - m) <= 1e-12 * m


def test_median_pairs_hand_examples():
    # pooled points 0, 1, 3, 7 on a line: distances 1, 3, 7, 2, 6, 4 -> sorted
    # 1 2 3 4 6 7, lower median 3; points 0, 1, 3: distances 1, 3, 2 -> median 2
    assert oracle.median_pairs(np.array([[0.0], [1.0]]), np.array([[3.0], [7.0]])) == 3.0
    assert oracle.median_pairs(np.array([[0.0], [1.0]]), np.array([[3.0]])) == 2.0


def test_median_pairs_matches_library_routine_and_ignores_the_split():
    from scipy.spatial.distance import pdist
    X, Y = _rand_pair(23, 18, 4, seed=21, shift=0.4)
    d = np.sort(pdist(np.concatenate([X, Y]).astype(np.float64)))
    want = d[(d.size - 1) // 2]
    assert abs(oracle.median_pairs(X, Y) - want) <= 1e-14 * want
    W = np.concatenate([X, Y])
    perm = np.random.default_rng(3).permutation(W.shape[0])
    W = W[perm]
    assert oracle.median_pairs(W[:10], W[10:]) == oracle.median_pairs(X, Y)
    assert oracle.median_pairs(Y, X) == oracle.median_pairs(X, Y)


def test_mask_packing_bit_order():
    # pooled row t is bit t % 32 of word t // 32 (the layout the library's relabeling
    # words use); unpacking inverts it, padding bits stay zero
    n = 70
    for t in (0, 1, 31, 32, 33, 63, 64, 69):
        sel = np.zeros((1, n), dtype=bool)
        sel[0, t] = True
        words = oracle.pack_masks(sel)
        assert words.shape == (1, 3) and words.dtype == np.uint32
        want = np.zeros(3, dtype=np.uint32)
        want[t // 32] = np.uint32(1) << np.uint32(t % 32)
        assert np.array_equal(words[0], want), t
    rng = np.random.default_rng(5)
    sel = rng.random((9, n)) < 0.4
    words = oracle.pack_masks(sel)
    assert np.array_equal(oracle.unpack_masks(words, n), sel)
    assert not (words[:, 2] >> np.uint32(n - 64)).any()   # rows 70..95 do not exist
