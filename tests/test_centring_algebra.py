"""CPU check of the centring algebra the CUDA path is built on, in FP64 numpy against
the oracle's direct statistic (Eq. 1 / Eq. 2 recomputed from the permuted rows).

The packed operand is C = W~ - kappa diag(r~), stored as its upper part with the
off-diagonal entries doubled, where W~ = W - u 1' - 1 u' and r~ = W~ 1; then
    stat = sign * (cT s'Cs + S~ / o^2),  S~ = 1'r~,
s marking the smaller group (size m; the other has size o), cT = (n / (nx ny))^2,
kappa = 2m/n, sign -1 for ED and +1 for MMD.  The identity holds for ANY u (the
library rounds its double-centring vector to FP32 and relies on that); these tests
check it for several u and both orders of nx, ny."""
import numpy as np
import pytest

import oracle
from paper_2406_06488_gb300 import workloads


def _pair(nx, ny, p, seed):
    return workloads.gaussian_pair(workloads.TwoSampleSpec(nx=nx, ny=ny, p=p, y_mean=0.3, data_seed=seed))


def _folded_stat(W, s, nx, ny, sign, u):
    n = nx + ny
    m = int(s.sum())
    o = n - m
    Wt = W - u[:, None] - u[None, :]
    rt = Wt.sum(axis=1)
    kappa = 2.0 * m / n
    P = 2.0 * np.triu(Wt, 1) + np.diag(np.diag(Wt) - kappa * rt)
    sf = s.astype(np.float64)
    cT = (n / (nx * ny)) ** 2
    return sign * (cT * (sf @ P @ sf) + rt.sum() / o ** 2)


def _double_centring_f32(W):
    n = W.shape[0]
    r = W.sum(axis=1)
    return (r / n - r.sum() / (2.0 * n * n)).astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("stat,sigma", [("ed", 1.0), ("mmd", 2.0), ("mmd_laplace", 3.0)])
@pytest.mark.parametrize("nx,ny", [(13, 29), (31, 9)])
def test_folded_formula_any_centring(stat, sigma, nx, ny):
    X, Y = _pair(nx, ny, 6, seed=nx * 3 + ny)
    Z = np.vstack([X, Y]).astype(np.float64)
    W = oracle.block_matrix(Z, Z, stat, sigma)
    sign = -1.0 if stat == "ed" else 1.0
    rng = np.random.default_rng(5)
    us = [np.zeros(nx + ny), _double_centring_f32(W), rng.normal(size=nx + ny), 1e3 * rng.normal(size=nx + ny)]
    sel = oracle.perm_select(4, nx, ny, 0, 6)
    for k in range(sel.shape[0]):
        ref = oracle.stat_select(X, Y, sel[k], stat, sigma)
        member = sel[k].astype(bool)
        s = member if nx <= ny else ~member   # the smaller group is contracted
        for u in us:
            got = _folded_stat(W, s, nx, ny, sign, u)
            scale = np.abs(W).max() * (1.0 + np.abs(u).max())
            assert abs(got - ref) <= 1e-11 * scale, (k, got, ref)


def test_double_centring_makes_residuals_small():
    # with the double-centring u the entries of W~ are residuals of the size of the
    # spread of the distances, not of their mean, and the row sums r~ vanish up to
    # the FP32 rounding of u (what keeps the FP16 split of C accurate)
    X, Y = _pair(200, 200, 50, seed=2)
    Z = np.vstack([X, Y]).astype(np.float64)
    W = oracle.block_matrix(Z, Z, "ed", 1.0)
    u = _double_centring_f32(W)
    Wt = W - u[:, None] - u[None, :]
    off = ~np.eye(400, dtype=bool)
    assert np.abs(Wt[off]).mean() < 0.1 * W[off].mean()
    assert np.abs(Wt.sum(axis=1)).max() < 1e-4 * W.sum(axis=1).max()
