"""Statistical validation on the batched path (the paper's Section 5 experiments as
many-test batches): under the null the p-values are uniform on {1, ..., B+1}/(B+1)
(the permutation test is exact), and under the alternatives the rejection rate at
alpha = 0.05 grows with the sample size."""
import numpy as np
import pytest
from scipy.stats import chisquare

from paper_2406_06488_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_06488_gb300 import ept
    c = ept.Context(0)
    yield c
    c.close()


def _pvalues(ctx, specs, chunk=500):
    out = []
    for k in range(0, len(specs), chunk):
        tests = []
        for sp in specs[k:k + chunk]:
            X, Y = workloads.gaussian_pair(sp)
            tests.append(dict(X=X, Y=Y, B=sp.B, seed=sp.seed, stat=sp.stat, sigma=sp.sigma))
        out += [r.p_value for r in ctx.test_batch(tests, want_stats=False)]
    return np.asarray(out)


@pytest.mark.parametrize("stat", ["ed", "mmd"])
def test_null_pvalues_are_uniform(ctx, stat):
    B, reps = 200, 1000
    p = _pvalues(ctx, workloads.null_specs(reps=reps, n=200, p=100, B=B, stat=stat))
    atoms = np.arange(1, B + 2) / (B + 1)
    assert np.all(np.isin(np.round(p * (B + 1)), np.arange(1, B + 2)))
    # ten bins of atoms; expected counts proportional to the atoms in each bin
    edges = np.linspace(0, 1, 11)
    idx_atoms = np.clip(np.searchsorted(edges, atoms, side="left") - 1, 0, 9)
    expect = np.bincount(idx_atoms, minlength=10) / atoms.size * reps
    got = np.bincount(np.clip(np.searchsorted(edges, p, side="left") - 1, 0, 9), minlength=10)
    assert chisquare(got, expect).pvalue > 1e-3, (got, expect)
    # level: P(p <= 0.05) = 10 / 201 under the null
    rate = np.mean(p <= 0.05)
    q = 10 / (B + 1)
    assert abs(rate - q) <= 4 * np.sqrt(q * (1 - q) / reps), rate


def test_power_grows_with_sample_size(ctx):
    pts = workloads.power_specs(1, reps=200, points=[60, 200, 360])
    power = [np.mean(_pvalues(ctx, specs) <= 0.05) for _, specs in pts]
    assert power[0] < power[1] < power[2], power
    assert power[0] > 0.05 and power[2] > 0.5, power
