"""The three tensor-core contraction kernels (EPT_OPT_CONTRACTION: 1 relabelings as
the shared-memory operand, 2 the same on pairs of SMs, 3 relabelings as the
tensor-memory operand) against the FP64 oracle (Algorithm 1 on the three blocks)
and against each other.

Shapes cover a single panel, ragged row panels, relabeling tiles that end inside
their first or second 128 relabelings or exactly on a tile edge, and a batched call
of uneven tests.  Every statistic within 1e-5 of the oracle (recomputation of
flagged statistics on, the product path); with recomputation off, the kernels'
fast values agree with each other to 2e-6 relative (the same unit decomposition,
summed in different orders)."""
import numpy as np
import pytest

import oracle
from paper_2406_06488_gb300 import workloads

pytestmark = pytest.mark.gpu

KERNELS = (1, 2, 3)


@pytest.fixture(scope="module")
def ctxs():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_06488_gb300 import ept
    out = {}
    for k in KERNELS:
        for refine in (0, 1):
            c = ept.Context(0)
            c.set_option("contraction", k)
            c.set_option("refine", refine)
            c.set_option("autotune", 0)
            out[(k, refine)] = c
    yield out
    for c in out.values():
        c.close()


def _pair(nx, ny, p, seed):
    return workloads.gaussian_pair(workloads.TwoSampleSpec(nx=nx, ny=ny, p=p, y_mean=0.2, data_seed=seed))


# (nx, ny, p, B, stat): B + 1 columns = 201 (inside the second 128 of one tile), 128
# (one sub-tile exactly), 129 (one column into the second), 256 (a tile edge), 300
CASES = [(70, 90, 12, 200, "ed"), (300, 517, 40, 127, "ed"), (1000, 1300, 64, 128, "mmd"),
         (777, 1500, 33, 255, "ed"), (2048, 1024, 100, 299, "mmd_laplace"), (1, 600, 5, 200, "ed")]


@pytest.mark.parametrize("nx,ny,p,B,stat", CASES)
def test_kernels_match_the_oracle_and_each_other(ctxs, nx, ny, p, B, stat):
    X, Y = _pair(nx, ny, p, seed=nx + ny)
    seed = 11 * nx + ny
    sigma = float(np.sqrt(p))
    ref = oracle.permutation_test(X, Y, B=B, seed=seed, stat=stat, sigma=sigma, method="blocks")
    want = np.concatenate([[ref["observed"]], ref["stats"]])
    fast = {}
    for k in KERNELS:
        r = ctxs[(k, 1)].test(X, Y, B=B, seed=seed, stat=stat, sigma=sigma)
        got = np.concatenate([[r.observed], r.stats])
        rel = np.abs(got - want) / np.abs(want)
        assert rel.max() <= 1e-5, (k, float(rel.max()), int(rel.argmax()))
        f = ctxs[(k, 0)].test(X, Y, B=B, seed=seed, stat=stat, sigma=sigma)
        fast[k] = np.concatenate([[f.observed], f.stats])
    for k in KERNELS[1:]:
        rel = np.abs(fast[k] - fast[1]) / np.abs(want)
        assert rel.max() <= 2e-6, (k, float(rel.max()), int(rel.argmax()))


def test_batched_uneven_tests(ctxs):
    tests, refs = [], []
    for j, (nx, ny, p, B) in enumerate([(50, 61, 7, 100), (400, 380, 30, 260), (1200, 900, 20, 130),
                                        (3, 5, 2, 64), (900, 1800, 50, 500)]):
        X, Y = _pair(nx, ny, p, seed=100 + j)
        tests.append(dict(X=X, Y=Y, B=B, seed=7 + j, stat="ed"))
        refs.append(oracle.permutation_test(X, Y, B=B, seed=7 + j, stat="ed", method="blocks"))
    for k in KERNELS:
        res = ctxs[(k, 1)].test_batch(tests)
        for r, ref in zip(res, refs):
            want = np.concatenate([[ref["observed"]], ref["stats"]])
            got = np.concatenate([[r.observed], r.stats])
            rel = np.abs(got - want) / np.abs(want)
            assert rel.max() <= 1e-5, (k, float(rel.max()))
