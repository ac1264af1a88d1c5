"""Runs that alternate between batch shapes in one context: the contraction reads its
work units from records that are uploaded once per plan and kept in the context's
scratch, so a shape that comes back after other shapes (another resident shape, the
streaming mode, a larger shape that grows the scratch, the plain path) must find its
records again.  Every result against the FP64 oracle (Algorithm 1 blocks; Section 3.1
p-value), and a repeated shape bit for bit equal to its first run."""
import numpy as np
import pytest

import oracle
from paper_2406_06488_gb300 import workloads

pytestmark = pytest.mark.gpu

REL_TOL = 1e-5


def _pair(nx, ny, p, seed):
    return workloads.gaussian_pair(workloads.TwoSampleSpec(nx=nx, ny=ny, p=p, y_mean=0.1, data_seed=seed))


def _check(r, X, Y, B, seed):
    ref = oracle.permutation_test(X, Y, B=B, seed=seed, stat="ed", method="blocks")
    got = np.concatenate([[r.observed], np.asarray(r.stats)])
    want = np.concatenate([[ref["observed"]], ref["stats"]])
    assert np.max(np.abs(got - want) / np.abs(want)) <= REL_TOL
    near = int(np.count_nonzero(np.abs(ref["stats"] - ref["observed"]) <= 1e-5 * abs(ref["observed"])))
    assert abs(r.n_ge - ref["n_ge"]) <= near


@pytest.mark.parametrize("graphs", [1, 0])
def test_shapes_alternate_in_one_context(graphs):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_06488_gb300 import ept
    A = _pair(600, 700, 30, 1)
    Bs = _pair(300, 1250, 12, 2)
    C = _pair(2500, 2200, 8, 3)   # larger: grows the context's scratch
    with ept.Context(0) as c:
        c.set_option("graphs", graphs)
        first = c.test(*A, B=500, seed=11)
        _check(first, *A, 500, 11)
        runs = [("B", Bs, 300, 12, {}), ("A", A, 500, 11, {}), ("stream", Bs, 300, 12, {"stream": True}),
                ("A", A, 500, 11, {}), ("C", C, 260, 13, {}), ("A", A, 500, 11, {}),
                ("plain", Bs, 300, 12, {"plain": True}), ("A", A, 500, 11, {})]
        for name, (X, Y), B, seed, kind in runs:
            if kind.get("stream"):
                c.set_option("stream_blocks", 1)
            r = c.test(X, Y, B=B, seed=seed, prec="plain_fp32" if kind.get("plain") else "split_bf16")
            if kind.get("stream"):
                assert r.n_windows > 1
                c.set_option("stream_blocks", 0)
            _check(r, X, Y, B, seed)
            if name == "A":
                assert r.observed == first.observed and np.array_equal(np.asarray(r.stats), np.asarray(first.stats))
