"""Debug checks (a stand-in for a memory checker, which is not available here): with
EPT_OPT_DEBUG_CHECKS every scratch region of a run is followed by a guard band that
is filled before the run and checked after it, and the plan's invariants are checked
on the host.  Every path must pass them and give the same results as without."""
import numpy as np
import pytest

from paper_2406_06488_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctxs():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_06488_gb300 import ept
    dbg, ref = ept.Context(0), ept.Context(0)
    dbg.set_option("debug_checks", 1)
    for c in (dbg, ref):   # the same chunk length in both, so the sums run in the same order
        c.set_option("autotune", 0)
    yield dbg, ref
    dbg.close()
    ref.close()


def _pair(nx, ny, p, seed):
    return workloads.gaussian_pair(workloads.TwoSampleSpec(nx=nx, ny=ny, p=p, y_mean=0.2, data_seed=seed))


@pytest.mark.parametrize("prec", ["split_bf16", "plain_fp32"])
@pytest.mark.parametrize("nx,ny,p,B,stat,sigma", [
    (1, 1, 1, 5, "ed", 1.0), (9, 1, 3, 40, "ed", 1.0), (255, 2, 5, 300, "mmd", 2.0), (300, 420, 70, 700, "ed", 1.0),
    (150, 170, 9, 333, "mmd_laplace", "median"), (2000, 3000, 1000, 2000, "ed", 1.0)])
def test_guards_hold_and_results_match(ctxs, prec, nx, ny, p, B, stat, sigma):
    dbg, ref = ctxs
    X, Y = _pair(nx, ny, p, seed=nx + ny + p)
    for _ in range(2):   # the second call replays a captured graph
        a = dbg.test(X, Y, B=B, seed=3, stat=stat, sigma=sigma, prec=prec)
    b = ref.test(X, Y, B=B, seed=3, stat=stat, sigma=sigma, prec=prec)
    assert a.observed == b.observed and a.n_ge == b.n_ge
    assert np.array_equal(np.asarray(a.stats), np.asarray(b.stats))


def test_guards_hold_for_batches_masks_and_ranges(ctxs):
    dbg, ref = ctxs
    r = np.random.default_rng(5)
    tests = []
    for k in range(20):
        X, Y = _pair(int(r.integers(1, 600)), int(r.integers(1, 600)), int(r.integers(1, 40)), seed=k)
        tests.append(dict(X=X, Y=Y, B=int(r.integers(0, 500)), seed=k))
    a = dbg.test_batch(tests)
    b = ref.test_batch(tests)
    for x, y in zip(a, b):
        assert x.observed == y.observed and x.n_ge == y.n_ge
    X, Y = _pair(40, 50, 4, seed=9)
    masks = dbg.perm_masks(seed=1, nx=40, ny=50, b0=1, count=64)
    assert dbg.test_masks(X, Y, masks).observed == ref.test_masks(X, Y, masks).observed
    assert dbg.test_range(X, Y, b_first=17, count=99, seed=2).n_ge == ref.test_range(X, Y, b_first=17, count=99,
                                                                                    seed=2).n_ge


@pytest.mark.parametrize("nx,ny,p,B,stat", [(9, 1, 3, 40, "ed"), (300, 420, 70, 700, "mmd"),
                                            (700, 900, 37, 300, "mmd_laplace")])
def test_guards_hold_in_streaming_mode(ctxs, nx, ny, p, B, stat):
    # windows of one panel each: every window's blocks, sums and partials reuse the
    # same guarded regions
    dbg, ref = ctxs
    X, Y = _pair(nx, ny, p, seed=nx + 2 * ny)
    try:
        for c in (dbg, ref):
            c.set_option("stream_blocks", 1)
        a = dbg.test(X, Y, B=B, seed=4, stat=stat, sigma=2.0)
        b = ref.test(X, Y, B=B, seed=4, stat=stat, sigma=2.0)
    finally:
        for c in (dbg, ref):
            c.set_option("stream_blocks", 0)
    assert a.n_windows == (nx + ny + 255) // 256
    assert a.observed == b.observed and a.n_ge == b.n_ge
    assert np.array_equal(np.asarray(a.stats), np.asarray(b.stats))


@pytest.mark.parametrize("nx,ny,p,B", [(1, 1, 1, 5), (255, 2, 5, 300), (600, 500, 40, 257)])
def test_guards_hold_for_the_precomputation_baseline(ctxs, nx, ny, p, B):
    dbg, ref = ctxs
    X, Y = _pair(nx, ny, p, seed=nx + 3 * ny)
    a = dbg.test(X, Y, B=B, seed=6, prec="pooled_fp32")
    b = ref.test(X, Y, B=B, seed=6, prec="pooled_fp32")
    assert a.observed == b.observed and a.n_ge == b.n_ge
    assert np.array_equal(np.asarray(a.stats), np.asarray(b.stats))
