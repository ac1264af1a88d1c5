"""Caller-supplied device memory (ept_create_ex / ept_allocator): every path of the
library runs on memory from PyTorch's caching allocator (a stream-ordered allocator)
and gives the same results as on its own memory; every allocation is given back;
a failing or misaligned allocator is reported, not used."""
import numpy as np
import pytest

from paper_2406_06488_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ept_mod():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_06488_gb300 import ept
    return ept


def _pair(nx, ny, p, seed):
    return workloads.gaussian_pair(workloads.TwoSampleSpec(nx=nx, ny=ny, p=p, y_mean=0.1, data_seed=seed))


def _torch_allocator(log, offset=0):
    import torch

    def alloc(nbytes, stream):
        p = torch.cuda.caching_allocator_alloc(nbytes + offset, device=0, stream=stream)
        log.append(("alloc", p + offset, nbytes))
        return p + offset

    def free(ptr, stream):
        log.append(("free", ptr))
        torch.cuda.caching_allocator_delete(ptr - offset)

    return alloc, free


def _same(a, b):
    assert a.observed == b.observed and a.n_ge == b.n_ge and a.n_windows == b.n_windows
    if a.stats is not None:
        assert np.array_equal(np.asarray(a.stats), np.asarray(b.stats))


def test_every_path_on_caller_memory(ept_mod):
    log = []
    own = ept_mod.Context(0)
    ext = ept_mod.Context(0, allocator=_torch_allocator(log))
    for c in (own, ext):
        c.set_option("autotune", 0)
    try:
        X, Y = _pair(700, 900, 37, seed=1)
        for prec in ("split_bf16", "plain_fp32", "pooled_fp32"):
            _same(ext.test(X, Y, B=500, seed=2, prec=prec), own.test(X, Y, B=500, seed=2, prec=prec))
        X2, Y2 = _pair(2000, 1500, 64, seed=2)   # a larger arena: the first one is given back
        _same(ext.test(X2, Y2, B=1000, seed=3), own.test(X2, Y2, B=1000, seed=3))
        for c in (own, ext):
            c.set_option("stream_blocks", 1)
        _same(ext.test(X, Y, B=300, seed=4, stat="mmd", sigma=3.0), own.test(X, Y, B=300, seed=4, stat="mmd",
                                                                                sigma=3.0))
        for c in (own, ext):
            c.set_option("stream_blocks", 0)
        tests = [dict(X=X, Y=Y, B=200, seed=k) for k in range(4)]
        for a, b in zip(ext.test_batch(tests), own.test_batch(tests)):
            _same(a, b)
        # serving: batches take their scratch from the allocator too
        tickets = [ext.submit(X, Y, B=200, seed=k) for k in range(6)]
        got = [ext.wait(t) for t in tickets]
        for k, r in enumerate(got):
            _same(r, own.test(X, Y, B=200, seed=k))
    finally:
        ext.close()
        own.close()
    allocs = [e[1] for e in log if e[0] == "alloc"]
    frees = [e[1] for e in log if e[0] == "free"]
    assert len(allocs) >= 3
    assert all(a % 256 == 0 for a in allocs)
    assert sorted(allocs) == sorted(frees)   # everything given back, once


def test_failing_allocator_reports_enomem(ept_mod):
    X, Y = _pair(100, 120, 5, seed=3)
    calls = []
    c = ept_mod.Context(0, allocator=(lambda n, s: calls.append(n) or 0, lambda p, s: None))
    try:
        with pytest.raises(ept_mod.EptError) as e:
            c.test(X, Y, B=50)
        assert e.value.status == 2   # EPT_ENOMEM
        assert calls
    finally:
        c.close()


def test_misaligned_allocator_is_refused(ept_mod):
    log = []
    X, Y = _pair(100, 120, 5, seed=3)
    c = ept_mod.Context(0, allocator=_torch_allocator(log, offset=16))
    try:
        with pytest.raises(ept_mod.EptError) as e:
            c.test(X, Y, B=50)
        assert e.value.status == 1   # EPT_EINVAL
    finally:
        c.close()
    assert [e[1] for e in log if e[0] == "alloc"] == [e[1] for e in log if e[0] == "free"]
