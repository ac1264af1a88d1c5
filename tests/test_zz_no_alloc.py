"""ept_test_static: the permutation test that allocates nothing (its scratch is one
fixed device array inside the library), for callers that cannot call cudaMalloc --
for example an application whose own memory pool owns the whole GPU, or a
latency-critical loop that must not enter the allocator.

Called through the C ABI with device buffers, it must give the statistics of the
allocating entry point (ept_test, split-BF16 path) within the tolerance of the
other parity tests, on two calls in a row (the second call reuses the array the
first one left behind), and reject tests too large for its array."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

REL_TOL = 1e-5


def _call_static(lib, ept, Xd, Yd, B, seed, stat, sigma, out):
    import torch
    r = ept._Result()
    st = lib.ept_test_static(Xd.data_ptr(), Xd.shape[0], Yd.data_ptr(), Yd.shape[0], Xd.shape[1], stat, sigma, B,
                             ctypes.c_uint64(seed), out.data_ptr() if out is not None else None, ctypes.byref(r),
                             torch.cuda.current_stream().cuda_stream)
    return st, r


def test_static_entry_point_matches_allocating_one():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_06488_gb300 import ept, workloads

    lib = ept.load()
    cases = [  # (spec, statistic code, sigma)
        (workloads.TwoSampleSpec(nx=300, ny=500, p=40, y_mean=0.2, B=2000, seed=7, data_seed=1), 0, 1.0),
        (workloads.TwoSampleSpec(nx=700, ny=250, p=17, y_var=1.2, B=3000, seed=9, data_seed=2), 1, 3.0),
    ]
    with ept.Context(0) as ctx:
        for spec, stat, sigma in cases:   # two calls in a row, different shapes
            X, Y = workloads.gaussian_pair(spec)
            Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
            ref = ctx.test(Xd, Yd, B=spec.B, seed=spec.seed, stat=["ed", "mmd"][stat], sigma=sigma,
                           prec="split_bf16")
            ref_stats = ref.stats.cpu().numpy()
            out = torch.full((spec.B,), float("nan"), dtype=torch.float64, device="cuda")
            st, r = _call_static(lib, ept, Xd, Yd, spec.B, spec.seed, stat, sigma, out)
            assert st == 0, lib.ept_last_error()
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            rel = np.abs(got - ref_stats) / np.abs(ref_stats)
            assert rel.max() <= REL_TOL
            assert abs(r.observed - ref.observed) <= REL_TOL * abs(ref.observed)
            near = int(np.count_nonzero(np.abs(ref_stats - ref.observed) <= 1e-5 * abs(ref.observed)))
            assert abs(r.n_ge - ref.n_ge) <= near
            assert r.p_value == (1.0 + r.n_ge) / (1.0 + spec.B)

    # a test whose scratch does not fit in the fixed array is refused, not truncated
    X, Y = workloads.gaussian_pair(workloads.TwoSampleSpec(nx=3000, ny=3000, p=8))
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    st, _ = _call_static(lib, ept, Xd, Yd, 1000, 0, 0, 1.0, None)
    assert st == 1
    assert b"EPT_STATIC_SCRATCH_BYTES" in lib.ept_last_error()
