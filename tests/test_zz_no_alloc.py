"""ept_test_static: the permutation test that allocates nothing (its scratch is one
fixed device array inside the library), for callers that cannot call cudaMalloc --
for example an application whose own memory pool owns the whole GPU, or a
latency-critical loop that must not enter the allocator.

Called through the C ABI with device buffers, on two calls in a row (the second
call reuses the array the first one left behind), its statistics must match the
FP64 oracle (Algorithm 1 on the three blocks, Section 3.1 p-value) within the
tolerance of the other parity tests and the allocating entry point's own results;
a warmed call must leave the device's free memory unchanged; a failing call (NaN
input) must leave the output buffer untouched; a test too large for the array is
rejected."""
import ctypes

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

REL_TOL = 1e-5


def _call_static(lib, ept, Xd, Yd, B, seed, stat, sigma, out):
    import torch
    r = ept._Result()
    st = lib.ept_test_static(Xd.data_ptr(), Xd.shape[0], Yd.data_ptr(), Yd.shape[0], Xd.shape[1], stat, sigma, B,
                             ctypes.c_uint64(seed), out.data_ptr() if out is not None else None, ctypes.byref(r),
                             torch.cuda.current_stream().cuda_stream)
    return st, r


def test_static_entry_point_matches_the_oracle():
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
            name = ["ed", "mmd"][stat]
            X, Y = workloads.gaussian_pair(spec)
            ref = oracle.permutation_test(X, Y, B=spec.B, seed=spec.seed, stat=name, sigma=sigma, method="blocks")
            Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
            out = torch.full((spec.B,), float("nan"), dtype=torch.float64, device="cuda")
            st, r = _call_static(lib, ept, Xd, Yd, spec.B, spec.seed, stat, sigma, out)
            assert st == 0, lib.ept_last_error()
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            rel = np.abs(got - ref["stats"]) / np.abs(ref["stats"])
            assert rel.max() <= REL_TOL, rel.max()
            assert abs(r.observed - ref["observed"]) <= REL_TOL * abs(ref["observed"])
            near = int(np.count_nonzero(np.abs(ref["stats"] - ref["observed"]) <= 1e-5 * abs(ref["observed"])))
            assert abs(r.n_ge - ref["n_ge"]) <= near
            assert r.p_value == (1.0 + r.n_ge) / (1.0 + spec.B)
            # the allocating entry point on the same device inputs agrees as well
            alloc = ctx.test(Xd, Yd, B=spec.B, seed=spec.seed, stat=name, sigma=sigma, prec="split_bf16")
            a = alloc.stats.cpu().numpy()
            assert (np.abs(got - a) / np.abs(a)).max() <= REL_TOL

        # a warmed call allocates nothing: the device's free memory is the same after it
        spec, stat, sigma = cases[0]
        X, Y = workloads.gaussian_pair(spec)
        Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
        out = torch.empty(spec.B, dtype=torch.float64, device="cuda")
        assert _call_static(lib, ept, Xd, Yd, spec.B, spec.seed, stat, sigma, out)[0] == 0
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        assert _call_static(lib, ept, Xd, Yd, spec.B, spec.seed, stat, sigma, out)[0] == 0
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0

        # a failing call leaves the output untouched
        Xbad = Xd.clone()
        Xbad[3, 1] = float("nan")
        keep = torch.full((spec.B,), float("nan"), dtype=torch.float64, device="cuda")
        st, _ = _call_static(lib, ept, Xbad, Yd, spec.B, spec.seed, stat, sigma, keep)
        assert st == 1
        torch.cuda.synchronize()
        assert torch.isnan(keep).all()

    # a test whose scratch does not fit in the fixed array is refused, not truncated
    X, Y = workloads.gaussian_pair(workloads.TwoSampleSpec(nx=3000, ny=3000, p=8))
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    st, _ = _call_static(lib, ept, Xd, Yd, 1000, 0, 0, 1.0, None)
    assert st == 1
    assert b"EPT_STATIC_SCRATCH_BYTES" in lib.ept_last_error()
