"""One test across ranks through the library (sharded.run_across_ranks): a single rank
equals the plain test, and two processes sharing the GPU (each with its own context
and range; the exchange runs on the host over gloo, and no kernel of one waits on the
other) give the whole test's statistics, count and p-value against the FP64 oracle."""
import os
import socket
import sys

import numpy as np
import pytest

import oracle
from paper_2406_06488_gb300 import workloads

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
REL_TOL = 1e-5
NX, NY, P, B, SEED = 300, 260, 12, 500, 11


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _inputs():
    return workloads.gaussian_pair(workloads.TwoSampleSpec(nx=NX, ny=NY, p=P, y_mean=0.15, data_seed=21))


@pytest.fixture(scope="module")
def ept_mod():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_06488_gb300 import ept
    return ept


def test_one_rank_equals_the_plain_test(ept_mod):
    import torch.distributed as dist
    from paper_2406_06488_gb300 import sharded
    X, Y = _inputs()
    dist.init_process_group("gloo", rank=0, world_size=1, init_method="tcp://127.0.0.1:%d" % _free_port())
    try:
        with ept_mod.Context(0) as ctx:
            plain = ctx.test(X, Y, B=B, seed=SEED)
            obs, stats, nge, near, p = sharded.run_across_ranks(ctx, X, Y, B=B, seed=SEED)
            assert obs == plain.observed and nge == plain.n_ge and p == plain.p_value
            assert np.max(np.abs(stats - np.asarray(plain.stats)) / np.abs(np.asarray(plain.stats))) <= 1e-9
            obs0, stats0, nge0, _, p0 = sharded.run_across_ranks(ctx, X, Y, B=0, seed=SEED)
            assert obs0 == obs and len(stats0) == 0 and nge0 == 0 and p0 == 1.0
    finally:
        dist.destroy_process_group()


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2406_06488_gb300 import ept, sharded
        X, Y = _inputs()
        with ept.Context(0) as ctx:
            obs, stats, nge, near, p = sharded.run_across_ranks(ctx, X, Y, B=B, seed=SEED)
        out[rank] = (obs, stats.tolist(), nge, near, p)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_give_the_whole_test(ept_mod):
    import torch.multiprocessing as mp
    X, Y = _inputs()
    ref = oracle.permutation_test(X, Y, B=B, seed=SEED, stat="ed")
    near_ref = int(np.count_nonzero(np.abs(ref["stats"] - ref["observed"]) <= 1e-5 * abs(ref["observed"])))
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1]
    obs, stats, nge, near, p = res[0]
    assert abs(obs - ref["observed"]) <= REL_TOL * abs(ref["observed"])
    stats = np.asarray(stats)
    assert np.max(np.abs(stats - ref["stats"]) / np.abs(ref["stats"])) <= REL_TOL
    assert abs(nge - ref["n_ge"]) <= near_ref and p == (1.0 + nge) / (1.0 + B)
