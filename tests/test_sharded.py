"""One permutation test across processes (paper_2406_06488_gb300/sharded.py), on the
CPU: the relabeling ranges cover 1..B once, and two or three gloo ranks, each
evaluating its range with the FP64 oracle, return after their single exchange
exactly the whole test's statistics, count and p-value (Section 3.1)."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2406_06488_gb300 import sharded  # noqa: E402

NX, NY, P, B, SEED = 60, 50, 4, 101, 7


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("B,world", [(0, 1), (1, 3), (101, 2), (101, 3), (5, 8), (10 ** 6, 7)])
def test_ranges_cover_every_relabeling_once(B, world):
    ranges = sharded.permutation_ranges(B, world)
    assert len(ranges) == world
    b = 1
    for b_first, count in ranges:
        assert b_first == b and count >= 0
        b += count
    assert b == B + 1
    sizes = [c for _, c in ranges]
    assert max(sizes) - min(sizes) <= 1


def test_range_arguments():
    with pytest.raises(ValueError):
        sharded.permutation_ranges(-1, 2)
    with pytest.raises(ValueError):
        sharded.permutation_ranges(10, 0)


def test_combine():
    obs, st, nge, near, p = sharded.combine(2.0, [[1.0, 3.0], [], [2.0]], 3)
    assert obs == 2.0 and list(st) == [1.0, 3.0, 2.0] and nge == 2 and near == 1 and p == 3.0 / 4.0
    with pytest.raises(ValueError):
        sharded.combine(2.0, [[1.0]], 2)


def test_combine_counts_against_one_observed():
    # the counts come from the gathered statistics and the observed statistic given,
    # not from per-range counts taken against slightly different observed values
    obs = 1.0
    parts = [[1.0 - 1e-16, 0.5], [1.0 + 1e-16, 2.0]]
    _, _, nge, near, p = sharded.combine(obs, parts, 4)
    assert nge == 2 and near == 2 and p == 3.0 / 5.0


def _inputs():
    from paper_2406_06488_gb300 import workloads
    return workloads.gaussian_pair(workloads.TwoSampleSpec(nx=NX, ny=NY, p=P, y_mean=0.3, data_seed=9))


def _oracle_range(b_first, count):
    import oracle
    X, Y = _inputs()
    observed = float(oracle.test_direct(X, Y, oracle.perm_select(SEED, NX, NY, 0, 1), "ed")[0])
    stats = oracle.test_direct(X, Y, oracle.perm_select(SEED, NX, NY, b_first, count), "ed") if count else np.zeros(0)
    n_ge = int(np.count_nonzero(stats >= observed))
    n_near = int(np.count_nonzero(np.abs(stats - observed) <= 1e-5 * abs(observed)))
    return observed, stats, n_ge, n_near


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), OMP_NUM_THREADS="1")
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2406_06488_gb300 import sharded as sh
        obs, stats, nge, near, p = sh.sharded_test(_oracle_range, B)
        out[rank] = (obs, stats.tolist(), nge, near, p)
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_ranks_reproduce_the_whole_test(world):
    import oracle
    import torch.multiprocessing as mp
    X, Y = _inputs()
    whole = oracle.permutation_test(X, Y, B=B, seed=SEED, stat="ed")
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == list(range(world))
    for r in range(world):
        obs, stats, nge, near, p = res[r]
        assert obs == whole["observed"]
        assert np.array_equal(np.asarray(stats), whole["stats"])
        assert nge == whole["n_ge"] and p == whole["p_value"]


def _failing_rank_main(rank, world, port, mode, out):
    import datetime
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), OMP_NUM_THREADS="1")
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    from paper_2406_06488_gb300 import sharded as sh

    def run_range(b_first, count):
        if rank == 1:
            if mode == "raise":
                raise ValueError("range evaluation failed")
            os._exit(3)                     # the process dies without a word
        return _oracle_range(b_first, count)

    import time
    t0 = time.time()
    try:
        sh.sharded_test(run_range, B)
        out[rank] = ("ok", time.time() - t0)
    except Exception as e:                  # noqa: BLE001 - the type is what the test checks
        out[rank] = (type(e).__name__, time.time() - t0)
    finally:
        try:
            dist.destroy_process_group()
        except Exception:                   # noqa: BLE001 - the group may be broken by a dead peer
            pass


@pytest.mark.parametrize("mode", ["raise", "exit"])
def test_a_failed_rank_ends_the_test_everywhere(mode):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_failing_rank_main, args=(r, 2, port, mode, out)) for r in range(2)]
        for pr in procs:
            pr.start()
        for pr in procs:
            pr.join(timeout=120)
        res = dict(out)
        codes = [pr.exitcode for pr in procs]
    # rank 0 learns of the failure in the status reduction (no result, no wait in the gather)
    assert res[0][0] == "RangeFailed" if mode == "raise" else res[0][0] != "ok", res
    assert res[0][1] < 30.0
    if mode == "raise":
        assert res[1][0] == "ValueError" and codes == [0, 0]
    else:
        assert 1 not in res and codes[1] == 3
