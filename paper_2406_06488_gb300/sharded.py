"""One permutation test across several processes (one GPU each): the relabelings
1..B of the test's counter-based stream are split into contiguous ranges, each
process evaluates its range (the observed statistic is relabeling 0 in every range),
and a single exchange at the end gathers the permuted statistics, which every
process then counts against rank 0's observed statistic; the p-value
(1 + #{stat* >= observed}) / (1 + B) (Section 3.1) is then that of the whole test.  Relabeling b is draw b of the stream whatever the number of
processes, so the result does not depend on it.  No collective runs inside a kernel.

The exchange uses torch.distributed on the process group given (tensors on the
current CUDA device for NCCL, on the CPU otherwise).  Failures: a rank whose range
raises reports it in a status reduction before the exchange and re-raises; the other
ranks then raise RangeFailed at once instead of waiting in the gather.  A rank that
dies outright is noticed by the process group (its timeout, or the broken
connection) in that same reduction."""
from __future__ import annotations

import numpy as np


def permutation_ranges(B: int, world: int):
    """Contiguous ranges (b_first, count) of relabelings 1..B for ranks 0..world-1,
    sizes differing by at most one (a rank may get none when world > B)."""
    if B < 0 or world < 1:
        raise ValueError("B must be >= 0 and world >= 1")
    base, extra = divmod(B, world)
    out, b = [], 1
    for r in range(world):
        c = base + (1 if r < extra else 0)
        out.append((b, c))
        b += c
    return out


def combine(observed: float, stats_parts, B: int):
    """The whole test from its ranges: (observed, stats[B] in relabeling order, n_ge,
    n_near_tie, p_value).  The counts are taken here, against the one observed
    statistic given (Section 3.1: #{stat* >= observed}; near-ties within 1e-5 of it),
    so that every rank compares every statistic with the same threshold even where
    the ranks' own evaluations of the observed statistic differ in the last bits."""
    stats = np.concatenate([np.asarray(s, dtype=np.float64) for s in stats_parts]) if B else np.zeros(0)
    if stats.shape[0] != B:
        raise ValueError("the ranges hold %d statistics, the test has %d" % (stats.shape[0], B))
    n_ge = int(np.count_nonzero(stats >= observed))
    n_near = int(np.count_nonzero(np.abs(stats - observed) <= 1e-5 * abs(observed)))
    return observed, stats, n_ge, n_near, (1.0 + n_ge) / (1.0 + B)


class RangeFailed(RuntimeError):
    """Another rank's range failed, so the test has no result."""


def sharded_test(run_range, B: int, group=None):
    """Run this rank's range with run_range(b_first, count) -> (observed, stats[count],
    n_ge, n_near_tie), then exchange once; every rank returns the whole test's
    (observed, stats[B], n_ge, n_near_tie, p_value)."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    ranges = permutation_ranges(B, world)
    b_first, count = ranges[rank]
    device = (torch.device("cuda", torch.cuda.current_device())
              if dist.get_backend(group) == "nccl" else torch.device("cpu"))
    error = None
    try:
        observed, stats, n_ge, n_near = run_range(b_first, count)
        stats = np.asarray(stats, dtype=np.float64).reshape(-1)
        if stats.shape[0] != count:
            raise ValueError("run_range returned %d statistics for a range of %d" % (stats.shape[0], count))
    except Exception as e:   # reported to the other ranks below, then re-raised here
        error = e
    # every rank's status before the exchange: a failed range ends the test everywhere
    failed = torch.tensor([0 if error is None else 1], dtype=torch.int64, device=device)
    dist.all_reduce(failed, group=group)
    if error is not None:
        raise error
    if int(failed.item()):
        raise RangeFailed("%d rank(s) failed to evaluate their range of relabelings" % int(failed.item()))
    width = max(c for _, c in ranges) if ranges else 0
    # one gather of the padded ranges (and of each rank's observed statistic, which
    # is the same relabeling 0 everywhere); every rank then counts the whole test's
    # statistics against rank 0's observed statistic
    mine = torch.zeros(width + 1, dtype=torch.float64, device=device)
    mine[0] = float(observed)
    if count:
        mine[1:count + 1] = torch.from_numpy(stats).to(device)
    parts = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    parts = [p.cpu().numpy() for p in parts]
    stats_parts = [parts[r][1:c + 1] for r, (_, c) in enumerate(ranges)]
    return combine(float(parts[0][0]), stats_parts, B)


def run_across_ranks(ctx, X, Y, B: int, seed: int = 0, stat="ed", sigma: float = 1.0, prec="split_bf16",
                      group=None):
    """sharded_test with this rank's range evaluated by ctx.test_range (the library)."""
    def run_range(b_first, count):
        if count == 0:   # no relabelings here: the observed statistic alone
            r = ctx.test(X, Y, B=0, seed=seed, stat=stat, sigma=sigma, prec=prec)
            return r.observed, np.zeros(0), 0, 0
        r = ctx.test_range(X, Y, b_first=b_first, count=count, seed=seed, stat=stat, sigma=sigma, prec=prec)
        st = r.stats.cpu().numpy() if hasattr(r.stats, "cpu") else r.stats
        return r.observed, st, r.n_ge, r.n_near_tie

    return sharded_test(run_range, B, group)
