"""Serving: requests submitted to the continuous-batching scheduler give the same
results as the same tests run alone, and the FP64 oracle's results when they arrive
(Poisson-timed, from a submitter thread) while earlier batches are running on other
lanes; tickets, cancellation, timeouts, per-request errors and the memory budget
behave as the C ABI states."""
import threading
import time

import numpy as np
import pytest

import oracle
from paper_2406_06488_gb300 import workloads

pytestmark = pytest.mark.gpu

REL_TOL = 1e-5


@pytest.fixture(scope="module")
def ept():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_06488_gb300 import ept as mod
    return mod


@pytest.fixture(scope="module")
def ctx(ept):
    c = ept.Context(0)
    yield c
    c.close()


def _requests(n, seed, max_n=700, max_p=60, max_B=600):
    r = np.random.default_rng(seed)
    out = []
    for k in range(n):
        nx, ny, p = int(r.integers(1, max_n)), int(r.integers(1, max_n)), int(r.integers(1, max_p))
        spec = workloads.TwoSampleSpec(nx=nx, ny=ny, p=p, y_mean=0.15 * (k % 2), data_seed=seed * 1000 + k)
        X, Y = workloads.gaussian_pair(spec)
        out.append(dict(X=X, Y=Y, B=int(r.integers(0, max_B)), seed=k + 3, stat="mmd" if k % 4 == 0 else "ed",
                        sigma=float(np.sqrt(p))))
    return out


@pytest.mark.parametrize("prec", ["split_bf16", "plain_fp32"])
def test_served_equals_alone(ctx, prec):
    reqs = _requests(40, seed=11)
    tickets = [ctx.submit(q["X"], q["Y"], B=q["B"], seed=q["seed"], stat=q["stat"], sigma=q["sigma"], prec=prec)
               for q in reqs]
    assert len(set(tickets)) == len(tickets)
    got = [ctx.wait(t) for t in tickets]
    for q, r in zip(reqs, got):
        alone = ctx.test(q["X"], q["Y"], B=q["B"], seed=q["seed"], stat=q["stat"], sigma=q["sigma"], prec=prec)
        assert abs(r.observed - alone.observed) <= REL_TOL * abs(alone.observed)
        if q["B"] > 0:
            a, b = np.asarray(r.stats), np.asarray(alone.stats)
            assert a.shape == b.shape and np.max(np.abs(a - b) / np.abs(b)) <= REL_TOL
        assert abs(r.n_ge - alone.n_ge) <= alone.n_near_tie
        assert r.p_value == (1.0 + r.n_ge) / (1.0 + q["B"])
        assert r.ms_total > 0.0


def test_mixed_precisions_in_queue(ctx):
    reqs = _requests(10, seed=12)
    precs = ["split_bf16" if k % 2 else "plain_fp32" for k in range(len(reqs))]
    tickets = [ctx.submit(q["X"], q["Y"], B=q["B"], seed=q["seed"], stat=q["stat"], sigma=q["sigma"], prec=pr)
               for q, pr in zip(reqs, precs)]
    for q, pr, t in zip(reqs, precs, tickets):
        r = ctx.wait(t)
        alone = ctx.test(q["X"], q["Y"], B=q["B"], seed=q["seed"], stat=q["stat"], sigma=q["sigma"], prec=pr)
        assert abs(r.observed - alone.observed) <= REL_TOL * abs(alone.observed)
        if q["B"] > 0:
            a, b = np.asarray(r.stats), np.asarray(alone.stats)
            assert a.shape == b.shape and np.max(np.abs(a - b) / np.abs(b)) <= REL_TOL
        assert abs(r.n_ge - alone.n_ge) <= alone.n_near_tie
        assert r.p_value == (1.0 + r.n_ge) / (1.0 + q["B"])


def test_overlapping_arrivals_match_the_oracle(ept):
    """A submitter thread feeds Poisson-timed requests (about 2000 per second) right
    after a large first one, so that requests arrive while earlier batches run on other
    lanes; every served result equals the FP64 oracle's whole test (Algorithm 1 on the
    three blocks; Section 3.1 p-value): statistics within 1e-5, counts equal except
    through near-ties."""
    c = ept.Context(0)
    try:
        r = np.random.default_rng(21)
        reqs = []
        big = workloads.TwoSampleSpec(nx=1000, ny=1000, p=400, y_mean=0.05, data_seed=2100)
        X, Y = workloads.gaussian_pair(big)
        reqs.append(dict(X=X, Y=Y, B=20000, seed=1, stat="ed", sigma=1.0))
        for k in range(31):
            nx, ny, p = int(r.integers(100, 1000)), int(r.integers(100, 1000)), int(r.integers(4, 120))
            spec = workloads.TwoSampleSpec(nx=nx, ny=ny, p=p, y_mean=0.1 * (k % 3), y_var=1.0 + 0.1 * (k % 2),
                                           data_seed=2200 + k)
            X, Y = workloads.gaussian_pair(spec)
            reqs.append(dict(X=X, Y=Y, B=int(r.choice([1000, 3000, 5000])), seed=100 + k,
                             stat=["ed", "mmd", "mmd_laplace"][k % 3], sigma=float(np.sqrt(p))))
        gaps = r.exponential(1.0 / 2000.0, size=len(reqs))
        tickets = [None] * len(reqs)

        def submitter():
            t0 = time.perf_counter()
            due = 0.0
            for k, q in enumerate(reqs):
                due += gaps[k] if k else 0.0
                delay = t0 + due - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                tickets[k] = c.submit(q["X"], q["Y"], B=q["B"], seed=q["seed"], stat=q["stat"], sigma=q["sigma"])

        th = threading.Thread(target=submitter)
        th.start()
        th.join()
        got = [c.wait(t) for t in tickets]
        lanes = c.serving_lanes()
        assert lanes["submits_while_busy"] >= 1, lanes
        assert lanes["peak_busy"] >= 2, lanes
        for q, res in zip(reqs, got):
            ref = oracle.permutation_test(q["X"], q["Y"], B=q["B"], seed=q["seed"], stat=q["stat"], sigma=q["sigma"],
                                          method="blocks")
            assert abs(res.observed - ref["observed"]) <= REL_TOL * abs(ref["observed"])
            rel = np.abs(np.asarray(res.stats) - ref["stats"]) / np.abs(ref["stats"])
            assert rel.max() <= REL_TOL, (q["stat"], float(rel.max()))
            near = int(np.count_nonzero(np.abs(ref["stats"] - ref["observed"]) <= 1e-5 * abs(ref["observed"])))
            assert abs(res.n_ge - ref["n_ge"]) <= near
            assert res.p_value == (1.0 + res.n_ge) / (1.0 + q["B"])
    finally:
        c.close()


def test_poll_timeout_and_unknown_ticket(ctx, ept):
    X, Y = workloads.gaussian_pair(workloads.HIGHDIM)
    t = ctx.submit(X, Y, B=10000, seed=5)
    with pytest.raises(ept.EptError) as e:
        ctx.wait(t, timeout_ms=0)
    assert e.value.status == 5          # not finished yet; the ticket stays valid
    r = ctx.wait(t)
    assert ctx.poll is not None and r.n_ge >= 0
    with pytest.raises(ept.EptError) as e:
        ctx.poll(t)                      # released by the wait
    assert e.value.status == 7
    with pytest.raises(ept.EptError) as e:
        ctx.wait(123456789)
    assert e.value.status == 7


def test_poll_reports_done(ctx):
    q = _requests(1, seed=13)[0]
    t = ctx.submit(q["X"], q["Y"], B=q["B"], seed=q["seed"], stat=q["stat"], sigma=q["sigma"])
    import time
    deadline = time.time() + 30
    while not ctx.poll(t):
        assert time.time() < deadline
        time.sleep(0.001)
    ctx.wait(t)


def test_cancel(ctx, ept):
    X, Y = workloads.gaussian_pair(workloads.HIGHDIM)
    tickets = [ctx.submit(X, Y, B=10000, seed=k) for k in range(8)]
    ctx.cancel(tickets[-1])              # queued behind the others, or running: discarded either way
    for t in tickets[:-1]:
        ctx.wait(t)
    with pytest.raises(ept.EptError) as e:
        ctx.wait(tickets[-1])
    assert e.value.status == 6


def test_bad_request_fails_alone(ctx, ept):
    reqs = _requests(6, seed=14)
    bad = dict(reqs[2])
    bad["X"] = bad["X"].copy()
    bad["X"][0, 0] = np.nan
    reqs[2] = bad
    tickets = [ctx.submit(q["X"], q["Y"], B=q["B"], seed=q["seed"], stat=q["stat"], sigma=q["sigma"]) for q in reqs]
    for k, (q, t) in enumerate(zip(reqs, tickets)):
        if k == 2:
            with pytest.raises(ept.EptError) as e:
                ctx.wait(t)
            assert e.value.status == 1
        else:
            r = ctx.wait(t)
            alone = ctx.test(q["X"], q["Y"], B=q["B"], seed=q["seed"], stat=q["stat"], sigma=q["sigma"])
            assert abs(r.observed - alone.observed) <= REL_TOL * abs(alone.observed)


def test_budget(ept):
    small = ept.Context(0, budget_bytes=64 << 20)
    try:
        X, Y = workloads.gaussian_pair(workloads.HIGHDIM)
        with pytest.raises(ept.EptError) as e:
            small.submit(X, Y, B=10000)     # needs far more than 64 MiB of scratch
        assert e.value.status == 2
        # small requests are queued and run within the budget, a few batches at a time
        reqs = _requests(30, seed=15, max_n=400, max_B=300)
        tickets = [small.submit(q["X"], q["Y"], B=q["B"], seed=q["seed"], stat=q["stat"], sigma=q["sigma"])
                   for q in reqs]
        for q, t in zip(reqs, tickets):
            r = small.wait(t)
            alone = small.test(q["X"], q["Y"], B=q["B"], seed=q["seed"], stat=q["stat"], sigma=q["sigma"])
            assert abs(r.observed - alone.observed) <= REL_TOL * abs(alone.observed)
    finally:
        small.close()


def test_destroy_with_requests_in_flight(ept):
    c = ept.Context(0)
    X, Y = workloads.gaussian_pair(workloads.SMALL)
    for k in range(20):
        c.submit(X, Y, B=2000, seed=k)
    c.close()                            # stops the scheduler, drains running batches, frees everything


def test_injected_allocation_failures_leave_no_leaks(ept):
    # host-side fault injection: the next scratch acquisitions fail with EPT_ENOMEM;
    # the context keeps working and the serving state drains back to zero
    c = ept.Context(0)
    try:
        X, Y = workloads.gaussian_pair(workloads.SMALL)
        c.set_option("fault_inject_alloc", 1)
        with pytest.raises(ept.EptError) as e:
            c.test(X, Y, B=100, seed=1)
        assert e.value.status == 2
        alone = c.test(X, Y, B=100, seed=1)
        c.set_option("serve_lanes", 1)
        c.set_option("fault_inject_alloc", 1)
        t1 = c.submit(X, Y, B=100, seed=1)
        with pytest.raises(ept.EptError) as e:
            c.wait(t1)
        assert e.value.status == 2
        t2 = c.submit(X, Y, B=100, seed=1)
        r2 = c.wait(t2)
        assert abs(r2.observed - alone.observed) <= REL_TOL * abs(alone.observed)
        a, b = np.asarray(r2.stats), np.asarray(alone.stats)
        assert np.max(np.abs(a - b) / np.abs(b)) <= REL_TOL
        assert c.serving_stats() == {"bytes_in_use": 0, "running": 0, "queued": 0, "finished": 0}
    finally:
        c.close()


def test_serving_stats_while_busy(ctx):
    X, Y = workloads.gaussian_pair(workloads.HIGHDIM)
    tickets = [ctx.submit(X, Y, B=10000, seed=k) for k in range(6)]
    st = ctx.serving_stats()
    assert st["running"] + st["queued"] + st["finished"] >= 1
    for t in tickets:
        ctx.wait(t)
    st = ctx.serving_stats()
    assert st["running"] == 0 and st["queued"] == 0 and st["bytes_in_use"] == 0
