"""The run planner of libept checked on the host alone (ept_plan_check, no GPU): its
geometry against closed forms of the packed upper storage (row panels of 256, K-blocks
of 64, chunks of at most unit_kb K-blocks that stop at the last K-block with real
columns, tiles of 256 relabelings, two row halves), the balance of the contraction
schedule, the streaming windows, agreement with ept_estimate_bytes, and the
argument checks.  The library's own invariant checks (the schedule covers every unit
once; windows cover the panels once, in order, within capacity) run inside each call."""
import math

import pytest

from paper_2406_06488_gb300 import ept, workloads


def _closed_form(nx, ny, B, unit_kb):
    n = nx + ny
    NP = math.ceil(n / 256)
    NKB = 4 * NP
    real_kb = math.ceil(n / 64)
    stored = sum(NKB - 4 * I for I in range(NP))
    chunks = sum(math.ceil((real_kb - 4 * I) / unit_kb) for I in range(NP))
    MT = math.ceil((B + 1) / 256)
    return dict(stored_blocks=stored, chunks=chunks, units=chunks * MT * 2, partials=2 * chunks)


@pytest.mark.parametrize("nx,ny,p,B", [(1, 1, 1, 0), (2, 3, 5, 255), (255, 1, 7, 256), (256, 256, 64, 1000),
                                       (2000, 3000, 1000, 10000), (10000, 10000, 100, 10000), (700, 5, 3, 70000)])
@pytest.mark.parametrize("unit_kb", [4, 8, 16, 32])
def test_geometry_matches_closed_forms(nx, ny, p, B, unit_kb):
    info = ept.plan_check([(nx, ny, p, B)], unit_kb=unit_kb)
    want = _closed_form(nx, ny, B, unit_kb)
    for k, v in want.items():
        assert info[k] == v, (k, info[k], v)
    assert info["windows"] == 0


def test_scratch_agrees_with_the_estimate():
    for nx, ny, p, B in [(100, 100, 10, 1000), (2000, 3000, 1000, 10000), (10000, 10000, 100, 10000)]:
        assert ept.plan_check([(nx, ny, p, B)])["scratch_bytes"] >= ept.estimate_bytes(nx, ny, p, B)


@pytest.mark.parametrize("shapes", [
    [(2000, 3000, 1000, 10000)],
    [(10000, 10000, 100, 10000)],
    [(s.nx, s.ny, s.p, s.B) for s in workloads.batched_specs(512)],
])
def test_schedule_is_balanced(shapes):
    info = ept.plan_check(shapes, num_sms=152)
    # sorted by length and dealt in snake order: the busiest CTA has at most about one
    # unit more than the least busy one
    assert info["cta_kblocks_max"] - info["cta_kblocks_min"] <= 16
    total = sum(_closed_form(nx, ny, B, 8)["units"] for nx, ny, _, B in shapes)
    assert info["units"] == total


def test_fewer_ctas_than_units_and_more():
    small = ept.plan_check([(10, 10, 3, 10)], num_sms=152)     # 2 units over 152 SMs: 2 CTAs
    assert small["units"] == 2 and small["cta_kblocks_min"] == small["cta_kblocks_max"] == 1
    one = ept.plan_check([(2000, 3000, 1000, 10000)], num_sms=1)
    assert one["cta_kblocks_max"] == one["cta_kblocks_min"]


@pytest.mark.parametrize("blocks", [1, 60, 200, 10 ** 9])
def test_streaming_windows(blocks):
    nx, ny = 1400, 1600
    NP = math.ceil((nx + ny) / 256)
    info = ept.plan_check([(nx, ny, 24, 700)], stream_blocks=blocks)
    want = _closed_form(nx, ny, 700, 8)
    assert info["units"] == want["units"] and info["stored_blocks"] == want["stored_blocks"]
    if blocks == 1:
        assert info["windows"] == NP            # one panel per window
    elif blocks >= want["stored_blocks"]:
        assert info["windows"] == 1
    else:
        assert 1 < info["windows"] <= NP
    resident = ept.plan_check([(nx, ny, 24, 700)])
    if info["windows"] > 1:
        assert info["scratch_bytes"] < resident["scratch_bytes"]


def test_streaming_large_test_fits_its_windows():
    # n = 60,000 in windows of at most 8000 blocks (the streaming profile's case)
    info = ept.plan_check([(30000, 30000, 8, 10000)], stream_blocks=8000)
    assert info["windows"] == 15 and info["stored_blocks"] == 110920


@pytest.mark.parametrize("shapes,kw", [
    ([], {}),
    ([(0, 5, 3, 10)], {}),
    ([(5, 5, 0, 10)], {}),
    ([(5, 5, (1 << 30) + 1, 10)], {}),
    ([(5, 5, 3, -1)], {}),
    ([(5, 5, 3, (1 << 31) + 1)], {}),
    ([(1 << 21, (1 << 21) + 1, 1, 1)], {}),
    ([(5, 5, 3, 10)], {"unit_kb": 0}),
    ([(5, 5, 3, 10)], {"num_sms": 0}),
    ([(5, 5, 3, 10), (6, 6, 3, 10)], {"stream_blocks": 4}),
])
def test_bad_arguments(shapes, kw):
    with pytest.raises(ept.EptError) as e:
        ept.plan_check(shapes, **kw)
    assert e.value.status == 1   # EPT_EINVAL
