"""Host-side parts of bench.py that need no GPU: the two CPU baselines it reports
(direct recomputation, Algorithm 4; the paper's Algorithm 1 on the three blocks),
timed on small workloads."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2406_06488_gb300 import workloads  # noqa: E402


def _small(nx, ny, p, B):
    spec = workloads.TwoSampleSpec(nx=nx, ny=ny, p=p, y_mean=0.2, B=B, seed=3, data_seed=4)
    X, Y = workloads.gaussian_pair(spec)
    return spec, X, Y


def test_paper_method_whole_test_when_sample_reaches_B():
    spec, X, Y = _small(60, 40, 5, 50)
    r = bench._cpu_paper_method(spec, X, Y, budget_s=2.0)
    assert r["value"] > 0 and r["cores"] >= 1
    assert "whole test" in r["sample"]
    assert abs(r["value"] - spec.B / r["test_s"]) <= 1e-9 * r["value"]


def test_paper_method_extrapolates_a_bounded_sample():
    spec, X, Y = _small(600, 500, 40, 10 ** 6)
    r = bench._cpu_paper_method(spec, X, Y, budget_s=0.5)
    assert r["ms_per_relabeling"] > 0 and r["build_s"] > 0
    assert abs(r["test_s"] - (r["build_s"] + spec.B * r["ms_per_relabeling"] / 1000.0)) <= 1e-6 * r["test_s"]
    assert "extrapolated" in r["sample"]


def test_paper_method_skips_large_n():
    spec = workloads.TwoSampleSpec(nx=5000, ny=5000, p=2, B=10)
    r = bench._cpu_paper_method(spec, np.zeros((5000, 2), np.float32), np.zeros((5000, 2), np.float32))
    assert r["value"] is None and "not timed" in r["sample"]


def test_direct_baseline_counts_what_it_timed():
    spec, X, Y = _small(80, 90, 6, 100)
    r, vals = bench._cpu_baseline(spec, X, Y, budget_s=5.0)
    assert r["kind"] == "oracle" and r["value"] > 0
    assert len(vals) == 64 and all(np.isfinite(vals))


def test_tuning_code_decodes_every_choice():
    # ept_result.tuning = 10000 kernel + 100 unit + 10 draw kernel + order (include/ept.h)
    class R:
        tune_candidates = 8

    for kernel in range(4):
        for unit in (0, 4, 8, 16, 32):
            for draw in range(4):
                for order in range(3):
                    R.tuning = 10000 * kernel + 100 * unit + 10 * draw + order
                    t = bench._tuning(R)
                    assert t["unit_kblocks"] == unit and t["candidates_timed"] == 8
                    assert t["contraction"] and t["draw_kernel"] and t["unit_order"]
    R.tuning = 10000 * 2 + 100 * 16 + 10 * 3 + 2
    t = bench._tuning(R)
    assert t["contraction"].startswith("pairs of SMs") and t["draw_kernel"].startswith("rank producers")
    assert t["unit_order"] == "by first K-block"
