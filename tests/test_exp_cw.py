"""The FP32 exponential the block builds use for kernel values (exp_cw in
csrc/ept_internal.cuh: Cody and Waite's range reduction and a degree-8 Taylor
polynomial), compiled for the host from the same header and checked against FP64
exp: at most 2 ulp anywhere on [-87, 0], and no smooth bias -- over narrow argument
windows (the spread of the entries of one block) the mean signed error is a small
fraction of an ulp, so that it averages out of block sums instead of shifting them."""
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SRC = r'''
#include <cmath>
#include <cstdio>
#include "ept_internal.cuh"
int main(int argc, char **argv) {
    const double lo = atof(argv[1]), hi = atof(argv[2]);
    const long n = atol(argv[3]);
    double max_ulp = 0.0, sum = 0.0;
    for (long i = 0; i < n; ++i) {
        const float x = (float)(lo + (hi - lo) * (i + 0.5) / n);
        const float y = ept::exp_cw(x);
        const double t = std::exp((double)x);
        const double ulp = std::ldexp(1.0, std::ilogb((float)t) - 23);
        const double e = ((double)y - t) / ulp;
        if (std::fabs(e) > max_ulp) max_ulp = std::fabs(e);
        sum += e;
    }
    printf("%.6f %.6f\n", max_ulp, sum / n);
    return 0;
}
'''


@pytest.fixture(scope="module")
def prog(tmp_path_factory):
    d = tmp_path_factory.mktemp("expcw")
    src = d / "exp_cw_check.cu"
    src.write_text(SRC)
    exe = d / "exp_cw_check"
    nvcc = os.environ.get("NVCC", "nvcc")
    inc = os.path.join(ROOT, "paper_2406_06488_gb300", "csrc")
    try:
        subprocess.run([nvcc, "-O2", "-std=c++17", "-I" + inc, "-o", str(exe), str(src)], check=True,
                       capture_output=True)
    except (OSError, subprocess.CalledProcessError) as e:
        pytest.skip("nvcc not usable here: %s" % e)
    return str(exe)


def _run(exe, lo, hi, n):
    out = subprocess.run([exe, repr(lo), repr(hi), str(n)], check=True, capture_output=True, text=True).stdout
    max_ulp, mean = (float(v) for v in out.split())
    return max_ulp, mean


def test_error_bound_on_the_whole_range(prog):
    max_ulp, _ = _run(prog, -87.0, 0.0, 2_000_000)
    assert max_ulp <= 2.0


@pytest.mark.parametrize("lo,hi", [(-0.05, -0.03), (-0.6, -0.4), (-1.2, -0.9), (-4.0, -3.5), (-12.0, -11.0)])
def test_no_smooth_bias_over_narrow_windows(prog, lo, hi):
    max_ulp, mean = _run(prog, lo, hi, 400_000)
    assert max_ulp <= 2.0
    assert abs(mean) <= 0.05, mean
