"""Where the statistic-level error of ill-conditioned tests comes from, shown with a
plain CPU model of the contraction's arithmetic (no GPU): the quadratic form s'Cs of
the centred pooled matrix (the form Algorithm 1's block sums reduce to), with

  * C rounded to FP32 and everything summed in FP64: the blocks' own precision;
  * C rounded to FP32 and each row summed in FP32 over units of 512 columns, the
    masked row sums added in FP32 over 128 rows, and the unit sums in FP64: the
    order and precision of the GPU contraction's accumulation.

A wide Gaussian kernel over one feature makes C nearly of rank one, so the FP32 row
sums of a unit carry roundings that do not average out across rows: the second
model loses an order of magnitude or more to the first, which stays within 1e-5.
A well-conditioned ED test loses nothing noticeable either way."""
import numpy as np

import oracle
from paper_2406_06488_gb300 import workloads

UNIT = 512
ROWS = 128


def _forms(X, Y, stat, sigma, seed, nperm=8):
    nx, ny = len(X), len(Y)
    Z = np.vstack([X, Y])
    W = oracle.block_matrix(Z, Z, stat, sigma)
    u = W.mean(1) - W.mean() / 2          # double centring: the statistic ignores W -> W - u1' - 1u'
    C = W - u[:, None] - u[None, :]
    C32 = C.astype(np.float32)
    e_blocks, e_accum = [], []
    for s in oracle.perm_select(seed, nx, ny, 1, nperm).astype(bool):
        sv = s.astype(np.float64)
        exact = sv @ C @ sv
        f = s.astype(np.float32)
        tot = 0.0
        for j0 in range(0, nx + ny, UNIT):
            rows = np.cumsum(C32[:, j0:j0 + UNIT] * f[None, j0:j0 + UNIT], axis=1, dtype=np.float32)[:, -1]
            for i0 in range(0, nx + ny, ROWS):
                tot += float(np.cumsum(rows[i0:i0 + ROWS] * f[i0:i0 + ROWS], dtype=np.float32)[-1])
        e_blocks.append(abs(sv @ C32.astype(np.float64) @ sv - exact) / abs(exact))
        e_accum.append(abs(tot - exact) / abs(exact))
    return max(e_blocks), max(e_accum)


def test_wide_kernel_few_features_loses_digits_in_fp32_accumulation():
    X, Y = workloads.gaussian_pair(workloads.TwoSampleSpec(nx=700, ny=600, p=1, y_mean=0.5, y_var=1.3,
                                                           data_seed=77))
    e_blocks, e_accum = _forms(X, Y, "mmd", 3.0, seed=5)
    assert e_blocks <= 1e-5
    assert e_accum > 10 * e_blocks and e_accum > 1e-5


def test_well_conditioned_ed_keeps_its_digits():
    X, Y = workloads.gaussian_pair(workloads.TwoSampleSpec(nx=700, ny=600, p=50, y_mean=0.1, data_seed=78))
    e_blocks, e_accum = _forms(X, Y, "ed", 1.0, seed=5)
    assert e_blocks <= 1e-7 and e_accum <= 1e-6
