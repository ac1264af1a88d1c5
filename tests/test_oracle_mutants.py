"""The pins have teeth: copies of the oracle with one planted mistake each (compiled
with the test-only switch EO_MUTANT) must fail at least one pin, while the oracle
itself passes them all (test_oracle_pins.py)."""
import numpy as np
import pytest

import oracle
import test_oracle_pins as pins

# each mutant: what it plants, and the pins that are expected to notice
MUTANTS = {
    1: ("Philox key not bumped between rounds", [pins.test_philox_known_answers]),
    2: ("selection sampling keeps slot when r <= need",
        [lambda: pins.test_stream_exact_count(37, 64)]),
    3: ("Gaussian kernel exp(-d^2/sigma^2)", [pins.test_distances_match_library_routine]),
    4: ("cross term 2/(nx nx) (the Algorithm 4/5 typo)", [lambda: pins.test_ed_p1_closed_form(300, 200)]),
    5: ("V-statistic diagonal dropped", [lambda: pins.test_three_implementations_agree("mmd", 7, 11, 3)]),
    6: ("block swap reads D_XY untransposed",
        [lambda: pins.test_block_swap_equals_recomputation_on_worked_example("ed")]),
    7: ("p-value without the +1 terms", [pins.test_pvalue_definition]),
    8: ("Laplacian kernel exp(-d^2/sigma)", [pins.test_laplace_kernel_matches_library_routine]),
    9: ("single-relabeling statistic skips the first y* row in the cross sum",
        [lambda: pins.test_stat_select_matches_recomputation("ed", 7, 11, 1)]),
    10: ("pooled trace taken along the first super-diagonal",
         [lambda: pins.test_pooled_moments_match_library_routine("mmd")]),
    11: ("exhaustive enumeration writes each index set mirrored",
         [lambda: pins.test_exhaustive_order_is_lexicographic(3, 5)]),
    12: ("permutation mean with pair inclusion (nx/n)^2",
         [lambda: pins.test_permutation_mean_equals_exhaustive_mean("ed")]),
}


@pytest.mark.parametrize("k", sorted(MUTANTS))
def test_mutant_is_caught(k):
    path = oracle.build_mutant(k)
    oracle.use_library(path)
    try:
        failures = 0
        for pin in MUTANTS[k][1]:
            try:
                pin()
            except AssertionError:
                failures += 1
        assert failures >= 1, "mutant %d (%s) passed its pins" % (k, MUTANTS[k][0])
    finally:
        oracle.use_library(None)
    # and the real oracle still passes the same pins
    for pin in MUTANTS[k][1]:
        pin()
