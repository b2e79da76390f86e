"""The oracle's pins catch plausible mistakes: each mutant build of the
oracle (one deliberate mistake planted on the CPU: a dropped term, a flipped
sign, a transposed operand, a wrong endpoint, an off-by-one in the overlap or
threshold test, a wrong bin origin, an ignored window, a wrong self-join
pair filter, a time sweep that prunes too much) must fail at least one pin
of tests/test_oracle_pins.py."""
import pytest

from oracle import oracle
from tests import test_oracle_pins as pins

MUTANTS = {
    1: "relative position does not change over the span (dropped term)",
    2: "sign of the linear coefficient flipped",
    3: "interpolation from the wrong endpoint",
    4: "segments touching at an instant counted as overlapping",
    5: "threshold exclusive instead of inclusive",
    6: "transposed operands in the second root",
    7: "bin index ignores the start of the extent",
    8: "query window ignored",
    9: "self-join keeps pairs of one trajectory",
    10: "self-join keeps both orders of a pair",
    11: "time sweep skips entries that start before the query segment",
}

PIN_CALLS = [
    lambda: [pins.test_stationary_point_query(f, h) for f, h in ((0.0, True), (0.5, True), (1.0 - 1e-6, True),
                                                                 (1.0 + 1e-6, False))],
    pins.test_parallel_motion_constant_offset,
    lambda: [pins.test_head_on_approach(*a) for a in ((10.0, 1.0, 2.0, 20.0), (7.5, 0.25, 0.1, 60.0),
                                                      (3.0, 2.0, 1.0, 1.6))],
    lambda: [pins.test_flyby_impact_parameter(b, d) for b, d in ((0.0, 1.0), (0.6, 1.0), (2.5, 3.0))],
    pins.test_touching_spans_are_not_pairs,
    pins.test_window_clips_the_span,
    pins.test_exact_crossing_with_zero_threshold,
    pins.test_identical_segment_is_in_range_over_its_extent,
    pins.test_invariants_on_random_pairs,
    pins.test_fig1_bin_table,
    pins.test_fig1_bin_table_time_shifted,
    pins.test_self_join_head_on_pair_once,
    lambda: [pins.test_self_join_is_the_filtered_full_search(s) for s in (1, 2)],
    pins.test_bruteforce_equals_sweep_on_random_sets,
]


@pytest.mark.parametrize("k", sorted(MUTANTS))
def test_pins_catch_mutant(k, tmp_path):
    path = oracle.build_mutant(k, str(tmp_path))
    prev = oracle.use_library(path)
    caught = []
    try:
        for call in PIN_CALLS:
            try:
                call()
            except AssertionError:
                caught.append(getattr(call, "__name__", "pin"))
    finally:
        oracle._lib = prev
    assert caught, f"no pin caught mutant {k}: {MUTANTS[k]}"


def test_unmutated_oracle_passes_the_same_pins():
    for call in PIN_CALLS:
        call()
