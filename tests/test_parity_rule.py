"""The rounding-envelope rule used to compare FP64 results with the oracle."""
import numpy as np
import pytest

from parity import check_counts, count_spread, image_bound, perturb


def test_perturbation_is_a_few_ulps():
    v = np.linspace(0.5, 2.0, 100).reshape(10, 10)
    d = np.abs(perturb(v, 1) / v - 1.0)
    assert 0 < d.max() < 1e-14


def test_counts_within_spread_plus_one_pass():
    ref = [10, 20, 30]
    spread = count_spread(ref, [[10, 21, 30], [10, 20, 29]])
    assert spread == [0, 1, 1]
    check_counts([11, 22, 31], ref, spread)


@pytest.mark.parametrize("gpu", [[13, 20, 30], [10, 23, 30], [10, 20, 27]])
def test_counts_outside_spread_fail(gpu):
    with pytest.raises(AssertionError):
        check_counts(gpu, [10, 20, 30], [0, 1, 0])


def test_count_bound_is_the_runs_largest_spread():
    # a step whose own spread is 0 gets the run's largest spread (2) plus one
    check_counts([13, 20, 30], [10, 20, 30], [0, 2, 0])
    with pytest.raises(AssertionError):
        check_counts([14, 20, 30], [10, 20, 30], [0, 2, 0])


def test_image_bound_scales_with_spread():
    ref = np.ones((4, 4))
    assert image_bound(ref, [ref + 1e-9]) == pytest.approx(10 * 1e-9 * 4 / 4, rel=1e-6)
    assert image_bound(ref, [ref]) == 1e-12
