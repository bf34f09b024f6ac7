"""The near-tie rule used to compare FP64 iteration counts with the oracle."""
import pytest

from parity import compare_counts


def test_equal_counts_have_no_tie():
    assert compare_counts([3, 4, 5], [3, 4, 5], [[1e-5, 9e-7]] * 3, 1e-6, 1e-2) is None


def test_off_by_one_at_a_near_tie_is_accepted():
    tails = [[2e-6, 5e-7], [1.7e-6, 0.9989e-6], [1.5e-6, 8e-7]]
    assert compare_counts([3, 50, 7], [3, 49, 8], tails, 1e-6, 1e-2) == 1


@pytest.mark.parametrize("gpu,ref", [([3, 48, 7], [3, 46, 7]), ([3, 50, 7], [3, 49, 7])])
def test_mismatch_away_from_tol_fails(gpu, ref):
    tails = [[2e-6, 5e-7], [1.7e-6, 0.5e-6], [1.5e-6, 8e-7]]
    with pytest.raises(AssertionError):
        compare_counts(gpu, ref, tails, 1e-6, 1e-2)
