"""The rounding-envelope rule used to compare FP64 results with the oracle."""
import numpy as np
import pytest

from parity import check_counts, count_spread, image_bound, perturb


def test_perturbation_is_a_few_ulps():
    v = np.linspace(0.5, 2.0, 100).reshape(10, 10)
    d = np.abs(perturb(v, 1) / v - 1.0)
    assert 0 < d.max() < 1e-14


def test_counts_within_the_runs_largest_spread_plus_one_pass():
    ref = [10, 20, 30]
    spread = count_spread(ref, [[10, 21, 30], [10, 20, 28]])
    assert spread == [0, 1, 2]
    check_counts([13, 17, 33], ref, spread)   # bound 3 at every step


@pytest.mark.parametrize("gpu", [[14, 20, 30], [10, 16, 30], [10, 20, 34]])
def test_counts_outside_the_bound_fail(gpu):
    with pytest.raises(AssertionError):
        check_counts(gpu, [10, 20, 30], [0, 1, 2])


def test_zero_envelope_requires_identical_counts():
    # perturbed runs that agree with the oracle at every step leave no slack
    check_counts([10, 20, 30], [10, 20, 30], [0, 0, 0])
    with pytest.raises(AssertionError):
        check_counts([10, 21, 30], [10, 20, 30], [0, 0, 0])


def test_heldout_runs_of_the_stored_sweep_pass_the_rule():
    """The measurement behind the rule: each perturbed oracle run of the stored 256 x 256 sweep, held
    out in turn, lies within the bound computed from the other perturbed runs."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "config2_oracle.json")
    runs = json.load(open(path))["runs"]
    for r in runs:
        ref, pert = r["inner_iters"], r["perturbed_iters"]
        assert len(pert) >= 6
        for h in range(len(pert)):
            others = [p for j, p in enumerate(pert) if j != h]
            check_counts(pert[h], ref, count_spread(ref, others))


def test_image_bound_scales_with_spread():
    ref = np.ones((4, 4))
    assert image_bound(ref, [ref + 1e-9]) == pytest.approx(10 * 1e-9 * 4 / 4, rel=1e-6)
    assert image_bound(ref, [ref]) == 1e-12
