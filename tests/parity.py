"""Comparison rules shared by the GPU parity tests.

CG residual trajectories are sensitive to rounding: the FP64 oracle itself,
run on x86 and on Arm numpy builds, gives relative residuals that differ by a
few percent after ~50 iterations, and stopping decisions near the tolerance
can go either way. The plain FP64 GPU path is therefore held to the oracle's
own rounding envelope: the oracle is re-run with every product with A and
every preconditioner output multiplied by (1 + 2^-50 xi), xi standard normal
(a few units in the last place, fresh noise each time: a model of rounding
that differs from numpy's in every operation), and the GPU result must lie as
close to the unperturbed oracle run as those runs do: iteration counts within
their largest per-step spread plus one, images within ten times their spread. Where the
perturbed runs agree exactly this is identical counts and images within
1e-12 relative (plus rounding).
"""
import numpy as np

EPS = 2.0 ** -50
N_PERTURBED = 3


def noise(j):
    """The oracle's noise hook for perturbed run j: (generator, relative size)."""
    return (np.random.default_rng(10_000 + j), EPS)


def perturb(v, j):
    """v (1 + 2^-50 xi), xi standard normal with seed j (input-only perturbation)."""
    rng = np.random.default_rng(10_000 + j)
    return np.asarray(v, dtype=np.float64) * (1.0 + EPS * rng.standard_normal(np.shape(v)))


def count_spread(ref, perturbed):
    """Per-step max |perturbed - ref| of the iteration counts."""
    return [max(abs(p[k] - ref[k]) for p in perturbed) for k in range(len(ref))]


def check_counts(gpu, ref, spread, slack=1):
    """Every step's count within the run's largest per-step spread plus slack.

    Three perturbed runs estimate the spread of each step poorly (a step can
    show 0 where its neighbours show 2); the operator, and so the sensitivity
    of the counts to rounding, is the same in every step of a run, so the
    largest spread over the steps bounds each of them.
    """
    assert len(gpu) == len(ref), (gpu, ref)
    bound = max(spread) + slack
    for k in range(len(ref)):
        assert abs(gpu[k] - ref[k]) <= bound, (k, gpu, ref, spread)


def image_bound(ref, perturbed_images, floor=1e-12):
    """Ten times the largest relative distance of a perturbed run from the reference run."""
    nr = np.linalg.norm(ref)
    spread = max(np.linalg.norm(p - ref) / nr for p in perturbed_images)
    return max(10.0 * spread, floor)
