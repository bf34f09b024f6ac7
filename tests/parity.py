"""Comparison rules shared by the GPU parity tests.

CG residual trajectories are sensitive to rounding: the FP64 oracle itself,
run on x86 and on Arm numpy builds, gives relative residuals that differ by a
few percent after ~50 iterations, and stopping decisions near the tolerance
can go either way. The plain FP64 GPU path is therefore held to the oracle's
own rounding envelope: the oracle is re-run on inputs perturbed at the level
of a few units in the last place (relative 2^-50), and the GPU result must lie
as close to the unperturbed oracle run as those perturbed runs do (iteration
counts within their spread plus one, images within ten times their spread).
Where the perturbed runs agree exactly, this is bit-identical counts and
images within 1e-12 relative (plus rounding).
"""
import numpy as np

EPS = 2.0 ** -50
N_PERTURBED = 3


def perturb(v, j):
    """v (1 + 2^-50 xi), xi standard normal with seed j."""
    rng = np.random.default_rng(10_000 + j)
    return np.asarray(v, dtype=np.float64) * (1.0 + EPS * rng.standard_normal(np.shape(v)))


def count_spread(ref, perturbed):
    """Per-step max |perturbed - ref| of the iteration counts."""
    return [max(abs(p[k] - ref[k]) for p in perturbed) for k in range(len(ref))]


def check_counts(gpu, ref, spread, slack=1):
    assert len(gpu) == len(ref), (gpu, ref)
    for k in range(len(ref)):
        assert abs(gpu[k] - ref[k]) <= spread[k] + slack, (k, gpu, ref, spread)


def image_bound(ref, perturbed_images, floor=1e-12):
    """Ten times the largest relative distance of a perturbed run from the reference run."""
    nr = np.linalg.norm(ref)
    spread = max(np.linalg.norm(p - ref) / nr for p in perturbed_images)
    return max(10.0 * spread, floor)
