"""Comparison rules shared by the GPU parity tests.

Iteration counts of the FP64 GPU path and the FP64 oracle are compared step by
step. Both sides decide "stop" with the same test, ||r_k|| / ||r_0|| < tol, in
double, but their residuals differ by the rounding order of every sum, and CG
amplifies such differences over its iterations. A count may therefore differ
by one only where the oracle's relative residual at the deciding iteration
lies within a narrow band of tol (a near tie); after such a step the two
trajectories start the next FP step from iterates that differ at the level of
the tolerance, so later counts and the final image are compared more loosely.
"""


def compare_counts(gpu, ref, tails, tol, band):
    """Return the index of the first near tie, or None if every count matches.

    ``tails[k]`` holds the oracle's relative residuals after its last two
    iterations of step k. A mismatch must be by one, and one of those two
    residuals must lie within ``band`` (relative) of ``tol``.
    """
    assert len(gpu) == len(ref), (gpu, ref)
    for k, (g, r) in enumerate(zip(gpu, ref)):
        if g == r:
            continue
        assert abs(g - r) == 1, (k, gpu, ref)
        near = min(abs(t / tol - 1.0) for t in tails[k])
        assert near < band, (k, gpu, ref, tails[k])
        return k
    return None
