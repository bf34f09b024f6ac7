"""Host-side pieces of the autograd wrapper (no GPU): the Gaussian PSF parameterisation."""
import numpy as np

from paper_1011_5964_gb300 import synth
from paper_1011_5964_gb300.autograd import gaussian_taps


def test_gaussian_taps_equal_the_input_generator():
    for sigma, m in [(1.0, 3), (2.0, 8), (2.5, 8)]:
        h, _ = gaussian_taps(sigma, m)
        assert np.abs(h - synth.gaussian_psf(sigma, half_width=m)).max() < 1e-15


def test_gaussian_tap_derivative_matches_central_differences():
    for sigma, m in [(1.3, 4), (2.0, 8)]:
        _, dh = gaussian_taps(sigma, m)
        e = 1e-6
        fd = (gaussian_taps(sigma + e, m)[0] - gaussian_taps(sigma - e, m)[0]) / (2 * e)
        assert np.abs(dh - fd).max() < 1e-8 * np.abs(fd).max()
        assert abs(dh.sum()) < 1e-14   # the taps stay normalised
