"""Seeded synthetic workloads for TV deblurring (inputs only).

This module draws the inputs that every side of the library uses: the
piecewise-constant ground truth, the symmetric point-spread functions and the
noise direction. It holds none of the deblurring arithmetic: blurring the
ground truth and scaling the noise to a given noise-to-signal ratio are left to
the caller, who applies its own blur operator and then ``add_noise``.

The workload shapes follow the paper's experiments (Sec. 5): a piecewise
constant true object (the paper's figures are not available, so shapes are
drawn at random), a symmetric out-of-focus (flat disk) or Gaussian PSF
normalised to sum 1 (Sec. 2, normalisation of the PSF; Sec. 5.1, eq. (of)),
and white Gaussian noise scaled so that ||eta||_2 / ||H u||_2 equals the noise
level (Sec. 5.1).

Only numpy is used, so the module imports on any host.
"""
from __future__ import annotations

import math

import numpy as np


def piecewise_constant_image(n_rows: int, n_cols: int, seed: int, n_shapes: int = 8) -> np.ndarray:
    """Piecewise-constant test object of shape (n_rows, n_cols), float64.

    Background intensity U[0,1]; then ``n_shapes`` shapes painted in order,
    each an axis-aligned rectangle or a disk with probability 1/2 and intensity
    U[0,1]. Rectangle: top-left corner uniform over the image, sides
    U[n/16, n/3] (clipped at the border). Disk: centre uniform, radius
    U[n/32, n/6]. Shapes may touch the border so that the boundary conditions
    matter.
    """
    rng = np.random.default_rng(seed)
    n = min(n_rows, n_cols)
    img = np.full((n_rows, n_cols), rng.uniform(0.0, 1.0), dtype=np.float64)
    rr, cc = np.meshgrid(np.arange(n_rows), np.arange(n_cols), indexing="ij")
    for _ in range(n_shapes):
        kind = rng.uniform() < 0.5
        val = rng.uniform(0.0, 1.0)
        if kind:
            r0 = int(rng.integers(0, n_rows))
            c0 = int(rng.integers(0, n_cols))
            hr = max(1, int(round(rng.uniform(n / 16.0, n / 3.0))))
            wc = max(1, int(round(rng.uniform(n / 16.0, n / 3.0))))
            img[r0:r0 + hr, c0:c0 + wc] = val
        else:
            cr = rng.uniform(0, n_rows)
            ccn = rng.uniform(0, n_cols)
            rad = rng.uniform(n / 32.0, n / 6.0)
            mask = (rr + 0.5 - cr) ** 2 + (cc + 0.5 - ccn) ** 2 <= rad * rad
            img[mask] = val
    return img


def gaussian_psf(sigma: float, half_width: int | None = None) -> np.ndarray:
    """Normalised isotropic Gaussian PSF, side 2m+1 with m = ceil(3 sigma) by default.

    h[m+a, m+b] proportional to exp(-(a^2+b^2) / (2 sigma^2)), sum 1. It is
    quadrantally symmetric and exactly rank one.
    """
    m = int(math.ceil(3.0 * sigma)) if half_width is None else int(half_width)
    a = np.arange(-m, m + 1, dtype=np.float64)
    g = np.exp(-(a * a) / (2.0 * sigma * sigma))
    h = np.outer(g, g)
    return h / h.sum()


def disk_psf(radius: float, side: int | None = None) -> np.ndarray:
    """Normalised out-of-focus (flat disk) PSF.

    Non-zero where a^2 + b^2 <= radius^2 (radius 7 gives 149 taps), zero padded
    to ``side`` x ``side`` (default 2*ceil(radius)+1), normalised to sum 1. The
    1D analogue is the paper's out-of-focus PSF of Sec. 5.1.
    """
    r = int(math.floor(radius))
    s = 2 * r + 1 if side is None else int(side)
    if s % 2 == 0 or s < 2 * r + 1:
        raise ValueError("disk PSF side must be odd and at least 2*floor(radius)+1")
    m = s // 2
    a = np.arange(-m, m + 1, dtype=np.float64)
    mask = (a[:, None] ** 2 + a[None, :] ** 2) <= radius * radius + 1e-12
    h = mask.astype(np.float64)
    return h / h.sum()


def noise_direction(n_rows: int, n_cols: int, seed: int) -> np.ndarray:
    """Standard normal field used as the noise direction (seeded, float64)."""
    rng = np.random.default_rng(seed + 7919)
    return rng.standard_normal((n_rows, n_cols))


def add_noise(blurred: np.ndarray, direction: np.ndarray, level: float) -> np.ndarray:
    """Return ``blurred + eta`` with eta = level * ||blurred|| * direction / ||direction||.

    The noise-to-signal ratio ||eta||_2 / ||blurred||_2 then equals ``level``
    exactly (up to rounding), as in the paper's experiments (Sec. 5.1).
    """
    blurred = np.asarray(blurred, dtype=np.float64)
    d = np.asarray(direction, dtype=np.float64)
    return blurred + level * np.linalg.norm(blurred) * d / np.linalg.norm(d)


def batch_items(count: int = 96, seed: int = 1000,
                sides=(128, 192, 256, 384, 512)) -> list[dict]:
    """Descriptions of a batch of independent deblurring problems.

    Item i has a side drawn uniformly from ``sides``, a Gaussian PSF with
    sigma ~ U[1,3] (half-width ceil(3 sigma)), alpha log-uniform in
    [1e-4, 1e-2], beta = 1e-2, 1% noise, and image / noise seeds seed+i.
    """
    rng = np.random.default_rng(seed)
    items = []
    for i in range(count):
        n = int(sides[int(rng.integers(0, len(sides)))])
        sigma = float(rng.uniform(1.0, 3.0))
        alpha = float(10.0 ** rng.uniform(-4.0, -2.0))
        items.append({"n": n, "sigma": sigma, "alpha": alpha, "beta": 1e-2,
                      "noise": 0.01, "seed": seed + i})
    return items


def piecewise_constant_signal(n: int, seed: int, margin: float = 0.125, n_jumps: int = 9) -> tuple[np.ndarray, slice]:
    """1D piecewise-constant signal on a support wider than the field of view.

    The paper's 1D experiment (Sec. 5.1) restores a signal on [0, 1] observed in
    the field of view [0.1, 0.9], the parts outside being left to the boundary
    conditions; its true signal is only shown in a figure, so the jumps are
    drawn at random. Returns (u_wide, fov): u_wide has n + 2 k samples, k =
    round(margin n), with ``n_jumps`` jump positions uniform over the support
    and levels U[0, 1] between them; fov = slice(k, k + n) selects the n
    samples of the field of view. Blur u_wide, then keep ``[fov]``: the
    observation then depends on the signal outside the field of view as a
    physical blur does, not on a boundary model (this needs the PSF half-width
    to be at most k).
    """
    k = int(round(margin * n))
    N = n + 2 * k
    rng = np.random.default_rng(seed)
    cuts = np.sort(rng.integers(1, N, size=n_jumps))
    levels = rng.uniform(0.0, 1.0, size=n_jumps + 1)
    u = np.empty(N)
    edges = np.concatenate([[0], cuts, [N]])
    for q in range(n_jumps + 1):
        u[edges[q]:edges[q + 1]] = levels[q]
    return u, slice(k, k + n)


def out_of_focus_psf_1d(m: int) -> np.ndarray:
    """The 1D out-of-focus PSF of eq. (of): h_i = c for |i| < m, else 0, sum 1,
    as a (1, 2m - 1) array (a PSF of one row for the 2D plans)."""
    if m < 1:
        raise ValueError("m must be at least 1")
    return np.full((1, 2 * m - 1), 1.0 / (2 * m - 1))


def alpha_grid(lo: float = 1e-6, hi: float = 1e-1, per_decade: int = 2) -> list[float]:
    """Log-spaced regularisation parameters from lo to hi (inclusive), ``per_decade``
    values per decade: the abscissa of an RRE-versus-alpha sweep (Sec. 5.1)."""
    k = int(round(math.log10(hi / lo) * per_decade))
    return [float(lo * 10.0 ** (i / per_decade)) for i in range(k + 1)]
