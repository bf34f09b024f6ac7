"""Pins of the oracle's functional and of its Newton finish of the fixed point.

* ``tv_functional`` (eq. (mp) discretised, data term 1/2 ||H u - v||^2) is the
  function whose gradient is ``euler_lagrange`` (eq. (el)): checked pixel by
  pixel by central differences, so a wrong weight on either term fails.
* ``newton_polish`` (Newton on g(u) = 0, not a step of the paper) must land on
  the limit of the paper's own FP iteration run to convergence, make g vanish,
  be a minimiser of the functional, and converge quadratically.
"""
import numpy as np
import pytest

import oracle as O
from paper_1011_5964_gb300 import synth


def _problem(n, bc, seed=5, sigma=1.2, m=2, noise=0.01):
    u_true = synth.piecewise_constant_image(n, n, seed=seed)
    h = synth.gaussian_psf(sigma, half_width=m)
    v = synth.add_noise(O.blur(u_true, h, bc), synth.noise_direction(n, n, seed), noise)
    return h, u_true, v


@pytest.mark.parametrize("bc", [O.AR, O.R])
def test_functional_gradient_is_the_euler_lagrange_residual(bc):
    rng = np.random.default_rng(31)
    h, _, v = _problem(7, bc)
    u = rng.uniform(0.0, 1.0, v.shape)
    alpha, beta, eps = 0.07, 0.2, 1e-6
    g = O.euler_lagrange(u, v, h, bc, alpha, beta)
    fd = np.zeros_like(u)
    for i in range(u.shape[0]):
        for j in range(u.shape[1]):
            e = np.zeros_like(u)
            e[i, j] = eps
            fd[i, j] = (O.tv_functional(u + e, v, h, bc, alpha, beta)
                        - O.tv_functional(u - e, v, h, bc, alpha, beta)) / (2 * eps)
    np.testing.assert_allclose(g, fd, rtol=0, atol=1e-8 * np.abs(g).max())


def test_functional_data_weight_is_one_half():
    """alpha = 0: T(u) = 1/2 ||H u - v||^2 exactly, so T(v + d) - T(v) is fixed by H alone."""
    h, _, v = _problem(6, O.AR)
    d = np.full(v.shape, 0.25)
    # AR blur reproduces constants (rows of H sum to sum(h) = 1): H d = d
    hd = O.blur(d, h, O.AR)
    assert np.allclose(hd, d, atol=1e-13)
    hv = O.blur(v, h, O.AR)
    assert O.tv_functional(v, hv, h, O.AR, 0.0, 1.0) == pytest.approx(0.0, abs=1e-24)
    got = O.tv_functional(v + d, hv, h, O.AR, 0.0, 1.0)
    assert got == pytest.approx(0.5 * 0.25 ** 2 * v.size, rel=1e-12)


def _fp_limit(v, h, bc, alpha, beta):
    u, st = O.tv_deblur(v, h, bc, alpha, beta, outer=4000, tol=1e-14, maxit=5000, kind=O.PC_NONE,
                        outer_tol=1e-15)
    return u


@pytest.mark.parametrize("bc", [O.AR, O.R])
def test_newton_polish_lands_on_the_fp_limit(bc):
    h, _, v = _problem(12, bc)
    alpha, beta = 0.05, 0.1
    u_fp = _fp_limit(v, h, bc, alpha, beta)
    u3, _ = O.tv_deblur(v, h, bc, alpha, beta, outer=3, tol=1e-10, maxit=5000)
    u_nt, st = O.newton_polish(u3, v, h, bc, alpha, beta, tol=1e-12)
    assert st["converged"]
    assert np.linalg.norm(u_nt - u_fp) <= 1e-10 * np.linalg.norm(u_fp)
    b = O.blur_adjoint(v, h, bc)
    assert st["g_norm_final"] <= 1e-12 * np.linalg.norm(b)
    assert np.linalg.norm(O.euler_lagrange(u_nt, v, h, bc, alpha, beta)) == pytest.approx(st["g_norm_final"],
                                                                                          rel=1e-9, abs=1e-300)


def test_newton_polish_minimises_the_functional():
    h, _, v = _problem(10, O.AR, seed=8)
    alpha, beta = 0.02, 0.05
    u3, _ = O.tv_deblur(v, h, O.AR, alpha, beta, outer=3, tol=1e-10, maxit=5000)
    u, st = O.newton_polish(u3, v, h, O.AR, alpha, beta, tol=1e-13)
    assert st["converged"]
    f0 = O.tv_functional(u, v, h, O.AR, alpha, beta)
    rng = np.random.default_rng(4)
    for _ in range(6):
        d = rng.standard_normal(u.shape)
        d /= np.linalg.norm(d)
        for eps in (1e-2, 1e-4):
            assert O.tv_functional(u + eps * d, v, h, O.AR, alpha, beta) > f0
            assert O.tv_functional(u - eps * d, v, h, O.AR, alpha, beta) > f0


def test_newton_polish_converges_quadratically():
    """Once steps are full and small, each relative change is at most C times the
    square of the previous one; the FP iteration's linear rate would not pass."""
    h, _, v = _problem(24, O.AR, seed=3, sigma=1.5, m=3)
    alpha, beta = 1e-3, 1e-2
    u5, _ = O.tv_deblur(v, h, O.AR, alpha, beta, outer=5, tol=1e-10, maxit=5000)
    _, st = O.newton_polish(u5, v, h, O.AR, alpha, beta, tol=1e-14)
    assert st["converged"]
    ch, t = st["rel_change"], st["t"]
    pairs = [(ch[k], ch[k + 1]) for k in range(len(ch) - 1)
             if t[k] == 1.0 and t[k + 1] == 1.0 and ch[k] < 1e-4 and ch[k + 1] > 1e-13]
    assert pairs, ch
    for a, b in pairs:
        assert b <= 1e4 * a * a, (a, b, ch)


def test_newton_polish_at_a_stationary_point_takes_no_step():
    h, _, v = _problem(8, O.R, seed=2)
    alpha, beta = 0.05, 0.1
    u = _fp_limit(v, h, O.R, alpha, beta)
    u2, st = O.newton_polish(u, v, h, O.R, alpha, beta, tol=1e-9)
    assert st["converged"] and len(st["rel_change"]) <= 1
    assert np.linalg.norm(u2 - u) <= 1e-12 * np.linalg.norm(u)


def test_newton_stats_count_the_cg_iterations():
    """The reported CG iterations of each Newton step are those of its Jacobian solve."""
    h, _, v = _problem(12, O.AR)
    alpha, beta = 0.05, 0.1
    u3, _ = O.tv_deblur(v, h, O.AR, alpha, beta, outer=3, tol=1e-10, maxit=5000)
    _, st = O.newton_polish(u3, v, h, O.AR, alpha, beta, tol=1e-12, kind=O.PC_NONE)
    g = O.euler_lagrange(u3, v, h, O.AR, alpha, beta)
    _, k, _, _ = O.adjoint_solve(u3, h, O.AR, alpha, beta, g, 1e-12, 20000, O.PC_NONE)
    assert st["cg_iters"][0] == k and k > 10
