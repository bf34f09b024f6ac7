"""Pins of the oracle's adjoint of the converged fixed point (a11).

The Euler-Lagrange residual g(u, theta) = H^T (H u - v) + alpha L(u) u of
eq. (el) vanishes at the fixed point of the lagged-diffusivity iteration; its
Jacobian J = H^T H + alpha nabla^2 J_beta(u) gives the gradient of a loss of
u* with respect to alpha, beta and the PSF taps through J lambda = dl/du.
These tests pin that against things other than the formulas themselves:
finite differences of the TV gradient and of g, a dense solve, and above all
central finite differences of the loss with u* re-converged by the FP
iteration for every perturbed parameter.
"""
import numpy as np
import pytest

import oracle as O
from paper_1011_5964_gb300 import synth


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


@pytest.fixture(scope="module")
def rng():
    return np.random.default_rng(2024)


def test_tv_hessian_is_the_derivative_of_the_tv_gradient(rng):
    u, x = rng.standard_normal((9, 11)), rng.standard_normal((9, 11))
    beta, eps = 0.3, 1e-6
    grad = lambda z: O.tv_apply(O.diffusivity(z, beta), z)   # grad J_beta = L(u) u
    fd = (grad(u + eps * x) - grad(u - eps * x)) / (2 * eps)
    assert rel(O.tv_hessian_apply(u, beta, x), fd) < 1e-8


def test_tv_hessian_is_symmetric_positive_semidefinite(rng):
    u = rng.standard_normal((6, 7))
    n = u.size
    Hm = np.column_stack([O.tv_hessian_apply(u, 0.2, np.eye(n)[:, k].reshape(6, 7)).ravel() for k in range(n)])
    assert np.abs(Hm - Hm.T).max() < 1e-12 * np.abs(Hm).max()
    assert np.linalg.eigvalsh(0.5 * (Hm + Hm.T)).min() > -1e-12 * np.abs(Hm).max()
    # constants are in its null space (only differences enter J_beta)
    assert np.abs(O.tv_hessian_apply(u, 0.2, np.ones((6, 7)))).max() < 1e-12


@pytest.mark.parametrize("bc", [O.AR, O.R])
def test_jacobian_is_the_derivative_of_the_euler_lagrange_residual(rng, bc):
    h = synth.gaussian_psf(1.0, half_width=2)
    u, v, x = (rng.standard_normal((10, 9)) for _ in range(3))
    alpha, beta, eps = 0.05, 0.2, 1e-6
    g = lambda z: O.euler_lagrange(z, v, h, bc, alpha, beta)
    fd = (g(u + eps * x) - g(u - eps * x)) / (2 * eps)
    assert rel(O.jacobian_apply(u, h, bc, alpha, beta, x), fd) < 1e-7


def test_adjoint_solve_matches_a_dense_solve(rng):
    h = synth.gaussian_psf(1.0, half_width=2)
    u, rhs = rng.standard_normal((7, 8)), rng.standard_normal((7, 8))
    alpha, beta = 0.05, 0.2
    n = u.size
    J = np.column_stack([O.jacobian_apply(u, h, O.AR, alpha, beta, np.eye(n)[:, k].reshape(7, 8)).ravel()
                         for k in range(n)])
    lam, it, rr, ok = O.adjoint_solve(u, h, O.AR, alpha, beta, rhs, tol=1e-13)
    assert ok
    assert rel(lam.ravel(), np.linalg.solve(J, rhs.ravel())) < 1e-10


def _problem(bc):
    nr, nc = 10, 12
    h = synth.gaussian_psf(1.0, half_width=2)
    ut = synth.piecewise_constant_image(nr, nc, seed=5)
    v = synth.add_noise(O.blur(ut, h, bc), synth.noise_direction(nr, nc, 5), 0.02)
    return h, ut, v


def _ustar(v, h, bc, alpha, beta):
    u, st = O.tv_deblur(v, h, bc, alpha, beta, outer=2000, tol=1e-14, maxit=5000, kind=O.PC_NONE, outer_tol=1e-15)
    return u


@pytest.mark.parametrize("bc,params", [(O.AR, ("alpha", "beta", (0, 0), (1, -1))), (O.R, ("alpha", (0, 1)))])
def test_gradients_match_finite_differences_of_the_converged_fixed_point(bc, params):
    h, ut, v = _problem(bc)
    alpha, beta = 0.05, 0.1
    loss = lambda u: float(np.sum((u - ut) ** 2))
    u = _ustar(v, h, bc, alpha, beta)
    assert np.abs(O.euler_lagrange(u, v, h, bc, alpha, beta)).max() < 1e-12
    lam, it, rr, ok = O.adjoint_solve(u, h, bc, alpha, beta, 2 * (u - ut), tol=1e-14)
    ga, gb, gh = O.fixed_point_gradients(u, v, h, bc, alpha, beta, lam)
    for p in params:
        if p == "alpha":
            e = 1e-5 * alpha
            fd = (loss(_ustar(v, h, bc, alpha + e, beta)) - loss(_ustar(v, h, bc, alpha - e, beta))) / (2 * e)
            got = ga
        elif p == "beta":
            e = 1e-5 * beta
            fd = (loss(_ustar(v, h, bc, alpha, beta + e)) - loss(_ustar(v, h, bc, alpha, beta - e))) / (2 * e)
            got = gb
        else:
            a, b = p
            E, e = O.unit_psf(h, a, b), 1e-6
            fd = (loss(_ustar(v, h + e * E, bc, alpha, beta)) - loss(_ustar(v, h - e * E, bc, alpha, beta))) / (2 * e)
            got = gh[2 + a, 2 + b]
        assert abs(got - fd) <= 1e-7 * abs(fd), (bc, p, got, fd)
