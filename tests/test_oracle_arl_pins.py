"""Pins of the oracle's L with anti-reflective BCs (L_AR, the "AR+Reblur+AR L"
columns of Tables 1-1 and 2-1; the remark after eq. (scalereb)).

* In 1D, L_AR is exactly the divergence-form stencil on the AR extension
  (eq. (anti1d)) of both y and u, the diffusivity taken from the extended u.
* For a constant diffusivity, L_AR is the anti-reflective blur (Sec. 2) with
  the 5-point Laplacian as its PSF: the AR algebra's own structure, which is
  why the paper expects the preconditioners to fit eq. (fpp) better.
* L_AR shares L's interior rows, so AR_2(L_AR) = AR_2(L); its preconditioners
  (P, D_P, P_D with D from diag(L_AR)) equal their dense definitions, and
  PBiCGstab solves the non-symmetric system.
"""
import numpy as np
import pytest

import oracle as O
from paper_1011_5964_gb300 import synth


def dense(op, nr, nc):
    n = nr * nc
    return np.column_stack([op(np.eye(n)[k].reshape(nr, nc)).ravel() for k in range(n)])


def test_1d_l_ar_is_the_stencil_on_the_ar_extension_of_u_and_y():
    rng = np.random.default_rng(1)
    n, beta = 12, 0.2
    u = rng.uniform(0, 1, n)
    y = rng.standard_normal(n)
    ue = np.concatenate([[2 * u[0] - u[1]], u, [2 * u[-1] - u[-2]]])     # eq. (anti1d), one ghost per side
    ye = np.concatenate([[2 * y[0] - y[1]], y, [2 * y[-1] - y[-2]]])
    wt = 1.0 / np.sqrt(np.diff(ue) ** 2 + beta * beta)                  # pairs (k, k+1), k = -1 .. n-1
    ref = np.array([wt[i] * (ye[i + 1] - ye[i]) - wt[i + 1] * (ye[i + 2] - ye[i + 1]) for i in range(n)])
    got = O.tv_apply_ar(O.diffusivity(u[None, :], beta), y[None, :])[0]
    np.testing.assert_allclose(got, ref, atol=1e-13)
    assert abs(got[0]) < 1e-13 and abs(got[-1]) < 1e-13      # the end rows vanish


@pytest.mark.parametrize("nr,nc", [(5, 7), (8, 6), (1, 9)])
def test_constant_diffusivity_l_ar_is_the_ar_blur_of_the_laplacian(nr, nc):
    c = 0.7
    w = np.full((nr, nc), c)
    lap = c * np.array([[0.0, -1.0, 0.0], [-1.0, 4.0, -1.0], [0.0, -1.0, 0.0]])
    if nr == 1:
        lap = c * np.array([[-1.0, 2.0, -1.0]])
    L = dense(lambda y: O.tv_apply_ar(w, y), nr, nc)
    Har = dense(lambda y: O.blur(y, lap, O.AR), nr, nc)
    np.testing.assert_allclose(L, Har, atol=1e-13)


def test_l_ar_has_the_interior_rows_of_l_and_is_not_symmetric():
    rng = np.random.default_rng(2)
    nr, nc = 6, 7
    w = O.diffusivity(rng.uniform(0, 1, (nr, nc)), 0.1)
    LA = dense(lambda y: O.tv_apply_ar(w, y), nr, nc)
    LN = dense(lambda y: O.tv_apply(w, y), nr, nc)
    interior = np.zeros((nr, nc), bool)
    interior[1:-1, 1:-1] = True
    idx = np.flatnonzero(interior.ravel())
    np.testing.assert_allclose(LA[idx], LN[idx], atol=1e-14)
    assert np.abs(LA - LA.T).max() > 1e-3
    np.testing.assert_allclose(np.diag(LA).reshape(nr, nc), O.tv_diag_ar(w), atol=1e-14)
    np.testing.assert_allclose(O.ar2_projection(LA, nr, nc), O.ar2_projection(LN, nr, nc), atol=1e-12)


@pytest.mark.parametrize("kind", [O.PC_FAST, O.PC_DFAST, O.PC_FASTD])
def test_arl_preconditioners_match_their_dense_definitions(kind):
    nr, nc, alpha, beta = 6, 7, 0.05, 0.1
    h = synth.gaussian_psf(1.0, half_width=1)
    rng = np.random.default_rng(3)
    u = rng.uniform(0, 1, (nr, nc))
    r = rng.standard_normal((nr, nc))
    w = O.diffusivity(u, beta)
    H = dense(lambda x: O.blur(x, h, O.AR), nr, nc)
    L = dense(lambda y: O.tv_apply_ar(w, y), nr, nc)
    D = 1.0 + alpha * np.diag(L)
    if kind == O.PC_FASTD:
        Dm = O.ar2_projection(np.diag(D ** -0.5), nr, nc)
        X = Dm @ H @ H @ Dm + alpha * O.ar2_projection((D ** -0.5)[:, None] * L * (D ** -0.5)[None, :], nr, nc)
    else:
        X = H @ H + alpha * O.ar2_projection(L, nr, nc)
    if kind != O.PC_FAST:
        X = np.sqrt(D)[:, None] * X * np.sqrt(D)[None, :]
    P = O.precond_setup(u, h, O.AR, alpha, beta, kind, method=O.METHOD_REBLUR_ARL)
    np.testing.assert_allclose(O.precond_apply(r, P).ravel(), np.linalg.solve(X, r.ravel()), rtol=1e-9,
                               atol=1e-10)


@pytest.mark.parametrize("kind", [O.PC_NONE, O.PC_DFAST, O.PC_FASTD])
def test_arl_bicgstab_solves_the_nonsymmetric_system(kind):
    nr, nc, alpha, beta = 7, 6, 0.02, 0.1
    h = synth.gaussian_psf(1.0, half_width=2)
    rng = np.random.default_rng(4)
    u = rng.uniform(0, 1, (nr, nc))
    b = rng.standard_normal((nr, nc))
    w = O.diffusivity(u, beta)
    A = dense(lambda x: O.reblur_apply(x, h, O.AR, w, alpha, arl=True), nr, nc)
    x, k, rr, ok = O.fp_step(u, b, h, O.AR, alpha, beta, kind, 1e-12, 500, method=O.METHOD_REBLUR_ARL)
    assert ok
    np.testing.assert_allclose(x.ravel(), np.linalg.solve(A, b.ravel()), rtol=1e-8, atol=1e-9)


def test_arl_needs_no_more_iterations_than_zero_neumann():
    """Table 2-1: with the same preconditioner family, AR BCs on L lower the PBiCGstab iterations
    per FP step (the system is closer to the AR algebra the preconditioner lives in)."""
    n = 32
    h = synth.gaussian_psf(1.5, half_width=4)
    ut = synth.piecewise_constant_image(n, n, seed=3)
    v = synth.add_noise(O.blur(ut, h, O.AR), synth.noise_direction(n, n, 3), 0.01)
    for kind in (O.PC_DFAST, O.PC_FASTD):
        avg = {}
        for method in (O.METHOD_REBLUR, O.METHOD_REBLUR_ARL):
            _, st = O.tv_deblur(v, h, O.AR, 1e-2, 1e-2, outer=10, tol=1e-5, maxit=5000, kind=kind, method=method)
            avg[method] = float(np.mean(st["inner_iters"]))
        assert avg[O.METHOD_REBLUR_ARL] <= avg[O.METHOD_REBLUR], (kind, avg)
