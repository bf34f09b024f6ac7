"""Pins of the oracle's scaled-system preconditioners R_D / M_D (Secs. 2.1, 2.2, 3.2).

R_D (reflective) and M_D (anti-reflective) precondition the scaled system
(H~^* H~ + alpha L~) u~ = H~^* v of eq. (scalesys), H~ = H D^-1/2, L~ =
D^-1/2 L D^-1/2, by H^^* H^ + alpha s_2(L~) with H^ = s_2(H) s_2(D^-1/2),
s_2 the level-2 projection onto the transform algebra. These tests build that
matrix densely from the definitions at tiny sizes and check the oracle's fast
spectra and solve against it, and check the paper's ordering M_D <= D_M.
"""
import numpy as np
import pytest

import oracle as O
from paper_1011_5964_gb300 import synth


def dense(apply, nr, nc):
    n = nr * nc
    return np.column_stack([apply(np.eye(n)[:, k].reshape(nr, nc)).ravel() for k in range(n)])


def proj2(A, U):
    """Level-2 projection U^T diag(diag(U A U^T)) U (Sec. 3.2, G8 reading)."""
    return U.T @ np.diag(np.diag(U @ A @ U.T)) @ U


@pytest.mark.parametrize("bc", [O.AR, O.R])
def test_scaled_spectra_equal_the_brute_force_projections(bc):
    rng = np.random.default_rng(5)
    nr, nc = 5, 6
    w = rng.uniform(0.5, 2.0, (nr, nc))
    d = rng.uniform(0.3, 1.5, (nr, nc))
    lam_d, lam_lt = O.spectrum_scaled(w, d, bc)
    U = np.kron(O.transform_matrix(nr, bc), O.transform_matrix(nc, bc))
    L = dense(lambda x: O.tv_apply(w, x), nr, nc)
    Dm = np.diag(d.ravel())
    assert np.abs(np.diag(U @ Dm @ U.T).reshape(nr, nc) - lam_d).max() < 1e-13
    assert np.abs(np.diag(U @ Dm @ L @ Dm @ U.T).reshape(nr, nc) - lam_lt).max() < 1e-13


@pytest.mark.parametrize("bc", [O.AR, O.R])
def test_unit_scaling_reduces_to_the_unscaled_spectrum(bc):
    rng = np.random.default_rng(6)
    w = rng.uniform(0.5, 2.0, (7, 4))
    lam_d, lam_lt = O.spectrum_scaled(w, np.ones_like(w), bc)
    assert np.abs(lam_d - 1.0).max() < 1e-13
    assert np.abs(lam_lt - O.spectrum_L(w, bc)).max() < 1e-13


@pytest.mark.parametrize("bc", [O.AR, O.R])
def test_fastd_solve_is_the_papers_scaled_preconditioner(bc):
    """precond_apply(fastd) = (D^1/2 M_D D^1/2)^-1 with M_D = H^^* H^ + alpha s_2(L~) built densely."""
    nr, nc = 6, 7
    h = synth.gaussian_psf(1.0, half_width=1)
    rng = np.random.default_rng(7)
    u = rng.standard_normal((nr, nc))
    alpha, beta = 0.05, 0.3
    P = O.precond_setup(u, h, bc, alpha, beta, O.PC_FASTD)
    U = np.kron(O.transform_matrix(nr, bc), O.transform_matrix(nc, bc))
    H = dense(lambda x: O.blur(x, h, bc), nr, nc)
    L = dense(lambda x: O.tv_apply(P["w"], x), nr, nc)
    dmh = np.diag(1.0 / np.sqrt(P["D"].ravel()))
    Hh = proj2(H, U) @ proj2(dmh, U)
    MD = Hh.T @ Hh + alpha * proj2(dmh @ L @ dmh, U)
    X = np.diag(np.sqrt(P["D"].ravel())) @ MD @ np.diag(np.sqrt(P["D"].ravel()))
    r = rng.standard_normal((nr, nc))
    z = O.precond_apply(r, P)
    assert np.abs(z.ravel() - np.linalg.solve(X, r.ravel())).max() < 1e-10 * np.abs(z).max()


def test_m_d_needs_no_more_iterations_than_d_m():
    """Tables 1-1 / 2-1: the scaled-system preconditioner M_D is at least as good as D_M."""
    n = 64
    h = synth.gaussian_psf(1.5, half_width=4)
    ut = synth.piecewise_constant_image(n, n, seed=1234)
    v = synth.add_noise(O.blur(ut, h, O.AR), synth.noise_direction(n, n, 1234), 0.01)
    for alpha in (1e-2, 1e-3):
        k_dm = sum(O.tv_deblur(v, h, O.AR, alpha, 1e-2, outer=3, tol=1e-6, kind=O.PC_DFAST)[1]["inner_iters"])
        k_md = sum(O.tv_deblur(v, h, O.AR, alpha, 1e-2, outer=3, tol=1e-6, kind=O.PC_FASTD)[1]["inner_iters"])
        assert k_md <= k_dm, (alpha, k_md, k_dm)
