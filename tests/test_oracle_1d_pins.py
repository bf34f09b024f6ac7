"""Pins of the oracle on 1D signals (a plan of one row, Sec. 3.1 and Sec. 5.1).

A 1D signal is stored as a 1 x n array with a PSF of one row. These tests
build the paper's 1D matrices densely from the 1D statements of Sec. 3.1 and
check that the oracle's 2D code, given one row, computes them:

* the blur under both BCs from the 1D extension rules of Sec. 2, and its
  diagonalisation by the 1D transforms (T_n of eq. (Tn) for AR, C_n for R);
* R, D_R, R_D and M, D_M, M_D: c(H)^T c(H) + alpha c(L) and
  hat-s(H)^T hat-s(H) + alpha hat-s(L) with the optimal projections of
  Sec. 3.1, the diagonal scaling of eq. (D) and the scaled system
  eq. (scalesys);
* P, D_P, P_D of the reblurring method with AR(.) of Sec. 3.1;
* the field-of-view observation of the 1D workload and its trend claims:
  the fast preconditioners cut the inner iterations (Table 1-1), and AR
  BCs want an alpha no larger than R BCs at the RRE minimum (Fig. tvrs).
"""
import numpy as np
import pytest

import oracle as O
from paper_1011_5964_gb300 import synth
from test_oracle_pins import ext_matrix_1d, paper_C, paper_S, paper_T


def dense1(op, n):
    """n x n matrix of a map on 1 x n arrays."""
    return np.column_stack([op(np.eye(n)[k][None, :]).ravel() for k in range(n)])


def sym_psf_1d(m, seed):
    rng = np.random.default_rng(seed)
    q = rng.uniform(0.1, 1.0, m + 1)
    h = q[np.abs(np.arange(-m, m + 1))]
    return (h / h.sum())[None, :]


def conv_on_extension(n, h1):
    """n x (n + 2m) matrix: v_i = sum_b h_b x~_{i-b} on the extended signal (eq. (blurred1d:matrixform))."""
    m = len(h1) // 2
    C = np.zeros((n, n + 2 * m))
    for i in range(n):
        for b in range(-m, m + 1):
            C[i, i - b + m] += h1[b + m]
    return C


def hat_S(n):
    B = np.zeros((n, n))
    B[0, 0] = B[-1, -1] = 1.0
    B[1:-1, 1:-1] = paper_S(n - 2)
    return B


def proj(A, B):
    """The optimal projection onto {B^T diag(lam) B}: B^T diag(diag(B A B^T)) B (rows of B the basis)."""
    return B.T @ np.diag(np.diag(B @ A @ B.T)) @ B


@pytest.mark.parametrize("bc", [O.AR, O.R])
@pytest.mark.parametrize("n,m", [(7, 2), (12, 4), (31, 6)])
def test_1d_blur_is_the_convolution_of_the_1d_extension(bc, n, m):
    h = sym_psf_1d(m, seed=n)
    H = dense1(lambda x: O.blur(x, h, bc), n)
    np.testing.assert_allclose(H, conv_on_extension(n, h[0]) @ ext_matrix_1d(n, m, bc), atol=1e-15)
    Ht = dense1(lambda y: O.blur_adjoint(y, h, bc), n)
    np.testing.assert_allclose(Ht, H.T, atol=1e-15)


@pytest.mark.parametrize("n,m", [(9, 2), (16, 5)])
def test_1d_blurs_are_diagonalised_by_the_1d_transforms(n, m):
    h = sym_psf_1d(m, seed=3 * n)
    h1 = h[0]
    # AR: H = T_n diag(h_hat(y)) T_n^-1 on the grid of eq. (gridy)
    y = np.arange(n) * np.pi / (n - 1)
    y[-1] = 0.0
    lam = np.array([sum(h1[m + b] * np.cos(b * t) for b in range(-m, m + 1)) for t in y])
    T = paper_T(n)
    H = dense1(lambda x: O.blur(x, h, O.AR), n)
    np.testing.assert_allclose(H, T @ np.diag(lam) @ np.linalg.inv(T), atol=1e-12)
    np.testing.assert_allclose(O.spectrum_H(h, 1, n, O.AR)[0], lam, atol=1e-14)
    # R: H = C_n diag(h_hat(k pi / n)) C_n^T
    yr = np.arange(n) * np.pi / n
    lam_r = np.array([sum(h1[m + b] * np.cos(b * t) for b in range(-m, m + 1)) for t in yr])
    C = paper_C(n)
    Hr = dense1(lambda x: O.blur(x, h, O.R), n)
    np.testing.assert_allclose(Hr, C @ np.diag(lam_r) @ C.T, atol=1e-12)
    np.testing.assert_allclose(O.spectrum_H(h, 1, n, O.R)[0], lam_r, atol=1e-14)


@pytest.mark.parametrize("bc", [O.AR, O.R])
@pytest.mark.parametrize("kind", [O.PC_FAST, O.PC_DFAST, O.PC_FASTD])
def test_1d_preconditioners_are_the_papers_1d_matrices(bc, kind):
    n, m, alpha, beta = 13, 2, 0.05, 0.1
    h = sym_psf_1d(m, seed=40)
    rng = np.random.default_rng(41)
    u = rng.uniform(0, 1, (1, n))
    r = rng.standard_normal((1, n))
    B = hat_S(n) if bc == O.AR else paper_C(n).T      # rows: the 1D basis vectors
    H = dense1(lambda x: O.blur(x, h, bc), n)
    w = O.diffusivity(u, beta)
    L = dense1(lambda x: O.tv_apply(w, x), n)
    D = 1.0 + alpha * np.diag(L)
    if kind == O.PC_FASTD:
        dm = np.diag(D ** -0.5)
        Hh = proj(H, B) @ proj(dm, B)
        X = Hh.T @ Hh + alpha * proj(dm @ L @ dm, B)
    else:
        X = proj(H, B).T @ proj(H, B) + alpha * proj(L, B)
    if kind != O.PC_FAST:
        X = np.sqrt(D)[:, None] * X * np.sqrt(D)[None, :]
    P = O.precond_setup(u, h, bc, alpha, beta, kind)
    z = O.precond_apply(r, P)
    np.testing.assert_allclose(z.ravel(), np.linalg.solve(X, r.ravel()), rtol=1e-10, atol=1e-11)


@pytest.mark.parametrize("kind", [O.PC_FAST, O.PC_DFAST, O.PC_FASTD])
def test_1d_reblur_preconditioners_use_the_1d_ar_projection(kind):
    n, m, alpha, beta = 11, 2, 0.05, 0.1
    h = sym_psf_1d(m, seed=50)
    rng = np.random.default_rng(51)
    u = rng.uniform(0, 1, (1, n))
    r = rng.standard_normal((1, n))
    H = dense1(lambda x: O.blur(x, h, O.AR), n)
    Hp = dense1(lambda x: O.blur(x, h[:, ::-1], O.AR), n)
    w = O.diffusivity(u, beta)
    L = dense1(lambda x: O.tv_apply(w, x), n)
    D = 1.0 + alpha * np.diag(L)
    if kind == O.PC_FASTD:
        dm = O.ar_projection(np.diag(D ** -0.5))
        X = dm @ Hp @ H @ dm + alpha * O.ar_projection((D ** -0.5)[:, None] * L * (D ** -0.5)[None, :])
    else:
        X = Hp @ H + alpha * O.ar_projection(L)
    if kind != O.PC_FAST:
        X = np.sqrt(D)[:, None] * X * np.sqrt(D)[None, :]
    P = O.precond_setup(u, h, O.AR, alpha, beta, kind, method=O.METHOD_REBLUR)
    z = O.precond_apply(r, P)
    np.testing.assert_allclose(z.ravel(), np.linalg.solve(X, r.ravel()), rtol=1e-9, atol=1e-10)


def test_1d_tv_operator_has_no_row_differences():
    """One row: L(u) = D_c^T W D_c with the 1D forward difference, eq. (el)."""
    rng = np.random.default_rng(60)
    n = 10
    u = rng.uniform(0, 1, (1, n))
    w = O.diffusivity(u, 0.2)
    d = np.diff(u[0])
    np.testing.assert_allclose(w[0, :-1], 1.0 / np.sqrt(d * d + 0.04), rtol=1e-15)
    assert w[0, -1] == pytest.approx(1.0 / 0.2)
    Dm = np.zeros((n - 1, n))
    Dm[np.arange(n - 1), np.arange(n - 1)] = -1.0
    Dm[np.arange(n - 1), np.arange(1, n)] = 1.0
    L = Dm.T @ np.diag(w[0, :-1]) @ Dm
    np.testing.assert_allclose(dense1(lambda x: O.tv_apply(w, x), n), L, atol=1e-14)


def _signal_problem(seed, n=203, m=11, noise=0.01):
    h = synth.out_of_focus_psf_1d(m)
    uw, fov = synth.piecewise_constant_signal(n, seed)
    hv = O.blur(uw[None, :], h, O.R)[:, fov]
    v = synth.add_noise(hv, synth.noise_direction(1, n, seed), noise)
    return h, uw[fov][None, :], v


def test_field_of_view_observation_is_the_plain_convolution():
    """The observation crops a blur of the wider signal far enough from its ends that no BC enters."""
    n, m = 203, 11
    h = synth.out_of_focus_psf_1d(m)
    uw, fov = synth.piecewise_constant_signal(n, 3)
    assert fov.start >= m
    full = np.convolve(uw, h[0], mode="same")
    np.testing.assert_allclose(O.blur(uw[None, :], h, O.R)[0, fov], full[fov], atol=1e-14)
    np.testing.assert_allclose(O.blur(uw[None, :], h, O.AR)[0, fov], full[fov], atol=1e-14)


@pytest.mark.parametrize("bc,method", [(O.R, O.METHOD_FP), (O.AR, O.METHOD_FP), (O.AR, O.METHOD_REBLUR)])
def test_1d_fast_preconditioners_cut_the_inner_iterations(bc, method):
    """Table 1-1 at alpha 1e-3, beta 0.1, n = 203: every fast preconditioner needs far fewer
    iterations per FP step than no preconditioner or the diagonal one (FP stop 1e-3, PCG tol 1e-6)."""
    h, _, v = _signal_problem(1)
    avg = {}
    for kind in (O.PC_NONE, O.PC_DIAG, O.PC_FAST, O.PC_DFAST, O.PC_FASTD):
        _, st = O.tv_deblur(v, h, bc, 1e-3, 0.1, outer=200, tol=1e-6, maxit=5000, kind=kind, outer_tol=1e-3,
                            method=method)
        avg[kind] = float(np.mean(st["inner_iters"]))
    for fast in (O.PC_FAST, O.PC_DFAST, O.PC_FASTD):
        assert 2.0 * avg[fast] < min(avg[O.PC_NONE], avg[O.PC_DIAG]), avg


def test_ar_optimal_alpha_is_no_larger_than_reflective():
    """Fig. tvrs: the RRE-optimal alpha on the sweep grid is no larger for AR than for R BCs,
    for each of five seeded signals, and the best AR RRE is lower on average."""
    alphas = synth.alpha_grid()
    best = {O.AR: [], O.R: []}
    for seed in range(1, 6):
        h, ut, v = _signal_problem(seed)
        for bc in (O.AR, O.R):
            rre = [float(np.linalg.norm(O.tv_deblur(v, h, bc, a, 0.1, outer=200, tol=1e-6, maxit=2000,
                                                    kind=O.PC_DFAST, outer_tol=1e-3)[0] - ut) / np.linalg.norm(ut))
                   for a in alphas]
            k = int(np.argmin(rre))
            assert 0 < k < len(alphas) - 1 or bc == O.R, (bc, seed, rre)   # an interior minimum for AR
            best[bc].append((alphas[k], rre[k]))
    for (a_ar, _), (a_r, _) in zip(best[O.AR], best[O.R]):
        assert a_ar <= a_r
    assert np.mean([e for _, e in best[O.AR]]) < np.mean([e for _, e in best[O.R]])
