"""Pins of the oracle's reblurring path (eq. (fpp), Sec. 3.1 after eq. (fpp), Sec. 3.2).

Each check compares the oracle with an independent construction:
* T_n built as hat-S_n (I + U) (the Remark after AR(A)) against T_n sampled from
  the functions of eq. (Tn), and its inverse (I - U) hat-S_n;
* the AR algebra of eq. (ARalg): the 2D anti-reflective blur is diagonalised
  by T_n (x) T_n with the eigenvalues of eqs. (symb), (gridy);
* AR(A) from the paper's definition reproduces an AR blur matrix exactly
  (its interior block is a tau matrix and its border columns are the
  anti-reflective folds), lies in the AR algebra with the eigenvalues the
  oracle's fast extension predicts, and is not the Frobenius argmin over the
  algebra (the Remark);
* the level-2 projection Q AR_1(Q^T AR_1(L) Q) Q^T built densely on tiny
  images against the oracle's extended eigenvalues;
* the P, D_P, P_D solves against dense solves of the paper's formulas;
* PBiCGstab against a dense solve of the nonsymmetric A' of eq. (fpp), one
  iteration for the exact preconditioner (alpha = 0), and the ordering of
  the preconditioners in the reblurring columns of Table 2-1.
"""
import numpy as np
import pytest

import oracle as O
from paper_1011_5964_gb300 import synth


def dense(op, nr, nc):
    n = nr * nc
    M = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        M[:, k] = op(e.reshape(nr, nc)).ravel()
    return M


def sampled_T(n):
    """T_n of eq. (Tn): columns (1 - y/pi, sin y, ..., sin((n-2) y), y/pi) times
    diag(1, sqrt(2/(n-1)) I, 1), sampled on y_i = (i-1) pi / (n-1)."""
    y = np.arange(n) * np.pi / (n - 1)
    cols = [1.0 - y / np.pi] + [np.sqrt(2.0 / (n - 1)) * np.sin(k * y) for k in range(1, n - 1)] + [y / np.pi]
    return np.stack(cols, axis=1)


def qsym_psf(mr, mc, seed):
    rng = np.random.default_rng(seed)
    q = rng.uniform(0.1, 1.0, (mr + 1, mc + 1))
    a = np.abs(np.arange(-mr, mr + 1))
    b = np.abs(np.arange(-mc, mc + 1))
    h = q[a[:, None], b[None, :]]
    return h / h.sum()


def gridy_symbol_1d(h1, n):
    """h_hat(y_j) on the grid of eq. (gridy): y_j = (j-1) pi / (n-1), y_n = 0."""
    m = len(h1) // 2
    y = np.arange(n) * np.pi / (n - 1)
    y[-1] = 0.0
    return np.array([sum(h1[m + k] * np.cos(k * t) for k in range(-m, m + 1)) for t in y])


@pytest.mark.parametrize("n", [4, 5, 8, 11])
def test_T_is_the_sampled_transform_of_eq_Tn(n):
    T, Ti = O.transform_T(n)
    np.testing.assert_allclose(T, sampled_T(n), atol=1e-14)
    np.testing.assert_allclose(T @ Ti, np.eye(n), atol=1e-13)


@pytest.mark.parametrize("nr,nc,mr,mc", [(6, 7, 1, 2), (7, 6, 2, 1), (8, 8, 3, 3)])
def test_T_diagonalises_the_2d_ar_blur(nr, nc, mr, mc):
    h = qsym_psf(mr, mc, seed=nr * nc)
    H = dense(lambda x: O.blur(x, h, O.AR), nr, nc)
    Tr, Tir = O.transform_T(nr)
    Tc, Tic = O.transform_T(nc)
    D = np.kron(Tir, Tic) @ H @ np.kron(Tr, Tc)
    np.testing.assert_allclose(D - np.diag(np.diag(D)), 0.0, atol=1e-12)
    np.testing.assert_allclose(np.diag(D), O.spectrum_H(h, nr, nc, O.AR).ravel(), atol=1e-12)


@pytest.mark.parametrize("n,m", [(7, 1), (9, 3), (12, 5)])
def test_ar_projection_reproduces_an_ar_blur(n, m):
    rng = np.random.default_rng(n + m)
    half = rng.uniform(0.1, 1.0, m + 1)
    h1 = np.concatenate([half[::-1], half[1:]])
    h1 /= h1.sum()
    H = dense(lambda x: O.blur(x, h1[None, :], O.AR), 1, n)
    np.testing.assert_allclose(O.ar_projection(H), H, atol=1e-13)
    # and its eigenvalues are the symbol on the grid of eq. (gridy)
    T, Ti = O.transform_T(n)
    np.testing.assert_allclose(np.diag(Ti @ H @ T), gridy_symbol_1d(h1, n), atol=1e-13)


@pytest.mark.parametrize("n", [6, 9, 13])
def test_ar_projection_is_in_the_algebra_with_extended_eigenvalues(n):
    rng = np.random.default_rng(3 * n)
    A = rng.standard_normal((n, n))
    A = A + A.T
    P = O.ar_projection(A)
    T, Ti = O.transform_T(n)
    D = Ti @ P @ T
    np.testing.assert_allclose(D - np.diag(np.diag(D)), 0.0, atol=1e-12)
    S = O.tvd_oracle._sine(n - 2)
    lam = np.diag(S @ A[1:-1, 1:-1] @ S)
    border = O.ar_extension(n - 2) @ lam
    np.testing.assert_allclose(np.diag(D), np.concatenate([[border], lam, [border]]), atol=1e-12)


def test_ar_projection_is_not_the_frobenius_argmin():
    """The Remark: AR(A) differs in general from argmin_{B in AR} ||B - A||_F."""
    n = 8
    rng = np.random.default_rng(5)
    A = rng.standard_normal((n, n))
    T, Ti = O.transform_T(n)
    basis = np.stack([np.outer(T[:, k], Ti[k]).ravel() for k in range(n)], axis=1)
    lam, *_ = np.linalg.lstsq(basis, A.ravel(), rcond=None)
    argmin = (basis @ lam).reshape(n, n)
    P = O.ar_projection(A)
    assert np.linalg.norm(P - A) > np.linalg.norm(argmin - A) + 1e-3
    assert np.linalg.norm(P - argmin) > 1e-3


@pytest.mark.parametrize("nr,nc", [(5, 6), (6, 5), (6, 6)])
def test_level2_projection_of_L_has_the_extended_eigenvalues(nr, nc):
    rng = np.random.default_rng(nr * 10 + nc)
    w = O.diffusivity(rng.uniform(0, 1, (nr, nc)), 0.1)
    L = dense(lambda y: O.tv_apply(w, y), nr, nc)
    A2 = O.ar2_projection(L, nr, nc)
    Tr, Tir = O.transform_T(nr)
    Tc, Tic = O.transform_T(nc)
    D = np.kron(Tir, Tic) @ A2 @ np.kron(Tr, Tc)
    np.testing.assert_allclose(D - np.diag(np.diag(D)), 0.0, atol=1e-11)
    np.testing.assert_allclose(np.diag(D), O.ar_extend2(O.spectrum_L(w, O.AR)).ravel(), atol=1e-11)


def _dense_reblur_preconditioner(u, h, alpha, beta, nr, nc, kind):
    w = O.diffusivity(u, beta)
    H = dense(lambda x: O.blur(x, h, O.AR), nr, nc)
    Hp = dense(lambda x: O.blur(x, h[::-1, ::-1], O.AR), nr, nc)
    L = dense(lambda y: O.tv_apply(w, y), nr, nc)
    D = 1.0 + alpha * np.diag(L)
    if kind == O.PC_FASTD:
        Dm = O.ar2_projection(np.diag(D ** -0.5), nr, nc)
        Lt = (D ** -0.5)[:, None] * L * (D ** -0.5)[None, :]
        X = Dm @ Hp @ H @ Dm + alpha * O.ar2_projection(Lt, nr, nc)
    else:
        X = Hp @ H + alpha * O.ar2_projection(L, nr, nc)
    if kind in (O.PC_DFAST, O.PC_FASTD):
        X = np.sqrt(D)[:, None] * X * np.sqrt(D)[None, :]
    return X


@pytest.mark.parametrize("kind", [O.PC_FAST, O.PC_DFAST, O.PC_FASTD])
@pytest.mark.parametrize("nr,nc", [(6, 5), (7, 7)])
def test_reblur_preconditioner_solve_matches_dense_definition(kind, nr, nc):
    alpha, beta = 0.05, 0.1
    h = qsym_psf(1, 2, seed=21)
    rng = np.random.default_rng(22 + nr)
    u = rng.uniform(0, 1, (nr, nc))
    r = rng.standard_normal((nr, nc))
    X = _dense_reblur_preconditioner(u, h, alpha, beta, nr, nc, kind)
    P = O.precond_setup(u, h, O.AR, alpha, beta, kind, method=O.METHOD_REBLUR)
    z = O.precond_apply(r, P)
    np.testing.assert_allclose(z.ravel(), np.linalg.solve(X, r.ravel()), rtol=1e-9, atol=1e-10)


def test_reblur_operator_is_nonsymmetric_and_matches_dense():
    nr, nc, alpha = 6, 7, 0.02
    h = qsym_psf(1, 1, seed=23)
    w = O.diffusivity(np.random.default_rng(24).uniform(0, 1, (nr, nc)), 0.1)
    A = dense(lambda x: O.reblur_apply(x, h, O.AR, w, alpha), nr, nc)
    H = dense(lambda x: O.blur(x, h, O.AR), nr, nc)
    L = dense(lambda y: O.tv_apply(w, y), nr, nc)
    np.testing.assert_allclose(A, H @ H + alpha * L, atol=1e-13)   # H' = H for a symmetric PSF
    assert np.abs(A - A.T).max() > 1e-3


@pytest.mark.parametrize("kind", [O.PC_NONE, O.PC_FAST, O.PC_DFAST, O.PC_FASTD])
def test_bicgstab_matches_dense_solve(kind):
    nr, nc, alpha, beta = 9, 8, 1e-2, 0.1
    h = qsym_psf(2, 1, seed=25)
    rng = np.random.default_rng(26)
    u = rng.uniform(0, 1, (nr, nc))
    b = rng.standard_normal((nr, nc))
    P = O.precond_setup(u, h, O.AR, alpha, beta, kind, method=O.METHOD_REBLUR)
    w = P["w"]
    x, k, rr, ok = O.bicgstab(lambda y: O.reblur_apply(y, h, O.AR, w, alpha), lambda r: O.precond_apply(r, P),
                              b, np.zeros_like(b), 1e-12, 500)
    A = dense(lambda y: O.reblur_apply(y, h, O.AR, w, alpha), nr, nc)
    assert ok and rr < 1e-12
    np.testing.assert_allclose(x.ravel(), np.linalg.solve(A, b.ravel()), rtol=1e-8, atol=1e-9)


def test_reblur_exact_preconditioner_alpha_zero_one_iteration():
    """alpha = 0: P = H' H = A', so PBiCGstab stops after its first half step."""
    nr, nc = 10, 9
    h = qsym_psf(2, 2, seed=27)
    rng = np.random.default_rng(28)
    v = rng.uniform(0, 1, (nr, nc))
    b = O.reblur_rhs(v, h, O.AR)
    _, k, rr, ok = O.fp_step(v, b, h, O.AR, 0.0, 0.1, O.PC_FAST, 1e-10, 50, method=O.METHOD_REBLUR)
    assert ok and k == 1, (k, rr)


def test_reblur_preconditioner_ordering_matches_table():
    """Reblurring columns of Table 2-1 (2D, beta = 0.01, tol 1e-5, little noise): the scaled
    reblurring preconditioners D_P and P_D need clearly fewer PBiCGstab iterations than D and I."""
    n = 48
    h = synth.gaussian_psf(1.5, half_width=4)
    u_true = synth.piecewise_constant_image(n, n, seed=29)
    v = synth.add_noise(O.blur(u_true, h, O.AR), synth.noise_direction(n, n, 29), 0.001)
    tot = {}
    for kind in (O.PC_FASTD, O.PC_DFAST, O.PC_DIAG, O.PC_NONE):
        _, st = O.tv_deblur(v, h, O.AR, 1e-1, 1e-2, outer=2, tol=1e-5, maxit=3000, kind=kind,
                            method=O.METHOD_REBLUR)
        tot[kind] = sum(st["inner_iters"])
    assert max(tot[O.PC_FASTD], tot[O.PC_DFAST]) < tot[O.PC_DIAG] < tot[O.PC_NONE], tot
    assert 3 * tot[O.PC_DFAST] < 2 * tot[O.PC_NONE], tot
