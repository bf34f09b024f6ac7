"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the paper's
closed-form eigendecompositions (eqs. (Tn), (lambda), (gridy), the DCT of
Sec. 3.1), its stated invariants (linear reproduction of AR BCs, symmetry of
reflective H, the Proposition on hat-s), textbook closed forms (the Neumann
Laplacian spectrum), finite differences of the TV functional, and dense brute
force on tiny images. Images are rectangular and PSFs quadrantally symmetric
with h_{a,b} != h_{b,a}, so that a transposed operand or a swapped axis fails.
"""
import numpy as np
import pytest

import oracle as O
from paper_1011_5964_gb300 import synth

SHAPES = [(7, 9, 2, 3), (6, 6, 4, 4), (5, 8, 3, 1), (8, 5, 1, 3)]


def qsym_psf(mr, mc, seed=0):
    """Random normalised quadrantally symmetric PSF, not separable, h_ab != h_ba."""
    rng = np.random.default_rng(seed)
    q = rng.uniform(0.1, 1.0, (mr + 1, mc + 1))
    a = np.abs(np.arange(-mr, mr + 1))
    b = np.abs(np.arange(-mc, mc + 1))
    h = q[a[:, None], b[None, :]]
    return h / h.sum()


def dense(op, nr, nc):
    n = nr * nc
    M = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        M[:, k] = op(e.reshape(nr, nc)).ravel()
    return M


def paper_T(n):
    """T_n of eq. (Tn): columns (1 - y/pi, sin y, ..., sin((n-2) y), y/pi) diag(1, sqrt(2/(n-1)) I, 1),
    sampled on y_i = (i-1) pi / (n-1)."""
    y = np.arange(n) * np.pi / (n - 1)
    T = np.zeros((n, n))
    T[:, 0] = 1.0 - y / np.pi
    T[:, n - 1] = y / np.pi
    for k in range(1, n - 1):
        T[:, k] = np.sqrt(2.0 / (n - 1)) * np.sin(k * y)
    return T


def paper_S(m):
    """S_m of eq. (lambda): sqrt(2/(m+1)) sin(i j pi / (m+1))."""
    i = np.arange(1, m + 1)
    return np.sqrt(2.0 / (m + 1)) * np.sin(np.outer(i, i) * np.pi / (m + 1))


def paper_C(n):
    """C_n of Sec. 3.1: [C_n]_{ij} = sqrt((2 - delta_j1)/n) cos((2i-1)(j-1) pi / (2n)), i spatial."""
    i = np.arange(1, n + 1)[:, None]
    j = np.arange(1, n + 1)[None, :]
    scale = np.sqrt((2.0 - (j == 1)) / n)
    return scale * np.cos((2 * i - 1) * (j - 1) * np.pi / (2 * n))


def ext_matrix_1d(n, m, bc):
    """(n + 2m) x n matrix of the 1D extension, written from the 1-based rules of Sec. 2."""
    E = np.zeros((n + 2 * m, n))
    for t in range(1 - m, n + m + 1):          # 1-based extended index
        row = t + m - 1
        if 1 <= t <= n:
            E[row, t - 1] = 1.0
        elif t <= 0:
            j = 1 - t                          # u_{1-j}
            if bc == O.AR:
                E[row, 0] += 2.0               # 2 u_1
                E[row, j] -= 1.0               # - u_{j+1}
            else:
                E[row, j - 1] += 1.0           # u_j
        else:
            j = t - n                          # u_{n+j}
            if bc == O.AR:
                E[row, n - 1] += 2.0           # 2 u_n
                E[row, n - j - 1] -= 1.0       # - u_{n-j}
            else:
                E[row, n - j] += 1.0           # u_{n+1-j}
    return E


# ---------------------------------------------------------------- extension

@pytest.mark.parametrize("bc", [O.AR, O.R])
@pytest.mark.parametrize("nr,nc,mr,mc", SHAPES)
def test_extension_is_tensor_product_of_1d_rules(nr, nc, mr, mc, bc):
    """The 2D extension (AR corners by the explicit formulas of Sec. 2) is E_r (x) E_c."""
    rng = np.random.default_rng(1)
    x = rng.standard_normal((nr, nc))
    Er, Ec = ext_matrix_1d(nr, mr, bc), ext_matrix_1d(nc, mc, bc)
    np.testing.assert_allclose(O.extend(x, mr, mc, bc), Er @ x @ Ec.T, atol=1e-13)


@pytest.mark.parametrize("bc", [O.AR, O.R])
@pytest.mark.parametrize("nr,nc,mr,mc", SHAPES)
def test_extension_adjoint(nr, nc, mr, mc, bc):
    rng = np.random.default_rng(2)
    x = rng.standard_normal((nr, nc))
    z = rng.standard_normal((nr + 2 * mr, nc + 2 * mc))
    lhs = float((O.extend(x, mr, mc, bc) * z).sum())
    rhs = float((x * O.extend_adjoint(z, mr, mc, bc)).sum())
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1.0)


# ---------------------------------------------------------------- blur operator

@pytest.mark.parametrize("nr,nc,mr,mc", SHAPES)
def test_ar_blur_diagonalised_by_paper_T(nr, nc, mr, mc):
    """H = (T_n (x) T_n) diag(h_hat(y_i, y_j)) (T_n (x) T_n)^{-1} (Sec. 2, [ADNS09] result)."""
    h = qsym_psf(mr, mc, seed=3)
    H = dense(lambda x: O.blur(x, h, O.AR), nr, nc)
    T = np.kron(paper_T(nr), paper_T(nc))
    Lam = np.linalg.solve(T, H @ T)
    yr = np.arange(nr) * np.pi / (nr - 1)
    yr[-1] = 0.0                                # eq. (gridy): y_n = 0
    yc = np.arange(nc) * np.pi / (nc - 1)
    yc[-1] = 0.0
    a = np.arange(-mr, mr + 1)
    b = np.arange(-mc, mc + 1)
    sym = np.einsum("ab,ia,jb->ij", h, np.cos(np.outer(yr, a)), np.cos(np.outer(yc, b)))
    np.testing.assert_allclose(Lam, np.diag(sym.ravel()), atol=1e-12)
    np.testing.assert_allclose(O.spectrum_H(h, nr, nc, O.AR), sym, atol=1e-13)


@pytest.mark.parametrize("nr,nc,mr,mc", SHAPES)
def test_r_blur_diagonalised_by_paper_dct(nr, nc, mr, mc):
    """Reflective H with quadrantally symmetric h is C^T Lambda C with C from Sec. 3.1, and symmetric."""
    h = qsym_psf(mr, mc, seed=4)
    H = dense(lambda x: O.blur(x, h, O.R), nr, nc)
    C = np.kron(paper_C(nr), paper_C(nc))      # columns are basis vectors
    Lam = C.T @ H @ C
    a = np.arange(-mr, mr + 1)
    b = np.arange(-mc, mc + 1)
    yr = np.arange(nr) * np.pi / nr
    yc = np.arange(nc) * np.pi / nc
    sym = np.einsum("ab,ia,jb->ij", h, np.cos(np.outer(yr, a)), np.cos(np.outer(yc, b)))
    np.testing.assert_allclose(Lam, np.diag(sym.ravel()), atol=1e-12)
    np.testing.assert_allclose(H, H.T, atol=1e-14)
    np.testing.assert_allclose(O.spectrum_H(h, nr, nc, O.R), sym, atol=1e-13)


def test_ar_blur_not_symmetric():
    h = qsym_psf(2, 2, seed=5)
    H = dense(lambda x: O.blur(x, h, O.AR), 7, 7)
    assert np.abs(H - H.T).max() > 1e-3


@pytest.mark.parametrize("nr,nc,mr,mc", SHAPES)
def test_ar_reproduces_bilinear(nr, nc, mr, mc):
    """AR BCs keep a + b i + c j + d i j unchanged under a normalised symmetric PSF (Sec. 2)."""
    h = qsym_psf(mr, mc, seed=6)
    I, J = np.meshgrid(np.arange(nr), np.arange(nc), indexing="ij")
    f = 0.3 + 0.7 * I - 0.2 * J + 0.05 * I * J
    np.testing.assert_allclose(O.blur(f, h, O.AR), f, atol=1e-12)


def test_reflective_does_not_reproduce_linear():
    h = qsym_psf(2, 2, seed=6)
    I, J = np.meshgrid(np.arange(8), np.arange(8), indexing="ij")
    f = 0.5 + 0.1 * I
    assert np.abs(O.blur(f, h, O.R) - f).max() > 1e-3


@pytest.mark.parametrize("bc", [O.AR, O.R])
@pytest.mark.parametrize("nr,nc,mr,mc", SHAPES)
def test_blur_adjoint_identity(nr, nc, mr, mc, bc):
    h = qsym_psf(mr, mc, seed=7)
    rng = np.random.default_rng(8)
    x = rng.standard_normal((nr, nc))
    y = rng.standard_normal((nr, nc))
    lhs = float((O.blur(x, h, bc) * y).sum())
    rhs = float((x * O.blur_adjoint(y, h, bc)).sum())
    assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + 1.0)


@pytest.mark.parametrize("bc", [O.AR, O.R])
def test_blur_at_matches_blur(bc):
    h = qsym_psf(3, 2, seed=9)
    rng = np.random.default_rng(10)
    x = rng.standard_normal((11, 9))
    y = O.blur(x, h, bc)
    for (i, j) in [(0, 0), (0, 8), (10, 0), (10, 8), (1, 4), (5, 5), (9, 1), (2, 7)]:
        assert abs(O.blur_at(x, h, bc, i, j) - y[i, j]) < 1e-13


@pytest.mark.parametrize("bc", [O.AR, O.R])
def test_zero_padded_disk_gives_same_blur(bc):
    """Zero padding the radius-7 disk from 15x15 to 31x31 leaves H unchanged."""
    x = synth.piecewise_constant_image(40, 36, seed=3)
    h15 = synth.disk_psf(7.0)
    h31 = synth.disk_psf(7.0, side=31)
    assert h15.shape == (15, 15) and int((h15 > 0).sum()) == 149
    np.testing.assert_allclose(O.blur(x, h15, bc), O.blur(x, h31, bc), atol=1e-14)


# ---------------------------------------------------------------- transforms

def test_dst1_matches_paper_matrix_and_is_involution():
    for m in (1, 2, 5, 8):
        S = paper_S(m)
        B = O.transform_matrix(m + 2, O.AR)
        np.testing.assert_allclose(B[1:-1, 1:-1], S, atol=1e-14)
        np.testing.assert_allclose(S @ S, np.eye(m), atol=1e-14)
        np.testing.assert_allclose(S, S.T, atol=0)


def test_dct_matches_paper_matrix_and_is_orthogonal():
    for n in (1, 2, 5, 8):
        C = paper_C(n)
        np.testing.assert_allclose(O.transform_matrix(n, O.R), C.T, atol=1e-14)
        np.testing.assert_allclose(C @ C.T, np.eye(n), atol=1e-14)


@pytest.mark.parametrize("bc", [O.AR, O.R])
def test_transform_roundtrip(bc):
    rng = np.random.default_rng(11)
    x = rng.standard_normal((6, 9))
    for ax in (0, 1):
        np.testing.assert_allclose(O.transform_inv(O.transform_fwd(x, bc, ax), bc, ax), x, atol=1e-14)
        B = O.transform_matrix(x.shape[ax], bc)
        ref = B @ x if ax == 0 else x @ B.T
        np.testing.assert_allclose(O.transform_fwd(x, bc, ax), ref, atol=1e-13)


# ---------------------------------------------------------------- TV operator

def test_tv_operator_is_gradient_of_tv_functional():
    """L(u) u = grad_u sum sqrt(|D u|^2 + beta^2), checked by central differences."""
    rng = np.random.default_rng(12)
    u = rng.uniform(0, 1, (6, 7))
    beta = 0.3

    def tv(v):
        return np.sqrt(O.grad_r(v) ** 2 + O.grad_c(v) ** 2 + beta * beta).sum()

    g = O.tv_apply(O.diffusivity(u, beta), u)
    eps = 1e-6
    fd = np.zeros_like(u)
    for i in range(u.shape[0]):
        for j in range(u.shape[1]):
            e = np.zeros_like(u)
            e[i, j] = eps
            fd[i, j] = (tv(u + e) - tv(u - e)) / (2 * eps)
    np.testing.assert_allclose(g, fd, atol=1e-7)


def test_tv_operator_symmetric_psd_kills_constants():
    rng = np.random.default_rng(13)
    u = rng.uniform(0, 1, (5, 8))
    w = O.diffusivity(u, 0.05)
    L = dense(lambda y: O.tv_apply(w, y), 5, 8)
    np.testing.assert_allclose(L, L.T, atol=1e-12)
    assert np.linalg.eigvalsh(L).min() > -1e-9
    np.testing.assert_allclose(L @ np.ones(40), 0.0, atol=1e-10)
    np.testing.assert_allclose(np.diag(L), O.tv_diag(w).ravel(), atol=1e-12)


def test_tv_constant_field_is_scaled_neumann_laplacian():
    """For constant u, w = 1/beta and L = beta^-1 (Neumann Laplacian), whose DCT-II eigenvalues
    are beta^-1 (4 sin^2(i pi / 2 n_r) + 4 sin^2(j pi / 2 n_c)) (textbook closed form)."""
    nr, nc, beta = 6, 9, 0.2
    w = O.diffusivity(np.full((nr, nc), 0.37), beta)
    L = dense(lambda y: O.tv_apply(w, y), nr, nc)
    C = np.kron(paper_C(nr), paper_C(nc))
    Lam = C.T @ L @ C
    i = np.arange(nr)[:, None]
    j = np.arange(nc)[None, :]
    closed = (4 * np.sin(i * np.pi / (2 * nr)) ** 2 + 4 * np.sin(j * np.pi / (2 * nc)) ** 2) / beta
    np.testing.assert_allclose(Lam, np.diag(closed.ravel()), atol=1e-11)
    np.testing.assert_allclose(O.spectrum_L(w, O.R), closed, atol=1e-11)


@pytest.mark.parametrize("bc", [O.AR, O.R])
@pytest.mark.parametrize("nr,nc", [(5, 8), (7, 6), (9, 9)])
def test_spectrum_L_is_diag_of_transformed_L(nr, nc, bc):
    rng = np.random.default_rng(14)
    w = O.diffusivity(rng.uniform(0, 1, (nr, nc)), 0.1)
    L = dense(lambda y: O.tv_apply(w, y), nr, nc)
    U = np.kron(O.transform_matrix(nr, bc), O.transform_matrix(nc, bc))
    np.testing.assert_allclose(O.spectrum_L(w, bc).ravel(), np.diag(U @ L @ U.T), atol=1e-12)


# ---------------------------------------------------------------- projections / preconditioners

def _argmin_in_algebra(A, U):
    """argmin_{B = U^T diag(lam) U} ||B - A||_F by least squares over the basis U^T e_k e_k^T U."""
    n = A.shape[0]
    basis = np.stack([np.outer(U[k], U[k]).ravel() for k in range(n)], axis=1)
    lam, *_ = np.linalg.lstsq(basis, A.ravel(), rcond=None)
    return U.T @ np.diag(lam) @ U


def test_proposition_hat_s():
    """hat-s(A) = blkdiag(A_11, s(A(2:n-1, 2:n-1)), A_nn), s(A) = S diag(S A S) S (Sec. 3.1)."""
    rng = np.random.default_rng(15)
    n = 7
    A = rng.standard_normal((n, n))
    hat = _argmin_in_algebra(A, O.transform_matrix(n, O.AR))
    S = paper_S(n - 2)
    inner = A[1:-1, 1:-1]
    s_inner = S @ np.diag(np.diag(S @ inner @ S)) @ S
    np.testing.assert_allclose(s_inner, _argmin_in_algebra(inner, S), atol=1e-12)
    expect = np.zeros((n, n))
    expect[0, 0] = A[0, 0]
    expect[-1, -1] = A[-1, -1]
    expect[1:-1, 1:-1] = s_inner
    np.testing.assert_allclose(hat, expect, atol=1e-12)


def _dense_preconditioner(u, h, bc, alpha, beta, nr, nc, scaled):
    """X = H_alg^T H_alg + alpha proj(L), optionally D^1/2 X D^1/2, with proj = Frobenius argmin."""
    U = np.kron(O.transform_matrix(nr, bc), O.transform_matrix(nc, bc))
    w = O.diffusivity(u, beta)
    H = dense(lambda x: O.blur(x, h, bc), nr, nc)
    L = dense(lambda y: O.tv_apply(w, y), nr, nc)
    Hp = _argmin_in_algebra(H, U)
    X = Hp.T @ Hp + alpha * _argmin_in_algebra(L, U)
    if scaled:
        d = np.sqrt(1.0 + alpha * np.diag(L))
        X = d[:, None] * X * d[None, :]
    return X


@pytest.mark.parametrize("bc", [O.AR, O.R])
@pytest.mark.parametrize("kind", [O.PC_FAST, O.PC_DFAST])
def test_preconditioner_solve_matches_dense_definition(bc, kind):
    nr, nc, alpha, beta = 6, 5, 0.05, 0.1
    h = qsym_psf(1, 2, seed=16)
    rng = np.random.default_rng(17)
    u = rng.uniform(0, 1, (nr, nc))
    r = rng.standard_normal((nr, nc))
    X = _dense_preconditioner(u, h, bc, alpha, beta, nr, nc, kind == O.PC_DFAST)
    P = O.precond_setup(u, h, bc, alpha, beta, kind)
    z = O.precond_apply(r, P)
    np.testing.assert_allclose(z.ravel(), np.linalg.solve(X, r.ravel()), rtol=1e-10, atol=1e-10)


def test_diag_preconditioner_is_eq_D():
    rng = np.random.default_rng(18)
    u = rng.uniform(0, 1, (5, 6))
    h = qsym_psf(1, 1)
    P = O.precond_setup(u, h, O.AR, 0.1, 0.2, O.PC_DIAG)
    r = rng.standard_normal((5, 6))
    d = 1.0 + 0.1 * O.tv_diag(O.diffusivity(u, 0.2))
    np.testing.assert_allclose(O.precond_apply(r, P), r / d, rtol=1e-14)


# ---------------------------------------------------------------- PCG and the FP loop

@pytest.mark.parametrize("bc", [O.AR, O.R])
def test_pcg_matches_dense_solve(bc):
    nr, nc, alpha, beta = 7, 6, 1e-2, 0.1
    h = qsym_psf(2, 1, seed=19)
    rng = np.random.default_rng(20)
    u = rng.uniform(0, 1, (nr, nc))
    b = rng.standard_normal((nr, nc))
    w = O.diffusivity(u, beta)
    A = dense(lambda x: O.normal_apply(x, h, bc, w, alpha), nr, nc)
    np.testing.assert_allclose(A, A.T, atol=1e-12)
    assert np.linalg.eigvalsh(A).min() > 0
    x, k, rr, ok = O.fp_step(u, b, h, bc, alpha, beta, O.PC_DFAST, 1e-13, 500)
    assert ok and k >= 1
    np.testing.assert_allclose(x.ravel(), np.linalg.solve(A, b.ravel()), rtol=1e-9, atol=1e-9)


def test_exact_preconditioner_alpha_zero_one_iteration():
    """Reflective BCs and alpha = 0: R = H^T H = A (Sec. 3.1), so PCG stops after one step."""
    v = synth.piecewise_constant_image(16, 12, seed=21)
    h = synth.gaussian_psf(1.0)
    b = O.blur_adjoint(v, h, O.R)
    x, k, rr, ok = O.fp_step(v * 0.5, b, h, O.R, 0.0, 0.1, O.PC_FAST, 1e-10, 50)
    assert ok and k == 1


def test_exact_preconditioner_constant_lag_one_iteration():
    """Reflective BCs and constant u_lag: L is in the cosine algebra, so R = A: one step."""
    h = synth.gaussian_psf(1.0)
    rng = np.random.default_rng(22)
    b = rng.standard_normal((12, 10))
    x, k, rr, ok = O.fp_step(np.full((12, 10), 0.4), b, h, O.R, 0.05, 0.1, O.PC_FAST, 1e-10, 50)
    assert ok and k == 1


def test_pcg_zero_residual_is_zero_iterations():
    h = synth.gaussian_psf(1.0)
    u = synth.piecewise_constant_image(10, 10, seed=23)
    w = O.diffusivity(u, 0.1)
    b = O.normal_apply(u, h, O.AR, w, 1e-2)
    x, k, rr, ok = O.fp_step(u, b, h, O.AR, 1e-2, 0.1, O.PC_DFAST, 1e-6, 50)
    assert k <= 1 and ok


@pytest.mark.parametrize("bc", [O.AR, O.R])
def test_fp_functional_decreases_and_gradient_shrinks(bc):
    """With near-exact inner solves each FP step does not increase the TV functional,
    and ||g(u)|| falls (Sec. 5 reports ||g(u^k)|| tending to small values)."""
    u_true = synth.piecewise_constant_image(16, 16, seed=24)
    h = synth.gaussian_psf(1.0)
    v = synth.add_noise(O.blur(u_true, h, bc), synth.noise_direction(16, 16, 24), 0.01)
    alpha, beta = 1e-2, 0.05
    b = O.blur_adjoint(v, h, bc)
    u = v.copy()
    f = [O.tv_functional(u, v, h, bc, alpha, beta)]
    g = [np.linalg.norm(O.euler_lagrange(u, v, h, bc, alpha, beta))]
    for _ in range(8):
        u, k, rr, ok = O.fp_step(u, b, h, bc, alpha, beta, O.PC_DFAST, 1e-12, 2000)
        assert ok
        f.append(O.tv_functional(u, v, h, bc, alpha, beta))
        g.append(np.linalg.norm(O.euler_lagrange(u, v, h, bc, alpha, beta)))
    assert all(f[i + 1] <= f[i] + 1e-12 * abs(f[i]) for i in range(len(f) - 1))
    assert g[-1] < 0.1 * g[0]


def test_preconditioner_ordering_matches_tables():
    """Trend of Tables 1-1 and 2-1: iterations fall from I to D to M to D_M."""
    n = 48
    u_true = synth.piecewise_constant_image(n, n, seed=1234)
    h = synth.gaussian_psf(1.5)
    v = synth.add_noise(O.blur(u_true, h, O.AR), synth.noise_direction(n, n, 1234), 0.01)
    tot = {}
    for kind in (O.PC_DFAST, O.PC_FAST, O.PC_DIAG, O.PC_NONE):
        _, st = O.tv_deblur(v, h, O.AR, 1e-3, 1e-2, outer=2, tol=1e-6, kind=kind)
        tot[kind] = sum(st["inner_iters"])
    assert tot[O.PC_DFAST] < tot[O.PC_FAST] < tot[O.PC_DIAG] < tot[O.PC_NONE]
    assert tot[O.PC_DFAST] * 1.5 < tot[O.PC_NONE]
