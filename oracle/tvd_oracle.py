"""Plain FP64 CPU oracle for the PCG inner step of lagged-diffusivity TV deblurring.

TEST INFRASTRUCTURE ONLY. This module is the slow, obviously correct reference
that the CUDA path is checked against. Only the test suite, the package smoke
check and the benchmark's CPU-baseline leg may import it; the library itself
never calls it and has no CPU fallback.

Everything is float64 numpy/scipy, written from the paper's definitions
(Bai, Donatelli, Serra-Capizzano, "Fast preconditioners for total variation
deblurring with anti-reflective boundary conditions"):

* boundary extension and blur: Sec. 2, eq. (blurred1d:matrixform), eq. (anti1d),
  the reflective rule of Sec. 2 and the 2D corner formulas of Sec. 2;
* lagged-diffusivity operator L(u) and the fixed-point step: Sec. 1, eqs. (el), (fp);
* optimal preconditioners R, D_R (cosine algebra, eqs. (R), (D), (R2), (DR2)) and
  M, D_M (sine algebra with hat-S, eqs. (M), (hats), the Proposition and the
  2D section 3.2), with eigenvalues from eqs. (symb), (lambda), (gridy);
* PCG: Golub & Van Loan, Algorithm 10.3.1, as cited in Sec. 1, with the stopping
  rule ||r_k|| / ||r_0|| < tol of Sec. 5.

Readings where the paper is silent or garbled:

* L(u) is discretised as D_r^T W D_r + D_c^T W D_c with forward differences that
  vanish on the last row / column (zero Neumann, eq. (el)), W = diag(psi^-1),
  psi = sqrt(|D u|^2 + beta^2) per pixel, unit grid spacing.
* The data term is read as 1/2 ||H u - v||^2; then eq. (fp) is exactly the
  lagged-diffusivity stationarity condition of the functional below.
* The AR transform T_n is sampled on y_i = (i-1) pi / (n-1), i = 1..n; the
  eigenvalue for the last basis vector (y/pi) is h_hat(0) as eq. (gridy) orders it.
* The cosine transform C is used as the frequency-by-space orthonormal DCT-II
  (scipy's ``dct(type=2, norm='ortho')``), with the algebra {C^T Lambda C}.
* Level-2 projections are computed as U^T diag(U A U^T) U with U the 2D
  transform (equal to the Q-permuted level-2 construction of Sec. 3.2).
* The diagonal ("D") preconditioner of the tables is D = I + alpha diag(L), eq. (D).
* PCG uses the Fletcher-Reeves beta of Algorithm 10.3.1, the recursive
  residual, and a strict ``<`` test after each residual update; ||r_0|| = 0
  means zero iterations. The iteration count is the number of products with A.

Index conventions: images are (n_rows, n_cols) float64 arrays, element (i, j)
row-major. A PSF is a (2 m_r + 1, 2 m_c + 1) array with h[m_r + a, m_c + b] =
h_{a,b}; it must be quadrantally symmetric for the fast preconditioners.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft

AR = "ar"   # anti-reflective boundary conditions
R = "r"     # reflective (Neumann) boundary conditions

PC_NONE = "none"     # I: no preconditioner
PC_DIAG = "diag"     # D = I + alpha diag(L(u)), eq. (D)
PC_FAST = "fast"     # R (reflective) or M (anti-reflective), eqs. (R2), (M)
PC_DFAST = "dfast"   # D_R = D^1/2 R D^1/2 or D_M = D^1/2 M D^1/2
PC_FASTD = "fastd"   # R_D / M_D: the optimal preconditioner of the scaled system, eq. (scalesys)


# --------------------------------------------------------------------------
# Boundary extension, Sec. 2
# --------------------------------------------------------------------------

def _ext_index_1d(t: int, n: int, bc: str):
    """Return [(index, coefficient), ...] giving x~_t as a combination of x_0..x_{n-1}.

    0-based form of eq. (anti1d): x~_{-j} = 2 x_0 - x_j and
    x~_{n-1+j} = 2 x_{n-1} - x_{n-1-j}; reflective rule of Sec. 2:
    x~_{-j} = x_{j-1} and x~_{n-1+j} = x_{n-j}.
    """
    if 0 <= t < n:
        return [(t, 1.0)]
    if bc == AR:
        if t < 0:
            return [(0, 2.0), (-t, -1.0)]
        return [(n - 1, 2.0), (2 * (n - 1) - t, -1.0)]
    if bc == R:
        if t < 0:
            return [(-t - 1, 1.0)]
        return [(2 * n - 1 - t, 1.0)]
    raise ValueError(bc)


def extend(x: np.ndarray, mr: int, mc: int, bc: str) -> np.ndarray:
    """Extended image x~ of shape (n_r + 2 m_r, n_c + 2 m_c); x~[i+m_r, j+m_c] = x~_{i,j}.

    Edges follow the 1D rules of Sec. 2 along the crossing direction. For AR,
    the four corner blocks follow the explicit corner formulas of Sec. 2, e.g.
    x~_{-i,-j} = 4 x_{0,0} - 2 x_{0,j} - 2 x_{i,0} + x_{i,j} (0-based). For R the
    corner blocks are the reflection in both directions.
    """
    x = np.asarray(x, dtype=np.float64)
    nr, nc = x.shape
    out = np.zeros((nr + 2 * mr, nc + 2 * mc))
    out[mr:mr + nr, mc:mc + nc] = x
    if bc == R:
        # reflection: x~_{-j} = x_{j-1}, x~_{n-1+j} = x_{n-j}, in each direction
        ir = np.concatenate([np.arange(mr - 1, -1, -1), np.arange(nr), np.arange(nr - 1, nr - 1 - mr, -1)])
        ic = np.concatenate([np.arange(mc - 1, -1, -1), np.arange(nc), np.arange(nc - 1, nc - 1 - mc, -1)])
        return x[np.ix_(ir, ic)].copy()
    if bc != AR:
        raise ValueError(bc)
    i = np.arange(1, mr + 1)          # distance outside, rows
    j = np.arange(1, mc + 1)          # distance outside, columns
    # edge strips, eq. (anti1d) along the crossing direction
    out[mr - i, mc:mc + nc] = 2.0 * x[0, :][None, :] - x[i, :]
    out[mr + nr - 1 + i, mc:mc + nc] = 2.0 * x[nr - 1, :][None, :] - x[nr - 1 - i, :]
    out[mr:mr + nr, mc - j] = 2.0 * x[:, 0][:, None] - x[:, j]
    out[mr:mr + nr, mc + nc - 1 + j] = 2.0 * x[:, nc - 1][:, None] - x[:, nc - 1 - j]
    # the four corner formulas of Sec. 2, with I, J the outside distances
    I, J = np.meshgrid(i, j, indexing="ij")
    for (bi, mi, oi) in ((0, I, mr - I), (nr - 1, nr - 1 - I, mr + nr - 1 + I)):
        for (bj, mj, oj) in ((0, J, mc - J), (nc - 1, nc - 1 - J, mc + nc - 1 + J)):
            out[oi, oj] = 4.0 * x[bi, bj] - 2.0 * x[bi, mj] - 2.0 * x[mi, bj] + x[mi, mj]
    return out


def extend_adjoint(z: np.ndarray, mr: int, mc: int, bc: str) -> np.ndarray:
    """Transpose of ``extend``: folds an extended array back onto the n_r x n_c grid.

    The extension acts separately on rows and columns (the AR corner formulas
    are the composition of the two 1D rules), so its transpose applies the
    transposed 1D rule along each axis in turn.
    """
    z = np.asarray(z, dtype=np.float64)
    nr = z.shape[0] - 2 * mr
    nc = z.shape[1] - 2 * mc
    # fold the row direction: (n_r + 2 m_r, n_c + 2 m_c) -> (n_r, n_c + 2 m_c)
    t = np.zeros((nr, z.shape[1]))
    for I in range(-mr, nr + mr):
        for (ii, ci) in _ext_index_1d(I, nr, bc):
            t[ii, :] += ci * z[I + mr, :]
    out = np.zeros((nr, nc))
    for J in range(-mc, nc + mc):
        for (jj, cj) in _ext_index_1d(J, nc, bc):
            out[:, jj] += cj * t[:, J + mc]
    return out


# --------------------------------------------------------------------------
# Blur operator H and its adjoint, Sec. 2, eq. (blurred1d:matrixform)
# --------------------------------------------------------------------------

def _psf_halfwidths(h: np.ndarray):
    pr, pc = h.shape
    if pr % 2 == 0 or pc % 2 == 0:
        raise ValueError("PSF sides must be odd")
    return pr // 2, pc // 2


def blur(x: np.ndarray, h: np.ndarray, bc: str) -> np.ndarray:
    """y = H x: extend x by the BC, then v_{ij} = sum_{a,b} h_{a,b} x~_{i-a, j-b}."""
    x = np.asarray(x, dtype=np.float64)
    mr, mc = _psf_halfwidths(h)
    nr, nc = x.shape
    xe = extend(x, mr, mc, bc)
    y = np.zeros((nr, nc))
    for a in range(-mr, mr + 1):
        for b in range(-mc, mc + 1):
            hab = h[mr + a, mc + b]
            if hab != 0.0:
                y += hab * xe[mr - a:mr - a + nr, mc - b:mc - b + nc]
    return y


def blur_adjoint(y: np.ndarray, h: np.ndarray, bc: str) -> np.ndarray:
    """x = H^T y = E^T C^T y, with C the convolution on the extended grid."""
    y = np.asarray(y, dtype=np.float64)
    mr, mc = _psf_halfwidths(h)
    nr, nc = y.shape
    z = np.zeros((nr + 2 * mr, nc + 2 * mc))
    for a in range(-mr, mr + 1):
        for b in range(-mc, mc + 1):
            hab = h[mr + a, mc + b]
            if hab != 0.0:
                z[mr - a:mr - a + nr, mc - b:mc - b + nc] += hab * y
    return extend_adjoint(z, mr, mc, bc)


def blur_at(x: np.ndarray, h: np.ndarray, bc: str, i: int, j: int) -> float:
    """(H x)_{i,j} for a single output pixel, evaluated directly from the definition.

    Used to check full-size results on sampled pixels without forming H x.
    """
    x = np.asarray(x, dtype=np.float64)
    mr, mc = _psf_halfwidths(h)
    nr, nc = x.shape
    acc = 0.0
    for a in range(-mr, mr + 1):
        for b in range(-mc, mc + 1):
            hab = h[mr + a, mc + b]
            if hab == 0.0:
                continue
            I, J = i - a, j - b
            r_in, c_in = 0 <= I < nr, 0 <= J < nc
            if bc == AR and not r_in and not c_in:
                bi, mi = (0, -I) if I < 0 else (nr - 1, 2 * (nr - 1) - I)
                bj, mj = (0, -J) if J < 0 else (nc - 1, 2 * (nc - 1) - J)
                val = 4.0 * x[bi, bj] - 2.0 * x[bi, mj] - 2.0 * x[mi, bj] + x[mi, mj]
            else:
                val = 0.0
                for (ii, ci) in _ext_index_1d(I, nr, bc):
                    for (jj, cj) in _ext_index_1d(J, nc, bc):
                        val += ci * cj * x[ii, jj]
            acc += hab * val
    return acc


# --------------------------------------------------------------------------
# Lagged-diffusivity TV operator, Sec. 1, eqs. (el), (fp)
# --------------------------------------------------------------------------

def grad_r(u: np.ndarray) -> np.ndarray:
    """Forward difference along rows, zero on the last row (zero Neumann)."""
    d = np.zeros_like(u, dtype=np.float64)
    d[:-1, :] = u[1:, :] - u[:-1, :]
    return d


def grad_c(u: np.ndarray) -> np.ndarray:
    """Forward difference along columns, zero on the last column (zero Neumann)."""
    d = np.zeros_like(u, dtype=np.float64)
    d[:, :-1] = u[:, 1:] - u[:, :-1]
    return d


def grad_r_T(g: np.ndarray) -> np.ndarray:
    """Transpose of ``grad_r``."""
    out = np.zeros_like(g, dtype=np.float64)
    out[:-1, :] -= g[:-1, :]
    out[1:, :] += g[:-1, :]
    return out


def grad_c_T(g: np.ndarray) -> np.ndarray:
    """Transpose of ``grad_c``."""
    out = np.zeros_like(g, dtype=np.float64)
    out[:, :-1] -= g[:, :-1]
    out[:, 1:] += g[:, :-1]
    return out


def diffusivity(u: np.ndarray, beta: float) -> np.ndarray:
    """w = psi^-1 = (|D u|^2 + beta^2)^(-1/2) per pixel (the lagged coefficient of L(u))."""
    u = np.asarray(u, dtype=np.float64)
    return 1.0 / np.sqrt(grad_r(u) ** 2 + grad_c(u) ** 2 + beta * beta)


def tv_apply(w: np.ndarray, y: np.ndarray) -> np.ndarray:
    """L y = D_r^T W D_r y + D_c^T W D_c y for the diffusivity field w."""
    y = np.asarray(y, dtype=np.float64)
    return grad_r_T(w * grad_r(y)) + grad_c_T(w * grad_c(y))


def tv_apply_ar(w: np.ndarray, y: np.ndarray) -> np.ndarray:
    """L_AR y: the lagged-diffusivity operator with anti-reflective BCs (the remark after
    eq. (scalereb); the "AR L" of Tables 1-1 and 2-1).

    Reading: y is extended by one pixel on every side with the rule of eq. (anti1d),
    y_{-1} = 2 y_0 - y_1 and y_n = 2 y_{n-1} - y_{n-2} along each axis, the diffusivity
    at a ghost pixel is that of its neighbour inside (in 1D this is exactly the AR
    extension of u, whose difference across the border repeats the first inner one),
    and every pixel of the image takes the full divergence-form stencil
    (L y)_i = w_{i-1} (y_i - y_{i-1}) - w_i (y_{i+1} - y_i) along each axis. On the
    first and last line of an axis the two differences are equal and the weights too,
    so that axis contributes nothing there: L_AR has the interior rows of L and is not
    symmetric.
    """
    w = np.asarray(w, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    nr, nc = y.shape
    out = np.zeros_like(y)

    def axis_terms(ya, wa):
        # ya, wa: lines along axis 0 of length n; returns the divergence-form terms
        n = ya.shape[0]
        if n == 1:
            return np.zeros_like(ya)
        ye = np.concatenate([2 * ya[:1] - ya[1:2], ya, 2 * ya[-1:] - ya[-2:-1]], axis=0)   # eq. (anti1d)
        # forward-difference weights w_k for k = -1 .. n-1 (pair (k, k+1)); ghosts copy the neighbour
        we = np.concatenate([wa[:1], wa[:-1], wa[-2:-1]], axis=0)
        fwd = we * (ye[1:] - ye[:-1])            # w_k (y_{k+1} - y_k), k = -1 .. n-1
        return fwd[:-1] - fwd[1:]                # w_{i-1}(y_i - y_{i-1}) - w_i(y_{i+1} - y_i)

    out += axis_terms(y, w)
    out += axis_terms(y.T, w.T).T
    return out


def tv_diag_ar(w: np.ndarray) -> np.ndarray:
    """diag(L_AR): the 5-point stencil's diagonal, each axis's pair of weights dropped on its first
    and last line (see ``tv_apply_ar``)."""
    w = np.asarray(w, dtype=np.float64)
    nr, nc = w.shape
    d = np.zeros_like(w)
    if nr > 2:
        d[1:-1, :] += w[1:-1, :] + w[:-2, :]
    if nc > 2:
        d[:, 1:-1] += w[:, 1:-1] + w[:, :-2]
    return d


def tv_diag(w: np.ndarray) -> np.ndarray:
    """diag(L) for the diffusivity w: the sum of the coefficients of the 5-point stencil."""
    w = np.asarray(w, dtype=np.float64)
    d = np.zeros_like(w)
    d[:-1, :] += w[:-1, :]
    d[1:, :] += w[:-1, :]
    d[:, :-1] += w[:, :-1]
    d[:, 1:] += w[:, :-1]
    return d


def tv_functional(u, v, h, bc, alpha, beta) -> float:
    """1/2 ||H u - v||^2 + alpha sum_pq sqrt(|D u|_pq^2 + beta^2), eq. (mp) discretised."""
    res = blur(u, h, bc) - v
    tv = np.sqrt(grad_r(u) ** 2 + grad_c(u) ** 2 + beta * beta).sum()
    return 0.5 * float((res * res).sum()) + alpha * float(tv)


def euler_lagrange(u, v, h, bc, alpha, beta) -> np.ndarray:
    """g(u) = H^T (H u - v) + alpha L(u) u, eq. (el) (the gradient of ``tv_functional``)."""
    w = diffusivity(u, beta)
    return blur_adjoint(blur(u, h, bc) - v, h, bc) + alpha * tv_apply(w, u)


# --------------------------------------------------------------------------
# Fast transforms, Secs. 2 and 3
# --------------------------------------------------------------------------

def transform_matrix(n: int, bc: str) -> np.ndarray:
    """Rows are the orthonormal basis vectors b_k of the 1D transform U.

    AR: hat-S_n = diag(1, S_{n-2}, 1) with S_m the DST-I of eq. (lambda).
    R: the DCT-II matrix C (frequency-by-space), so that C x = dct(x, 2, 'ortho').
    """
    eye = np.eye(n)
    if bc == AR:
        B = np.zeros((n, n))
        B[0, 0] = 1.0
        B[n - 1, n - 1] = 1.0
        if n > 2:
            B[1:n - 1, 1:n - 1] = sfft.dst(np.eye(n - 2), type=1, norm="ortho", axis=0)
        return B
    if bc == R:
        return sfft.dct(eye, type=2, norm="ortho", axis=0)
    raise ValueError(bc)


def transform_fwd(x: np.ndarray, bc: str, axis: int) -> np.ndarray:
    """Apply U along ``axis``: hat-S (AR, DST-I on the interior) or the DCT-II (R)."""
    x = np.asarray(x, dtype=np.float64)
    if bc == AR:
        out = x.copy()
        n = x.shape[axis]
        if n > 2:
            sl = [slice(None)] * x.ndim
            sl[axis] = slice(1, n - 1)
            out[tuple(sl)] = sfft.dst(x[tuple(sl)], type=1, norm="ortho", axis=axis)
        return out
    return sfft.dct(x, type=2, norm="ortho", axis=axis)


def transform_inv(x: np.ndarray, bc: str, axis: int) -> np.ndarray:
    """Apply U^{-1} along ``axis``: hat-S again (it is an involution) or the DCT-III (R)."""
    if bc == AR:
        return transform_fwd(x, bc, axis)
    return sfft.idct(np.asarray(x, dtype=np.float64), type=2, norm="ortho", axis=axis)


def symbol_grid(n: int, bc: str) -> np.ndarray:
    """Frequencies at which the PSF symbol gives the eigenvalues of H.

    AR, eq. (gridy): basis vector 0 (the 1 - y/pi column) and n-1 (the y/pi
    column) take y = 0; interior basis vector k (DST-I frequency k) takes
    y = k pi / (n-1). R: DCT-II frequency k takes y = k pi / n.
    """
    k = np.arange(n, dtype=np.float64)
    if n == 1:
        return np.zeros(1)     # a single sample (a 1D signal's row axis): the constant, y = 0
    if bc == AR:
        y = k * np.pi / (n - 1)
        y[0] = 0.0
        y[n - 1] = 0.0
        return y
    return k * np.pi / n


def psf_symbol(h: np.ndarray, yr: np.ndarray, yc: np.ndarray) -> np.ndarray:
    """h_hat(y_i, y_j) = sum_{a,b} h_{a,b} exp(i (a y_i + b y_j)), eq. (symb), real part.

    For a quadrantally symmetric h the imaginary part vanishes.
    """
    mr, mc = _psf_halfwidths(h)
    ar = np.arange(-mr, mr + 1)
    ac = np.arange(-mc, mc + 1)
    Er = np.exp(1j * np.outer(yr, ar))
    Ec = np.exp(1j * np.outer(yc, ac))
    return np.real(Er @ h @ Ec.T)


def spectrum_H(h: np.ndarray, nr: int, nc: int, bc: str) -> np.ndarray:
    """Eigenvalues Lambda_H[i, j] of H in the 2D transform basis (n_r x n_c)."""
    return psf_symbol(h, symbol_grid(nr, bc), symbol_grid(nc, bc))


def _E_G(n: int, bc: str):
    """E[k,p] = b_k(p)^2 and G[k,p] = ((D_1 b_k)_p)^2, with D_1 the Neumann forward difference."""
    B = transform_matrix(n, bc)
    E = B * B
    D = np.zeros_like(B)
    D[:, :-1] = B[:, 1:] - B[:, :-1]
    return E, D * D


def spectrum_L(w: np.ndarray, bc: str) -> np.ndarray:
    """Lambda_L = diag(U L U^T) for L = D_r^T W D_r + D_c^T W D_c and U = B_r (x) B_c.

    (b_i (x) b_j)^T L (b_i (x) b_j) = sum_pq w_pq [G_r(i,p) E_c(j,q) + E_r(i,p) G_c(j,q)],
    i.e. Lambda_L = G_r W E_c^T + E_r W G_c^T. These are the eigenvalues of the
    level-2 projection c_2(L) (R) or hat-s_2(L) (AR) of Sec. 3.2.
    """
    w = np.asarray(w, dtype=np.float64)
    nr, nc = w.shape
    Er, Gr = _E_G(nr, bc)
    Ec, Gc = _E_G(nc, bc)
    return Gr @ w @ Ec.T + Er @ w @ Gc.T


def _E_F(n: int, bc: str):
    """E[k,p] = b_k(p)^2 and F[k,p] = b_k(p) b_k(p+1) (0 for p = n-1)."""
    B = transform_matrix(n, bc)
    F = np.zeros_like(B)
    F[:, :-1] = B[:, :-1] * B[:, 1:]
    return B * B, F


def spectrum_scaled(w: np.ndarray, d: np.ndarray, bc: str):
    """(Lambda_D, Lambda_L~) of R_D / M_D (Secs. 2.1, 2.2, 3.2), d = D^-1/2 per pixel.

    Lambda_D = diag(U diag(d) U^T) = E_r d E_c^T, the eigenvalues of the level-2
    projection of D^-1/2. Lambda_L~ = diag(U L~ U^T) with L~ = D^-1/2 L D^-1/2:
    for x = d o (b_i (x) b_j), x^T L x = sum_pq w_pq [(D_r x)_pq^2 + (D_c x)_pq^2],
    and expanding (D_r x)_pq^2 = b_j(q)^2 [d_{p+1,q}^2 b_i(p+1)^2 + d_pq^2 b_i(p)^2
    - 2 d_{p+1,q} d_pq b_i(p) b_i(p+1)] (and the column analogue) gives
    Lambda_L~ = E_r S E_c^T - 2 F_r gamma E_c^T - 2 E_r delta F_c^T with
    S = the D-weighted stencil diagonal, gamma_pq = w_pq d_{p+1,q} d_pq,
    delta_pq = w_pq d_{p,q+1} d_pq.
    """
    w = np.asarray(w, dtype=np.float64)
    d = np.asarray(d, dtype=np.float64)
    nr, nc = w.shape
    Er, Fr = _E_F(nr, bc)
    Ec, Fc = _E_F(nc, bc)
    d2 = d * d
    S = np.zeros_like(w)
    S[1:, :] += w[:-1, :] * d2[1:, :]
    S[:-1, :] += w[:-1, :] * d2[:-1, :]
    S[:, 1:] += w[:, :-1] * d2[:, 1:]
    S[:, :-1] += w[:, :-1] * d2[:, :-1]
    gam = np.zeros_like(w)
    gam[:-1, :] = w[:-1, :] * d[1:, :] * d[:-1, :]
    dlt = np.zeros_like(w)
    dlt[:, :-1] = w[:, :-1] * d[:, 1:] * d[:, :-1]
    lam_d = Er @ d @ Ec.T
    lam_lt = Er @ S @ Ec.T - 2.0 * (Fr @ gam @ Ec.T) - 2.0 * (Er @ dlt @ Fc.T)
    return lam_d, lam_lt


# --------------------------------------------------------------------------
# Preconditioners, Sec. 3
# --------------------------------------------------------------------------

def precond_setup(u_lag, h, bc, alpha, beta, kind, method="fp"):
    """Everything the preconditioner solve needs for the FP step at u_lag.

    Returns a dict with the diffusivity ``w``, ``D`` = 1 + alpha diag(L) (eq. (D)),
    and ``spec`` = Lambda_H^2 + alpha Lambda_L, the eigenvalues of R (eq. (R2)) or
    M (2D form of eq. (M)); D_R / D_M scale these by D^1/2 on both sides.
    With method = METHOD_REBLUR (eq. (fpp), AR BCs) the fast kinds are the
    reblurring preconditioners P, D_P, P_D of Sec. 3 (see reblur_setup).
    """
    if method in REBLUR_METHODS:
        return reblur_setup(u_lag, h, bc, alpha, beta, kind, arl=method == METHOD_REBLUR_ARL)
    w = diffusivity(u_lag, beta)
    nr, nc = w.shape
    D = 1.0 + alpha * tv_diag(w)
    P = {"kind": kind, "bc": bc, "w": w, "D": D, "alpha": alpha}
    if kind in (PC_FAST, PC_DFAST, PC_FASTD):
        lam_h = spectrum_H(h, nr, nc, bc)
        if kind == PC_FASTD:
            # R_D / M_D = H^^* H^ + alpha s_2(L~), H^ = s_2(H) s_2(D^-1/2): eigenvalues
            # Lambda_H^2 Lambda_D^2 + alpha Lambda_L~; applied to the original system as
            # D^1/2 M_D D^1/2 (PCG on eq. (scalesys) is PCG on eq. (fp) with that preconditioner)
            lam_d, lam_lt = spectrum_scaled(w, 1.0 / np.sqrt(D), bc)
            spec = lam_h * lam_h * lam_d * lam_d + alpha * lam_lt
        else:
            spec = lam_h * lam_h + alpha * spectrum_L(w, bc)
        if np.min(spec) <= 1e-300:
            raise ValueError("preconditioner spectrum is not positive")
        P["spec"] = spec
    return P


def precond_apply(r: np.ndarray, P) -> np.ndarray:
    """z = X^{-1} r for X in {I, D, R|M, D_R|D_M, R_D|M_D}.

    X^{-1} r = D^{-1/2} U^{-1} diag(spec)^{-1} U D^{-1/2} r for the scaled
    variants, with U = B_r (x) B_c applied as the 1D transform along each axis.
    """
    kind, bc = P["kind"], P["bc"]
    r = np.asarray(r, dtype=np.float64)
    if kind == PC_NONE:
        return r.copy()
    if kind == PC_DIAG:
        return r / P["D"]
    scaled = kind in (PC_DFAST, PC_FASTD)
    t = r / np.sqrt(P["D"]) if scaled else r.copy()
    if "Tr" in P:
        # reblurring preconditioners: (T_r (x) T_c) diag(spec) (T_r (x) T_c)^{-1}
        t = P["Tinv_r"] @ t @ P["Tinv_c"].T
        t = t / P["spec"]
        t = P["Tr"] @ t @ P["Tc"].T
        return t / np.sqrt(P["D"]) if scaled else t
    t = transform_fwd(transform_fwd(t, bc, 1), bc, 0)
    t = t / P["spec"]
    t = transform_inv(transform_inv(t, bc, 0), bc, 1)
    if scaled:
        t = t / np.sqrt(P["D"])
    return t


def normal_apply(x, h, bc, w, alpha) -> np.ndarray:
    """A x = H^T H x + alpha L(w) x, the matrix of the FP step, eq. (fp)."""
    return blur_adjoint(blur(x, h, bc), h, bc) + alpha * tv_apply(w, x)


# --------------------------------------------------------------------------
# PCG (Golub & Van Loan, Algorithm 10.3.1) and the FP loop, Secs. 1 and 5
# --------------------------------------------------------------------------

def pcg(apply_A, apply_M, b, x0, tol, maxit, hist=None, noise=None):
    """Preconditioned CG on A x = b from x0.

    Stops when ||r_k||_2 / ||r_0||_2 < tol (Sec. 5) or after ``maxit`` products
    with A. Returns (x, iterations, relres, converged). If ``hist`` is a list,
    the relative residual after each iteration is appended to it.

    ``noise = (rng, eps)`` (test hook, off by default) multiplies every product
    with A and every preconditioner output by (1 + eps xi), xi standard normal:
    it models rounding that differs from this implementation's, to measure how
    sensitive the iteration is to it.
    """
    if noise is not None:
        rng, eps = noise
        A0, M0 = apply_A, apply_M

        def apply_A(y):
            q = A0(y)
            return q * (1.0 + eps * rng.standard_normal(q.shape))

        def apply_M(r):
            z = M0(r)
            return z * (1.0 + eps * rng.standard_normal(z.shape))
    x = np.array(x0, dtype=np.float64, copy=True)
    r = b - apply_A(x)
    r0 = float(np.sqrt((r * r).sum()))
    if r0 == 0.0:
        return x, 0, 0.0, True
    k = 0
    rho_old = None
    p = None
    relres = 1.0
    while k < maxit:
        z = apply_M(r)
        rho = float((r * z).sum())
        k += 1
        if k == 1:
            p = z.copy()
        else:
            p = z + (rho / rho_old) * p
        q = apply_A(p)
        a = rho / float((p * q).sum())
        x = x + a * p
        r = r - a * q
        rho_old = rho
        relres = float(np.sqrt((r * r).sum())) / r0
        if hist is not None:
            hist.append(relres)
        if relres < tol:
            return x, k, relres, True
    return x, k, relres, False


def fp_step(u, b, h, bc, alpha, beta, kind, tol, maxit, hist=None, noise=None, method="fp"):
    """One lagged-diffusivity step from x0 = u: solve (H^T H + alpha L(u)) x = H^T v by PCG
    (eq. (fp)), or with method = METHOD_REBLUR (H' H + alpha L(u)) x = H' v by PBiCGstab
    (eq. (fpp)); METHOD_REBLUR_ARL puts L_AR(u) in place of L(u). b is the right-hand side."""
    P = precond_setup(u, h, bc, alpha, beta, kind, method)
    w = P["w"]
    if method in REBLUR_METHODS:
        arl = method == METHOD_REBLUR_ARL
        return bicgstab(lambda y: reblur_apply(y, h, bc, w, alpha, arl),
                        lambda r: precond_apply(r, P), b, u, tol, maxit, hist, noise)
    return pcg(lambda y: normal_apply(y, h, bc, w, alpha),
               lambda r: precond_apply(r, P), b, u, tol, maxit, hist, noise)


def tv_deblur(v, h, bc, alpha, beta, outer=10, tol=1e-6, maxit=1000,
              kind=PC_DFAST, outer_tol=0.0, noise=None, method="fp"):
    """Lagged-diffusivity FP iteration with PCG inner solves, u^0 = v (Sec. 5).

    Runs ``outer`` FP steps, or stops earlier when ||u^k - u^{k-1}|| / ||u^k||
    < outer_tol (if outer_tol > 0). Returns (u, stats) where stats holds the
    per-step inner iteration counts, residuals, relative changes and the
    relative residuals of the last two inner iterations of each step. With
    method = METHOD_REBLUR each step solves eq. (fpp) by PBiCGstab (Sec. 5); METHOD_REBLUR_ARL
    does the same with L_AR in place of L (``tv_apply_ar``).
    """
    v = np.asarray(v, dtype=np.float64)
    b = reblur_rhs(v, h, bc) if method in REBLUR_METHODS else blur_adjoint(v, h, bc)
    u = v.copy()
    stats = {"inner_iters": [], "relres": [], "rel_change": [], "converged": [], "relres_tail": []}
    for _ in range(outer):
        hist = []
        x, k, rr, ok = fp_step(u, b, h, bc, alpha, beta, kind, tol, maxit, hist, noise, method)
        stats["relres_tail"].append(hist[-2:])
        change = float(np.linalg.norm(x - u) / max(np.linalg.norm(x), 1e-300))
        stats["inner_iters"].append(k)
        stats["relres"].append(rr)
        stats["rel_change"].append(change)
        stats["converged"].append(ok)
        u = x
        if outer_tol > 0.0 and change < outer_tol:
            break
    return u, stats


# --------------------------------------------------------------------------
# Reblurring, eq. (fpp): (H' H + alpha L(u^k)) u^{k+1} = H' v with H' the AR
# blur of the PSF rotated by 180 degrees, solved by PBiCGstab; the AR algebra
# of eq. (ARalg), the projection AR(.) and the preconditioners P, D_P, P_D
# (Sec. 3.1 after eq. (fpp), the Remark on T_n, eq. (scalereb); 2D forms in
# Sec. 3.2)
# --------------------------------------------------------------------------

METHOD_FP = "fp"
METHOD_REBLUR = "reblur"
METHOD_REBLUR_ARL = "reblur_arl"     # eq. (fpp) with L_AR (the "AR+Reblur+AR L" columns)
REBLUR_METHODS = (METHOD_REBLUR, METHOD_REBLUR_ARL)


def rotated_psf(h: np.ndarray) -> np.ndarray:
    """The PSF rotated by 180 degrees (h'_{a,b} = h_{-a,-b})."""
    return np.asarray(h, dtype=np.float64)[::-1, ::-1].copy()


def reblur_apply(x, h, bc, w, alpha, arl=False) -> np.ndarray:
    """A' x = H' H x + alpha L(w) x, the matrix of eq. (fpp); with arl, L is L_AR (``tv_apply_ar``)."""
    return blur(blur(x, h, bc), rotated_psf(h), bc) + alpha * (tv_apply_ar(w, x) if arl else tv_apply(w, x))


def reblur_rhs(v, h, bc) -> np.ndarray:
    """H' v, the right-hand side of eq. (fpp)."""
    return blur(v, rotated_psf(h), bc)


def _sine(m: int) -> np.ndarray:
    """S_m of eq. (lambda) (the orthonormal DST-I, symmetric)."""
    return sfft.dst(np.eye(m), type=1, norm="ortho", axis=0)


def transform_T(n: int):
    """(T_n, T_n^{-1}) from the Remark after AR(A): T_n = hat-S_n (I + U), T_n^{-1} = (I - U) hat-S_n,
    U = [0 0 0; S p 0 S J p; 0 0 0] with p_j = 1 - j/(n-1), j = 1..n-2 (the interior of the sampled 1 - x)."""
    Sh = transform_matrix(n, AR)
    U = np.zeros((n, n))
    if n > 2:
        S = _sine(n - 2)
        p = 1.0 - np.arange(1, n - 1) / (n - 1)
        U[1:-1, 0] = S @ p
        U[1:-1, -1] = S @ p[::-1]
    I = np.eye(n)
    return Sh @ (I + U), (I - U) @ Sh


def _tau_generator(first_col: np.ndarray) -> np.ndarray:
    """z of a tau matrix T(z) - H(sigma^2 z, J sigma^2 z) from its first column c_k = z_k - z_{k+2}."""
    m = first_col.shape[0]
    z = np.zeros(m)
    for k in range(m - 1, -1, -1):
        z[k] = first_col[k] + (z[k + 2] if k + 2 < m else 0.0)
    return z


def ar_projection(A: np.ndarray) -> np.ndarray:
    """AR(A) of Sec. 3.1 for an n x n matrix A: interior block s(A(2:n-1, 2:n-1)) (the optimal sine
    projection s(B) = S diag(S B S) S), first column z_{i} + 2 sum_{k > i} z_k (1-based, rows 1..n-1)
    with z the Toeplitz generator of that interior block, last column its flip, first and last rows
    zero but for the corners."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    if n == 1:
        return A.copy()        # every 1 x 1 matrix is in the algebra (T_1 = 1)
    m = n - 2
    S = _sine(m)
    inner = A[1:-1, 1:-1]
    s_in = S @ np.diag(np.diag(S @ inner @ S)) @ S
    z = np.concatenate([_tau_generator(s_in[:, 0]), [0.0, 0.0]])
    out = np.zeros((n, n))
    out[1:-1, 1:-1] = s_in
    for i in range(n):
        out[i, 0] = z[i] + 2.0 * z[i + 1:].sum()
    out[:, -1] = out[::-1, 0]
    return out


def _swap_levels(A: np.ndarray, nr: int, nc: int) -> np.ndarray:
    """Q^T A Q of Sec. 3.2: the (i, j) entry of block (k, l) becomes the (k, l) entry of block (i, j)."""
    return A.reshape(nr, nc, nr, nc).transpose(1, 0, 3, 2).reshape(nr * nc, nr * nc)


def ar2_projection(A: np.ndarray, nr: int, nc: int) -> np.ndarray:
    """AR_2(A) = Q AR_1(Q^T AR_1(A) Q) Q^T (Sec. 3.2) for an (nr nc) x (nr nc) matrix; AR_1 applies
    AR(.) to every block."""
    def ar1(B, nb, bs):
        out = np.empty_like(B)
        for a in range(nb):
            for b in range(nb):
                out[a * bs:(a + 1) * bs, b * bs:(b + 1) * bs] = ar_projection(B[a * bs:(a + 1) * bs,
                                                                                b * bs:(b + 1) * bs])
        return out
    A1 = ar1(np.asarray(A, dtype=np.float64), nr, nc)
    A2 = ar1(_swap_levels(A1, nr, nc), nc, nr)
    return _swap_levels(A2, nc, nr)


def ar_extension(m: int) -> np.ndarray:
    """c with h_hat_z(0) = c . lam: the border eigenvalue of AR(A) from the eigenvalues lam of its
    interior sine projection (lam -> tau first column S diag(lam) S e_1 -> z -> z_1 + 2 sum z_k)."""
    S = _sine(m)
    cols = S * S[0][None, :]                   # column i: S diag(e_i) S e_1
    Z = np.stack([_tau_generator(cols[:, i]) for i in range(m)], axis=1)
    wts = np.full(m, 2.0)
    wts[0] = 1.0
    return wts @ Z


def ar_extend2(lam: np.ndarray) -> np.ndarray:
    """Eigenvalues of AR_2 from the interior ones: border rows / columns are the c-weighted sums of
    the interior along that dimension (AR(.) per level), corners along both. A dimension of length
    1 (a 1D signal's row axis) has no border to extend: there the projection is the identity."""
    nr, nc = lam.shape
    out = np.array(lam, dtype=np.float64, copy=True)
    rows = slice(1, nr - 1) if nr > 1 else slice(0, 1)
    cc = ar_extension(nc - 2)
    out[rows, 0] = out[rows, -1] = out[rows, 1:-1] @ cc
    if nr > 1:
        cr = ar_extension(nr - 2)
        out[0, :] = out[-1, :] = cr @ out[1:-1, :]
    return out


def reblur_setup(u_lag, h, bc, alpha, beta, kind, arl=False):
    """Preconditioner of eq. (fpp) (AR BCs): P = H' H + alpha AR_2(L) (eigenvalues Lambda_H^2 +
    alpha Lambda_AR2(L) in the T_n (x) T_n basis: H' = H for a symmetric PSF and H is in the AR
    algebra), D_P = D^1/2 P D^1/2, or P_D = H^' H^ + alpha AR_2(L~), H^ = H AR_2(D^-1/2), applied as
    D^1/2 P_D D^1/2 (eigenvalues Lambda_H^2 Lambda_D^2 + alpha Lambda_L~).

    With arl (L_AR of ``tv_apply_ar`` in the system): D = I + alpha diag(L_AR), eq. (D) for that
    L. AR_2(.) reads only the interior block of its argument, where L_AR equals L, so the
    eigenvalues are those of the Neumann L."""
    if bc != AR:
        raise ValueError("the reblurring preconditioners are defined for anti-reflective BCs")
    w = diffusivity(u_lag, beta)
    nr, nc = w.shape
    D = 1.0 + alpha * (tv_diag_ar(w) if arl else tv_diag(w))
    P = {"kind": kind, "bc": bc, "w": w, "D": D, "alpha": alpha,
         "method": METHOD_REBLUR_ARL if arl else METHOD_REBLUR}
    if kind in (PC_FAST, PC_DFAST, PC_FASTD):
        lam_h = spectrum_H(h, nr, nc, AR)
        if kind == PC_FASTD:
            lam_d, lam_lt = spectrum_scaled(w, 1.0 / np.sqrt(D), AR)
            spec = lam_h * lam_h * ar_extend2(lam_d) ** 2 + alpha * ar_extend2(lam_lt)
        else:
            spec = lam_h * lam_h + alpha * ar_extend2(spectrum_L(w, AR))
        if np.min(spec) <= 1e-300:
            raise ValueError("preconditioner spectrum is not positive")
        P["spec"] = spec
        P["Tr"], P["Tinv_r"] = transform_T(nr)
        P["Tc"], P["Tinv_c"] = transform_T(nc)
    return P


def bicgstab(apply_A, apply_M, b, x0, tol, maxit, hist=None, noise=None):
    """Preconditioned BiCGstab (van der Vorst 1992, cited as [V92]) on A x = b from x0, with the
    preconditioned directions p^ = M^-1 p and s^ = M^-1 s and the shadow residual r^ = r_0.

    Stops when ||r_k||_2 / ||r_0||_2 < tol (Sec. 5), tested on the half-step residual s and on
    r after each iteration, or after ``maxit`` iterations (one iteration = two products with A).
    Returns (x, iterations, relres, converged); ``hist`` and ``noise`` as for pcg.
    """
    if noise is not None:
        rng, eps = noise
        A0, M0 = apply_A, apply_M

        def apply_A(y):
            q = A0(y)
            return q * (1.0 + eps * rng.standard_normal(q.shape))

        def apply_M(r):
            z = M0(r)
            return z * (1.0 + eps * rng.standard_normal(z.shape))
    x = np.array(x0, dtype=np.float64, copy=True)
    r = b - apply_A(x)
    r0 = float(np.sqrt((r * r).sum()))
    if r0 == 0.0:
        return x, 0, 0.0, True
    rhat = r.copy()
    rho_old = alpha = omega = 1.0
    v = np.zeros_like(r)
    p = np.zeros_like(r)
    k = 0
    relres = 1.0
    while k < maxit:
        k += 1
        rho = float((rhat * r).sum())
        if rho == 0.0:
            return x, k, relres, False
        if k == 1:
            p = r.copy()
        else:
            beta = (rho / rho_old) * (alpha / omega)
            p = r + beta * (p - omega * v)
        phat = apply_M(p)
        v = apply_A(phat)
        alpha = rho / float((rhat * v).sum())
        s = r - alpha * v
        relres = float(np.sqrt((s * s).sum())) / r0
        if relres < tol:
            x = x + alpha * phat
            if hist is not None:
                hist.append(relres)
            return x, k, relres, True
        shat = apply_M(s)
        t = apply_A(shat)
        tt = float((t * t).sum())
        if tt == 0.0:
            return x, k, relres, False
        omega = float((t * s).sum()) / tt
        x = x + alpha * phat + omega * shat
        r = s - omega * t
        relres = float(np.sqrt((r * r).sum())) / r0
        if hist is not None:
            hist.append(relres)
        if relres < tol:
            return x, k, relres, True
        if omega == 0.0:
            return x, k, relres, False
        rho_old = rho
    return x, k, relres, False


# --------------------------------------------------------------------------
# Adjoint of the converged fixed point (implicit differentiation of the
# Euler-Lagrange equation g(u*, theta) = 0, eq. (el); not a construction of
# the paper: it differentiates the paper's method with respect to alpha,
# beta and the PSF)
# --------------------------------------------------------------------------

def tv_hessian_apply(u, beta, x):
    """nabla^2 J_beta(u) x for J_beta(u) = sum_pq psi_pq, psi = sqrt(|D u|^2 + beta^2).

    The gradient of J_beta is D^T (psi^-1 D u) = L(u) u; differentiating it
    once more per cell gives D^T [psi^-1 D x - psi^-3 (D u . D x) D u] with
    the forward differences D = (D_r, D_c) of ``grad_r`` / ``grad_c``.
    """
    u = np.asarray(u, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    dr, dc = grad_r(u), grad_c(u)
    psi = np.sqrt(dr * dr + dc * dc + beta * beta)
    xr, xc = grad_r(x), grad_c(x)
    s = (dr * xr + dc * xc) / psi ** 3
    return grad_r_T(xr / psi - s * dr) + grad_c_T(xc / psi - s * dc)


def jacobian_apply(u, h, bc, alpha, beta, x):
    """J x = H^T H x + alpha nabla^2 J_beta(u) x: the derivative of g(u) of eq. (el) in u (SPD)."""
    return blur_adjoint(blur(x, h, bc), h, bc) + alpha * tv_hessian_apply(u, beta, x)


def adjoint_solve(u, h, bc, alpha, beta, rhs, tol=1e-12, maxit=20000, kind=PC_NONE):
    """lambda with J(u) lambda = rhs, by the PCG of Algorithm 10.3.1, from 0.

    ``kind`` picks the preconditioner: the FP step's one at u (``precond_setup``,
    built for H^T H + alpha L(u), which bounds J from above); PC_NONE by default.
    Returns (lambda, iterations, ||r|| / ||r_0||, converged).
    """
    rhs = np.asarray(rhs, dtype=np.float64)
    P = precond_setup(u, h, bc, alpha, beta, kind)
    return pcg(lambda y: jacobian_apply(u, h, bc, alpha, beta, y), lambda r: precond_apply(r, P), rhs,
               np.zeros_like(rhs), tol, maxit)


def newton_polish(u, v, h, bc, alpha, beta, tol=1e-10, max_steps=30, cg_tol=1e-12, maxit=20000,
                  kind=PC_DFAST):
    """Finish the fixed point of eq. (fp) by Newton's method on g(u) = 0, eq. (el).

    Not a step of the paper: the lagged-diffusivity iteration converges only
    linearly, and the adjoint needs u* to a tolerance it reaches slowly. From an
    FP iterate u each step solves J(u) d = g(u) (``adjoint_solve`` with the FP
    step's preconditioner at u, to ||r|| / ||r_0|| < cg_tol) and moves to
    u - t d, where t = 1, halved while ||g(u - t d)|| >= ||g(u)|| (at most 10
    times; a step that never lowers ||g|| ends the loop, unconverged). A full
    step with ||d|| / ||u - d|| < tol is taken as it is: there ||g|| sits at
    its rounding floor and need not fall. The loop stops after the step with
    ||t d|| / ||u - t d|| < tol (converged), or after max_steps. Returns
    (u, stats): per step the relative change, ||g|| before the step, the step
    length t and the CG iterations; ``converged``; and ``g_norm_final`` of the
    returned u.
    """
    u = np.array(u, dtype=np.float64, copy=True)
    v = np.asarray(v, dtype=np.float64)
    g = euler_lagrange(u, v, h, bc, alpha, beta)
    gn = float(np.linalg.norm(g))
    stats = {"rel_change": [], "g_norm": [], "t": [], "cg_iters": [], "converged": False}
    for _ in range(max_steps):
        if gn == 0.0:
            stats["converged"] = True
            break
        d, k, _, _ = adjoint_solve(u, h, bc, alpha, beta, g, cg_tol, maxit, kind)
        t = 1.0
        for halving in range(11):
            u_new = u - t * d
            g_new = euler_lagrange(u_new, v, h, bc, alpha, beta)
            gn_new = float(np.linalg.norm(g_new))
            tiny = halving == 0 and float(np.linalg.norm(d)) < tol * float(np.linalg.norm(u_new))
            if gn_new < gn or tiny:
                break
            t *= 0.5
        else:
            break
        change = t * float(np.linalg.norm(d)) / max(float(np.linalg.norm(u_new)), 1e-300)
        stats["rel_change"].append(change)
        stats["g_norm"].append(gn)
        stats["t"].append(t)
        stats["cg_iters"].append(k)
        u, g, gn = u_new, g_new, gn_new
        if change < tol:
            stats["converged"] = True
            break
    stats["g_norm_final"] = gn
    return u, stats


def unit_psf(h, a, b):
    """The PSF with a single 1 at tap (a, b) (offsets from the centre): dH/dh_ab."""
    e = np.zeros_like(np.asarray(h, dtype=np.float64))
    mr, mc = _psf_halfwidths(e)
    e[mr + a, mc + b] = 1.0
    return e


def fixed_point_gradients(u, v, h, bc, alpha, beta, lam):
    """d loss / d theta = -lam^T dF/dtheta at the fixed point u of F(u, theta) = g(u) = 0.

    F = H^T (H u - v) + alpha grad J_beta(u) (eq. (el)), lam solves J lam = d loss / d u. Then
      dF/dalpha = grad J_beta(u) = L(u) u,
      dF/dbeta  = alpha D^T [ d(psi^-1)/d beta D u ] = alpha D^T [ -beta psi^-3 D u ],
      dF/dh_ab  = E_ab^T (H u - v) + H^T E_ab u with E_ab = dH/dh_ab (H is linear in h),
    so lam^T dF/dh_ab = (E_ab lam) . (H u - v) + (H lam) . (E_ab u).
    Returns (dl_dalpha, dl_dbeta, dl_dh) with dl_dh shaped like h (every tap free).
    """
    u = np.asarray(u, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    w = diffusivity(u, beta)
    dl_dalpha = -float(np.sum(lam * tv_apply(w, u)))
    dr, dc = grad_r(u), grad_c(u)
    psi3 = (1.0 / w) ** 3
    dF_dbeta = alpha * (grad_r_T(-beta * dr / psi3) + grad_c_T(-beta * dc / psi3))
    dl_dbeta = -float(np.sum(lam * dF_dbeta))
    res = blur(u, h, bc) - np.asarray(v, dtype=np.float64)
    hlam = blur(lam, h, bc)
    mr, mc = _psf_halfwidths(h)
    dl_dh = np.zeros_like(np.asarray(h, dtype=np.float64))
    for a in range(-mr, mr + 1):
        for b in range(-mc, mc + 1):
            e = unit_psf(h, a, b)
            dl_dh[mr + a, mc + b] = -(float(np.sum(blur(lam, e, bc) * res)) + float(np.sum(hlam * blur(u, e, bc))))
    return dl_dalpha, dl_dbeta, dl_dh
