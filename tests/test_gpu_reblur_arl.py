"""GPU parity of the reblurring method with anti-reflective BCs on L as well
(TVD_METHOD_REBLUR_ARL, the "AR+Reblur+AR L" columns of Tables 1-1 and 2-1).

* L_AR (tv_operator_apply on such a plan) element by element against the
  oracle's ``tv_apply_ar``: FP64 1e-12, float 1e-5 of the largest entry, on
  images and on 1D signals.
* The P, D_P, P_D solves (D from diag(L_AR)) against the oracle, with the
  tolerances of the REBLUR method's tests.
* PBiCGstab on one FP step and a 10-step deblur in FP64, held to the oracle's
  rounding envelope (tests/parity.py); MIXED deblurs with both sides solving
  each step to 1e-10 within 1e-5 of the oracle.
* The eq. (fpp) residual norm that tv_deblur reports per step (with L_AR).
"""
import numpy as np
import pytest

import oracle as O
from paper_1011_5964_gb300 import synth
from parity import N_PERTURBED, check_counts, count_spread, image_bound, noise

pytestmark = pytest.mark.gpu
ARL = O.METHOD_REBLUR_ARL


@pytest.fixture(scope="module")
def tdev():
    import torch
    import paper_1011_5964_gb300 as pkg
    pkg.load_library()
    return torch, pkg, torch.device("cuda:0")


def observe(n_rows, n_cols, h, noise_level, seed):
    u_true = synth.piecewise_constant_image(n_rows, n_cols, seed=seed)
    return synth.add_noise(O.blur(u_true, h, O.AR), synth.noise_direction(n_rows, n_cols, seed), noise_level)


def maxrel(z, ref):
    return float(np.abs(z - ref).max() / np.abs(ref).max())


@pytest.mark.parametrize("nr,nc", [(5, 6), (37, 53), (64, 64), (1, 203), (130, 3)])
@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_l_ar_matches_the_oracle(tdev, nr, nc, mode):
    torch, pkg, dev = tdev
    rng = np.random.default_rng(nr * 7 + nc)
    u, x = rng.uniform(0, 1, (nr, nc)), rng.standard_normal((nr, nc))
    if mode == "mixed":
        u, x = (a.astype(np.float32).astype(np.float64) for a in (u, x))
    dt = torch.float64 if mode == "fp64" else torch.float32
    h = np.ones((1, 1))
    with pkg.Plan(nr, nc, h, bc="ar", pc="dfast", mode=mode, method="reblur_arl") as plan:
        assert plan.method == "reblur_arl"
        y = plan.tv_operator(torch.tensor(u, dtype=dt, device=dev), 0.1,
                             torch.tensor(x, dtype=dt, device=dev)).double().cpu().numpy()
    ref = O.tv_apply_ar(O.diffusivity(u, 0.1), x)
    assert maxrel(y, ref) < (1e-12 if mode == "fp64" else 1e-5)


SHAPES = [(37, 53), (64, 64), (5, 6), (130, 128), (1, 203)]
FORMS = [("fp64", "fft", 1e-10), ("mixed", "fft", 1e-3), ("mixed", "gemm", 3e-2)]


@pytest.mark.parametrize("mode,transform,tol", FORMS)
@pytest.mark.parametrize("kind", ["fast", "dfast", "fastd"])
@pytest.mark.parametrize("nr,nc", SHAPES)
def test_arl_preconditioner_solve(tdev, nr, nc, kind, mode, transform, tol):
    torch, pkg, dev = tdev
    if nr == 1 and transform == "gemm":
        pytest.skip("1D plans use the FFT form only")
    h = synth.gaussian_psf(1.0, half_width=min(3, max(nr - 2, 0), nc - 2)) if nr > 1 else \
        synth.out_of_focus_psf_1d(4)
    rng = np.random.default_rng(nr + 17 * nc)
    u = synth.piecewise_constant_image(nr, nc, seed=nr) if nr > 1 else rng.uniform(0, 1, (1, nc))
    r = rng.standard_normal((nr, nc))
    dt = torch.float64 if mode == "fp64" else torch.float32
    if mode == "mixed":
        u = u.astype(np.float32).astype(np.float64)
        r = r.astype(np.float32).astype(np.float64)
    with pkg.Plan(nr, nc, h, bc="ar", pc=kind, mode=mode, method="reblur_arl",
                  transform=None if (mode == "fp64" or nr == 1) else transform) as plan:
        plan.precond_setup(torch.tensor(u, dtype=dt, device=dev), 1e-2, 0.05)
        z = plan.precond_solve(torch.tensor(r, dtype=dt, device=dev)).double().cpu().numpy()
    ref = O.precond_apply(r, O.precond_setup(u, h, O.AR, 1e-2, 0.05, kind, method=ARL))
    err = maxrel(z, ref)
    assert err < tol, err


@pytest.mark.parametrize("kind", ["dfast", "fastd", "none"])
def test_arl_pbicgstab_fp64_matches_oracle(tdev, kind):
    torch, pkg, dev = tdev
    nr, nc = 45, 70
    h = synth.gaussian_psf(1.5)
    v = observe(nr, nc, h, 0.01, 11)
    b = O.reblur_rhs(v, h, O.AR)
    args = (v, b, h, O.AR, 1e-3, 1e-2, kind, 1e-6, 3000)
    x_ref, k_ref, rr_ref, ok = O.fp_step(*args, method=ARL)
    pert = [O.fp_step(*args, noise=noise(j), method=ARL) for j in range(1, N_PERTURBED + 1)]
    with pkg.Plan(nr, nc, h, bc="ar", pc=kind, mode="fp64", method="reblur_arl") as plan:
        vt = torch.tensor(v, dtype=torch.float64, device=dev)
        x = vt.clone()
        k, rr, st = plan.pbicgstab_solve(vt, 1e-3, 1e-2, torch.tensor(b, dtype=torch.float64, device=dev), x,
                                         tol=1e-6, maxit=3000)
        x = x.cpu().numpy()
    assert st == pkg.TVD_OK and ok and rr < 1e-6
    check_counts([k], [k_ref], count_spread([k_ref], [[p[1]] for p in pert]))
    err = np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref)
    assert err < image_bound(x_ref, [p[0] for p in pert]), err


@pytest.mark.parametrize("kind", ["dfast", "fastd"])
def test_arl_deblur_fp64_counts(tdev, kind):
    """64 x 64, Gaussian sigma 1.5 on 9 x 9, 1% noise, alpha 1e-3, beta 1e-2, 10 FP steps of eq. (fpp), L_AR."""
    torch, pkg, dev = tdev
    n = 64
    h = synth.gaussian_psf(1.5, half_width=4)
    v = observe(n, n, h, 0.01, 1234)
    kw = dict(outer=10, tol=1e-6, maxit=3000, kind=kind, method=ARL)
    u_ref, st_ref = O.tv_deblur(v, h, O.AR, 1e-3, 1e-2, **kw)
    pert = [O.tv_deblur(v, h, O.AR, 1e-3, 1e-2, noise=noise(j), **kw) for j in range(1, N_PERTURBED + 1)]
    with pkg.Plan(n, n, h, bc="ar", pc=kind, mode="fp64", method="reblur_arl") as plan:
        u, st = plan.deblur(torch.tensor(v, dtype=torch.float64, device=dev), 1e-3, 1e-2, max_outer=10,
                            inner_tol=1e-6, inner_maxit=3000)
        u = u.cpu().numpy()
    assert st["status"] == pkg.TVD_OK
    spread = count_spread(st_ref["inner_iters"], [p[1]["inner_iters"] for p in pert])
    check_counts(st["inner_iters"], st_ref["inner_iters"], spread)
    err = np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref)
    assert err < image_bound(u_ref, [p[0] for p in pert]), (err, spread)


@pytest.mark.parametrize("transform", ["gemm", "fft"])
@pytest.mark.parametrize("kind", ["dfast", "fastd"])
def test_arl_mixed_deblur_within_1e5_of_oracle(tdev, kind, transform):
    torch, pkg, dev = tdev
    n = 96
    h = synth.gaussian_psf(2.0, half_width=7)
    v = observe(n, n, h, 0.01, 77)
    u_ref, _ = O.tv_deblur(v, h, O.AR, 1e-3, 1e-2, outer=4, tol=1e-10, maxit=20000, kind=kind, method=ARL)
    with pkg.Plan(n, n, h, bc="ar", pc=kind, mode="mixed", method="reblur_arl", transform=transform) as plan:
        u, st = plan.deblur(torch.tensor(v, dtype=torch.float64, device=dev), 1e-3, 1e-2, max_outer=4,
                            inner_tol=1e-10, inner_maxit=20000)
        u = u.cpu().numpy()
    assert st["status"] == pkg.TVD_OK
    err = np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref)
    assert err < 1e-5, err


def test_arl_tracked_residual_is_the_fpp_residual_with_l_ar(tdev):
    torch, pkg, dev = tdev
    n, alpha, beta, K = 40, 2e-3, 2e-2, 4
    h = synth.gaussian_psf(1.5, half_width=4)
    v = observe(n, n, h, 0.01, 9)
    b = O.reblur_rhs(v, h, O.AR)
    u = v.copy()
    g_ref = []
    for _ in range(K):
        w = O.diffusivity(u, beta)
        g_ref.append(float(np.linalg.norm(b - O.reblur_apply(u, h, O.AR, w, alpha, arl=True))))
        u, _, _, _ = O.fp_step(u, b, h, O.AR, alpha, beta, "dfast", 1e-12, 20000, method=ARL)
    with pkg.Plan(n, n, h, bc="ar", pc="dfast", mode="fp64", method="reblur_arl") as plan:
        _, st = plan.deblur(torch.tensor(v, device=dev), alpha, beta, max_outer=K, inner_tol=1e-12,
                            inner_maxit=20000, track=True)
    np.testing.assert_allclose(st["g_norm"], g_ref, rtol=1e-6)


def test_arl_refusals(tdev):
    torch, pkg, dev = tdev
    h = synth.gaussian_psf(1.0, half_width=2)
    with pytest.raises(pkg.TvdError):
        pkg.Plan(16, 16, h, bc="r", method="reblur_arl")
    with pkg.Plan(16, 16, h, bc="ar", pc="dfast", mode="fp64", method="reblur_arl") as plan:
        x = torch.zeros(16, 16, dtype=torch.float64, device=dev)
        with pytest.raises(pkg.TvdError):
            plan.pcg_solve(x, 1e-3, 1e-2, x, x.clone())
        with pytest.raises(pkg.TvdError):
            plan.newton(x.clone(), x, 1e-3, 1e-2)
