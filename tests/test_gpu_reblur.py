"""GPU parity of the reblurring method (eq. (fpp), Sec. 3) against the FP64 oracle.

* The P, D_P, P_D preconditioner solves (T_n (x) T_n with the AR_2 spectrum;
  FP64 and MIXED plans in the FFT form with the rank-2 corrections of
  T_n = hat-S (I + U), MIXED plans in the GEMM form with the dense T_n^-1 and
  T_n), element by element against the oracle: FP64 within 1e-10 of the
  largest entry, float FFT form 1e-3, GEMM form 1e-2 (tf32) / 3e-2 (bf16), as
  for the sine-algebra preconditioners.
* PBiCGstab on one FP step and a 10-step reblurring deblur in FP64, held to
  the oracle's rounding envelope (tests/parity.py); MIXED deblurs with both
  sides solving each step to 1e-10 within 1e-5 of the oracle.
* The ordering of the reblurring columns of Table 2-1 on the GPU, and the
  entry points' refusals (PCG on a reblurring plan, PBiCGstab on an eq. (fp)
  plan, reblurring with reflective BCs).
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_1011_5964_gb300 import synth
from parity import N_PERTURBED, check_counts, count_spread, image_bound, noise

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tdev():
    import torch
    import paper_1011_5964_gb300 as pkg
    pkg.load_library()
    return torch, torch.device("cuda:0")


class _env:
    def __init__(self, **kv):
        self.kv = {k: v for k, v in kv.items() if v is not None}

    def __enter__(self):
        self.old = {k: os.environ.get(k) for k in self.kv}
        os.environ.update(self.kv)

    def __exit__(self, *exc):
        for k, v in self.old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def observe(n_rows, n_cols, h, noise_level, seed):
    u_true = synth.piecewise_constant_image(n_rows, n_cols, seed=seed)
    return synth.add_noise(O.blur(u_true, h, O.AR), synth.noise_direction(n_rows, n_cols, seed), noise_level)


def maxrel(z, ref):
    return float(np.abs(z - ref).max() / np.abs(ref).max())


SHAPES = [(37, 53), (64, 64), (5, 6), (96, 33), (130, 128)]
FORMS = [("fp64", "fft", None, 1e-10), ("mixed", "fft", None, 1e-3), ("mixed", "gemm", "f32", 1e-2),
         ("mixed", "gemm", "bf16", 3e-2)]


@pytest.mark.parametrize("mode,transform,storage,tol", FORMS)
@pytest.mark.parametrize("kind", ["fast", "dfast", "fastd"])
@pytest.mark.parametrize("nr,nc", SHAPES)
def test_reblur_preconditioner_solve(tdev, nr, nc, kind, mode, transform, storage, tol):
    torch, dev = tdev
    import paper_1011_5964_gb300 as pkg
    h = synth.gaussian_psf(1.0, half_width=min(3, nr - 2, nc - 2))
    rng = np.random.default_rng(nr + 17 * nc)
    u = synth.piecewise_constant_image(nr, nc, seed=nr)
    r = rng.standard_normal((nr, nc))
    dt = torch.float64 if mode == "fp64" else torch.float32
    if mode == "mixed":
        u = u.astype(np.float32).astype(np.float64)
        r = r.astype(np.float32).astype(np.float64)
    with _env(TVD_GEMM_STORAGE=storage):
        with pkg.Plan(nr, nc, h, bc="ar", pc=kind, mode=mode, method="reblur",
                      transform=None if mode == "fp64" else transform) as plan:
            assert plan.method == "reblur"
            plan.precond_setup(torch.tensor(u, dtype=dt, device=dev), 1e-2, 0.05)
            z = plan.precond_solve(torch.tensor(r, dtype=dt, device=dev)).double().cpu().numpy()
    ref = O.precond_apply(r, O.precond_setup(u, h, O.AR, 1e-2, 0.05, kind, method=O.METHOD_REBLUR))
    err = maxrel(z, ref)
    assert err < tol, err


@pytest.mark.parametrize("kind", ["dfast", "fastd", "none", "diag"])
def test_pbicgstab_fp64_matches_oracle(tdev, kind):
    torch, dev = tdev
    import paper_1011_5964_gb300 as pkg
    nr, nc = 45, 70
    h = synth.gaussian_psf(1.5)
    v = observe(nr, nc, h, 0.01, 11)
    b = O.reblur_rhs(v, h, O.AR)
    args = (v, b, h, O.AR, 1e-3, 1e-2, kind, 1e-6, 3000)
    x_ref, k_ref, rr_ref, ok = O.fp_step(*args, method=O.METHOD_REBLUR)
    pert = [O.fp_step(*args, noise=noise(j), method=O.METHOD_REBLUR) for j in range(1, N_PERTURBED + 1)]
    with pkg.Plan(nr, nc, h, bc="ar", pc=kind, mode="fp64", method="reblur") as plan:
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
def test_reblur_deblur_fp64_counts(tdev, kind):
    """64 x 64, Gaussian sigma 1.5 on 9 x 9, 1% noise, alpha 1e-3, beta 1e-2, 10 FP steps of eq. (fpp)."""
    torch, dev = tdev
    import paper_1011_5964_gb300 as pkg
    n = 64
    h = synth.gaussian_psf(1.5, half_width=4)
    v = observe(n, n, h, 0.01, 1234)
    kw = dict(outer=10, tol=1e-6, maxit=3000, kind=kind, method=O.METHOD_REBLUR)
    u_ref, st_ref = O.tv_deblur(v, h, O.AR, 1e-3, 1e-2, **kw)
    pert = [O.tv_deblur(v, h, O.AR, 1e-3, 1e-2, noise=noise(j), **kw) for j in range(1, N_PERTURBED + 1)]
    with pkg.Plan(n, n, h, bc="ar", pc=kind, mode="fp64", method="reblur") as plan:
        u, st = plan.deblur(torch.tensor(v, dtype=torch.float64, device=dev), 1e-3, 1e-2, max_outer=10,
                            inner_tol=1e-6, inner_maxit=3000)
        u = u.cpu().numpy()
    assert st["status"] == pkg.TVD_OK
    spread = count_spread(st_ref["inner_iters"], [p[1]["inner_iters"] for p in pert])
    check_counts(st["inner_iters"], st_ref["inner_iters"], spread)
    err = np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref)
    assert err < image_bound(u_ref, [p[0] for p in pert]), (err, spread)


@pytest.mark.parametrize("transform", ["gemm", "fft"])
@pytest.mark.parametrize("kind", ["dfast", "fastd", "fast"])
def test_reblur_mixed_deblur_within_1e5_of_oracle(tdev, kind, transform):
    torch, dev = tdev
    import paper_1011_5964_gb300 as pkg
    n = 96
    h = synth.gaussian_psf(2.0, half_width=7)
    v = observe(n, n, h, 0.01, 77)
    u_ref, _ = O.tv_deblur(v, h, O.AR, 1e-3, 1e-2, outer=4, tol=1e-10, maxit=20000, kind=kind,
                           method=O.METHOD_REBLUR)
    with pkg.Plan(n, n, h, bc="ar", pc=kind, mode="mixed", method="reblur", transform=transform) as plan:
        u, st = plan.deblur(torch.tensor(v, dtype=torch.float64, device=dev), 1e-3, 1e-2, max_outer=4,
                            inner_tol=1e-10, inner_maxit=20000)
        u = u.cpu().numpy()
    assert st["status"] == pkg.TVD_OK
    err = np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref)
    assert err < 1e-5, err


def test_reblur_ordering_on_gpu(tdev):
    """Table 2-1's reblurring columns: D_P and P_D need fewer PBiCGstab iterations than D and I."""
    torch, dev = tdev
    import paper_1011_5964_gb300 as pkg
    n = 48
    h = synth.gaussian_psf(1.5, half_width=4)
    v = observe(n, n, h, 0.001, 29)
    tot = {}
    for kind in ("fastd", "dfast", "diag", "none"):
        with pkg.Plan(n, n, h, bc="ar", pc=kind, mode="fp64", method="reblur") as plan:
            _, st = plan.deblur(torch.tensor(v, dtype=torch.float64, device=dev), 1e-1, 1e-2, max_outer=2,
                                inner_tol=1e-5, inner_maxit=3000)
            tot[kind] = st["total_inner_iters"]
    assert max(tot["fastd"], tot["dfast"]) < tot["diag"] < tot["none"], tot


def test_reblur_refusals(tdev):
    torch, dev = tdev
    import paper_1011_5964_gb300 as pkg
    h = synth.gaussian_psf(1.0, half_width=2)
    with pkg.Plan(16, 16, h, bc="r", pc="dfast", mode="fp64") as plan:
        with pytest.raises(pkg.TvdError):
            plan.set_method("reblur")
        assert plan.method == "fp"
    x = torch.zeros(16, 16, dtype=torch.float64, device=dev)
    with pkg.Plan(16, 16, h, bc="ar", pc="dfast", mode="fp64") as plan:
        with pytest.raises(pkg.TvdError):
            plan.pbicgstab_solve(x + 1.0, 1e-3, 1e-2, x, x.clone())
        plan.set_method("reblur")
        with pytest.raises(pkg.TvdError):
            plan.pcg_solve(x + 1.0, 1e-3, 1e-2, x, x.clone())
        plan.set_method("fp")
        assert plan.method == "fp"
