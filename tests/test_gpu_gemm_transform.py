"""GPU parity of the GEMM form of the preconditioner transforms (MIXED plans).

The fast preconditioners' 2D transform U = B_r (x) B_c (Secs. 2-3: hat-S_n for
AR, the DCT-II C_n for R) is applied as four dense products on the tensor
cores by the library's own kernel (TMA tiles, tcgen05.mma, float
accumulation). Checks, against the FP64 oracle on the same seeded inputs:

* the preconditioner solve z = X^{-1} r for R, M, D_R, D_M, R_D, M_D on square,
  rectangular, tiny and ragged images (sizes that span several 128-row tiles
  with a ragged tail), element by element: max |z - z_ref| / max |z_ref|.
  Tolerances: with float operands (tf32 products, unit roundoff 2^-11) four
  products each add about 2^-11 relative, so 1e-2; with bf16 operands (unit
  roundoff 2^-9 for each of the matrices and the four product inputs) about
  eight roundings of 2e-3, so 3e-2;
* the GEMM form against the FFT form of the same plan;
* MIXED deblurs with both sides at inner tol 1e-10 within 1e-5 of the
  oracle (the preconditioner only shapes the iteration; the double residual
  decides convergence);
* one FP step of the 1024 x 1024 workload reaching its tolerance, measured
  with the oracle's operator;
* argument validation of tvd_plan_set_transform; the operand storage.

Operand storage: float (tf32 products) below sides of 1024, bf16 from 1024
on; the tests set TVD_GEMM_STORAGE to cover both at every size.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_1011_5964_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tdev():
    import torch
    import paper_1011_5964_gb300 as pkg
    pkg.load_library()
    return torch, torch.device("cuda:0")


def observe(n_rows, n_cols, h, bc, noise, seed):
    u_true = synth.piecewise_constant_image(n_rows, n_cols, seed=seed)
    return synth.add_noise(O.blur(u_true, h, bc), synth.noise_direction(n_rows, n_cols, seed), noise)


SHAPES = [(37, 53), (64, 64), (3, 3), (4, 7), (128, 130), (96, 33), (300, 200), (257, 129)]
TOL = {"f32": 1e-2, "bf16": 3e-2}


def maxrel(z, ref):
    return float(np.abs(z - ref).max() / np.abs(ref).max())


class _env:
    """Set environment variables for the plan set-up inside the block (read by the library then)."""

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


def _solve(torch, dev, nr, nc, bc, kind, transform, storage=None):
    import paper_1011_5964_gb300 as pkg
    h = synth.gaussian_psf(1.0, half_width=min(3, nr - 2, nc - 2))
    rng = np.random.default_rng(nr + 17 * nc)
    u = synth.piecewise_constant_image(nr, nc, seed=nr).astype(np.float32).astype(np.float64)
    r = rng.standard_normal((nr, nc)).astype(np.float32).astype(np.float64)
    alpha, beta = 1e-2, 0.05
    with _env(TVD_GEMM_STORAGE=storage):
        with pkg.Plan(nr, nc, h, bc=bc, pc=kind, mode="mixed", transform=transform) as plan:
            assert plan.transform == transform
            if storage is not None:
                assert plan.gemm_storage == storage
            plan.precond_setup(torch.tensor(u, dtype=torch.float32, device=dev), alpha, beta)
            z = plan.precond_solve(torch.tensor(r, dtype=torch.float32, device=dev)).double().cpu().numpy()
    P = O.precond_setup(u, h, bc, alpha, beta, kind)
    return z, O.precond_apply(r, P)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("kind", ["dfast", "fast", "fastd"])
@pytest.mark.parametrize("bc", ["ar", "r"])
@pytest.mark.parametrize("nr,nc", SHAPES)
def test_gemm_preconditioner_solve(tdev, nr, nc, bc, kind, storage):
    torch, dev = tdev
    z, ref = _solve(torch, dev, nr, nc, bc, kind, "gemm", storage=storage)
    err = maxrel(z, ref)
    assert err < TOL[storage], err


@pytest.mark.parametrize("bc", ["ar", "r"])
def test_gemm_form_matches_fft_form(tdev, bc):
    torch, dev = tdev
    z_g, _ = _solve(torch, dev, 100, 90, bc, "dfast", "gemm", storage="f32")
    z_f, _ = _solve(torch, dev, 100, 90, bc, "dfast", "fft")
    assert maxrel(z_g, z_f) < TOL["f32"]


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("bc,kind", [("ar", "dfast"), ("r", "dfast"), ("ar", "fastd"), ("ar", "fast")])
def test_mixed_deblur_gemm_within_1e5_of_oracle(tdev, bc, kind, storage):
    torch, dev = tdev
    import paper_1011_5964_gb300 as pkg
    n = 96
    h = synth.gaussian_psf(2.0, half_width=7)
    v = observe(n, n, h, bc, 0.01, 77)
    u_ref, _ = O.tv_deblur(v, h, bc, 1e-3, 1e-2, outer=4, tol=1e-10, maxit=5000, kind=kind)
    with _env(TVD_GEMM_STORAGE=storage), pkg.Plan(n, n, h, bc=bc, pc=kind, mode="mixed", transform="gemm") as plan:
        u, st = plan.deblur(torch.tensor(v, dtype=torch.float64, device=dev), 1e-3, 1e-2, max_outer=4,
                            inner_tol=1e-10, inner_maxit=5000)
        u = u.cpu().numpy()
    assert st["status"] == pkg.TVD_OK
    err = np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref)
    assert err < 1e-5, err


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_gemm_full_size_step_residual(tdev, storage):
    """1024 x 1024, AR, radius-7 disk on 31 x 31, 1% noise, alpha 1e-3, GEMM transforms: one FP step
    from u^0 = v reaches the tolerance, measured with the oracle's operator at full size."""
    torch, dev = tdev
    import paper_1011_5964_gb300 as pkg
    n = 1024
    h = synth.disk_psf(7.0, side=31)
    v = observe(n, n, h, "ar", 0.01, 1234)
    b = O.blur_adjoint(v, h, "ar")
    tol = 1e-6
    with _env(TVD_GEMM_STORAGE=storage), pkg.Plan(n, n, h, bc="ar", pc="dfast", mode="mixed",
                                                  transform="gemm") as plan:
        vt = torch.tensor(v, dtype=torch.float64, device=dev)
        x = vt.clone()
        k, rr, st = plan.pcg_solve(vt, 1e-3, 1e-2, torch.tensor(b, dtype=torch.float64, device=dev), x,
                                   tol=tol, maxit=3000)
        x = x.cpu().numpy()
    assert st == pkg.TVD_OK and k > 0
    w = O.diffusivity(v, 1e-2)
    r0 = np.linalg.norm(b - O.normal_apply(v, h, "ar", w, 1e-3))
    r1 = np.linalg.norm(b - O.normal_apply(x, h, "ar", w, 1e-3))
    assert r1 / r0 < tol * 1.01


def test_set_transform_validation(tdev):
    torch, dev = tdev
    import paper_1011_5964_gb300 as pkg
    h = synth.gaussian_psf(1.0, half_width=2)
    with pkg.Plan(16, 16, h, bc="ar", pc="dfast", mode="fp64") as plan:
        with pytest.raises(pkg.TvdError):
            plan.set_transform("gemm")
        assert plan.transform == "fft"
    with pkg.Plan(16, 16, h, bc="ar", pc="diag", mode="mixed") as plan:
        with pytest.raises(pkg.TvdError):
            plan.set_transform("gemm")
    with pkg.Plan(16, 16, h, bc="ar", pc="dfast", mode="mixed") as plan:
        assert plan.lib.tvd_plan_set_transform(plan.handle, 7, None) == pkg.TVD_EINVAL
        for kind in ("gemm", "fft", "gemm"):
            plan.set_transform(kind)
            assert plan.transform == kind
        assert plan.gemm_storage == "f32"   # float operands below sides of 1024
    with _env(TVD_GEMM_STORAGE="bf16"), pkg.Plan(16, 16, h, bc="r", pc="fast", mode="mixed", transform="gemm") as plan:
        assert plan.gemm_storage == "bf16"


def test_batched_gemm_plans_equal_individual_calls(tdev):
    """Items whose plans use the GEMM form give their own tv_deblur result bit for bit (one algorithm per
    plan product, fixed at set-up)."""
    torch, dev = tdev
    import paper_1011_5964_gb300 as pkg
    items = [(64, 64, 2.0, 3e-4), (96, 80, 2.5, 1e-3), (72, 72, 1.5, 1e-2)]
    plans, vs = [], []
    for i, (nr, nc, sigma, _) in enumerate(items):
        h = synth.gaussian_psf(sigma, half_width=int(np.ceil(3 * sigma)))
        plans.append(pkg.Plan(nr, nc, h, bc="ar", pc="dfast", mode="mixed", transform="gemm"))
        vs.append(torch.tensor(observe(nr, nc, h, "ar", 0.01, 2000 + i), dtype=torch.float64, device=dev))
    try:
        ref = []
        for (nr, nc, sigma, alpha), p, v in zip(items, plans, vs):
            u, st = p.deblur(v, alpha, 1e-2, max_outer=3, inner_tol=1e-6, inner_maxit=2000)
            ref.append((u.clone(), st["inner_iters"]))
        torch.cuda.synchronize()
        us, stats = pkg.deblur_batched(plans, vs, [it[3] for it in items], [1e-2] * len(items), max_outer=3,
                                       inner_tol=1e-6, inner_maxit=2000, workers=3)
        torch.cuda.synchronize()
        for i, ((u_ref, it_ref), u, st) in enumerate(zip(ref, us, stats)):
            assert st["status"] == 0, (i, st)
            assert st["inner_iters"] == it_ref, (i, st["inner_iters"], it_ref)
            assert torch.equal(u, u_ref), (i, float((u - u_ref).abs().max()))
    finally:
        for p in plans:
            p.close()


@pytest.mark.parametrize("nr,nc", [(256, 256), (512, 256), (256, 768)])
@pytest.mark.parametrize("kind", ["dfast", "fast", "fastd"])
@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_folded_products_match_the_oracle(tdev, nr, nc, kind, storage):
    """Anti-reflective plans with sides multiples of 256 run the folded products (each
    transform split into its sum and difference halves, half the K per product): the solve
    matches the oracle like the full products do, and the two forms agree."""
    torch, dev = tdev
    z, ref = _solve(torch, dev, nr, nc, "ar", kind, "gemm", storage=storage)
    assert maxrel(z, ref) < TOL[storage]
    with _env(TVD_GEMM_FOLD="0"):
        z0, _ = _solve(torch, dev, nr, nc, "ar", kind, "gemm", storage=storage)
    assert maxrel(z0, ref) < TOL[storage]
    assert maxrel(z, z0) < TOL[storage]


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("kind", ["dfast", "fastd"])
def test_folded_mixed_deblur_within_1e5_of_oracle(tdev, kind, storage):
    torch, dev = tdev
    import paper_1011_5964_gb300 as pkg
    n = 256
    h = synth.gaussian_psf(2.0, half_width=7)
    v = observe(n, n, h, "ar", 0.01, 78)
    u_ref, _ = O.tv_deblur(v, h, "ar", 1e-3, 1e-2, outer=3, tol=1e-10, maxit=5000, kind=kind)
    with _env(TVD_GEMM_STORAGE=storage), pkg.Plan(n, n, h, bc="ar", pc=kind, mode="mixed", transform="gemm") as plan:
        u, st = plan.deblur(torch.tensor(v, dtype=torch.float64, device=dev), 1e-3, 1e-2, max_outer=3,
                            inner_tol=1e-10, inner_maxit=5000)
        u = u.cpu().numpy()
    assert st["status"] == pkg.TVD_OK
    err = np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref)
    assert err < 1e-5, err


def test_folded_form_is_reported(tdev):
    torch, dev = tdev
    import paper_1011_5964_gb300 as pkg
    h = synth.gaussian_psf(1.0, half_width=2)
    cases = [((256, 512), "ar", "fp", True), ((300, 256), "ar", "fp", False), ((256, 256), "r", "fp", False),
             ((256, 256), "ar", "reblur", False)]
    for (nr, nc), bc, method, folded in cases:
        with pkg.Plan(nr, nc, h, bc=bc, pc="dfast", mode="mixed", transform="gemm", method=method) as plan:
            assert plan.gemm_folded == folded, (nr, nc, bc, method)
    with _env(TVD_GEMM_FOLD="0"), pkg.Plan(256, 256, h, bc="ar", pc="dfast", mode="mixed", transform="gemm") as plan:
        assert not plan.gemm_folded
    with pkg.Plan(256, 256, h, bc="ar", pc="dfast", mode="mixed", transform="fft") as plan:
        assert not plan.gemm_folded
