"""The preconditioner-form autotuner (tvd_plan_tune) on MIXED plans.

* It times every form the plan admits -- the FFT form, the transform products
  with 64- and with 128-column tiles, and the folded products where the plan
  allows them (anti-reflective eq. (fp), sides multiples of 256) -- reports
  each, and leaves the plan in the fastest.
* The tuned plan's preconditioner solve still matches the oracle element by
  element (max |z - z_ref| / max |z_ref|: 1e-4 in the FFT form, the float
  rounding of the line passes; 1e-2 in the GEMM form with float operands,
  the tf32 products), and a MIXED deblur of a tuned plan with both sides
  solving each FP step to 1e-10 stays within 1e-5 of the oracle.
* The choice outlasts a change of method (eq. (fpp) cannot fold, eq. (fp)
  folds again).
* FP64, 1D and I / D plans have nothing to tune and are refused.
"""
import math

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
    return torch, pkg, torch.device("cuda:0")


def maxrel(z, ref):
    return float(np.abs(z - ref).max() / np.abs(ref).max())


def check_report(plan, rep, count):
    cands = rep["candidates"]
    assert len(cands) == count
    forms = {(c["transform"], c["tile_n"], c["folded"]) for c in cands}
    want = {("fft", 0, False), ("gemm", 64, False), ("gemm", 128, False)} | (
        {("gemm", 64, True)} if count == 4 else set())
    assert forms == want
    times = [c["us_per_solve"] for c in cands]
    assert all(math.isfinite(t) and t > 0 for t in times), times
    assert rep["chosen"] == int(np.argmin(times))
    c = cands[rep["chosen"]]
    assert plan.transform == c["transform"]
    assert plan.gemm_tile == c["tile_n"]
    assert plan.gemm_folded == c["folded"]
    return c


@pytest.mark.parametrize("nr,nc,bc,kind,count", [(256, 256, "ar", "dfast", 4), (130, 128, "r", "dfast", 3),
                                                 (64, 96, "ar", "fastd", 3), (256, 512, "ar", "fast", 4)])
def test_tune_keeps_the_fastest_form_and_its_solve_matches_the_oracle(tdev, nr, nc, bc, kind, count):
    torch, pkg, dev = tdev
    h = synth.gaussian_psf(1.0, half_width=3)
    rng = np.random.default_rng(nr + 17 * nc)
    u = synth.piecewise_constant_image(nr, nc, seed=nr).astype(np.float32).astype(np.float64)
    r = rng.standard_normal((nr, nc)).astype(np.float32).astype(np.float64)
    alpha, beta = 1e-2, 0.05
    with pkg.Plan(nr, nc, h, bc=bc, pc=kind, mode="mixed") as plan:
        c = check_report(plan, plan.tune(reps=2), count)
        plan.precond_setup(torch.tensor(u, dtype=torch.float32, device=dev), alpha, beta)
        z = plan.precond_solve(torch.tensor(r, dtype=torch.float32, device=dev)).double().cpu().numpy()
    ref = O.precond_apply(r, O.precond_setup(u, h, bc, alpha, beta, kind))
    assert maxrel(z, ref) < (1e-4 if c["transform"] == "fft" else 1e-2), (c, maxrel(z, ref))


def test_tuned_plan_deblur_within_1e5_of_oracle(tdev):
    torch, pkg, dev = tdev
    n = 96
    h = synth.gaussian_psf(2.0, half_width=7)
    u_true = synth.piecewise_constant_image(n, n, seed=79)
    v = synth.add_noise(O.blur(u_true, h, O.AR), synth.noise_direction(n, n, 79), 0.01)
    u_ref, _ = O.tv_deblur(v, h, O.AR, 1e-3, 1e-2, outer=4, tol=1e-10, maxit=5000, kind=O.PC_DFAST)
    with pkg.Plan(n, n, h, bc="ar", pc="dfast", mode="mixed") as plan:
        check_report(plan, plan.tune(), 3)
        u, st = plan.deblur(torch.tensor(v, dtype=torch.float64, device=dev), 1e-3, 1e-2, max_outer=4,
                            inner_tol=1e-10, inner_maxit=5000)
        u = u.cpu().numpy()
    assert st["status"] == pkg.TVD_OK
    assert np.linalg.norm(u - u_ref) <= 1e-5 * np.linalg.norm(u_ref)


def test_tuned_choice_outlasts_a_change_of_method(tdev):
    torch, pkg, dev = tdev
    h = synth.gaussian_psf(1.0, half_width=2)
    with pkg.Plan(256, 256, h, bc="ar", pc="dfast", mode="mixed") as plan:
        c = check_report(plan, plan.tune(reps=2), 4)
        plan.set_method("reblur")
        assert plan.transform == c["transform"] and not plan.gemm_folded
        if c["transform"] == "gemm":
            assert plan.gemm_tile == c["tile_n"]
        plan.set_method("fp")
        assert (plan.transform, plan.gemm_tile, plan.gemm_folded) == (c["transform"], c["tile_n"], c["folded"])


def test_tune_refusals(tdev):
    torch, pkg, dev = tdev
    h = synth.gaussian_psf(1.0, half_width=2)
    for kw in (dict(mode="fp64", pc="dfast"), dict(mode="mixed", pc="diag"), dict(mode="mixed", pc="none")):
        with pkg.Plan(32, 32, h, bc="ar", **kw) as plan:
            with pytest.raises(pkg.TvdError):
                plan.tune()
    with pkg.Plan(1, 64, synth.out_of_focus_psf_1d(3), bc="ar", pc="dfast", mode="mixed") as plan:
        with pytest.raises(pkg.TvdError):
            plan.tune()
