"""GPU parity of pcg_solve and tv_deblur against the FP64 oracle.

* FP64 plans: held to the oracle's own rounding envelope (tests/parity.py):
  each FP step's inner iteration count within that step's own spread over
  oracle runs whose operator outputs are perturbed at a relative 2^-50 (equal
  counts where those runs agree); restored images within ten times their
  spread (at least 1e-12 relative).
* MIXED plans: both sides solve each FP step to ||r||/||r_0|| < 1e-10; the
  restored images agree within 1e-5 relative.
* Error paths: NaN data (breakdown), maxit too small (no convergence),
  asymmetric PSF, PSF wider than the image allows.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_1011_5964_gb300 import synth
from parity import N_PERTURBED, check_counts, count_spread, image_bound, noise

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "config2_oracle.json")


@pytest.fixture(scope="module")
def tdev():
    import torch
    import paper_1011_5964_gb300 as pkg
    pkg.load_library()
    return torch, torch.device("cuda:0")


def observe(n_rows, n_cols, h, bc, noise, seed):
    u_true = synth.piecewise_constant_image(n_rows, n_cols, seed=seed)
    return synth.add_noise(O.blur(u_true, h, bc), synth.noise_direction(n_rows, n_cols, seed), noise)


@pytest.mark.parametrize("bc,kind", [("ar", "dfast"), ("ar", "fast"), ("r", "dfast"), ("ar", "fastd"), ("r", "fastd"), ("ar", "none"),
                                     ("r", "diag")])
def test_pcg_solve_fp64_matches_oracle(tdev, bc, kind):
    torch, dev = tdev
    import paper_1011_5964_gb300 as pkg
    nr, nc = 45, 70
    h = synth.gaussian_psf(1.5)
    v = observe(nr, nc, h, bc, 0.01, 11)
    b = O.blur_adjoint(v, h, bc)
    x_ref, k_ref, rr_ref, ok = O.fp_step(v, b, h, bc, 1e-3, 1e-2, kind, 1e-6, 2000)
    pert = [O.fp_step(v, b, h, bc, 1e-3, 1e-2, kind, 1e-6, 2000, noise=noise(j)) for j in range(1, N_PERTURBED + 1)]
    with pkg.Plan(nr, nc, h, bc=bc, pc=kind, mode="fp64") as plan:
        vt = torch.tensor(v, dtype=torch.float64, device=dev)
        bt = torch.tensor(b, dtype=torch.float64, device=dev)
        x = vt.clone()
        k, rr, st = plan.pcg_solve(vt, 1e-3, 1e-2, bt, x, tol=1e-6, maxit=2000)
        x = x.cpu().numpy()
    assert st == pkg.TVD_OK and ok and rr < 1e-6
    check_counts([k], [k_ref], count_spread([k_ref], [[p[1]] for p in pert]))
    err = np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref)
    assert err < image_bound(x_ref, [p[0] for p in pert]), err


@pytest.mark.parametrize("kind", ["dfast", "fast", "fastd"])
def test_config1_deblur_fp64_iteration_counts(tdev, kind):
    """64 x 64, AR, Gaussian sigma 1.5 on 9 x 9, 1% noise, alpha 1e-3, beta 1e-2, 10 FP steps, tol 1e-6."""
    torch, dev = tdev
    import paper_1011_5964_gb300 as pkg
    n = 64
    h = synth.gaussian_psf(1.5, half_width=4)
    v = observe(n, n, h, "ar", 0.01, 1234)
    kw = dict(outer=10, tol=1e-6, kind=kind)
    u_ref, st_ref = O.tv_deblur(v, h, "ar", 1e-3, 1e-2, **kw)
    pert = [O.tv_deblur(v, h, "ar", 1e-3, 1e-2, noise=noise(j), **kw) for j in range(1, N_PERTURBED + 1)]
    with pkg.Plan(n, n, h, bc="ar", pc=kind, mode="fp64") as plan:
        u, st = plan.deblur(torch.tensor(v, dtype=torch.float64, device=dev), 1e-3, 1e-2, max_outer=10,
                            inner_tol=1e-6)
        u = u.cpu().numpy()
    spread = count_spread(st_ref["inner_iters"], [p[1]["inner_iters"] for p in pert])
    check_counts(st["inner_iters"], st_ref["inner_iters"], spread)
    err = np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref)
    assert err < image_bound(u_ref, [p[0] for p in pert]), (err, spread)


@pytest.mark.skipif(not os.path.exists(GOLDEN), reason="golden file not generated")
@pytest.mark.parametrize("bc", ["r", "ar"])
@pytest.mark.parametrize("kind", ["dfast", "none"])
def test_config2_sweep_iteration_counts(tdev, bc, kind):
    """256 x 256, sigma 2 on 15 x 15, noise {0.5%, 2%}, alpha {1e-4, 1e-3, 1e-2}, 10 FP steps: per-step
    counts and sampled pixels within the oracle's rounding envelope (stored by tests/golden/make_config2.py)."""
    torch, dev = tdev
    import paper_1011_5964_gb300 as pkg
    data = json.load(open(GOLDEN))
    meta = data["meta"]
    n = meta["n"]
    idx = np.array(meta["sample_index"])
    h = synth.gaussian_psf(2.0, half_width=7)
    runs = [r for r in data["runs"] if r["bc"] == bc and r["kind"] == kind]
    assert len(runs) == 6
    with pkg.Plan(n, n, h, bc=bc, pc=kind, mode="fp64") as plan:
        for run in runs:
            v = observe(n, n, h, bc, run["noise"], meta["seed"])
            u, st = plan.deblur(torch.tensor(v, dtype=torch.float64, device=dev), run["alpha"], 1e-2,
                                max_outer=meta["outer"], inner_tol=meta["tol"], inner_maxit=5000)
            check_counts(st["inner_iters"], run["inner_iters"], run["count_spread"])
            u = u.cpu().numpy()
            un = float(np.linalg.norm(u))
            assert abs(un - run["u_norm"]) <= max(10 * run["image_spread"], 1e-12) * run["u_norm"], run
            d = np.abs(u[idx[:, 0], idx[:, 1]] - np.array(run["samples"])).max()
            assert d <= 10 * run["sample_spread"] + 1e-12, (d, run["sample_spread"])


@pytest.mark.parametrize("bc", ["ar", "r"])
def test_mixed_deblur_within_1e5_of_oracle(tdev, bc):
    torch, dev = tdev
    import paper_1011_5964_gb300 as pkg
    n = 96
    h = synth.gaussian_psf(2.0, half_width=7)
    v = observe(n, n, h, bc, 0.01, 77)
    u_ref, st_ref = O.tv_deblur(v, h, bc, 1e-3, 1e-2, outer=4, tol=1e-10, maxit=5000, kind="dfast")
    with pkg.Plan(n, n, h, bc=bc, pc="dfast", mode="mixed") as plan:
        u, st = plan.deblur(torch.tensor(v, dtype=torch.float64, device=dev), 1e-3, 1e-2, max_outer=4,
                            inner_tol=1e-10, inner_maxit=5000)
        u = u.cpu().numpy()
    assert st["status"] == pkg.TVD_OK
    err = np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref)
    assert err < 1e-5, err


def test_mixed_pcg_solve_reaches_double_tolerance(tdev):
    """A MIXED solve's stopping test is on the double residual: check it with the oracle's operator."""
    torch, dev = tdev
    import paper_1011_5964_gb300 as pkg
    nr, nc = 80, 72
    h = synth.disk_psf(3.0)
    v = observe(nr, nc, h, "ar", 0.01, 5)
    b = O.blur_adjoint(v, h, "ar")
    with pkg.Plan(nr, nc, h, bc="ar", pc="dfast", mode="mixed") as plan:
        vt = torch.tensor(v, dtype=torch.float64, device=dev)
        x = vt.clone()
        k, rr, st = plan.pcg_solve(vt, 1e-3, 1e-2, torch.tensor(b, dtype=torch.float64, device=dev), x,
                                   tol=1e-9, maxit=3000)
        x = x.cpu().numpy()
    assert st == pkg.TVD_OK and rr < 1e-9
    w = O.diffusivity(v, 1e-2)
    r0 = np.linalg.norm(b - O.normal_apply(v, h, "ar", w, 1e-3))
    r1 = np.linalg.norm(b - O.normal_apply(x, h, "ar", w, 1e-3))
    assert r1 / r0 < 1.5e-9


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_full_size_step_residual(tdev, mode):
    """1024 x 1024, AR, radius-7 disk on 31 x 31, 1% noise, alpha 1e-3: one FP step from u^0 = v
    reaches the tolerance, measured with the oracle's operator at full size."""
    torch, dev = tdev
    import paper_1011_5964_gb300 as pkg
    n = 1024
    h = synth.disk_psf(7.0, side=31)
    v = observe(n, n, h, "ar", 0.01, 1234)
    b = O.blur_adjoint(v, h, "ar")
    tol = 1e-6
    with pkg.Plan(n, n, h, bc="ar", pc="dfast", mode=mode) as plan:
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


def test_nan_data_is_breakdown(tdev):
    torch, dev = tdev
    import paper_1011_5964_gb300 as pkg
    n = 32
    h = synth.gaussian_psf(1.0)
    v = observe(n, n, h, "ar", 0.01, 3)
    v[5, 7] = np.nan
    with pkg.Plan(n, n, h, bc="ar", pc="dfast", mode="fp64") as plan:
        vt = torch.tensor(v, dtype=torch.float64, device=dev)
        with pytest.raises(pkg.TvdError) as e:
            plan.deblur(vt, 1e-3, 1e-2, max_outer=2)
        assert e.value.status in (pkg.TVD_EBREAKDOWN, pkg.TVD_EINVAL)


def test_maxit_reports_no_convergence(tdev):
    torch, dev = tdev
    import paper_1011_5964_gb300 as pkg
    n = 40
    h = synth.gaussian_psf(1.5)
    v = observe(n, n, h, "ar", 0.01, 4)
    b = O.blur_adjoint(v, h, "ar")
    with pkg.Plan(n, n, h, bc="ar", pc="dfast", mode="fp64") as plan:
        vt = torch.tensor(v, dtype=torch.float64, device=dev)
        x = vt.clone()
        k, rr, st = plan.pcg_solve(vt, 1e-3, 1e-2, torch.tensor(b, dtype=torch.float64, device=dev), x,
                                   tol=1e-12, maxit=3)
    assert st == pkg.TVD_ENOCONV and k == 3
    _, k_ref, rr_ref, ok = O.fp_step(v, b, h, "ar", 1e-3, 1e-2, "dfast", 1e-12, 3)
    assert not ok and abs(rr - rr_ref) < 1e-9 * rr_ref


def test_plan_validation(tdev):
    torch, dev = tdev
    import paper_1011_5964_gb300 as pkg
    h = synth.gaussian_psf(1.0)
    h_asym = h.copy()
    h_asym[0, 1] += 1e-3
    with pytest.raises(pkg.TvdError) as e:
        pkg.Plan(16, 16, h_asym)
    assert e.value.status == pkg.TVD_EPSF_ASYM
    with pytest.raises(pkg.TvdError) as e:
        pkg.Plan(4, 16, synth.gaussian_psf(1.0))        # m_r = 3 > n_r - 2
    assert e.value.status == pkg.TVD_EPSF_SIZE
    with pytest.raises(pkg.TvdError) as e:
        pkg.Plan(16, 16, np.ones((4, 3)) / 12)
    assert e.value.status == pkg.TVD_EPSF_SIZE
    # zero padding is trimmed: a 31 x 31 disk works on a 17 x 17 image (effective m = 7 <= 15)
    with pkg.Plan(17, 17, synth.disk_psf(7.0, side=31)) as plan:
        x = torch.ones(17, 17, dtype=torch.float64, device=dev)
        y = plan.blur(x)
        assert torch.allclose(y, x)
