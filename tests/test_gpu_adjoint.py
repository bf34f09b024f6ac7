"""GPU parity of the adjoint of the converged fixed point (tv_hessian_apply, tv_deblur_adjoint).

The oracle's adjoint is pinned against finite differences of the re-converged
fixed point (tests/test_oracle_adjoint_pins.py). Here the CUDA path gets the
oracle's u*, v and dl/du = 2 (u* - u_true) and must return the same lambda and
gradients: both sides solve J lambda = dl/du to ||r|| / ||r_0|| < 1e-13
(the GPU with the plan's preconditioner, the oracle without), so they agree to
rounding times the conditioning; the bound is 1e-9 relative.
"""
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


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


@pytest.mark.parametrize("nr,nc", [(3, 3), (7, 12), (33, 17), (64, 64)])
@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_tv_hessian_apply_matches_the_oracle(tdev, nr, nc, mode):
    torch, pkg, dev = tdev
    rng = np.random.default_rng(nr * 100 + nc)
    u, x = rng.standard_normal((nr, nc)), rng.standard_normal((nr, nc))
    h = np.ones((1, 1))
    with pkg.Plan(nr, nc, h, bc="ar", pc="none", mode=mode) as plan:
        y = plan.hessian(torch.tensor(u, device=dev), 0.3, torch.tensor(x, device=dev)).cpu().numpy()
    assert rel(y, O.tv_hessian_apply(u, 0.3, x)) < 1e-12


CASES = [  # nr, nc, sigma, half-width, bc, alpha, beta, preconditioner
    (10, 12, 1.0, 2, "ar", 0.05, 0.1, "dfast"),
    (11, 9, 1.2, 3, "r", 0.02, 0.05, "dfast"),
    (12, 10, 1.0, 2, "ar", 0.05, 0.1, "none"),
    (12, 10, 1.0, 2, "ar", 0.05, 0.1, "diag"),
    (40, 48, 1.5, 4, "ar", 2e-3, 2e-2, "dfast"),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}-{c[4]}-{c[7]}")
@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_adjoint_gradients_match_the_oracle(tdev, case, mode):
    torch, pkg, dev = tdev
    nr, nc, sigma, hw, bc, alpha, beta, pc = case
    h = synth.gaussian_psf(sigma, half_width=hw)
    ut = synth.piecewise_constant_image(nr, nc, seed=5)
    v = synth.add_noise(O.blur(ut, h, bc), synth.noise_direction(nr, nc, 5), 0.02)
    kind = O.PC_DFAST if nr * nc > 400 else O.PC_NONE
    u, _ = O.tv_deblur(v, h, bc, alpha, beta, outer=3000, tol=1e-14, maxit=20000, kind=kind, outer_tol=1e-15)
    g = 2.0 * (u - ut)
    lam, it, rr, ok = O.adjoint_solve(u, h, bc, alpha, beta, g, tol=1e-14)
    ga, gb, gh = O.fixed_point_gradients(u, v, h, bc, alpha, beta, lam)
    T = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    with pkg.Plan(nr, nc, h, bc=bc, pc=pc, mode=mode) as plan:
        assert plan.psf_size() == h.shape
        lam_g, da, db, dh, st = plan.adjoint(T(u), T(v), alpha, beta, T(g), tol=1e-13, maxit=20000)
    assert st["status"] == 0 and st["relres"] < 1e-13, st
    assert rel(lam_g.cpu().numpy(), lam) < 1e-9
    assert abs(da - ga) <= 1e-9 * abs(ga)
    assert abs(db - gb) <= 1e-9 * abs(gb)
    assert rel(dh, gh) < 1e-9


def test_adjoint_rejects_bad_arguments(tdev):
    torch, pkg, dev = tdev
    h = synth.gaussian_psf(1.0, half_width=2)
    z = torch.zeros((8, 8), dtype=torch.float64, device=dev)
    with pkg.Plan(8, 8, h, bc="ar", pc="dfast", mode="fp64") as plan:
        with pytest.raises(pkg.TvdError):
            plan.adjoint(z, z, -1.0, 0.1, z)
        with pytest.raises(pkg.TvdError):
            plan.adjoint(z, z, 0.1, 0.0, z)


def test_adjoint_of_zero_loss_gradient_is_zero(tdev):
    torch, pkg, dev = tdev
    h = synth.gaussian_psf(1.0, half_width=2)
    rng = np.random.default_rng(3)
    u = torch.tensor(rng.standard_normal((9, 9)), device=dev)
    with pkg.Plan(9, 9, h, bc="ar", pc="dfast", mode="fp64") as plan:
        lam, da, db, dh, st = plan.adjoint(u, u, 0.01, 0.1, torch.zeros_like(u))
    assert st["iters"] == 0 and float(lam.abs().max()) == 0.0 and da == 0.0 and db == 0.0 and not dh.any()
