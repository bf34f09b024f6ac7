"""GPU parity of the Newton finish of the fixed point (tv_deblur_newton) and of
the per-step ||g(u^k)|| and functional that tv_deblur reports on request.

* Newton: both sides run the FP iteration for a few steps, then Newton steps
  on g(u) = 0 (eq. (el)) to a relative change below 1e-12; the minimiser of
  the strictly convex functional is unique, so both land on it. The bound on
  the restored images is 1e-9 relative (the Jacobian solves stop at 1e-12 on
  both sides; what remains is rounding times the conditioning of J).
* Tracking: the FP iterates of the two sides agree to about the inner
  tolerance (1e-12 here), so ||g(u^k)|| agrees to 1e-6 relative and the
  functional T(u^k) to 1e-10.
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


def _problem(nr, nc, sigma, hw, bc, seed=5, noise=0.01):
    h = synth.gaussian_psf(sigma, half_width=hw)
    ut = synth.piecewise_constant_image(nr, nc, seed=seed)
    v = synth.add_noise(O.blur(ut, h, bc), synth.noise_direction(nr, nc, seed), noise)
    return h, ut, v


CASES = [  # nr, nc, sigma, half-width, bc, alpha, beta, preconditioner, FP steps before Newton
    (12, 10, 1.0, 2, "ar", 0.05, 0.1, "dfast", 3),
    (11, 9, 1.2, 3, "r", 0.02, 0.05, "dfast", 3),
    (12, 10, 1.0, 2, "ar", 0.05, 0.1, "diag", 3),
    (48, 40, 1.5, 4, "ar", 1e-3, 1e-2, "dfast", 8),
    (37, 53, 1.5, 4, "r", 1e-3, 1e-2, "fast", 8),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}-{c[4]}-{c[7]}")
@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_newton_finish_matches_the_oracle(tdev, case, mode):
    torch, pkg, dev = tdev
    nr, nc, sigma, hw, bc, alpha, beta, pc, steps = case
    h, _, v = _problem(nr, nc, sigma, hw, bc)
    u0, _ = O.tv_deblur(v, h, bc, alpha, beta, outer=steps, tol=1e-10, maxit=20000, kind=pc)
    u_ref, ost = O.newton_polish(u0, v, h, bc, alpha, beta, tol=1e-12, cg_tol=1e-12, kind=pc)
    assert ost["converged"]
    vt = torch.tensor(v, dtype=torch.float64, device=dev)
    with pkg.Plan(nr, nc, h, bc=bc, pc=pc, mode=mode) as plan:
        u, _ = plan.deblur(vt, alpha, beta, max_outer=steps, inner_tol=1e-10, inner_maxit=20000)
        st = plan.newton(u, vt, alpha, beta, tol=1e-12, cg_tol=1e-12)
        u = u.cpu().numpy()
    assert st["status"] == pkg.TVD_OK, st
    assert st["last_rel_change"] < 1e-12 and st["steps"] >= 1
    assert st["g_norm"] <= 1e-10 * st["g_norm_initial"]
    assert np.linalg.norm(u - u_ref) <= 1e-9 * np.linalg.norm(u_ref)
    b = np.linalg.norm(O.blur_adjoint(v, h, bc))
    assert st["g_norm"] <= 1e-11 * b


def test_newton_from_a_stationary_point_takes_one_tiny_step(tdev):
    torch, pkg, dev = tdev
    h, _, v = _problem(16, 16, 1.0, 2, "ar")
    vt = torch.tensor(v, dtype=torch.float64, device=dev)
    with pkg.Plan(16, 16, h, bc="ar", pc="dfast", mode="fp64") as plan:
        u, _ = plan.deblur(vt, 0.05, 0.1, max_outer=5, inner_tol=1e-10)
        st1 = plan.newton(u, vt, 0.05, 0.1, tol=1e-12, cg_tol=1e-12)
        u1 = u.clone()
        st2 = plan.newton(u, vt, 0.05, 0.1, tol=1e-10, cg_tol=1e-12)
    assert st1["status"] == pkg.TVD_OK and st2["status"] == pkg.TVD_OK
    assert st2["steps"] <= 1 and st2["halvings"] == 0
    assert float((u - u1).norm()) <= 1e-10 * float(u1.norm())


def test_newton_zero_steps_only_evaluates_g(tdev):
    torch, pkg, dev = tdev
    h, _, v = _problem(9, 13, 1.0, 2, "r")
    alpha, beta = 0.05, 0.1
    vt = torch.tensor(v, dtype=torch.float64, device=dev)
    u = vt.clone()
    with pkg.Plan(9, 13, h, bc="r", pc="dfast", mode="fp64") as plan:
        st = plan.newton(u, vt, alpha, beta, max_steps=0)
    assert st["status"] == pkg.TVD_OK and st["steps"] == 0
    assert torch.equal(u, vt)
    g = np.linalg.norm(O.euler_lagrange(v, v, h, "r", alpha, beta))
    assert abs(st["g_norm_initial"] - g) <= 1e-12 * g


def test_newton_rejects_invalid_arguments_and_reblurring_plans(tdev):
    torch, pkg, dev = tdev
    h, _, v = _problem(9, 9, 1.0, 2, "ar")
    vt = torch.tensor(v, dtype=torch.float64, device=dev)
    u = vt.clone()
    with pkg.Plan(9, 9, h, bc="ar", pc="dfast", mode="fp64") as plan:
        with pytest.raises(pkg.TvdError):
            plan.newton(u, vt, 0.05, 0.1, tol=0.0)
        with pytest.raises(pkg.TvdError):
            plan.newton(u, vt, 0.05, -1.0)
        with pytest.raises(pkg.TvdError):
            plan.newton(vt, vt, 0.05, 0.1)
    with pkg.Plan(9, 9, h, bc="ar", pc="dfast", mode="fp64", method="reblur") as plan:
        with pytest.raises(pkg.TvdError):
            plan.newton(u, vt, 0.05, 0.1)
    assert torch.equal(u, vt)


@pytest.mark.parametrize("bc,pc,mode", [("ar", "dfast", "fp64"), ("r", "fast", "mixed"), ("ar", "fastd", "mixed")])
def test_tracked_g_norm_and_functional_match_the_oracle(tdev, bc, pc, mode):
    torch, pkg, dev = tdev
    nr, nc, alpha, beta, K = 40, 36, 2e-3, 2e-2, 6
    h, _, v = _problem(nr, nc, 1.5, 4, bc, seed=11)
    b = O.blur_adjoint(v, h, bc)
    u = v.copy()
    g_ref, f_ref = [], []
    for _ in range(K):
        g_ref.append(float(np.linalg.norm(O.euler_lagrange(u, v, h, bc, alpha, beta))))
        f_ref.append(O.tv_functional(u, v, h, bc, alpha, beta))
        u, _, _, _ = O.fp_step(u, b, h, bc, alpha, beta, pc, 1e-12, 20000)
    g_fin = float(np.linalg.norm(O.euler_lagrange(u, v, h, bc, alpha, beta)))
    f_fin = O.tv_functional(u, v, h, bc, alpha, beta)
    vt = torch.tensor(v, dtype=torch.float64, device=dev)
    with pkg.Plan(nr, nc, h, bc=bc, pc=pc, mode=mode) as plan:
        _, st = plan.deblur(vt, alpha, beta, max_outer=K, inner_tol=1e-12, inner_maxit=20000, track=True)
        _, st0 = plan.deblur(vt, alpha, beta, max_outer=K, inner_tol=1e-12, inner_maxit=20000)
    assert st["inner_iters"] == st0["inner_iters"]   # tracking changes nothing in the iteration
    np.testing.assert_allclose(st["g_norm"], g_ref, rtol=1e-6)
    np.testing.assert_allclose(st["functional"], f_ref, rtol=1e-10)
    assert st["final_g_norm"] == pytest.approx(g_fin, rel=1e-6)
    assert st["final_functional"] == pytest.approx(f_fin, rel=1e-10)
    # the lagged-diffusivity iteration lowers the functional at every step (near-exact solves)
    assert all(f_ref[k + 1] < f_ref[k] for k in range(K - 1))
