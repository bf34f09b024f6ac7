"""The differentiation workload at its own size: 512 x 512, anti-reflective
BCs, observation blurred with a Gaussian sigma 2.5 on 17 x 17 and 1% noise,
model PSF a Gaussian sigma 2.0 on the same support, alpha 1e-3, beta 1e-2,
loss l = ||u* - u_true||^2.

* The fixed point: FP steps until the relative change falls below 1e-4, then
  Newton steps (tv_deblur_newton) to a relative change below 1e-12, on both
  sides; the GPU's u* at the stored pixel sample within 1e-9 (RMS, relative
  to ||u*|| / sqrt(N)) of the oracle's (tests/golden/adjoint512_oracle.json,
  written by make_adjoint512.py from the oracle alone).
* The adjoint gradients dl/dalpha, dl/dbeta, every dl/dh_ab and dl/dsigma
  within 1e-7 relative of the oracle's. Both sides stop the Newton steps at
  1e-12 and the adjoint PCG at ||r|| / ||r_0|| < 1e-12; what separates them
  is that residual times the conditioning of J (about 1e4-1e5 here), so
  1e-7 leaves a margin over the expected 1e-8.
* Through torch.autograd (tv_fixed_point, MIXED), the gradient in
  (log alpha, log beta, sigma) against central finite differences with step
  1e-4, each fixed point re-converged: within 1e-5 relative (truncation about
  1e-8, the fixed points' own accuracy about 1e-7 of each difference).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1011_5964_gb300 import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "adjoint512_oracle.json")


@pytest.fixture(scope="module")
def case():
    import torch
    import paper_1011_5964_gb300 as pkg
    pkg.load_library()
    g = json.load(open(GOLDEN))
    m = g["meta"]
    n, hw = m["n"], m["half_width"]
    ut = synth.piecewise_constant_image(n, n, seed=m["seed"])
    h_true = synth.gaussian_psf(m["sigma_true"], half_width=hw)
    v = synth.add_noise(O.blur(ut, h_true, "ar"), synth.noise_direction(n, n, m["seed"]), m["noise"])
    return torch, pkg, torch.device("cuda:0"), g, ut, v


def sampled_rel(u, ref_samples, idx, ref_norm):
    d = u.ravel()[idx] - np.asarray(ref_samples)
    return float(np.sqrt(np.mean(d * d)) / (ref_norm / np.sqrt(u.size)))


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_fixed_point_and_gradients_match_the_oracle(case, mode):
    torch, pkg, dev, g, ut, v = case
    m = g["meta"]
    n, hw, alpha, beta = m["n"], m["half_width"], m["alpha"], m["beta"]
    h = synth.gaussian_psf(m["sigma"], half_width=hw)
    vt = torch.tensor(v, device=dev)
    utt = torch.tensor(ut, device=dev)
    with pkg.Plan(n, n, h, bc="ar", pc="dfast", mode=mode) as plan:
        u, st = plan.deblur(vt, alpha, beta, max_outer=400, outer_tol=1e-4, inner_tol=1e-8, inner_maxit=20000)
        nst = plan.newton(u, vt, alpha, beta, tol=1e-12, cg_tol=1e-12, cg_maxit=20000)
        lam, da, db, dh, ast = plan.adjoint(u, vt, alpha, beta, 2.0 * (u - utt), tol=1e-12, maxit=20000)
        un = u.cpu().numpy()
    assert nst["status"] == pkg.TVD_OK and nst["last_rel_change"] < 1e-12, nst
    assert ast["status"] == pkg.TVD_OK, ast
    idx = np.array(g["sample_idx"])
    assert sampled_rel(un, g["u_samples"], idx, g["u_norm"]) < 1e-9
    assert abs(float(np.sum((un - ut) ** 2)) - g["loss"]) <= 1e-9 * g["loss"]
    assert abs(da - g["dl_dalpha"]) <= 1e-7 * abs(g["dl_dalpha"])
    assert abs(db - g["dl_dbeta"]) <= 1e-7 * abs(g["dl_dbeta"])
    ref_h = np.array(g["dl_dh"])
    assert np.abs(dh - ref_h).max() <= 1e-7 * np.abs(ref_h).max()
    eps = 1e-6
    dh_ds = (synth.gaussian_psf(m["sigma"] + eps, half_width=hw) - synth.gaussian_psf(m["sigma"] - eps, half_width=hw))
    dsigma = float(np.sum(dh * dh_ds / (2 * eps)))
    assert abs(dsigma - g["dl_dsigma"]) <= 1e-7 * abs(g["dl_dsigma"])


def test_autograd_gradient_matches_central_differences(case):
    torch, pkg, dev, g, ut, v = case
    from paper_1011_5964_gb300.autograd import tv_fixed_point
    m = g["meta"]
    hw = m["half_width"]
    vt = torch.tensor(v, device=dev)
    utt = torch.tensor(ut, device=dev)

    def loss(la, lb, s, grad):
        p = [torch.tensor(x, dtype=torch.float64, device=dev, requires_grad=grad) for x in (la, lb, s)]
        u = tv_fixed_point(vt, p[0].exp(), p[1].exp(), p[2], hw, bc="ar", mode="mixed", max_outer=400,
                           outer_tol=1e-12, inner_tol=1e-10, adjoint_tol=1e-12, newton_from=1e-4)
        val = ((u - utt) ** 2).sum()
        if not grad:
            return float(val), None
        val.backward()
        return float(val), np.array([float(q.grad) for q in p])

    p0 = [math.log(m["alpha"]), math.log(m["beta"]), m["sigma"]]
    l0, grad = loss(*p0, True)
    assert abs(l0 - g["loss"]) <= 1e-8 * g["loss"]
    step = 1e-4
    for k in range(3):
        pp, pm = list(p0), list(p0)
        pp[k] += step
        pm[k] -= step
        fd = (loss(*pp, False)[0] - loss(*pm, False)[0]) / (2 * step)
        assert abs(grad[k] - fd) <= 1e-5 * abs(fd), (k, grad[k], fd)
