"""The differentiable fixed point (torch.autograd.Function over tv_deblur / tv_deblur_adjoint).

Loss ||u*(v, alpha, beta, sigma) - u_true||^2 with learnable log alpha, log
beta and the Gaussian width sigma (the differentiation configuration, at a
size where the fixed point converges to 1e-13 in seconds). Checked against
central finite differences with step 1e-4 in (log alpha, log beta, sigma)
(FP iteration re-converged for every step) and against the FP64 oracle's
adjoint gradient (itself pinned by finite differences of the oracle's fixed
point).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1011_5964_gb300 import synth

pytestmark = pytest.mark.gpu

N, M, SEED = 24, 6, 77
SIGMA_TRUE, SIGMA0, ALPHA0, BETA0 = 1.5, 1.2, 0.02, 0.1


@pytest.fixture(scope="module")
def prob():
    import torch
    from paper_1011_5964_gb300.autograd import gaussian_taps
    ut = synth.piecewise_constant_image(N, N, seed=SEED)
    h_true, _ = gaussian_taps(SIGMA_TRUE, M)
    v = synth.add_noise(O.blur(ut, h_true, "ar"), synth.noise_direction(N, N, SEED), 0.01)
    dev = torch.device("cuda:0")
    return torch, dev, ut, v


def loss_and_grads(prob, mode, la, lb, s, want_grad=True):
    torch, dev, ut, v = prob
    from paper_1011_5964_gb300.autograd import tv_fixed_point
    vt = torch.tensor(v, dtype=torch.float64, device=dev)
    ut_t = torch.tensor(ut, dtype=torch.float64, device=dev)
    la_t = torch.tensor(la, dtype=torch.float64, device=dev, requires_grad=want_grad)
    lb_t = torch.tensor(lb, dtype=torch.float64, device=dev, requires_grad=want_grad)
    s_t = torch.tensor(s, dtype=torch.float64, device=dev, requires_grad=want_grad)
    u = tv_fixed_point(vt, la_t.exp(), lb_t.exp(), s_t, M, bc="ar", mode=mode, max_outer=3000, outer_tol=1e-13,
                       inner_tol=1e-13, adjoint_tol=1e-13)
    loss = ((u - ut_t) ** 2).sum()
    if not want_grad:
        return float(loss), None
    loss.backward()
    return float(loss), np.array([float(la_t.grad), float(lb_t.grad), float(s_t.grad)])


def test_gradients_match_central_differences(prob):
    p0 = [math.log(ALPHA0), math.log(BETA0), SIGMA0]
    _, g = loss_and_grads(prob, "fp64", *p0)
    step = 1e-4
    for k in range(3):
        pp, pm = list(p0), list(p0)
        pp[k] += step
        pm[k] -= step
        fd = (loss_and_grads(prob, "fp64", *pp, want_grad=False)[0]
              - loss_and_grads(prob, "fp64", *pm, want_grad=False)[0]) / (2 * step)
        assert abs(g[k] - fd) <= 1e-5 * abs(fd) + 1e-9, (k, g[k], fd)


def test_gradients_match_the_oracle(prob):
    torch, dev, ut, v = prob
    from paper_1011_5964_gb300.autograd import gaussian_taps
    la, lb, s = math.log(ALPHA0), math.log(BETA0), SIGMA0
    _, g = loss_and_grads(prob, "fp64", la, lb, s)
    alpha, beta = math.exp(la), math.exp(lb)
    h, dh = gaussian_taps(s, M)
    u, _ = O.tv_deblur(v, h, "ar", alpha, beta, outer=3000, tol=1e-14, maxit=20000, kind=O.PC_DFAST, outer_tol=1e-15)
    lam, it, rr, ok = O.adjoint_solve(u, h, "ar", alpha, beta, 2 * (u - ut), tol=1e-14)
    ga, gb, gh = O.fixed_point_gradients(u, v, h, "ar", alpha, beta, lam)
    ref = np.array([ga * alpha, gb * beta, float(np.sum(gh * dh))])   # chain rule to log alpha, log beta, sigma
    assert np.abs(g - ref).max() <= 1e-7 * np.abs(ref).max(), (g, ref)


def test_mixed_form_gradients_agree_with_fp64(prob):
    p0 = [math.log(ALPHA0), math.log(BETA0), SIGMA0]
    l64, g64 = loss_and_grads(prob, "fp64", *p0)
    lmx, gmx = loss_and_grads(prob, "mixed", *p0)
    assert abs(lmx - l64) <= 1e-6 * abs(l64)
    assert np.abs(gmx - g64).max() <= 1e-5 * np.abs(g64).max(), (gmx, g64)


def test_gradient_with_respect_to_the_observation(prob):
    """dl/dv = H lambda: checked by a directional central difference."""
    torch, dev, ut, v = prob
    from paper_1011_5964_gb300.autograd import tv_fixed_point
    rng = np.random.default_rng(1)
    d = rng.standard_normal(v.shape)
    ut_t = torch.tensor(ut, dtype=torch.float64, device=dev)
    def run(vv, grad):
        vt = torch.tensor(vv, dtype=torch.float64, device=dev, requires_grad=grad)
        u = tv_fixed_point(vt, torch.tensor(ALPHA0, dtype=torch.float64), torch.tensor(BETA0, dtype=torch.float64),
                           torch.tensor(SIGMA0, dtype=torch.float64), M, max_outer=3000, outer_tol=1e-13,
                           inner_tol=1e-13, adjoint_tol=1e-13)
        loss = ((u - ut_t) ** 2).sum()
        if grad:
            loss.backward()
            return float(loss), vt.grad.cpu().numpy()
        return float(loss), None
    _, gv = run(v, True)
    e = 1e-5
    fd = (run(v + e * d, False)[0] - run(v - e * d, False)[0]) / (2 * e)
    assert abs(float(np.sum(gv * d)) - fd) <= 1e-5 * abs(fd)
