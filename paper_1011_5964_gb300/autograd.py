"""torch.autograd.Function over tv_deblur and tv_deblur_adjoint.

The forward pass runs the lagged-diffusivity FP iteration of libtvd (eq. (fp))
until its relative change falls below ``newton_from``, then finishes the fixed
point u* by Newton steps on g(u) = 0 (tv_deblur_newton) to ``outer_tol``
(``newton_from`` = 0: the FP iteration alone to ``outer_tol``); the backward pass runs
the adjoint of that fixed point (tv_deblur_adjoint: one preconditioned solve
with J = H^T H + alpha nabla^2 J_beta(u*)), so no outer iterate is stored,
only u*. Gradients flow to the observation v, alpha, beta and the width sigma
of a Gaussian PSF on a fixed (2m + 1)^2 support. This module only marshals
arguments; the fixed point and the adjoint run in the library's kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import Plan


def gaussian_taps(sigma: float, half_width: int):
    """h(sigma) = g g^T / (sum g)^2 with g_a = exp(-a^2 / (2 sigma^2)), and dh/dsigma."""
    a = np.arange(-half_width, half_width + 1, dtype=np.float64)
    g = np.exp(-(a * a) / (2.0 * sigma * sigma))
    G = g.sum()
    h = np.outer(g, g) / (G * G)
    dg = g * (a * a) / sigma ** 3
    dG = dg.sum()
    dh = (np.outer(dg, g) + np.outer(g, dg)) / (G * G) - 2.0 * h * dG / G
    return h, dh


class GaussianTVFixedPoint(torch.autograd.Function):
    """u* = the TV-deblurring fixed point of v for a Gaussian PSF, differentiable in (v, alpha, beta, sigma)."""

    @staticmethod
    def forward(ctx, v, alpha, beta, sigma, half_width: int, bc: str, mode: str, max_outer: int, outer_tol: float,
                inner_tol: float, adjoint_tol: float, newton_from: float):
        a, b, s = float(alpha), float(beta), float(sigma)
        h, dh = gaussian_taps(s, half_width)
        v64 = v.detach().to(torch.float64).contiguous()
        plan = Plan(v64.shape[0], v64.shape[1], h, bc=bc, pc="dfast", mode=mode)
        fp_tol = newton_from if newton_from > 0.0 else outer_tol
        u, stats = plan.deblur(v64, a, b, max_outer=max_outer, outer_tol=fp_tol, inner_tol=inner_tol,
                               inner_maxit=20000)
        if newton_from > 0.0:
            stats["newton"] = plan.newton(u, v64, a, b, tol=outer_tol, cg_tol=inner_tol)
        ctx.plan = plan
        ctx.pdev = [x.device if torch.is_tensor(x) else v.device for x in (alpha, beta, sigma)]
        ctx.params = (a, b, dh, adjoint_tol)
        ctx.stats = stats
        ctx.save_for_backward(v64, u)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        v64, u = ctx.saved_tensors
        a, b, dh, tol = ctx.params
        plan = ctx.plan
        g = grad_u.detach().to(torch.float64).contiguous()
        lam, da, db, dpsf, st = plan.adjoint(u, v64, a, b, g, tol=tol, maxit=20000)
        ctx.adjoint_stats = st
        dv = None
        if ctx.needs_input_grad[0]:
            # F(u, v) = H^T (H u - v) + ...: dF/dv = -H^T, so dl/dv = H lambda
            x = lam if plan.mode == "fp64" else lam.to(torch.float32)
            dv = plan.blur(x).to(grad_u.dtype)
        if dpsf.shape != dh.shape:
            raise RuntimeError("the plan trimmed the Gaussian support; use a half-width with non-zero outer taps")
        dsigma = float(np.sum(dpsf * dh))
        scal = lambda x, k: (torch.tensor(x, dtype=torch.float64, device=ctx.pdev[k - 1])
                             if ctx.needs_input_grad[k] else None)
        return dv, scal(da, 1), scal(db, 2), scal(dsigma, 3), None, None, None, None, None, None, None, None


def tv_fixed_point(v, alpha, beta, sigma, half_width: int, bc: str = "ar", mode: str = "fp64",
                   max_outer: int = 500, outer_tol: float = 1e-10, inner_tol: float = 1e-10,
                   adjoint_tol: float = 1e-10, newton_from: float = 1e-4):
    """Differentiable u*(v, alpha, beta, sigma): alpha, beta, sigma are 0-dim tensors (requires_grad as needed)."""
    return GaussianTVFixedPoint.apply(v, alpha, beta, sigma, half_width, bc, mode, max_outer, outer_tol, inner_tol,
                                      adjoint_tol, newton_from)
