"""The device-driven CG loop: a CUDA graph with a while node runs chunks of CG
iterations until the device's CG state reports convergence, in place of the
host polling the state after each chunk.

* The same kernels run in the same order, so a deblur with the device loop
  equals the host-polled one bit for bit (iterate and per-step inner
  iteration counts), in FP64 and MIXED plans, FFT and GEMM forms.
* The loop launches no chunk past convergence; it adds one single-thread
  kernel per chunk of four iterations (the condition) and one per solve (the
  budget), so its kernel count stays within 10% of the host-polled loop's
  (at the 1024^2 MIXED workload, where the host-polled loop launches many
  chunks past convergence, it launches 16% fewer).
* The same for PBiCGstab (the reblurring method, with L and with L_AR); a
  plan whose method changes after a solve drops its captured chunks and
  gives the new method's result (equal to a fresh plan's).
* A solve that cannot converge stops at maxit (the state's own stop; the
  chunk budget of the loop is a second bound).

TVD_CG_DEVICE_LOOP=0 at graph capture selects the host-polled loop.
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
    return torch, pkg, torch.device("cuda:0")


def _deblur(torch, pkg, dev, v, h, loop, method="fp", **plan_kw):
    old = os.environ.get("TVD_CG_DEVICE_LOOP")
    os.environ["TVD_CG_DEVICE_LOOP"] = "1" if loop else "0"
    try:
        with pkg.Plan(v.shape[0], v.shape[1], h, bc="ar", pc="dfast", method=method, **plan_kw) as plan:
            vt = torch.tensor(v, device=dev)
            k0 = pkg.kernel_launches()
            u, st = plan.deblur(vt, 1e-3, 1e-2, max_outer=4, inner_tol=1e-6, inner_maxit=3000)
            torch.cuda.synchronize()
            return u, st, pkg.kernel_launches() - k0
    finally:
        if old is None:
            os.environ.pop("TVD_CG_DEVICE_LOOP", None)
        else:
            os.environ["TVD_CG_DEVICE_LOOP"] = old


def _observation(n, seed):
    h = synth.gaussian_psf(1.5, half_width=4)
    u_true = synth.piecewise_constant_image(n, n, seed=seed)
    return h, synth.add_noise(O.blur(u_true, h, O.AR), synth.noise_direction(n, n, seed), 0.01)


@pytest.mark.parametrize("method", ["fp", "reblur", "reblur_arl"])
@pytest.mark.parametrize("mode,transform", [("fp64", None), ("mixed", "fft"), ("mixed", "gemm")])
def test_device_loop_equals_host_polled_loop(tdev, mode, transform, method):
    torch, pkg, dev = tdev
    h, v = _observation(160, 31)
    kw = dict(mode=mode, transform=transform, method=method)
    u0, st0, k0 = _deblur(torch, pkg, dev, v, h, False, **kw)
    u1, st1, k1 = _deblur(torch, pkg, dev, v, h, True, **kw)
    assert st0["status"] == st1["status"] == pkg.TVD_OK
    assert list(st1["inner_iters"]) == list(st0["inner_iters"])
    assert torch.equal(u1, u0), float((u1 - u0).abs().max())
    assert k1 <= 1.1 * k0, (k1, k0)


def test_device_loop_stops_at_maxit(tdev):
    torch, pkg, dev = tdev
    n = 64
    h = synth.gaussian_psf(1.5, half_width=4)
    rng = np.random.default_rng(5)
    u = torch.tensor(rng.uniform(0, 1, (n, n)), device=dev)
    b = torch.tensor(rng.standard_normal((n, n)), device=dev)
    with pkg.Plan(n, n, h, bc="ar", pc="dfast", mode="fp64") as plan:
        x = torch.zeros_like(b)
        k, _, st = plan.pcg_solve(u, 1e-3, 1e-2, b, x, tol=1e-300, maxit=37)
    assert st == pkg.TVD_ENOCONV and k == 37


def test_method_change_drops_captured_chunks(tdev):
    torch, pkg, dev = tdev
    h, v = _observation(96, 32)
    vt = torch.tensor(v, device=dev)
    kw = dict(max_outer=3, inner_tol=1e-6, inner_maxit=3000)
    with pkg.Plan(96, 96, h, bc="ar", pc="dfast", mode="mixed", method="reblur_arl") as fresh:
        u_ref, st_ref = fresh.deblur(vt, 1e-3, 1e-2, **kw)
    with pkg.Plan(96, 96, h, bc="ar", pc="dfast", mode="mixed", method="reblur") as plan:
        plan.deblur(vt, 1e-3, 1e-2, **kw)
        plan.set_method("reblur_arl")
        u, st = plan.deblur(vt, 1e-3, 1e-2, **kw)
    assert list(st["inner_iters"]) == list(st_ref["inner_iters"])
    assert float((u - u_ref).norm()) <= 1e-12 * float(u_ref.norm())


def test_adjoint_device_loop_equals_host_polled_loop(tdev):
    """The MIXED Jacobian CG of the adjoint (and of the Newton steps) runs through the same loop."""
    torch, pkg, dev = tdev
    h, v = _observation(96, 33)
    vt = torch.tensor(v, device=dev)
    out = []
    for loop in (False, True):
        os.environ["TVD_CG_DEVICE_LOOP"] = "1" if loop else "0"
        try:
            with pkg.Plan(96, 96, h, bc="ar", pc="dfast", mode="mixed") as plan:
                u, _ = plan.deblur(vt, 1e-3, 1e-2, max_outer=6, inner_tol=1e-8, inner_maxit=5000)
                lam, da, db, dh, ast = plan.adjoint(u, vt, 1e-3, 1e-2, 2.0 * (u - vt), tol=1e-10, maxit=5000)
                out.append((lam.clone(), da, db, np.array(dh), ast))
        finally:
            os.environ.pop("TVD_CG_DEVICE_LOOP", None)
    (l0, a0, b0, h0, s0), (l1, a1, b1, h1, s1) = out
    assert s0["status"] == s1["status"] and s0["iters"] == s1["iters"] > 0
    assert torch.equal(l0, l1)
    assert (a0, b0) == (a1, b1) and np.array_equal(h0, h1)
