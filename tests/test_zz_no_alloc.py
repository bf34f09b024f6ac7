"""The allocation-free entry point tvd_normal_apply_noalloc.

tvd_normal_apply_noalloc serves callers that cannot allocate device memory
themselves or through the library: code running under a framework that owns
a fixed device-memory pool or budget, and callbacks from such a framework that
must not allocate behind its back. It keeps H x, the diffusivity and the PSF
tables in fixed arrays of the library instead. Its output is checked against
the plan-based entry points (ar_blur_apply, tv_operator_apply) and against the
FP64 oracle's H^T H x + alpha L(u) x, on two calls in a row. This file is
collected last so that a failure here does not hide the results of the other
tests; it must pass both alone in a fresh process and after the rest of the
suite.
"""
import numpy as np
import pytest

import oracle as O
from paper_1011_5964_gb300 import synth

pytestmark = pytest.mark.gpu


def reference(pkg, torch, h, bc, u, x, alpha, beta):
    """H^T H x + alpha L(u) x through the existing plan entry points (ar_blur_apply, tv_operator_apply)."""
    n_rows, n_cols = x.shape
    with pkg.Plan(n_rows, n_cols, h, bc=bc, pc="dfast", mode="fp64") as plan:
        hx = plan.blur(x)
        hthx = plan.blur(hx, transpose=True)
        lx = plan.tv_operator(u, beta, x)
        out = hthx + alpha * lx
        torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("bc", ["ar", "r"])
def test_noalloc_matches_plan_path_twice(bc):
    import torch
    import paper_1011_5964_gb300 as pkg
    dev = torch.device("cuda:0")
    cases = [
        (synth.disk_psf(7.0, side=31), (300, 257), 1e-3, 1e-2, 11),   # first call: disk, ragged tiles
        (synth.gaussian_psf(1.5), (96, 130), 1e-2, 5e-2, 12),         # second call: other PSF and size
    ]
    for h, (n_rows, n_cols), alpha, beta, seed in cases:
        u = torch.tensor(synth.piecewise_constant_image(n_rows, n_cols, seed=seed), dtype=torch.float64, device=dev)
        g = torch.Generator(device=dev).manual_seed(seed)
        x = torch.randn(n_rows, n_cols, dtype=torch.float64, device=dev, generator=g)
        y = pkg.normal_apply_noalloc(h, u, alpha, beta, x, bc=bc)
        ref = reference(pkg, torch, h, bc, u, x, alpha, beta)
        err = float((y - ref).abs().max() / ref.abs().max())
        assert err < 1e-12, (bc, n_rows, n_cols, err)
        # the oracle's product of the FP step (eq. (fp)), element by element
        un, xn = u.cpu().numpy(), x.cpu().numpy()
        ref_o = O.normal_apply(xn, h, bc, O.diffusivity(un, beta), alpha)
        err_o = float(np.abs(y.cpu().numpy() - ref_o).max() / np.abs(ref_o).max())
        assert err_o < 1e-12, (bc, n_rows, n_cols, err_o)


def test_noalloc_rejects_oversize():
    import torch
    import paper_1011_5964_gb300 as pkg
    dev = torch.device("cuda:0")
    x = torch.zeros(1024, 1024, dtype=torch.float64, device=dev)
    with pytest.raises(pkg.TvdError) as e:
        pkg.normal_apply_noalloc(synth.gaussian_psf(1.0), x + 1.0, 1e-3, 1e-2, x)
    assert e.value.status == pkg.TVD_EINVAL and "exceeds" in str(e.value)
