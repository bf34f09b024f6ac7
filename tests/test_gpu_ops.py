"""GPU parity of the operator entry points against the FP64 oracle.

Each case calls the C ABI (through the binding) and compares element by element
with the oracle on the same seeded inputs. Sizes span several 32 x 32 tiles
with ragged tails, rectangular images, the smallest image (3 x 3), PSF
half-widths up to n - 2, non-separable PSFs with h_ab != h_ba, the zero-padded
31 x 31 disk, and transform lengths with large prime factors (generic radix).

Tolerances: float64 plans 1e-12 relative (max-norm) for the stencils and 1e-10
for the transform solve (rounding of O(n log n) sums and of the spectral
divide); float32 plans 5e-6 (stencils) and 1e-3 (preconditioner solve, whose
spectrum spans several decades, so relative rounding is amplified).
"""
import numpy as np
import pytest

import oracle as O
from paper_1011_5964_gb300 import synth

pytestmark = pytest.mark.gpu


def qsym_psf(mr, mc, seed=0):
    rng = np.random.default_rng(seed)
    q = rng.uniform(0.1, 1.0, (mr + 1, mc + 1))
    a = np.abs(np.arange(-mr, mr + 1))
    b = np.abs(np.arange(-mc, mc + 1))
    h = q[a[:, None], b[None, :]]
    return h / h.sum()


def rel_maxerr(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    import paper_1011_5964_gb300 as pkg
    pkg.load_library()
    return torch, torch.device("cuda:0")


CASES = [
    # (nr, nc, psf)
    (37, 53, "gauss1.5"),
    (64, 64, "gauss1.5"),
    (70, 45, "qsym3x2"),
    (100, 90, "disk31"),
    (3, 3, "qsym1x1"),
    (5, 40, "qsym3x2"),
    (129, 66, "qsym2x4"),
]


def make_psf(name):
    if name == "gauss1.5":
        return synth.gaussian_psf(1.5)
    if name == "disk31":
        return synth.disk_psf(7.0, side=31)
    mr, mc = name[4:].split("x")
    return qsym_psf(int(mr), int(mc), seed=int(mr) * 7 + int(mc))


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
@pytest.mark.parametrize("bc", ["ar", "r"])
@pytest.mark.parametrize("nr,nc,psf", CASES)
def test_blur_forward_and_transpose(torch_dev, nr, nc, psf, bc, mode):
    torch, dev = torch_dev
    import paper_1011_5964_gb300 as pkg
    h = make_psf(psf)
    rng = np.random.default_rng(nr * 1000 + nc)
    x = rng.standard_normal((nr, nc))
    dt = torch.float64 if mode == "fp64" else torch.float32
    tol = 1e-12 if mode == "fp64" else 5e-6
    with pkg.Plan(nr, nc, h, bc=bc, pc="dfast", mode=mode) as plan:
        xt = torch.tensor(x, dtype=dt, device=dev)
        y = plan.blur(xt).double().cpu().numpy()
        yt = plan.blur(xt, transpose=True).double().cpu().numpy()
    xr = x.astype(np.float32).astype(np.float64) if mode == "mixed" else x
    assert rel_maxerr(y, O.blur(xr, h, bc)) < tol
    assert rel_maxerr(yt, O.blur_adjoint(xr, h, bc)) < tol


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
@pytest.mark.parametrize("nr,nc", [(37, 53), (3, 3), (64, 65), (130, 33)])
def test_tv_operator(torch_dev, nr, nc, mode):
    torch, dev = torch_dev
    import paper_1011_5964_gb300 as pkg
    rng = np.random.default_rng(5)
    u = rng.uniform(0, 1, (nr, nc))
    x = rng.standard_normal((nr, nc))
    dt = torch.float64 if mode == "fp64" else torch.float32
    with pkg.Plan(nr, nc, synth.gaussian_psf(0.5, half_width=1), mode=mode) as plan:
        y = plan.tv_operator(torch.tensor(u, dtype=dt, device=dev), 0.05,
                             torch.tensor(x, dtype=dt, device=dev)).double().cpu().numpy()
    if mode == "mixed":
        u = u.astype(np.float32).astype(np.float64)
        x = x.astype(np.float32).astype(np.float64)
    ref = O.tv_apply(O.diffusivity(u, 0.05), x)
    assert rel_maxerr(y, ref) < (1e-12 if mode == "fp64" else 2e-5)


PC_SHAPES = [(37, 53), (64, 64), (3, 3), (4, 7), (128, 130), (96, 33)]


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
@pytest.mark.parametrize("kind", ["dfast", "fast", "fastd", "diag", "none"])
@pytest.mark.parametrize("bc", ["ar", "r"])
@pytest.mark.parametrize("nr,nc", PC_SHAPES)
def test_preconditioner_solve(torch_dev, nr, nc, bc, kind, mode):
    torch, dev = torch_dev
    import paper_1011_5964_gb300 as pkg
    h = synth.gaussian_psf(1.0, half_width=min(3, nr - 2, nc - 2))
    rng = np.random.default_rng(nr + 17 * nc)
    u = synth.piecewise_constant_image(nr, nc, seed=nr)
    r = rng.standard_normal((nr, nc))
    alpha, beta = 1e-2, 0.05
    dt = torch.float64 if mode == "fp64" else torch.float32
    if mode == "mixed":
        u = u.astype(np.float32).astype(np.float64)
        r = r.astype(np.float32).astype(np.float64)
    # the FFT form of the transforms (the GEMM form has its own tests in test_gpu_gemm_transform.py)
    with pkg.Plan(nr, nc, h, bc=bc, pc=kind, mode=mode, transform="fft") as plan:
        plan.precond_setup(torch.tensor(u, dtype=dt, device=dev), alpha, beta)
        z = plan.precond_solve(torch.tensor(r, dtype=dt, device=dev)).double().cpu().numpy()
    P = O.precond_setup(u, h, bc, alpha, beta, kind)
    ref = O.precond_apply(r, P)
    # element by element: max |z - z_ref| / max |z_ref|
    err = float(np.abs(z - ref).max() / np.abs(ref).max())
    assert err < (1e-10 if mode == "fp64" else 1e-3), err


def test_blur_full_size_sampled(torch_dev):
    """1024 x 1024, anti-reflective, the 31 x 31 zero-padded disk (the benchmark
    workload): sampled outputs, including every corner and border, against the
    oracle's single-pixel evaluation, in both arithmetic modes."""
    torch, dev = torch_dev
    import paper_1011_5964_gb300 as pkg
    n = 1024
    h = synth.disk_psf(7.0, side=31)
    x = synth.piecewise_constant_image(n, n, seed=1234)
    pts = [(0, 0), (0, n - 1), (n - 1, 0), (n - 1, n - 1), (0, 500), (n - 1, 3), (6, 0), (700, n - 1),
           (3, 4), (1020, 1017), (511, 512), (7, 7), (8, 1016), (1016, 8), (300, 301)]
    for mode, tol in (("fp64", 1e-12), ("mixed", 5e-6)):
        dt = torch.float64 if mode == "fp64" else torch.float32
        with pkg.Plan(n, n, h, bc="ar", pc="dfast", mode=mode) as plan:
            xt = torch.tensor(x, dtype=dt, device=dev)
            y = plan.blur(xt).double().cpu().numpy()
        xr = x.astype(np.float32).astype(np.float64) if mode == "mixed" else x
        for (i, j) in pts:
            ref = O.blur_at(xr, h, "ar", i, j)
            assert abs(y[i, j] - ref) <= tol * max(1.0, abs(ref)), (mode, i, j, y[i, j], ref)


def test_adjoint_identity_full_size(torch_dev):
    """<H x, y> = <x, H^T y> at 2048 x 2048 (a property that holds at any size)."""
    torch, dev = torch_dev
    import paper_1011_5964_gb300 as pkg
    n = 2048
    h = synth.disk_psf(7.0, side=31)
    g = torch.Generator(device=dev).manual_seed(3)
    x = torch.randn(n, n, dtype=torch.float64, device=dev, generator=g)
    y = torch.randn(n, n, dtype=torch.float64, device=dev, generator=g)
    with pkg.Plan(n, n, h, bc="ar", pc="dfast", mode="fp64") as plan:
        lhs = float((plan.blur(x) * y).sum())
        rhs = float((x * plan.blur(y, transpose=True)).sum())
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + float(x.abs().sum()))
