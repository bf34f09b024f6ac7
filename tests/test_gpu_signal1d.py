"""GPU parity on 1D signals (plans of one row, Sec. 5.1) and of the alpha sweep.

The workload is the paper's 1D experiment with synthetic inputs: a seeded
piecewise-constant signal of n = 203 samples in the field of view [0.1, 0.9]
of a wider support, blurred by the out-of-focus PSF of eq. (of) with m = 11
(21 taps) on that support and cropped, 1% noise, beta = 0.1, FP stop 1e-3,
PCG tol 1e-6 (Sec. 5). The observation is built with the oracle's blur.

* Operators (blur, its transpose, L, every preconditioner solve): element by
  element against the oracle on signals of several lengths, 1e-12 (FP64)
  and 1e-5 relative to the largest entry (MIXED: float arithmetic).
* Deblurring: the FP64 GPU path's per-step iteration counts against the
  oracle's, with the envelope of six oracle runs under rounding noise
  (tests/parity.py), and the restored signal within ten times their spread.
* Alpha sweep (Fig. tvrs): the GPU's RRE at every alpha of the grid within
  1e-6 relative of the oracle's when both sides solve each FP step to 1e-10,
  and the same RRE-optimal alpha.
"""
import numpy as np
import pytest

import oracle as O
from paper_1011_5964_gb300 import synth
from parity import N_PERTURBED, check_counts

pytestmark = pytest.mark.gpu

N, M, BETA = 203, 11, 0.1


@pytest.fixture(scope="module")
def tdev():
    import torch
    import paper_1011_5964_gb300 as pkg
    pkg.load_library()
    return torch, pkg, torch.device("cuda:0")


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def signal_problem(seed, n=N, m=M):
    h = synth.out_of_focus_psf_1d(m)
    uw, fov = synth.piecewise_constant_signal(n, seed)
    hv = O.blur(uw[None, :], h, O.R)[:, fov]
    v = synth.add_noise(hv, synth.noise_direction(1, n, seed), 0.01)
    return h, uw[fov][None, :], v


def sym_psf_1d(m, seed):
    rng = np.random.default_rng(seed)
    q = rng.uniform(0.1, 1.0, m + 1)
    h = q[np.abs(np.arange(-m, m + 1))]
    return (h / h.sum())[None, :]


SHAPES = [(3, 1), (7, 2), (64, 7), (203, 10), (257, 20), (1000, 31)]


@pytest.mark.parametrize("n,m", SHAPES)
@pytest.mark.parametrize("bc", ["ar", "r"])
@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_1d_blur_and_transpose_match_the_oracle(tdev, n, m, bc, mode):
    torch, pkg, dev = tdev
    h = sym_psf_1d(m, seed=n + m) if m % 2 else synth.out_of_focus_psf_1d(m)
    m_eff = h.shape[1] // 2
    if m_eff > n - 2:
        pytest.skip("PSF wider than the signal allows")
    x = np.random.default_rng(n).standard_normal((1, n))
    dt = torch.float64 if mode == "fp64" else torch.float32
    tol = 1e-12 if mode == "fp64" else 2e-6
    with pkg.Plan(1, n, h, bc=bc, pc="dfast", mode=mode) as plan:
        xt = torch.tensor(x, dtype=dt, device=dev)
        y = plan.blur(xt).double().cpu().numpy()
        yt = plan.blur(xt, transpose=True).double().cpu().numpy()
    assert rel(y, O.blur(x, h, bc)) < tol
    assert rel(yt, O.blur_adjoint(x, h, bc)) < tol


@pytest.mark.parametrize("bc", ["ar", "r"])
@pytest.mark.parametrize("pc", ["fast", "dfast", "fastd"])
@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_1d_preconditioner_solve_matches_the_oracle(tdev, bc, pc, mode):
    torch, pkg, dev = tdev
    h, _, v = signal_problem(2)
    alpha = 1e-3
    u = v + 0.05 * np.random.default_rng(3).standard_normal(v.shape)
    r = np.random.default_rng(4).standard_normal(v.shape)
    dt = torch.float64 if mode == "fp64" else torch.float32
    with pkg.Plan(1, N, h, bc=bc, pc=pc, mode=mode) as plan:
        plan.precond_setup(torch.tensor(u, dtype=dt, device=dev), alpha, BETA)
        z = plan.precond_solve(torch.tensor(r, dtype=dt, device=dev)).double().cpu().numpy()
    ref = O.precond_apply(r, O.precond_setup(u, h, bc, alpha, BETA, pc))
    assert rel(z, ref) < (1e-11 if mode == "fp64" else 2e-4), rel(z, ref)


@pytest.mark.parametrize("pc", ["fast", "dfast", "fastd"])
def test_1d_reblur_preconditioner_matches_the_oracle(tdev, pc):
    torch, pkg, dev = tdev
    h, _, v = signal_problem(5)
    alpha = 1e-3
    u = v + 0.05 * np.random.default_rng(6).standard_normal(v.shape)
    r = np.random.default_rng(7).standard_normal(v.shape)
    with pkg.Plan(1, N, h, bc="ar", pc=pc, mode="fp64", method="reblur") as plan:
        plan.precond_setup(torch.tensor(u, device=dev), alpha, BETA)
        z = plan.precond_solve(torch.tensor(r, device=dev)).cpu().numpy()
    ref = O.precond_apply(r, O.precond_setup(u, h, "ar", alpha, BETA, pc, method=O.METHOD_REBLUR))
    assert rel(z, ref) < 1e-10, rel(z, ref)


def _oracle_runs(v, h, bc, alpha, kind, method):
    runs = []
    for j in range(N_PERTURBED + 1):
        noise = (np.random.default_rng(10_000 + j), 2.0 ** -50) if j else None
        runs.append(O.tv_deblur(v, h, bc, alpha, BETA, outer=100, tol=1e-6, maxit=5000, kind=kind, outer_tol=1e-3,
                                noise=noise, method=method))
    return runs


@pytest.mark.parametrize("bc,pc,method", [("ar", "dfast", "fp"), ("r", "dfast", "fp"), ("ar", "fastd", "fp"),
                                          ("ar", "none", "fp"), ("ar", "dfast", "reblur")])
def test_1d_deblur_counts_and_signal_match_the_oracle(tdev, bc, pc, method):
    torch, pkg, dev = tdev
    h, _, v = signal_problem(1)
    alpha = 1e-3
    runs = _oracle_runs(v, h, bc, alpha, pc, method)
    (u0, st0), pert = runs[0], runs[1:]
    ref = st0["inner_iters"]
    K = len(ref)
    assert all(len(p[1]["inner_iters"]) == K for p in pert)   # the FP step count is stable under rounding
    spread = [max(abs(p[1]["inner_iters"][k] - ref[k]) for p in pert) for k in range(K)]
    img = max(float(np.linalg.norm(p[0] - u0)) / float(np.linalg.norm(u0)) for p in pert)
    with pkg.Plan(1, N, h, bc=bc, pc=pc, mode="fp64", method=method) as plan:
        u, st = plan.deblur(torch.tensor(v, device=dev), alpha, BETA, max_outer=100, outer_tol=1e-3, inner_tol=1e-6,
                            inner_maxit=5000)
        u = u.cpu().numpy()
    assert st["outer_iters"] == K
    check_counts(st["inner_iters"], ref, spread)
    assert np.linalg.norm(u - u0) <= max(10.0 * img, 1e-12) * np.linalg.norm(u0)


@pytest.mark.parametrize("bc", ["ar", "r"])
def test_alpha_sweep_rre_matches_the_oracle(tdev, bc):
    torch, pkg, dev = tdev
    h, ut, v = signal_problem(4)
    alphas = synth.alpha_grid()
    us, stats = pkg.alpha_sweep(torch.tensor(v, device=dev), h, alphas, BETA, bc=bc, pc="dfast", mode="fp64",
                                outer_tol=1e-3, inner_tol=1e-10, inner_maxit=20000)
    rre = [float(np.linalg.norm(u.cpu().numpy() - ut) / np.linalg.norm(ut)) for u in us]
    ref = []
    for a in alphas:
        u, _ = O.tv_deblur(v, h, bc, a, BETA, outer=100, tol=1e-10, maxit=20000, kind=O.PC_DFAST, outer_tol=1e-3)
        ref.append(float(np.linalg.norm(u - ut) / np.linalg.norm(ut)))
    assert all(s["status"] == pkg.TVD_OK for s in stats)
    np.testing.assert_allclose(rre, ref, rtol=1e-6)
    assert int(np.argmin(rre)) == int(np.argmin(ref))


def test_one_row_plan_validation(tdev):
    torch, pkg, dev = tdev
    with pytest.raises(pkg.TvdError):
        pkg.Plan(1, N, synth.gaussian_psf(1.0, half_width=2), bc="ar")    # a 2D PSF on a 1D signal
    with pytest.raises(pkg.TvdError):
        pkg.Plan(2, N, synth.out_of_focus_psf_1d(3), bc="ar")             # two rows are not a plan size
    with pkg.Plan(1, N, synth.out_of_focus_psf_1d(M), bc="ar", pc="dfast", mode="mixed") as plan:
        assert plan.transform == "fft"
        with pytest.raises(pkg.TvdError):
            plan.set_transform("gemm")
