"""Write tests/golden/config2_oracle.json: FP64 oracle results for the 256 x 256 sweep
(reflective D_R and anti-reflective D_M preconditioners, plus unpreconditioned CG;
noise 0.5% and 2%; alpha in {1e-4, 1e-3, 1e-2}; beta 1e-2; Gaussian PSF sigma 2 on
15 x 15; 10 FP steps; PCG tol 1e-6).

For each case: the per-step inner iteration counts, the norm of the restored
image and 64 sampled pixels of it, and the rounding envelope of the oracle
itself (six more runs with every operator output perturbed by a relative
2^-50, see tests/parity.py): their per-step counts, the per-step spread of the
counts and the spread of the sampled pixels and of the image. Calls only the oracle, the input generator
and the perturbation helper. Run:  python tests/golden/make_config2.py
"""
import json
import multiprocessing as mp
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

N = 256
SEED = 1234
OUTER = 10
TOL = 1e-6


def cases():
    out = []
    for bc in ("r", "ar"):
        for kind in ("dfast", "none"):
            for noise in (0.005, 0.02):
                for alpha in (1e-4, 1e-3, 1e-2):
                    out.append({"bc": bc, "kind": kind, "noise": noise, "alpha": alpha})
    return out


def sample_index():
    import numpy as np
    rng = np.random.default_rng(99)
    return rng.integers(0, N, size=(64, 2))


def run(case):
    import numpy as np
    import oracle as O
    from paper_1011_5964_gb300 import synth
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from parity import N_PERTURBED, count_spread, noise
    h = synth.gaussian_psf(2.0, half_width=7)
    u_true = synth.piecewise_constant_image(N, N, seed=SEED)
    v = synth.add_noise(O.blur(u_true, h, case["bc"]), synth.noise_direction(N, N, SEED), case["noise"])
    args = (h, case["bc"], case["alpha"], 1e-2)
    kw = dict(outer=OUTER, tol=TOL, maxit=5000, kind=case["kind"])
    u, st = O.tv_deblur(v, *args, **kw)
    pert = [O.tv_deblur(v, *args, noise=noise(j), **kw) for j in range(1, N_PERTURBED + 1)]
    idx = sample_index()
    samp = u[idx[:, 0], idx[:, 1]]
    nu = float(np.linalg.norm(u))
    return dict(case, inner_iters=st["inner_iters"],
                perturbed_iters=[p[1]["inner_iters"] for p in pert],
                count_spread=count_spread(st["inner_iters"], [p[1]["inner_iters"] for p in pert]),
                u_norm=nu, samples=samp.tolist(),
                sample_spread=float(max(np.abs(p[0][idx[:, 0], idx[:, 1]] - samp).max() for p in pert)),
                image_spread=float(max(np.linalg.norm(p[0] - u) / nu for p in pert)))


if __name__ == "__main__":
    ctx = mp.get_context("spawn")
    with ctx.Pool(max(1, (os.cpu_count() or 2) - 1)) as pool:
        results = pool.map(run, cases())
    meta = {"n": N, "seed": SEED, "outer": OUTER, "tol": TOL, "beta": 1e-2, "psf": "gaussian sigma=2, 15x15",
            "source": "oracle/tvd_oracle.py (FP64 numpy/scipy)", "sample_index": sample_index().tolist()}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "config2_oracle.json")
    with open(path, "w") as f:
        json.dump({"meta": meta, "runs": results}, f, indent=1)
    print("wrote", path)
