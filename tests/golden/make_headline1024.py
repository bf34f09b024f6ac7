"""Write tests/golden/headline1024_oracle.json: the FP64 oracle on the 1024 x 1024
headline workload (piecewise-constant image, seed 1234, anti-reflective BCs,
radius-7 disk PSF zero-padded to 31 x 31, 1% noise, alpha 1e-3, beta 1e-2,
10 FP steps, D_M preconditioner), for the GPU parity tests at that size:

* "fp64": the run at PCG tol 1e-6 (the plain method's setting) and six runs
  with the oracle's rounding-noise hook (every product with A and every
  preconditioner output times 1 + 2^-50 xi, the same hook and seeds as
  tests/parity.py), giving each FP step's count spread and the image spread;
* "tight": the run at PCG tol 1e-10 (both sides solve each FP step to 1e-10
  for the chosen-form gate of 1e-5 relative on the restored image).

Each run stores the per-step inner iteration counts, the norm of the restored
image and its values at a fixed seeded sample of pixels (all four corners,
pixels on each border line, and uniformly drawn interior pixels). Calls only
the oracle and the input generator; the eight runs go to separate processes:
    python tests/golden/make_headline1024.py
"""
import concurrent.futures as cf
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

N, SEED, ALPHA, BETA, OUTER = 1024, 1234, 1e-3, 1e-2, 10
EPS = 2.0 ** -50


def sample_indices(n):
    import numpy as np
    rng = np.random.default_rng(4321)
    pts = {(0, 0), (0, n - 1), (n - 1, 0), (n - 1, n - 1)}
    for k in rng.integers(1, n - 1, size=32):
        pts |= {(0, int(k)), (n - 1, int(k)), (int(k), 0), (int(k), n - 1)}
    for i, j in zip(rng.integers(0, n, size=2048), rng.integers(0, n, size=2048)):
        pts.add((int(i), int(j)))
    return sorted(i * n + j for i, j in pts)


def inputs():
    import oracle as O
    from paper_1011_5964_gb300 import synth
    h = synth.disk_psf(7.0, side=31)
    u_true = synth.piecewise_constant_image(N, N, seed=SEED)
    v = synth.add_noise(O.blur(u_true, h, "ar"), synth.noise_direction(N, N, SEED), 0.01)
    return v, h


def run(tol, j):
    """One oracle deblur; j >= 1 selects the perturbed run with noise seed 10000 + j."""
    import numpy as np
    import oracle as O
    v, h = inputs()
    noise = (np.random.default_rng(10_000 + j), EPS) if j else None
    t0 = time.time()
    u, st = O.tv_deblur(v, h, "ar", ALPHA, BETA, outer=OUTER, tol=tol, maxit=20000, kind="dfast", noise=noise)
    return u, st["inner_iters"], time.time() - t0


if __name__ == "__main__":
    import numpy as np
    idx = sample_indices(N)
    jobs = [(1e-6, j) for j in range(7)] + [(1e-10, 0)]
    with cf.ProcessPoolExecutor(max_workers=len(jobs), mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(run, *zip(*jobs)))
    (u0, it0, s0), pert, (ut, itt, st_) = res[0], res[1:7], res[7]
    nrm = float(np.linalg.norm(u0))
    spread = [max(abs(p[1][k] - it0[k]) for p in pert) for k in range(OUTER)]
    img_spread = max(float(np.linalg.norm(p[0] - u0)) / nrm for p in pert)
    flat0, flatt = u0.ravel(), ut.ravel()
    out = {
        "meta": {"n": N, "seed": SEED, "psf": "disk r=7 on 31x31", "bc": "ar", "noise": 0.01, "alpha": ALPHA,
                 "beta": BETA, "outer": OUTER, "kind": "dfast", "perturbation": "2^-50, seeds 10001-10006",
                 "source": "oracle/tvd_oracle.py (FP64 numpy/scipy)",
                 "seconds": {"fp64": s0, "tight": st_}},
        "sample_idx": idx,
        "fp64": {"tol": 1e-6, "inner_iters": it0, "perturbed_iters": [p[1] for p in pert],
                 "step_spread": spread, "image_spread": img_spread, "u_norm": nrm,
                 "u_samples": [float(flat0[i]) for i in idx]},
        "tight": {"tol": 1e-10, "inner_iters": itt, "u_norm": float(np.linalg.norm(ut)),
                  "u_samples": [float(flatt[i]) for i in idx]},
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "headline1024_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print("wrote", path, "fp64 iters", it0, "spread", spread, "tight iters", itt)
