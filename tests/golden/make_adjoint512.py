"""Write tests/golden/adjoint512_oracle.json: the FP64 oracle's converged fixed
point and its adjoint gradients on the 512 x 512 differentiation workload
(piecewise-constant ground truth, seed 77; observation blurred with a Gaussian
sigma 2.5 on 17 x 17 under anti-reflective BCs, 1% noise; the model's PSF a
Gaussian sigma 2.0 on the same support; alpha 1e-3, beta 1e-2; loss
l(u*) = ||u* - u_true||^2):

* u*: the FP iteration with the D_M preconditioner (PCG tol 1e-8) until the
  relative change falls below 1e-4, then ``newton_polish`` (preconditioned CG
  to 1e-12 per Newton step) until it falls below 1e-12;
* lambda = J(u*)^-1 dl/du by ``adjoint_solve`` (D_M, tol 1e-12), then
  ``fixed_point_gradients``: dl/dalpha, dl/dbeta and dl/dh for every tap, and
  dl/dsigma = sum dl/dh * dh/dsigma with dh/dsigma by central differences
  (step 1e-6) of the input generator's Gaussian.

Stores the norms of u* and lambda, their values at a seeded pixel sample (the
four corners, pixels on each border line, uniform interior pixels), the norm
of g(u*) and the iteration counts. Calls only the oracle and the input
generator (about an hour on one core):
    python tests/golden/make_adjoint512.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1011_5964_gb300 import synth  # noqa: E402

N, SEED, M, SIGMA_TRUE, SIGMA, ALPHA, BETA, NOISE = 512, 77, 8, 2.5, 2.0, 1e-3, 1e-2, 0.01


def sample_indices(n):
    rng = np.random.default_rng(8642)
    pts = {(0, 0), (0, n - 1), (n - 1, 0), (n - 1, n - 1)}
    for k in rng.integers(1, n - 1, size=24):
        pts |= {(0, int(k)), (n - 1, int(k)), (int(k), 0), (int(k), n - 1)}
    for i, j in zip(rng.integers(0, n, size=1024), rng.integers(0, n, size=1024)):
        pts.add((int(i), int(j)))
    return sorted(i * n + j for i, j in pts)


def main():
    u_true = synth.piecewise_constant_image(N, N, seed=SEED)
    h_true = synth.gaussian_psf(SIGMA_TRUE, half_width=M)
    h = synth.gaussian_psf(SIGMA, half_width=M)
    v = synth.add_noise(O.blur(u_true, h_true, "ar"), synth.noise_direction(N, N, SEED), NOISE)
    t0 = time.time()
    u_fp, fst = O.tv_deblur(v, h, "ar", ALPHA, BETA, outer=400, tol=1e-8, maxit=20000, kind=O.PC_DFAST,
                            outer_tol=1e-4)
    t1 = time.time()
    print("FP", len(fst["inner_iters"]), fst["rel_change"][-1], t1 - t0, flush=True)
    u, nst = O.newton_polish(u_fp, v, h, "ar", ALPHA, BETA, tol=1e-12, max_steps=40, cg_tol=1e-12,
                             kind=O.PC_DFAST)
    t2 = time.time()
    print("Newton", nst, t2 - t1, flush=True)
    dl_du = 2.0 * (u - u_true)
    lam, ait, arel, aok = O.adjoint_solve(u, h, "ar", ALPHA, BETA, dl_du, tol=1e-12, maxit=50000, kind=O.PC_DFAST)
    ga, gb, gh = O.fixed_point_gradients(u, v, h, "ar", ALPHA, BETA, lam)
    t3 = time.time()
    eps = 1e-6
    dh = (synth.gaussian_psf(SIGMA + eps, half_width=M) - synth.gaussian_psf(SIGMA - eps, half_width=M)) / (2 * eps)
    idx = sample_indices(N)
    out = {
        "meta": {"n": N, "seed": SEED, "half_width": M, "sigma_true": SIGMA_TRUE, "sigma": SIGMA, "bc": "ar",
                 "noise": NOISE, "alpha": ALPHA, "beta": BETA, "loss": "||u* - u_true||^2",
                 "fp": {"kind": "dfast", "tol": 1e-8, "outer_tol": 1e-4, "steps": len(fst["inner_iters"]),
                        "inner_iters": fst["inner_iters"], "last_rel_change": fst["rel_change"][-1]},
                 "newton": {"tol": 1e-12, "cg_tol": 1e-12, "rel_change": nst["rel_change"], "t": nst["t"],
                            "cg_iters": nst["cg_iters"], "g_norm": nst["g_norm"], "converged": nst["converged"]},
                 "adjoint": {"kind": "dfast", "tol": 1e-12, "iters": ait, "relres": arel, "converged": aok},
                 "source": "oracle/tvd_oracle.py (FP64 numpy/scipy)",
                 "seconds": {"fp": t1 - t0, "newton": t2 - t1, "adjoint": t3 - t2}},
        "sample_idx": idx,
        "u_norm": float(np.linalg.norm(u)),
        "u_samples": [float(x) for x in u.ravel()[idx]],
        "g_norm": nst["g_norm_final"],
        "b_norm": float(np.linalg.norm(O.blur_adjoint(v, h, "ar"))),
        "loss": float(np.sum((u - u_true) ** 2)),
        "lambda_norm": float(np.linalg.norm(lam)),
        "lambda_samples": [float(x) for x in lam.ravel()[idx]],
        "dl_dalpha": ga,
        "dl_dbeta": gb,
        "dl_dh": gh.tolist(),
        "dl_dsigma": float(np.sum(gh * dh)),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "adjoint512_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print("wrote", path, flush=True)


if __name__ == "__main__":
    main()
