"""Write tests/golden/config2_oracle.json: FP64 oracle inner-iteration counts for the
256 x 256 sweep (reflective D_R and anti-reflective D_M preconditioners, plus
unpreconditioned CG; noise 0.5% and 2%; alpha in {1e-4, 1e-3, 1e-2}; beta 1e-2;
Gaussian PSF sigma 2 on 15 x 15; 10 FP steps; PCG tol 1e-6).

Calls only the oracle and the input generator. Run:  python tests/golden/make_config2.py
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


def run(case):
    import oracle as O
    from paper_1011_5964_gb300 import synth
    h = synth.gaussian_psf(2.0, half_width=7)
    u_true = synth.piecewise_constant_image(N, N, seed=SEED)
    v = synth.add_noise(O.blur(u_true, h, case["bc"]), synth.noise_direction(N, N, SEED), case["noise"])
    u, st = O.tv_deblur(v, h, case["bc"], case["alpha"], 1e-2, outer=OUTER, tol=TOL, maxit=5000, kind=case["kind"])
    return dict(case, inner_iters=st["inner_iters"], relres_tail=st["relres_tail"],
                u_norm=float((u * u).sum() ** 0.5))


if __name__ == "__main__":
    ctx = mp.get_context("spawn")
    with ctx.Pool(max(1, (os.cpu_count() or 2) - 1)) as pool:
        results = pool.map(run, cases())
    meta = {"n": N, "seed": SEED, "outer": OUTER, "tol": TOL, "beta": 1e-2, "psf": "gaussian sigma=2, 15x15",
            "source": "oracle/tvd_oracle.py (FP64 numpy/scipy)"}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "config2_oracle.json")
    with open(path, "w") as f:
        json.dump({"meta": meta, "runs": results}, f, indent=1)
    print("wrote", path)
