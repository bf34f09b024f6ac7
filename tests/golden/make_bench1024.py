"""Write tests/golden/bench1024_oracle.json: the FP64 oracle's run of the benchmark
workload (1024 x 1024 piecewise-constant image, seed 1234, anti-reflective BCs,
radius-7 disk PSF zero-padded to 31 x 31, 1% noise, alpha 1e-3, beta 1e-2,
10 FP steps, PCG tol 1e-6, D_M preconditioner).

Records per-step inner iteration counts, the last two relative residuals of
each step and the norm of the restored image. The benchmark's CPU baseline
uses the total iteration count to turn its sampled oracle iteration rate into
deblurs per second. Calls only the oracle and the input generator:
    python tests/golden/make_bench1024.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

if __name__ == "__main__":
    import oracle as O
    from paper_1011_5964_gb300 import synth
    n, seed = 1024, 1234
    h = synth.disk_psf(7.0, side=31)
    u_true = synth.piecewise_constant_image(n, n, seed=seed)
    v = synth.add_noise(O.blur(u_true, h, "ar"), synth.noise_direction(n, n, seed), 0.01)
    t0 = time.time()
    u, st = O.tv_deblur(v, h, "ar", 1e-3, 1e-2, outer=10, tol=1e-6, maxit=5000, kind="dfast")
    out = {"meta": {"n": n, "seed": seed, "psf": "disk r=7 on 31x31", "bc": "ar", "noise": 0.01, "alpha": 1e-3,
                    "beta": 1e-2, "outer": 10, "tol": 1e-6, "kind": "dfast",
                    "source": "oracle/tvd_oracle.py (FP64 numpy/scipy)", "seconds": time.time() - t0},
           "inner_iters": st["inner_iters"], "relres_tail": st["relres_tail"],
           "u_norm": float((u * u).sum() ** 0.5)}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "bench1024_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)
