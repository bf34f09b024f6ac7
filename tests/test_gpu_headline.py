"""GPU parity at the headline workload: 1024 x 1024, anti-reflective BCs, radius-7
disk PSF zero-padded to 31 x 31, 1% noise, alpha 1e-3, beta 1e-2, 10 FP steps,
D_M preconditioner, against the FP64 oracle's runs stored in
tests/golden/headline1024_oracle.json (written by make_headline1024.py, which
calls only the oracle and the input generator).

* Plain FP64 GPU form at PCG tol 1e-6: each FP step's inner iteration count
  within that step's own spread over the oracle runs with rounding noise
  (tests/parity.py; identical where those runs agree); the restored image's
  norm and its sampled pixels within ten times the image spread of those runs.
* Chosen (MIXED) form with both sides solving each FP step to 1e-10: the
  restored image within 1e-5 relative of the oracle's, estimated from the
  stored pixel sample (all corners, border pixels, uniform interior pixels)
  as the root-mean-square difference over the sample against ||u|| / sqrt(N),
  and on the norm.

The observation v is built on the host with the oracle's own blur, exactly
as the golden script builds it.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_1011_5964_gb300 import synth
from parity import check_counts

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "headline1024_oracle.json")


@pytest.fixture(scope="module")
def case():
    import torch
    import paper_1011_5964_gb300 as pkg
    pkg.load_library()
    data = json.load(open(GOLDEN))
    m = data["meta"]
    n = m["n"]
    h = synth.disk_psf(7.0, side=31)
    u_true = synth.piecewise_constant_image(n, n, seed=m["seed"])
    v = synth.add_noise(O.blur(u_true, h, "ar"), synth.noise_direction(n, n, m["seed"]), m["noise"])
    return torch, torch.device("cuda:0"), pkg, data, h, v


def sampled_rel(u, ref_samples, idx, ref_norm):
    """Root-mean-square difference over the sample, relative to the RMS value ||u_ref|| / sqrt(N)."""
    d = u.ravel()[idx] - np.asarray(ref_samples)
    return float(np.sqrt(np.mean(d * d)) / (ref_norm / np.sqrt(u.size)))


def test_plain_fp64_1024_counts_and_image(case):
    torch, dev, pkg, data, h, v = case
    m, g = data["meta"], data["fp64"]
    with pkg.Plan(m["n"], m["n"], h, bc="ar", pc="dfast", mode="fp64") as plan:
        u, st = plan.deblur(torch.tensor(v, dtype=torch.float64, device=dev), m["alpha"], m["beta"],
                            max_outer=m["outer"], inner_tol=g["tol"], inner_maxit=5000)
        u = u.cpu().numpy()
    assert st["status"] == pkg.TVD_OK
    check_counts(st["inner_iters"], g["inner_iters"], g["step_spread"])
    bound = max(10.0 * g["image_spread"], 1e-12)
    assert abs(float(np.linalg.norm(u)) - g["u_norm"]) <= bound * g["u_norm"]
    err = sampled_rel(u, g["u_samples"], np.array(data["sample_idx"]), g["u_norm"])
    assert err < bound, (err, bound)


@pytest.mark.parametrize("transform", ["gemm", "fft"])
def test_mixed_1024_tight_within_1e5(case, transform):
    torch, dev, pkg, data, h, v = case
    m, g = data["meta"], data["tight"]
    with pkg.Plan(m["n"], m["n"], h, bc="ar", pc="dfast", mode="mixed", transform=transform) as plan:
        u, st = plan.deblur(torch.tensor(v, dtype=torch.float64, device=dev), m["alpha"], m["beta"],
                            max_outer=m["outer"], inner_tol=g["tol"], inner_maxit=20000)
        u = u.cpu().numpy()
    assert st["status"] == pkg.TVD_OK
    assert abs(float(np.linalg.norm(u)) - g["u_norm"]) <= 1e-5 * g["u_norm"]
    err = sampled_rel(u, g["u_samples"], np.array(data["sample_idx"]), g["u_norm"])
    assert err < 1e-5, err
