"""GPU tests of tv_deblur_batched: independent problems solved concurrently.

Each item must give exactly the result of its own tv_deblur call (same plan
configuration, deterministic kernels), whatever the worker count and order;
items sharing a plan run one after another; one small FP64 item is also held
to the oracle.
"""
import numpy as np
import pytest

import oracle as O
from paper_1011_5964_gb300 import synth

pytestmark = pytest.mark.gpu

ITEMS = [  # (n_rows, n_cols, sigma, alpha, mode)
    (48, 40, 1.2, 1e-3, "fp64"),
    (64, 64, 2.0, 3e-4, "mixed"),
    (33, 57, 1.5, 1e-2, "fp64"),
    (96, 80, 2.5, 1e-3, "mixed"),
    (40, 40, 1.0, 5e-3, "fp64"),
]


def problem(i, nr, nc, sigma):
    h = synth.gaussian_psf(sigma, half_width=int(np.ceil(3 * sigma)))
    u = synth.piecewise_constant_image(nr, nc, seed=1000 + i)
    v = synth.add_noise(O.blur(u, h, "ar"), synth.noise_direction(nr, nc, 1000 + i), 0.01)
    return h, v


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    import paper_1011_5964_gb300 as pkg
    pkg.load_library()
    return torch, torch.device("cuda:0")


@pytest.fixture(scope="module")
def setup(torch_dev):
    torch, dev = torch_dev
    import paper_1011_5964_gb300 as pkg
    probs = [problem(i, *it[:3]) for i, it in enumerate(ITEMS)]
    plans = [pkg.Plan(it[0], it[1], h, bc="ar", pc="dfast", mode=it[4]) for it, (h, v) in zip(ITEMS, probs)]
    vs = [torch.tensor(v, dtype=torch.float64, device=dev) for h, v in probs]
    yield torch, pkg, probs, plans, vs
    for p in plans:
        p.close()


def individual(setup):
    torch, pkg, probs, plans, vs = setup
    out = []
    for it, p, v in zip(ITEMS, plans, vs):
        u, st = p.deblur(v, it[3], 1e-2, max_outer=4, inner_tol=1e-6, inner_maxit=2000)
        out.append((u.clone(), st["inner_iters"]))
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("workers", [1, 3, 8])
def test_batched_equals_individual_calls(setup, workers):
    torch, pkg, probs, plans, vs = setup
    ref = individual(setup)
    us, stats = pkg.deblur_batched(plans, vs, [it[3] for it in ITEMS], [1e-2] * len(ITEMS), max_outer=4,
                                   inner_tol=1e-6, inner_maxit=2000, workers=workers)
    torch.cuda.synchronize()
    for i, ((u_ref, it_ref), u, st) in enumerate(zip(ref, us, stats)):
        assert st["status"] == 0, (i, st)
        assert st["inner_iters"] == it_ref, (i, st["inner_iters"], it_ref)
        assert torch.equal(u, u_ref), (i, float((u - u_ref).abs().max()))


def test_items_sharing_a_plan_run_in_turn(setup):
    torch, pkg, probs, plans, vs = setup
    p, v = plans[0], vs[0]
    alphas = [1e-3, 1e-2, 3e-3]
    ref = []
    for a in alphas:
        u, st = p.deblur(v, a, 1e-2, max_outer=3, inner_tol=1e-6, inner_maxit=2000)
        ref.append((u.clone(), st["inner_iters"]))
    us, stats = pkg.deblur_batched([p, p, p], [v, v, v], alphas, [1e-2] * 3, max_outer=3, inner_tol=1e-6,
                                   inner_maxit=2000, workers=4)
    torch.cuda.synchronize()
    for (u_ref, it_ref), u, st in zip(ref, us, stats):
        assert st["inner_iters"] == it_ref
        assert torch.equal(u, u_ref)


def test_batched_fp64_item_matches_the_oracle(setup):
    torch, pkg, probs, plans, vs = setup
    i = 4
    h, v = probs[i]
    u_ref, st_ref = O.tv_deblur(v, h, "ar", ITEMS[i][3], 1e-2, outer=4, tol=1e-6, kind=O.PC_DFAST)
    us, stats = pkg.deblur_batched([plans[i]], [vs[i]], [ITEMS[i][3]], [1e-2], max_outer=4, inner_tol=1e-6,
                                   inner_maxit=2000, workers=2)
    u = us[0].cpu().numpy()
    assert max(abs(a - b) for a, b in zip(stats[0]["inner_iters"], st_ref["inner_iters"])) <= 1
    assert np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref) < 1e-9


def test_batched_rejects_a_bad_item(setup):
    torch, pkg, probs, plans, vs = setup
    with pytest.raises(pkg.TvdError):
        pkg.deblur_batched(plans[:2], vs[:2], [1e-3, -1.0], [1e-2, 1e-2])
