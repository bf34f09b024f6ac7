"""Benchmark: TV deblurring at 1024 x 1024 on one GB300 (or N independent replicas).

Workload (one "step" = one full deblur through the C ABI, every row of the PCG
hot path): 1024 x 1024 seeded piecewise-constant image, anti-reflective BCs,
radius-7 out-of-focus disk PSF zero-padded to 31 x 31, 1% Gaussian noise,
alpha 1e-3, beta 1e-2, 10 lagged-diffusivity FP steps from u^0 = v, each solved
by PCG with the D_M (hat-S / DST-I) preconditioner to ||r|| / ||r_0|| < 1e-6.

Arms:
  --impl ours (default): the chosen form (MIXED: float kernels, double CG
      scalars, double iterative refinement) is the headline ``value``
      (deblurs/s); the plain FP64 GPU form is measured beside it; PCG
      iterations/s are reported for both.
  --impl reference: the FP64 CPU oracle as it stands, timed on the host cores
      on a bounded sample of the same workload.

Timing: inputs resident in HBM, W untimed warm-up steps, then K steps, each
bracketed by CUDA events on the launch stream, with the L2 cache flushed (a
512 MiB write) between steps; barrier + synchronize on both sides; the max over
ranks. ``e2e`` repeats the step through the public API with pinned host
buffers (host->device copy of v, deblur, device->host copy of u inside the
timed region). Under torchrun (N > 1) every rank deblurs its own image
(replicas only, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "PCG iters/s and deblurs/s at 1024², chosen vs plain FP64 GPU, rel err ≤1e-5"
N_SIDE = 1024
SEED = 1234
ALPHA, BETA, OUTER, TOL, NOISE = 1e-3, 1e-2, 10, 1e-6, 0.01
WORKLOAD = "tv_deblur 1024x1024 AR disk-r7(31x31) 1% noise alpha=1e-3 beta=1e-2 10 FP steps tol=1e-6 D_M"

# Algorithmic bytes per launch of each kernel class, in words of the kernel's
# type per pixel: the arrays each kernel must read and write once.
WORDS_PER_PIXEL = {
    "blur_forward": 4,          # read z, p; write p = z + beta p, t = H p (the fused direction update)
    "blur_adjoint_L": 4,        # read t, p, w; write q = H^T t + alpha L p
    "precond_row_forward": 8,   # read r, q, p, x, D^-1/2; write r, x, t (the fused CG x / r update)
    "precond_column_solve": 3,  # read t, 1/spectrum; write t
    "precond_row_inverse": 4,   # read t, D^-1/2, r; write z
    "spectrum_row": 3,          # read w; write E w, G w
    "spectrum_column": 4,       # read E w, G w, Lambda_H^2; write 1/spectrum
    "cg_init": 3,               # read b, A x; write r
    "cg_p_update": 3,           # read z, p; write p
    "cg_xr_update": 6,          # read x, p, r, q; write x, r
    "cg_simple_precond": 3,
    "tv_coefficients": 2,
    "vector_misc": 2,
    "precond_gemm_vector": 8,   # the GEMM form's vector pass: read r, q, p, x, D^-1/2; write r, x, S
}

# DRAM bytes per launch (read + write) of kernels captured with ncu on this
# workload, each with the SHA-256 (first 16 hex digits) of the source file of
# its kernel at capture time: an entry is used only while that file is
# unchanged, so a stale figure is reported as null.
NCU_TRAFFIC = {
    # the four folded products of one CG iteration, averaged (3.16, 7.36, 3.16, 11.57 MB)
    "precond_gemm_tc.f32": {"source": "tc_gemm.cuh", "sha16": "0e21a148903b6e71", "bytes": 6312384},
    "blur_forward.f32": {"source": "blur.cu", "sha16": "613b0e8572161374", "bytes": 8476928},
    "blur_adjoint_L.f32": {"source": "blur.cu", "sha16": "613b0e8572161374", "bytes": 12658944},
}


def traffic_of(name):
    entry = NCU_TRAFFIC.get(name)
    if not entry:
        return None
    import hashlib
    path = os.path.join(ROOT, "paper_1011_5964_gb300", "csrc", entry["source"])
    try:
        digest = hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    return entry["bytes"] if digest == entry["sha16"] else None


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def make_inputs():
    import numpy as np
    from paper_1011_5964_gb300 import synth
    h = synth.disk_psf(7.0, side=31)
    u_true = synth.piecewise_constant_image(N_SIDE, N_SIDE, seed=SEED)
    z = synth.noise_direction(N_SIDE, N_SIDE, SEED)
    return np, synth, h, u_true, z


BATCH = 96
BATCH_WORKERS = 16


def batched_leg(pkg, torch, dev, synth):
    """Config of many independent images: BATCH items (sides from {128, ..., 512},
    Gaussian sigma ~ U[1,3], alpha log-uniform in [1e-4, 1e-2], 1% noise, AR,
    D_M, MIXED, 10 FP steps) through tv_deblur_batched, plans made beforehand.
    Timed by the host clock around the call (which returns when every item is
    done), after one untimed pass that captures each plan's CUDA graphs."""
    import math
    from paper_1011_5964_gb300.replicas import reduce_over_ranks, shard
    ws, rank, _ = dist_env()
    every = synth.batch_items(BATCH, seed=1000)
    # with several ranks each takes its share of the items (no exchange between them)
    items = [every[i] for i in shard([it["n"] ** 2 for it in every], rank, ws)]
    t0 = time.perf_counter()
    plans, vs = [], []
    for it in items:
        n = it["n"]
        h = synth.gaussian_psf(it["sigma"], half_width=int(math.ceil(3.0 * it["sigma"])))
        u_true = torch.tensor(synth.piecewise_constant_image(n, n, seed=it["seed"]), dtype=torch.float64, device=dev)
        with pkg.Plan(n, n, h, bc="ar", pc="dfast", mode="fp64") as p64:
            hu = p64.blur(u_true).cpu().numpy()
        v = synth.add_noise(hu, synth.noise_direction(n, n, it["seed"]), it["noise"])
        vs.append(torch.tensor(v, dtype=torch.float64, device=dev))
        plans.append(pkg.Plan(n, n, h, bc="ar", pc="dfast", mode="mixed"))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    alphas = [it["alpha"] for it in items]
    betas = [it["beta"] for it in items]
    outs = [torch.empty_like(v) for v in vs]
    res = {}

    def timed(key, workers):
        pkg.deblur_batched(plans, vs, alphas, betas, OUTER, TOL, 5000, outs, workers)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, stats = pkg.deblur_batched(plans, vs, alphas, betas, OUTER, TOL, 5000, outs, workers)
        torch.cuda.synchronize()
        res[key] = (reduce_over_ranks(time.perf_counter() - t0, "max", dev),
                    reduce_over_ranks(sum(sum(st["inner_iters"]) for st in stats), "sum", dev))

    timed("default_1", 1)
    timed("default", BATCH_WORKERS)
    # the library's autotuner picks each plan's preconditioner form (FFT, 64- or
    # 128-column product tiles, folded products) by timing them
    t0 = time.perf_counter()
    forms = {}
    for p in plans:
        rep = p.tune()
        c = rep["candidates"][rep["chosen"]]
        key = "fft" if c["transform"] == "fft" else f"gemm{c['tile_n']}" + ("_folded" if c["folded"] else "")
        forms[key] = forms.get(key, 0) + 1
    torch.cuda.synchronize()
    tune_s = time.perf_counter() - t0
    timed("tuned", BATCH_WORKERS)
    for p in plans:
        p.close()
    pixels = sum(it["n"] * it["n"] for it in every)
    return {"workload": f"{BATCH} independent tv_deblur, sides from {{128,192,256,384,512}} "
                        f"({pixels / 1e6:.2f} Mpixel in all), Gaussian sigma U[1,3], alpha log-U[1e-4,1e-2], "
                        f"beta 1e-2, 1% noise, AR, D_M, MIXED, 10 FP steps, tol 1e-6",
            "deblurs_per_s": BATCH / res["tuned"][0], "workers": BATCH_WORKERS,
            "pcg_iters_per_s": res["tuned"][1] / res["tuned"][0],
            "untuned_deblurs_per_s": BATCH / res["default"][0],
            "one_stream_deblurs_per_s": BATCH / res["default_1"][0], "plan_setup_s": setup_s,
            "tune_s": tune_s, "tuned_forms": forms,
            "timing": "host clock around the call, inputs resident"}


def size_leg(pkg, torch, dev, synth, n, steps=2, warmup=1, pc="dfast", transform=None, method="fp"):
    """The same workload at n x n (radius-7 disk on 31 x 31, AR, MIXED, 10 FP steps) with
    preconditioner pc (D_M, or M_D for 'fastd') and the plan's default transform form
    (or `transform`); with method 'reblur' each FP step solves eq. (fpp) by PBiCGstab (D_P / P_D).
    Device time per deblur by CUDA events, L2 flushed before each step."""
    h = synth.disk_psf(7.0, side=31)
    u_true = torch.tensor(synth.piecewise_constant_image(n, n, seed=SEED), dtype=torch.float64, device=dev)
    with pkg.Plan(n, n, h, bc="ar", pc="dfast", mode="fp64") as p64:
        hu = p64.blur(u_true).cpu().numpy()
    v = torch.tensor(synth.add_noise(hu, synth.noise_direction(n, n, SEED), NOISE), dtype=torch.float64, device=dev)
    u = torch.empty_like(v)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    ms, iters = 0.0, 0
    with pkg.Plan(n, n, h, bc="ar", pc=pc, mode="mixed", transform=transform, method=method) as plan:
        form = plan.transform
        for s_ in range(warmup + steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, st = plan.deblur(v, ALPHA, BETA, max_outer=OUTER, inner_tol=TOL, inner_maxit=5000, out=u)
            e1.record(stream)
            e1.synchronize()
            if s_ >= warmup:
                ms += e0.elapsed_time(e1)
                iters += st["total_inner_iters"]
    if method in ("reblur", "reblur_arl"):
        name = "P_D" if pc == "fastd" else "D_P"
        eq = "reblurring eq. (fpp), PBiCGstab" + (", AR BCs on L" if method == "reblur_arl" else "")
    else:
        name = "M_D" if pc == "fastd" else "D_M"
        eq = "eq. (fp), PCG"
    return {"workload": f"tv_deblur {n}x{n} AR disk-r7(31x31) 1% noise alpha=1e-3 beta=1e-2 10 FP steps tol=1e-6 "
                        f"{eq}, {name}, MIXED, {form} transforms", "deblurs_per_s": 1000.0 * steps / ms,
            "ms_per_step": ms / steps,
            "pcg_iters_per_s": iters / (ms / 1000.0), "inner_iters_per_deblur": iters / steps}


def signal_leg(pkg, torch, dev, synth):
    """The 1D experiment (Sec. 5.1): a 203-sample signal in the field of view of a wider support,
    out-of-focus PSF (21 taps), 1% noise, beta 0.1, FP stop 1e-3, PCG tol 1e-6, D_M / D_R, FP64;
    the RRE-versus-alpha sweep over 11 alphas (1e-6 .. 1e-1) for AR and R BCs, each sweep one batch
    of plans. The observation is blurred on the wider support with the library's own FP64 H (no BC
    reaches the field of view). Host clock around each sweep (plan set-up included)."""
    import numpy as np
    n, m, seed = 203, 11, 4
    h = synth.out_of_focus_psf_1d(m)
    uw, fov = synth.piecewise_constant_signal(n, seed)
    with pkg.Plan(1, uw.size, h, bc="r", pc="dfast", mode="fp64") as pw:
        hv = pw.blur(torch.tensor(uw[None, :], device=dev)).cpu().numpy()[:, fov]
    v = torch.tensor(synth.add_noise(hv, synth.noise_direction(1, n, seed), 0.01), device=dev)
    ut = uw[fov][None, :]
    alphas = synth.alpha_grid()
    out = {"workload": "1D signal n=203 (field of view of 253 samples), out-of-focus PSF 21 taps, 1% noise, "
                       "beta 0.1, FP stop 1e-3, PCG tol 1e-6, D_M (AR) / D_R (R), FP64, alpha sweep 1e-6..1e-1",
           "alphas": alphas}
    for bc in ("ar", "r"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        us, stats = pkg.alpha_sweep(v, h, alphas, 0.1, bc=bc, pc="dfast", mode="fp64", outer_tol=1e-3,
                                    inner_tol=1e-6)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        rre = [float(np.linalg.norm(u.cpu().numpy() - ut) / np.linalg.norm(ut)) for u in us]
        k = int(np.argmin(rre))
        out[bc] = {"sweep_s": dt, "rre": rre, "best_alpha": alphas[k], "best_rre": rre[k],
                   "fp_steps": [st["outer_iters"] for st in stats],
                   "inner_per_step": [float(np.mean(st["inner_iters"])) for st in stats]}
    return out


def adjoint_leg(pkg, torch, dev, synth):
    """Adjoint of the converged fixed point at 512 x 512: the observation blurred
    with a Gaussian sigma = 2.5, the plan's PSF sigma = 2.0 on a 17 x 17 support
    (half-width ceil(3 x 2.5)), alpha 1e-3, beta 1e-2, AR, D_M, MIXED. u* from
    tv_deblur run to ||u^k - u^{k-1}|| / ||u^k|| < 1e-4, then Newton steps on
    g(u) = 0 (tv_deblur_newton) to a relative change below 1e-12; then one
    adjoint solve (tol 1e-10) for l = ||u* - u_true||^2 and dl/dsigma by the
    chain rule through the PSF taps. Device time by CUDA events."""
    import numpy as np
    n, seed, m = 512, 77, 8
    u_true = synth.piecewise_constant_image(n, n, seed=seed)
    h_true = synth.gaussian_psf(2.5, half_width=m)
    h = synth.gaussian_psf(2.0, half_width=m)
    ut = torch.tensor(u_true, dtype=torch.float64, device=dev)
    with pkg.Plan(n, n, h_true, bc="ar", pc="dfast", mode="fp64") as p64:
        hu = p64.blur(ut).cpu().numpy()
    v = torch.tensor(synth.add_noise(hu, synth.noise_direction(n, n, seed), 0.01), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    with pkg.Plan(n, n, h, bc="ar", pc="dfast", mode="mixed") as plan:
        e0, e1, e2, e3 = (torch.cuda.Event(enable_timing=True) for _ in range(4))
        e0.record(stream)
        u, st = plan.deblur(v, ALPHA, BETA, max_outer=400, outer_tol=1e-4, inner_tol=1e-8, inner_maxit=5000)
        e1.record(stream)
        nst = plan.newton(u, v, ALPHA, BETA, tol=1e-12, cg_tol=1e-12, cg_maxit=20000)
        e2.record(stream)
        lam, da, db, dh, ast = plan.adjoint(u, v, ALPHA, BETA, 2.0 * (u - ut), tol=1e-10, maxit=5000)
        e3.record(stream)
        e3.synchronize()
    eps = 1e-6
    dh_dsigma = (synth.gaussian_psf(2.0 + eps, half_width=m) - synth.gaussian_psf(2.0 - eps, half_width=m)) / (2 * eps)
    return {"workload": "adjoint of the converged fixed point, 512x512 AR, plan PSF Gaussian sigma 2.0 on 17x17, "
                        "data blurred with sigma 2.5, alpha 1e-3, beta 1e-2, D_M, MIXED",
            "fixed_point_ms": e0.elapsed_time(e1), "fp_steps": st["outer_iters"],
            "fp_inner_iters": st["total_inner_iters"], "fp_last_rel_change": st["last_rel_change"],
            "newton_ms": e1.elapsed_time(e2), "newton_steps": nst["steps"], "newton_cg_iters": nst["total_cg_iters"],
            "newton_halvings": nst["halvings"], "last_rel_change": nst["last_rel_change"],
            "g_norm_initial": nst["g_norm_initial"], "g_norm": nst["g_norm"], "newton_status": nst["status"],
            "adjoint_ms": e2.elapsed_time(e3), "adjoint_iters": ast["iters"], "adjoint_relres": ast["relres"],
            "dl_dalpha": da, "dl_dbeta": db, "dl_dsigma": float(np.sum(dh * dh_dsigma))}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# TF32 / bf16 dense tensor rate of GB300 (nominal 1.1 / 2.25 PFLOP/s): the TF32
# peak is the measured bf16 figure times this ratio.
TF32_OVER_BF16 = 1.1 / 2.25


def tf32_peak():
    """TF32 tensor peak (TFLOP/s) for a kernel timed inside a long step: the measured sustained
    bf16 cuBLAS rate x the nominal TF32 / bf16 ratio."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["bf16_tflops_sustained"]) * TF32_OVER_BF16, "measured (bf16 sustained x 1.1/2.25)"
    except Exception:
        return 1700.0 * TF32_OVER_BF16, "fallback (bf16 sustained 1.7 PF x 1.1/2.25)"


def bf16_peak():
    """bf16 tensor peak (TFLOP/s) for a kernel timed inside a long step: the measured sustained cuBLAS rate."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(path))["bf16_tflops_sustained"]), "measured (bf16 sustained)"
    except Exception:
        return 1700.0, "fallback (bf16 sustained 1.7 PF)"


def setup_ms_of(plan, u_lag, stream, reps=20):
    """Average device time (ms) of one FP step's set-up (tau_precond_setup: diffusivity, D and
    the preconditioner spectrum) at u_lag, or None if it cannot be taken."""
    import torch
    try:
        for _ in range(3):
            plan.precond_setup(u_lag, ALPHA, BETA)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            plan.precond_setup(u_lag, ALPHA, BETA)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps
    except Exception as exc:   # a failed side measurement leaves the headline intact
        print(f"set-up timing skipped: {exc}", file=sys.stderr)
        return None


def steady_rate(iters, ms, deblurs, setup_ms):
    """Inner PCG iterations per second with the per-FP-step set-up taken out of the deblur time."""
    if setup_ms is None:
        return None
    loop_ms = ms - deblurs * OUTER * setup_ms
    return iters / (loop_ms / 1000.0) if loop_ms > 0 else None


def path_roofline(pcg_iters_per_s, prec_bytes=4):
    """The whole PCG iteration against HBM: the floor of the standard recurrence, 15 words per pixel
    (matvec 3, x / r update 6, preconditioner 3, p update 3), times the iteration rate."""
    bytes_per_iter = 15 * prec_bytes * N_SIDE * N_SIDE
    achieved = bytes_per_iter * pcg_iters_per_s / 1e9
    peak, src = peaks()
    return {"bound": "hbm", "words_per_pixel": 15, "bytes_per_iteration": bytes_per_iter, "achieved": achieved,
            "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_source": src}


def rooflines_of(prof, total_ms, storage, folded=False):
    """Roofline entry of every kernel class of the step with a known algorithmic work per launch."""
    out = {}
    for name, (kms, kl) in prof.items():
        base = name.rsplit(".", 1)[0]
        if kl and (base in WORDS_PER_PIXEL or base == "precond_gemm_tc"):
            out[name] = roofline_of(name, kms, kl, total_ms, storage, folded)
    return out


def roofline_of(name, kms, klaunch, total_ms, storage=None, folded=False):
    """Roofline entry of one kernel class from its summed device time and launch count."""
    base, prec = name.rsplit(".", 1)
    avg_s = kms / 1000.0 / max(klaunch, 1)
    share = kms / max(total_ms, 1e-12)
    if base == "precond_gemm_tc":
        # one n x n x n product of the transform form (the library's tcgen05 kernel): 2 n^3 flops
        # (bf16 or tf32 operands, float accumulation); n^3 for the folded products (two half-length
        # transforms of n lines each)
        flops = (1.0 if folded else 2.0) * N_SIDE ** 3
        peak, src = bf16_peak() if storage == "bf16" else tf32_peak()
        achieved = flops / avg_s / 1e12
        kind = "folded transform product" if folded else "transform product"
        return {"bound": "tensor", "kernel": f"{name} ({storage} {kind}, tcgen05)", "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic_of(name), "peak_source": src,
                "flops_per_launch": flops, "avg_launch_us": avg_s * 1e6, "launches": klaunch, "share": share}
    word = 4 if prec == "f32" else 8
    bytes_per_launch = WORDS_PER_PIXEL.get(base, 2) * word * N_SIDE * N_SIDE
    achieved = bytes_per_launch / avg_s / 1e9
    peak, peak_src = peaks()
    return {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic_of(name), "peak_source": peak_src,
            "bytes_per_launch": bytes_per_launch, "avg_launch_us": avg_s * 1e6, "launches": klaunch, "share": share}


def cpu_sample(h, v, sample_iters: int):
    """Oracle as it stands: FP-step set-up plus `sample_iters` PCG iterations of the first
    FP step at the full workload. Returns (setup_s, seconds per iteration)."""
    import numpy as np
    import oracle as O
    b = O.blur_adjoint(v, h, "ar")
    t0 = time.perf_counter()
    P = O.precond_setup(v, h, "ar", ALPHA, BETA, "dfast")
    t1 = time.perf_counter()
    w = P["w"]
    O.pcg(lambda y: O.normal_apply(y, h, "ar", w, ALPHA), lambda r: O.precond_apply(r, P), b, v, 1e-300,
          sample_iters)
    t2 = time.perf_counter()
    # pcg also applies A once to form r_0: charge it as one iteration
    return (t1 - t0) + (t2 - t1) / (sample_iters + 1), (t2 - t1) / (sample_iters + 1)


def cpu_full_deblur(n):
    """One complete oracle deblur of the workload at n x n (disk r7, AR, D_M, 10 FP steps, tol 1e-6),
    wall-clock seconds and its inner iterations."""
    import oracle as O
    from paper_1011_5964_gb300 import synth
    h = synth.disk_psf(7.0, side=31)
    u_true = synth.piecewise_constant_image(n, n, seed=SEED)
    v = synth.add_noise(O.blur(u_true, h, "ar"), synth.noise_direction(n, n, SEED), NOISE)
    t0 = time.perf_counter()
    _, st = O.tv_deblur(v, h, "ar", ALPHA, BETA, outer=OUTER, tol=TOL, maxit=5000, kind="dfast")
    return time.perf_counter() - t0, int(sum(st["inner_iters"]))


def oracle_iters_per_deblur():
    path = os.path.join(ROOT, "tests", "golden", "bench1024_oracle.json")
    try:
        d = json.load(open(path))
        return int(sum(d["inner_iters"])), "stored FP64 oracle run (tests/golden/bench1024_oracle.json)"
    except Exception:
        return None, "no stored oracle run"


def run_reference(args):
    """The FP64 CPU oracle, timed on the host cores on a bounded sample of the workload."""
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        if rank != 0:
            dist.barrier()
            dist.destroy_process_group()
            return
    import numpy as np
    import oracle as O
    _, synth, h, u_true, z = make_inputs()
    v = synth.add_noise(O.blur(u_true, h, "ar"), z, NOISE)
    iters_per_deblur, src = oracle_iters_per_deblur()
    if iters_per_deblur is None:
        iters_per_deblur, src = 10 * 60, "assumed 60 inner iterations per FP step (no stored oracle run)"
    sample_iters = 2
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        setup_s, it_s = cpu_sample(h, v, sample_iters)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append((setup_s, it_s, dt))
    setup_s = statistics.median(t[0] for t in times)
    it_s = statistics.median(t[1] for t in times)
    deblur_s = OUTER * setup_s + iters_per_deblur * it_s
    value = 1.0 / deblur_s
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "deblurs/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * statistics.median(t[2] for t in times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD},
            "pcg_iters_per_s": 1.0 / it_s,
            "cpu_baseline": {"value": value, "unit": "deblurs/s", "cores": cores, "kind": "oracle",
                             "sample": f"per step: FP-step set-up + {sample_iters} PCG iterations of the first FP "
                                       f"step at 1024x1024; deblur time = 10 x set-up + {iters_per_deblur} "
                                       f"iterations ({src})"},
            "e2e": {"value": value, "unit": "deblurs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


def run_ours(args):
    import numpy as np
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    import paper_1011_5964_gb300 as pkg
    pkg.load_library()
    _, synth, h, u_true, z = make_inputs()
    stream = torch.cuda.current_stream()

    mixed = pkg.Plan(N_SIDE, N_SIDE, h, bc="ar", pc="dfast", mode="mixed")
    plain = pkg.Plan(N_SIDE, N_SIDE, h, bc="ar", pc="dfast", mode="fp64")
    # observation v = H u_true + eta, blurred by this library's FP64 operator
    hu = plain.blur(torch.tensor(u_true, dtype=torch.float64, device=dev)).cpu().numpy()
    v_host = synth.add_noise(hu, z, NOISE)
    v = torch.tensor(v_host, dtype=torch.float64, device=dev)
    u = torch.empty_like(v)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    def timed(plan, steps, warmup, out):
        stats = []
        for _ in range(warmup):
            plan.deblur(v, ALPHA, BETA, max_outer=OUTER, inner_tol=TOL, inner_maxit=5000, out=out)
        barrier()
        ms = 0.0
        launches0 = pkg.kernel_launches()
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, st = plan.deblur(v, ALPHA, BETA, max_outer=OUTER, inner_tol=TOL, inner_maxit=5000, out=out)
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
            stats.append(st)
        launches = pkg.kernel_launches() - launches0
        barrier()
        return ms, stats, launches

    from paper_1011_5964_gb300.replicas import reduce_over_ranks

    def max_over_ranks(x):
        return reduce_over_ranks(x, "max", device=dev)

    sampler = ClockSampler(local)
    sampler.start()
    ms_mixed, st_mixed, launches = timed(mixed, args.steps, args.warmup, u)
    clocks = sampler.stop()
    if args.only_chosen:
        # profiler runs: the chosen form's warm-up and timed steps only
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": ws * 1000.0 * args.steps / max_over_ranks(ms_mixed),
                              "unit": "deblurs/s", "only_chosen": True, "gpu_launches": launches}))
        mixed.close()
        plain.close()
        return
    ms_mixed = max_over_ranks(ms_mixed)
    u_mixed = u.clone()
    iters_mixed = sum(s["total_inner_iters"] for s in st_mixed)
    ms_per_step = ms_mixed / args.steps
    value = ws * 1000.0 / ms_per_step

    # plain FP64 GPU form (fewer steps: it is much slower)
    u64 = torch.empty_like(v)
    p_steps = max(1, min(2, args.steps))
    ms_plain, st_plain, _ = timed(plain, p_steps, 1, u64)
    ms_plain = max_over_ranks(ms_plain)
    iters_plain = sum(s["total_inner_iters"] for s in st_plain)
    rel_err = float(torch.linalg.norm(u_mixed - u64) / torch.linalg.norm(u64))
    # the per-FP-step set-up alone, so the inner loop's steady rate can be reported without it
    setup_mixed = setup_ms_of(mixed, u_mixed.float(), stream)
    setup_plain = setup_ms_of(plain, u64, stream)
    steady_mixed = steady_rate(iters_mixed, ms_mixed, args.steps, setup_mixed)
    steady_plain = steady_rate(iters_plain, ms_plain, p_steps, setup_plain)

    # per-kernel device time of one more chosen-form step (CUDA events around every launch)
    pkg.profile_enable(True)
    flush.zero_()
    mixed.deblur(v, ALPHA, BETA, max_outer=OUTER, inner_tol=TOL, inner_maxit=5000, out=u)
    torch.cuda.synchronize()
    prof = pkg.profile_read()
    pkg.profile_enable(False)
    if rank == 0:
        table = {k: {"ms": round(v_[0], 4), "launches": v_[1]} for k, v_ in sorted(prof.items(), key=lambda kv: -kv[1][0])
                 if v_[1]}
        print("per-kernel-class device time of one chosen-form step: " + json.dumps(table), file=sys.stderr)
    total_ms = sum(v_[0] for v_ in prof.values())
    # every kernel is the library's own: the dominant class by device time, and all classes
    top = max(prof.items(), key=lambda kv: kv[1][0])
    roofline = roofline_of(top[0], top[1][0], top[1][1], total_ms, mixed.gemm_storage, mixed.gemm_folded)
    rooflines = rooflines_of(prof, total_ms, mixed.gemm_storage, mixed.gemm_folded)

    # end to end through the public API with pinned host buffers
    v_pin = torch.tensor(v_host, dtype=torch.float64).pin_memory()
    u_pin = torch.empty_like(v_pin).pin_memory()
    v_dev = torch.empty_like(v)
    barrier()
    e2e_ms = 0.0
    for s in range(args.warmup + args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        v_dev.copy_(v_pin, non_blocking=True)
        mixed.deblur(v_dev, ALPHA, BETA, max_outer=OUTER, inner_tol=TOL, inner_maxit=5000, out=u)
        u_pin.copy_(u, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        if s >= args.warmup:
            e2e_ms += e0.elapsed_time(e1)
    barrier()
    e2e_ms = max_over_ranks(e2e_ms)
    nbytes = N_SIDE * N_SIDE * 8

    line = {"metric": METRIC, "value": value, "unit": "deblurs/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "form": "mixed (float kernels, double scalars + refinement)",
                       "l2": "flushed between steps (512 MiB write)", "parallelism": f"replicas x{ws}"},
            "pcg_iters_per_s": ws * iters_mixed / (ms_mixed / 1000.0),
            "inner_iters_per_deblur": iters_mixed / args.steps,
            "setup_ms_per_fp_step": setup_mixed,
            "pcg_iters_per_s_steady": None if steady_mixed is None else ws * steady_mixed,
            "plain_fp64": {"deblurs_per_s": ws * 1000.0 * p_steps / ms_plain,
                           "pcg_iters_per_s": ws * iters_plain / (ms_plain / 1000.0),
                           "setup_ms_per_fp_step": setup_plain,
                           "pcg_iters_per_s_steady": None if steady_plain is None else ws * steady_plain,
                           "inner_iters_per_deblur": iters_plain / p_steps, "ms_per_step": ms_plain / p_steps},
            "rel_err_vs_plain_fp64": rel_err,
            "gpu_launches": launches,
            "roofline": roofline,
            "rooflines": rooflines,
            "path_roofline": path_roofline(ws * iters_mixed / (ms_mixed / 1000.0)),
            "transform_form": mixed.transform,
            "gemm_operands": mixed.gemm_storage, "gemm_folded": mixed.gemm_folded,
            "clocks": clocks,
            "e2e": {"value": ws * 1000.0 * args.steps / e2e_ms, "unit": "deblurs/s",
                    "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}}

    if not args.no_batch:
        line["batched"] = batched_leg(pkg, torch, dev, synth)
        line["adjoint"] = adjoint_leg(pkg, torch, dev, synth)
        line["size_2048"] = size_leg(pkg, torch, dev, synth, 2048)
        line["m_d_1024"] = size_leg(pkg, torch, dev, synth, 1024, steps=3, pc="fastd")
        line["fft_form_1024"] = size_leg(pkg, torch, dev, synth, 1024, steps=3, transform="fft")
        line["reblur_1024"] = size_leg(pkg, torch, dev, synth, 1024, steps=3, method="reblur")
        line["reblur_arl_1024"] = size_leg(pkg, torch, dev, synth, 1024, steps=3, method="reblur_arl")
        line["signal_1d"] = signal_leg(pkg, torch, dev, synth)

    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        iters_per_deblur, src = oracle_iters_per_deblur()
        if iters_per_deblur is None:
            iters_per_deblur, src = int(round(iters_plain / p_steps)), "iteration count of the FP64 GPU form"
        setup_s, it_s = cpu_sample(h, v_host, 8)
        deblur_s = OUTER * setup_s + iters_per_deblur * it_s
        full_s, full_iters = cpu_full_deblur(256)
        line["cpu_baseline"] = {"value": 1.0 / deblur_s, "unit": "deblurs/s", "cores": os.cpu_count(),
                                "kind": "oracle", "pcg_iters_per_s": 1.0 / it_s,
                                "sample": f"extrapolated: FP-step set-up + 8 PCG iterations of the first FP step at "
                                          f"1024x1024 (numpy/scipy default threading); deblur time = 10 x set-up + "
                                          f"{iters_per_deblur} iterations ({src})",
                                "full_256": {"measured_s": full_s, "deblurs_per_s": 1.0 / full_s,
                                             "inner_iters": full_iters,
                                             "sample": "measured: one complete oracle tv_deblur of the same "
                                                       "workload at 256x256 (wall clock)"}}
    if rank == 0:
        print(json.dumps(line))
    mixed.close()
    plain.close()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batch-of-independent-images and adjoint legs")
    ap.add_argument("--only-chosen", action="store_true",
                    help="time the chosen form only (no plain FP64, e2e, per-kernel or CPU legs); for profiler runs")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
