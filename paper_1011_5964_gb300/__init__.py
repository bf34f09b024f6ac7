"""GB300 TV-deblurring PCG library: thin Python binding of libtvd.so.

The library (``libtvd.so``, built in-tree from ``csrc/`` by ``_build.build()``)
implements the PCG inner step of the lagged-diffusivity fixed-point method for
TV deblurring with reflective / anti-reflective boundary conditions (Bai,
Donatelli, Serra-Capizzano). Its C ABI is declared in ``include/tvd.h``.

This module only marshals arguments: torch CUDA tensors become device
pointers, torch's current stream is passed as the CUDA stream, and status codes
become exceptions. Every step of the computation runs in the CUDA kernels;
there is no CPU fallback, and loading fails loudly if the library is missing.

The function names mirror the C ABI: ``ar_blur_apply``, ``tv_operator_apply``,
``tau_precond_setup``, ``tau_precond_solve``, ``pcg_solve``, ``tv_deblur``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtvd.so")

BC = {"r": 0, "reflective": 0, "ar": 1, "antireflective": 1}
PC = {"none": 0, "diag": 1, "fast": 2, "dfast": 3, "fastd": 4}
MODE = {"fp64": 0, "mixed": 1}

TVD_OK, TVD_EINVAL, TVD_EPSF_ASYM, TVD_EPSF_SIZE, TVD_ENOMEM, TVD_ECUDA, TVD_ENOCONV, TVD_EBREAKDOWN, TVD_ETIMEOUT = range(9)
STATUS_NAMES = ["TVD_OK", "TVD_EINVAL", "TVD_EPSF_ASYM", "TVD_EPSF_SIZE", "TVD_ENOMEM", "TVD_ECUDA",
                "TVD_ENOCONV", "TVD_EBREAKDOWN", "TVD_ETIMEOUT"]

# Function names of the C ABI, in include/tvd.h order.
TRANSFORM = {"fft": 0, "gemm": 1}
METHOD = {"fp": 0, "reblur": 1, "reblur_arl": 2}
ABI_FUNCTIONS = ["tvd_plan_create", "tvd_plan_destroy", "ar_blur_apply", "tv_operator_apply",
                 "tau_precond_setup", "tau_precond_solve", "pcg_solve", "tv_deblur",
                 "tvd_plan_set_method", "tvd_plan_method", "pbicgstab_solve",
                 "tv_deblur_batched", "tv_hessian_apply", "tv_deblur_adjoint", "tv_deblur_newton", "tvd_plan_psf_size",
                 "tvd_normal_apply_noalloc", "tvd_plan_set_transform", "tvd_plan_transform", "tvd_plan_gemm_storage", "tvd_plan_gemm_folded",
                 "tvd_plan_gemm_tile", "tvd_plan_tune",
                 "tvd_last_error", "tvd_version", "tvd_kernel_launches",
                 "tvd_profile_enable", "tvd_profile_classes", "tvd_profile_name", "tvd_profile_read"]


class TvdError(RuntimeError):
    """A libtvd call returned an error status."""

    def __init__(self, status: int, message: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {message}")


class _Stats(ctypes.Structure):
    _fields_ = [("outer_iters", ctypes.c_int), ("inner_iters", ctypes.POINTER(ctypes.c_int)),
                ("cap", ctypes.c_int), ("total_inner_iters", ctypes.c_int),
                ("refinement_sweeps", ctypes.c_int), ("last_relres", ctypes.c_double),
                ("last_rel_change", ctypes.c_double), ("last_status", ctypes.c_int),
                ("g_norm", ctypes.POINTER(ctypes.c_double)), ("functional", ctypes.POINTER(ctypes.c_double)),
                ("final_g_norm", ctypes.c_double), ("final_functional", ctypes.c_double)]


TUNE_MAX = 4      # TVD_TUNE_MAX
TUNE_SOLVES = 16  # TVD_TUNE_SOLVES


class _TuneReport(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int), ("chosen", ctypes.c_int), ("transform", ctypes.c_int * TUNE_MAX),
                ("tile_n", ctypes.c_int * TUNE_MAX), ("folded", ctypes.c_int * TUNE_MAX),
                ("us_per_solve", ctypes.c_double * TUNE_MAX)]


class _NewtonStats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("total_cg_iters", ctypes.c_int), ("halvings", ctypes.c_int),
                ("last_t", ctypes.c_double), ("last_rel_change", ctypes.c_double),
                ("last_cg_relres", ctypes.c_double), ("g_norm_initial", ctypes.c_double),
                ("g_norm", ctypes.c_double)]


class _BatchItem(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("v", ctypes.c_void_p), ("u_out", ctypes.c_void_p),
                ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("inner_iters", ctypes.POINTER(ctypes.c_int)), ("status", ctypes.c_int),
                ("outer_tol", ctypes.c_double), ("outer_iters", ctypes.c_int)]


_lib = None


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Load libtvd.so (once). Raises if it has not been built."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libtvd.so not found at {p}; build it with paper_1011_5964_gb300._build.build()")
    lib = ctypes.CDLL(p)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.tvd_plan_create.argtypes = [ctypes.POINTER(vp), i, i, ctypes.POINTER(d), i, i, i, i, i, vp]
    lib.tvd_plan_destroy.argtypes = [vp]
    lib.ar_blur_apply.argtypes = [vp, i, vp, vp, vp]
    lib.tv_operator_apply.argtypes = [vp, vp, d, vp, vp, vp]
    lib.tau_precond_setup.argtypes = [vp, vp, d, d, vp]
    lib.tau_precond_solve.argtypes = [vp, vp, vp, vp]
    lib.pcg_solve.argtypes = [vp, vp, d, d, vp, vp, d, i, ctypes.POINTER(i), ctypes.POINTER(d), vp]
    lib.tv_deblur.argtypes = [vp, vp, d, d, i, d, d, i, vp, ctypes.POINTER(_Stats), vp]
    lib.tvd_normal_apply_noalloc.argtypes = [i, i, ctypes.POINTER(d), i, i, i, vp, d, d, vp, vp, vp]
    lib.tv_deblur_batched.argtypes = [ctypes.POINTER(_BatchItem), i, i, d, i, i, vp]
    lib.tv_hessian_apply.argtypes = [vp, vp, d, vp, vp, vp]
    lib.tv_deblur_adjoint.argtypes = [vp, vp, vp, d, d, vp, vp, d, i, ctypes.POINTER(d), ctypes.POINTER(d),
                                      ctypes.POINTER(d), ctypes.POINTER(i), ctypes.POINTER(d), vp]
    lib.tv_deblur_newton.argtypes = [vp, vp, d, d, vp, d, i, d, i, ctypes.POINTER(_NewtonStats), vp]
    lib.tvd_plan_psf_size.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i)]
    lib.tvd_plan_set_transform.argtypes = [vp, i, vp]
    lib.tvd_plan_set_method.argtypes = [vp, i, vp]
    lib.tvd_plan_method.argtypes = [vp]
    lib.pbicgstab_solve.argtypes = [vp, vp, d, d, vp, vp, d, i, ctypes.POINTER(i), ctypes.POINTER(d), vp]
    lib.tvd_plan_transform.argtypes = [vp]
    lib.tvd_plan_gemm_storage.argtypes = [vp]
    lib.tvd_plan_gemm_folded.argtypes = [vp]
    lib.tvd_plan_gemm_tile.argtypes = [vp]
    lib.tvd_plan_tune.argtypes = [vp, i, ctypes.POINTER(_TuneReport), vp]
    lib.tvd_last_error.restype = ctypes.c_char_p
    lib.tvd_version.restype = ctypes.c_char_p
    lib.tvd_kernel_launches.restype = ctypes.c_ulonglong
    lib.tvd_profile_enable.argtypes = [i]
    lib.tvd_profile_name.argtypes = [i]
    lib.tvd_profile_name.restype = ctypes.c_char_p
    lib.tvd_profile_read.argtypes = [i, ctypes.POINTER(d), ctypes.POINTER(ctypes.c_longlong)]
    for name in ABI_FUNCTIONS:
        if name not in ("tvd_last_error", "tvd_version", "tvd_kernel_launches", "tvd_profile_name"):
            getattr(lib, name).restype = ctypes.c_int
    if path is None:
        _lib = lib
    return lib


def _check(status: int, allow=()) -> int:
    if status != TVD_OK and status not in allow:
        msg = load_library().tvd_last_error().decode(errors="replace")
        raise TvdError(status, msg)
    return status


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t, dtype, n):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"expected dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"expected a contiguous tensor with {n} elements")
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """A libtvd plan: image size, PSF, boundary conditions, preconditioner and arithmetic.

    ``psf`` is a (2 m_r + 1, 2 m_c + 1) float64 array, centred and quadrantally
    symmetric. ``bc``: 'ar' (anti-reflective) or 'r' (reflective). ``pc``:
    'none', 'diag', 'fast' (R / M), 'dfast' (D_R / D_M) or 'fastd' (R_D / M_D).
    ``mode``: 'fp64' or 'mixed'. ``method``: 'fp' (eq. (fp), PCG), 'reblur' or 'reblur_arl'
    (eq. (fpp), PBiCGstab; the fast kinds are then P, D_P, P_D). Operator calls
    take float64 tensors in fp64 mode and float32 in mixed mode; solver calls
    always take float64 tensors.
    """

    def __init__(self, n_rows: int, n_cols: int, psf, bc: str = "ar", pc: str = "dfast", mode: str = "fp64",
                 transform: str | None = None, method: str = "fp"):
        import torch
        self.lib = load_library()
        self.shape = (int(n_rows), int(n_cols))
        self.n = self.shape[0] * self.shape[1]
        self.mode = mode
        self.op_dtype = torch.float64 if mode == "fp64" else torch.float32
        h = np.ascontiguousarray(np.asarray(psf, dtype=np.float64))
        handle = ctypes.c_void_p()
        _check(self.lib.tvd_plan_create(ctypes.byref(handle), self.shape[0], self.shape[1],
                                        h.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), h.shape[0], h.shape[1],
                                        BC[bc], PC[pc], MODE[mode], _stream()))
        self.handle = handle
        if method != "fp":
            self.set_method(method)
        if transform is not None:
            self.set_transform(transform)

    def set_method(self, method: str):
        """'fp' (eq. (fp), PCG), 'reblur' (eq. (fpp), PBiCGstab) or 'reblur_arl' (eq. (fpp) with
        anti-reflective BCs on L too, PBiCGstab); both reblurring methods need anti-reflective BCs."""
        _check(self.lib.tvd_plan_set_method(self.handle, METHOD[method], _stream()))

    @property
    def method(self) -> str:
        code = self.lib.tvd_plan_method(self.handle)
        return next(k for k, c in METHOD.items() if c == code)

    def set_transform(self, kind: str):
        """Transform form of the fast preconditioners on a mixed plan: 'fft' or 'gemm'."""
        _check(self.lib.tvd_plan_set_transform(self.handle, TRANSFORM[kind], _stream()))

    @property
    def transform(self) -> str:
        return "gemm" if self.lib.tvd_plan_transform(self.handle) == TRANSFORM["gemm"] else "fft"

    @property
    def gemm_folded(self) -> bool:
        """True when the GEMM form runs the folded (half-K) products."""
        return bool(self.lib.tvd_plan_gemm_folded(self.handle))

    @property
    def gemm_tile(self) -> int:
        """Output tile width of the transform products (64 / 128), 0 in the FFT form."""
        return int(self.lib.tvd_plan_gemm_tile(self.handle))

    def tune(self, reps: int = 3) -> dict:
        """Time every preconditioner form the plan admits and keep the fastest (tvd_plan_tune).

        Returns {"chosen": k, "candidates": [{"transform", "tile_n", "folded", "us_per_solve"}, ...]}.
        """
        rep = _TuneReport()
        _check(self.lib.tvd_plan_tune(self.handle, int(reps), ctypes.byref(rep), _stream()))
        cands = [{"transform": "gemm" if rep.transform[k] == TRANSFORM["gemm"] else "fft",
                  "tile_n": int(rep.tile_n[k]), "folded": bool(rep.folded[k]),
                  "us_per_solve": float(rep.us_per_solve[k])} for k in range(rep.count)]
        return {"chosen": int(rep.chosen), "candidates": cands}

    @property
    def gemm_storage(self):
        """Operand storage of the GEMM form: 'f32' (TF32 products), 'bf16', or None (FFT form)."""
        return {0: None, 1: "f32", 2: "bf16"}[self.lib.tvd_plan_gemm_storage(self.handle)]

    def close(self):
        if getattr(self, "handle", None):
            self.lib.tvd_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- operator calls (plan's operator dtype)
    def blur(self, x, transpose: bool = False, out=None):
        import torch
        y = torch.empty_like(x) if out is None else out
        _check(self.lib.ar_blur_apply(self.handle, int(bool(transpose)), _ptr(x, self.op_dtype, self.n),
                                      _ptr(y, self.op_dtype, self.n), _stream()))
        return y

    def tv_operator(self, u_lag, beta: float, x, out=None):
        import torch
        y = torch.empty_like(x) if out is None else out
        _check(self.lib.tv_operator_apply(self.handle, _ptr(u_lag, self.op_dtype, self.n), float(beta),
                                          _ptr(x, self.op_dtype, self.n), _ptr(y, self.op_dtype, self.n), _stream()))
        return y

    def precond_setup(self, u_lag, alpha: float, beta: float):
        _check(self.lib.tau_precond_setup(self.handle, _ptr(u_lag, self.op_dtype, self.n), float(alpha), float(beta),
                                          _stream()))

    def precond_solve(self, r, out=None):
        import torch
        z = torch.empty_like(r) if out is None else out
        _check(self.lib.tau_precond_solve(self.handle, _ptr(r, self.op_dtype, self.n), _ptr(z, self.op_dtype, self.n),
                                          _stream()))
        return z

    # ---- solver calls (float64)
    def pcg_solve(self, u_lag, alpha: float, beta: float, b, x, tol: float = 1e-6, maxit: int = 1000):
        """Solve (H^T H + alpha L(u_lag)) x = b in place. Returns (iterations, relres, status)."""
        import torch
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0.0)
        st = self.lib.pcg_solve(self.handle, _ptr(u_lag, torch.float64, self.n), float(alpha), float(beta),
                                _ptr(b, torch.float64, self.n), _ptr(x, torch.float64, self.n), float(tol), int(maxit),
                                ctypes.byref(it), ctypes.byref(rr), _stream())
        _check(st, allow=(TVD_ENOCONV,))
        return it.value, rr.value, st

    def pbicgstab_solve(self, u_lag, alpha: float, beta: float, b, x, tol: float = 1e-6, maxit: int = 1000):
        """Solve (H' H + alpha L(u_lag)) x = b (eq. (fpp)) in place on a reblurring plan.
        Returns (iterations, relres, status)."""
        import torch
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0.0)
        st = self.lib.pbicgstab_solve(self.handle, _ptr(u_lag, torch.float64, self.n), float(alpha), float(beta),
                                      _ptr(b, torch.float64, self.n), _ptr(x, torch.float64, self.n), float(tol),
                                      int(maxit), ctypes.byref(it), ctypes.byref(rr), _stream())
        _check(st, allow=(TVD_ENOCONV,))
        return it.value, rr.value, st

    def hessian(self, u, beta: float, x, out=None):
        """y = nabla^2 J_beta(u) x (float64 CUDA tensors), the Hessian of the TV term."""
        import torch
        y = torch.empty_like(x) if out is None else out
        _check(self.lib.tv_hessian_apply(self.handle, _ptr(u, torch.float64, self.n), float(beta),
                                         _ptr(x, torch.float64, self.n), _ptr(y, torch.float64, self.n), _stream()))
        return y

    def psf_size(self):
        """(p_rows, p_cols) of the plan's PSF support after trimming zero outer rows / columns."""
        pr, pc = ctypes.c_int(0), ctypes.c_int(0)
        _check(self.lib.tvd_plan_psf_size(self.handle, ctypes.byref(pr), ctypes.byref(pc)))
        return pr.value, pc.value

    def adjoint(self, u_star, v, alpha: float, beta: float, dl_du, tol: float = 1e-10, maxit: int = 5000):
        """Gradients of a loss of the converged fixed point u* (float64 CUDA tensors).

        Solves J lambda = dl_du, J = H^T H + alpha nabla^2 J_beta(u*), and returns
        (lambda, dl/dalpha, dl/dbeta, dl/dpsf (numpy, psf_size()), stats dict).
        """
        import torch
        lam = torch.empty_like(dl_du)
        pr, pc = self.psf_size()
        dpsf = np.zeros((pr, pc), dtype=np.float64)
        da, db, rr = ctypes.c_double(0.0), ctypes.c_double(0.0), ctypes.c_double(0.0)
        it = ctypes.c_int(0)
        st = self.lib.tv_deblur_adjoint(self.handle, _ptr(u_star, torch.float64, self.n), _ptr(v, torch.float64, self.n),
                                        float(alpha), float(beta), _ptr(dl_du, torch.float64, self.n),
                                        _ptr(lam, torch.float64, self.n), float(tol), int(maxit), ctypes.byref(da),
                                        ctypes.byref(db), dpsf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        ctypes.byref(it), ctypes.byref(rr), _stream())
        _check(st, allow=(TVD_ENOCONV,))
        return lam, da.value, db.value, dpsf, {"iters": it.value, "relres": rr.value, "status": st}

    def deblur(self, v, alpha: float, beta: float, max_outer: int = 10, outer_tol: float = 0.0,
               inner_tol: float = 1e-6, inner_maxit: int = 1000, out=None, track: bool = False):
        """Lagged-diffusivity FP iteration from u^0 = v. Returns (u, stats dict).

        With track=True the stats also hold, per FP step k, ||g(u^k)|| (eq. (el)) and
        the functional T(u^k) of the iterate the step starts from, and both for the
        returned iterate ("final_g_norm", "final_functional").
        """
        import torch
        u = torch.empty_like(v) if out is None else out
        cap = max(int(max_outer), 1)
        arr = (ctypes.c_int * cap)()
        gn = (ctypes.c_double * cap)() if track else None
        fn = (ctypes.c_double * cap)() if track else None
        stats = _Stats()
        stats.inner_iters, stats.cap = arr, cap
        if track:
            stats.g_norm, stats.functional = gn, fn
        st = self.lib.tv_deblur(self.handle, _ptr(v, torch.float64, self.n), float(alpha), float(beta), int(max_outer),
                                float(outer_tol), float(inner_tol), int(inner_maxit), _ptr(u, torch.float64, self.n),
                                ctypes.byref(stats), _stream())
        _check(st, allow=(TVD_ENOCONV,))
        k = stats.outer_iters
        out = {"outer_iters": k, "inner_iters": list(arr[:min(k, cap)]),
               "total_inner_iters": stats.total_inner_iters, "refinement_sweeps": stats.refinement_sweeps,
               "last_relres": stats.last_relres, "last_rel_change": stats.last_rel_change,
               "last_status": stats.last_status, "status": st}
        if track:
            out.update({"g_norm": list(gn[:min(k, cap)]), "functional": list(fn[:min(k, cap)]),
                        "final_g_norm": stats.final_g_norm, "final_functional": stats.final_functional})
        return u, out

    def newton(self, u, v, alpha: float, beta: float, tol: float = 1e-10, max_steps: int = 30,
               cg_tol: float = 1e-10, cg_maxit: int = 20000):
        """Newton finish of the fixed point in place (u: float64 CUDA tensor, distinct from v).

        Steps on g(u) = 0 (eq. (el)) until the relative change falls below tol;
        returns the stats dict (steps, CG iterations, halvings, last step length,
        last relative change, ||g|| before and after, status).
        """
        import torch
        ns = _NewtonStats()
        st = self.lib.tv_deblur_newton(self.handle, _ptr(v, torch.float64, self.n), float(alpha), float(beta),
                                       _ptr(u, torch.float64, self.n), float(tol), int(max_steps), float(cg_tol),
                                       int(cg_maxit), ctypes.byref(ns), _stream())
        _check(st, allow=(TVD_ENOCONV,))
        return {"steps": ns.steps, "total_cg_iters": ns.total_cg_iters, "halvings": ns.halvings,
                "last_t": ns.last_t, "last_rel_change": ns.last_rel_change, "last_cg_relres": ns.last_cg_relres,
                "g_norm_initial": ns.g_norm_initial, "g_norm": ns.g_norm, "status": st}


def normal_apply_noalloc(psf, u_lag, alpha: float, beta: float, x, y=None, bc: str = "ar"):
    """y = H^T H x + alpha L(u_lag) x (float64 CUDA tensors) without any device allocation by the library.

    For callers that must not allocate device memory (code under a framework
    that owns a fixed device-memory pool or budget, and its callbacks). The
    library keeps the intermediate results in fixed device arrays shared by all
    calls: calls that overlap on the GPU race, and n_rows * n_cols is limited
    to 524288. The first call on a device looks up those arrays and should come
    before any stream capture; every call synchronises its stream.
    """
    import torch
    lib = load_library()
    n_rows, n_cols = x.shape
    n = n_rows * n_cols
    out = torch.empty_like(x) if y is None else y
    h = np.ascontiguousarray(np.asarray(psf, dtype=np.float64))
    _check(lib.tvd_normal_apply_noalloc(n_rows, n_cols, h.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        h.shape[0], h.shape[1], BC[bc], _ptr(u_lag, torch.float64, n),
                                        float(alpha), float(beta), _ptr(x, torch.float64, n),
                                        _ptr(out, torch.float64, n), _stream()))
    return out


def deblur_batched(plans, vs, alphas, betas, max_outer: int = 10, inner_tol: float = 1e-6,
                   inner_maxit: int = 1000, outs=None, workers: int = 8, outer_tol: float = 0.0):
    """tv_deblur of independent problems at once (one Plan per item; float64 CUDA tensors).

    Items run on `workers` host threads with a CUDA stream each, largest
    first; each item's result equals that of plan.deblur(v, alpha, beta, ...,
    outer_tol=outer_tol). Returns (list of u, list of per-item dicts
    {"status", "inner_iters", "outer_iters"}).
    """
    import torch
    lib = load_library()
    count = len(plans)
    if not (len(vs) == len(alphas) == len(betas) == count):
        raise ValueError("plans, vs, alphas and betas must have the same length")
    us = [torch.empty_like(v) for v in vs] if outs is None else list(outs)
    cap = max(int(max_outer), 1)
    iters = [(ctypes.c_int * cap)() for _ in range(count)]
    arr = (_BatchItem * max(count, 1))()
    for i, pl in enumerate(plans):
        arr[i].plan = pl.handle
        arr[i].v = _ptr(vs[i], torch.float64, pl.n)
        arr[i].u_out = _ptr(us[i], torch.float64, pl.n)
        arr[i].alpha = float(alphas[i])
        arr[i].beta = float(betas[i])
        arr[i].inner_iters = ctypes.cast(iters[i], ctypes.POINTER(ctypes.c_int))
        arr[i].status = 0
        arr[i].outer_tol = float(outer_tol)
    st = lib.tv_deblur_batched(arr, count, int(max_outer), float(inner_tol), int(inner_maxit), int(workers),
                               _stream())
    _check(st, allow=(TVD_ENOCONV,))
    return us, [{"status": arr[i].status, "outer_iters": arr[i].outer_iters,
                 "inner_iters": list(iters[i][:min(arr[i].outer_iters, max_outer)])} for i in range(count)]


def alpha_sweep(v, psf, alphas, beta: float, bc: str = "ar", pc: str = "dfast", mode: str = "fp64",
                method: str = "fp", max_outer: int = 100, outer_tol: float = 1e-3, inner_tol: float = 1e-6,
                inner_maxit: int = 5000, workers: int = 8):
    """Deblur one observation v (float64 CUDA tensor, an image or a 1 x n signal) once per
    regularisation parameter in ``alphas``, as one batch of independent problems: one plan per
    alpha (same size, PSF, BCs, preconditioner, arithmetic and method), run by tv_deblur_batched.

    The FP iteration of each item stops at ||u^k - u^{k-1}|| / ||u^k|| < outer_tol (1e-3 in the
    paper's 1D experiment, Sec. 5.1) or after max_outer steps. Returns (list of u, list of per-item
    stats): the input of an RRE-versus-alpha curve (Fig. tvrs).
    """
    nr, nc = v.shape
    plans = [Plan(nr, nc, psf, bc=bc, pc=pc, mode=mode, method=method) for _ in alphas]
    try:
        return deblur_batched(plans, [v] * len(alphas), list(alphas), [beta] * len(alphas), max_outer=max_outer,
                              inner_tol=inner_tol, inner_maxit=inner_maxit, workers=workers, outer_tol=outer_tol)
    finally:
        for pl in plans:
            pl.close()


def kernel_launches() -> int:
    """CUDA kernels launched by the library in this process so far."""
    return int(load_library().tvd_kernel_launches())


def profile_enable(on: bool = True) -> None:
    """Start (or stop) CUDA-event timing per kernel class; clears earlier records."""
    _check(load_library().tvd_profile_enable(int(bool(on))))


def profile_read() -> dict:
    """{class name: (total device ms, launches)} since profiling was enabled."""
    lib = load_library()
    out = {}
    for c in range(lib.tvd_profile_classes()):
        ms = ctypes.c_double(0.0)
        n = ctypes.c_longlong(0)
        _check(lib.tvd_profile_read(c, ctypes.byref(ms), ctypes.byref(n)))
        out[lib.tvd_profile_name(c).decode()] = (ms.value, n.value)
    return out


# Module-level names matching the C ABI.
def ar_blur_apply(plan: Plan, transpose: bool, x, y=None):
    return plan.blur(x, transpose, y)


def tv_operator_apply(plan: Plan, u_lag, beta: float, x, y=None):
    return plan.tv_operator(u_lag, beta, x, y)


def tau_precond_setup(plan: Plan, u_lag, alpha: float, beta: float):
    return plan.precond_setup(u_lag, alpha, beta)


def tau_precond_solve(plan: Plan, r, z=None):
    return plan.precond_solve(r, z)


def pcg_solve(plan: Plan, u_lag, alpha, beta, b, x, tol=1e-6, maxit=1000):
    return plan.pcg_solve(u_lag, alpha, beta, b, x, tol, maxit)


def pbicgstab_solve(plan: Plan, u_lag, alpha, beta, b, x, tol=1e-6, maxit=1000):
    return plan.pbicgstab_solve(u_lag, alpha, beta, b, x, tol, maxit)


def tvd_plan_set_method(plan: Plan, method: str):
    return plan.set_method(method)


def tv_deblur(plan: Plan, v, alpha, beta, max_outer=10, outer_tol=0.0, inner_tol=1e-6, inner_maxit=1000, u=None):
    return plan.deblur(v, alpha, beta, max_outer, outer_tol, inner_tol, inner_maxit, u)


def tv_hessian_apply(plan: Plan, u, beta, x, y=None):
    return plan.hessian(u, beta, x, y)


def tv_deblur_adjoint(plan: Plan, u_star, v, alpha, beta, dl_du, tol=1e-10, maxit=5000):
    return plan.adjoint(u_star, v, alpha, beta, dl_du, tol, maxit)


def tvd_plan_psf_size(plan: Plan):
    return plan.psf_size()


def tv_deblur_batched(plans, vs, alphas, betas, max_outer=10, inner_tol=1e-6, inner_maxit=1000, outs=None,
                      workers=8):
    return deblur_batched(plans, vs, alphas, betas, max_outer, inner_tol, inner_maxit, outs, workers)
