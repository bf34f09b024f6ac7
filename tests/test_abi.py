"""The C-ABI library loads and exports every function that include/tvd.h declares.

No compute call is made here (no GPU is needed). The library is built first if
it is missing.
"""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tvd.h")


def header_functions():
    """Names of the functions declared in the header (declarations end with ');')."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = "\n".join(ln for ln in text.splitlines() if not ln.lstrip().startswith("#"))
    names = []
    for stmt in text.split(";"):
        stmt = stmt.strip()
        if not stmt.endswith(")") or "typedef" in stmt or "{" in stmt:
            continue
        m = re.search(r"([A-Za-z_][A-Za-z0-9_]*)\s*\(", stmt)
        if m:
            names.append(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    import paper_1011_5964_gb300 as pkg
    if not os.path.exists(pkg.LIB_PATH):
        from paper_1011_5964_gb300 import _build
        _build.build()
    return pkg.load_library()


def test_header_declares_the_abi():
    import paper_1011_5964_gb300 as pkg
    names = header_functions()
    assert set(names) == set(pkg.ABI_FUNCTIONS), names


def test_library_exports_every_declared_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), name


def test_version_and_error_without_gpu(lib):
    assert lib.tvd_version().decode().startswith("tvd-gb300")
    assert lib.tvd_last_error() is not None


def test_plan_create_rejects_bad_arguments_before_touching_the_gpu(lib):
    """Argument validation is host logic: a NULL out-pointer and a too-small image are refused."""
    import ctypes
    import numpy as np
    import paper_1011_5964_gb300 as pkg
    h = np.ones((3, 3)) / 9.0
    hp = h.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert lib.tvd_plan_create(None, 16, 16, hp, 3, 3, 1, 3, 0, None) == pkg.TVD_EINVAL
    out = ctypes.c_void_p()
    assert lib.tvd_plan_create(ctypes.byref(out), 2, 16, hp, 3, 3, 1, 3, 0, None) == pkg.TVD_EINVAL
    assert lib.tvd_plan_create(ctypes.byref(out), 16, 16, hp, 3, 3, 7, 3, 0, None) == pkg.TVD_EINVAL


def test_batched_argument_checks_without_gpu(lib):
    """tv_deblur_batched validates before any CUDA call: nothing to do, or invalid arguments."""
    import paper_1011_5964_gb300 as pkg
    assert lib.tv_deblur_batched(None, 0, 10, 1e-6, 100, 0, None) == pkg.TVD_OK
    assert lib.tv_deblur_batched(None, -1, 10, 1e-6, 100, 0, None) == pkg.TVD_EINVAL
    assert lib.tv_deblur_batched(None, 2, 10, 1e-6, 100, 0, None) == pkg.TVD_EINVAL
    items = (pkg._BatchItem * 1)()
    assert lib.tv_deblur_batched(items, 1, 10, 1e-6, 100, 0, None) == pkg.TVD_EINVAL   # null plan
    assert lib.tv_deblur_batched(items, 1, 10, 0.0, 100, 0, None) == pkg.TVD_EINVAL    # tol <= 0
    assert lib.tv_deblur_batched(items, 1, 10, 1e-6, 100, 65, None) == pkg.TVD_EINVAL  # workers > 64


def test_reblur_entry_points_validate_without_gpu(lib):
    """The reblurring entry points refuse a NULL plan or an unknown method before any CUDA call."""
    import ctypes
    import paper_1011_5964_gb300 as pkg
    assert lib.tvd_plan_set_method(None, 1, None) == pkg.TVD_EINVAL
    assert lib.tvd_plan_method(None) == pkg.METHOD["fp"]
    it, rr = ctypes.c_int(), ctypes.c_double()
    assert lib.pbicgstab_solve(None, None, 1e-3, 1e-2, None, None, 1e-6, 10, ctypes.byref(it), ctypes.byref(rr),
                               None) == pkg.TVD_EINVAL


def test_newton_entry_point_validates_without_gpu(lib):
    import ctypes
    import paper_1011_5964_gb300 as pkg
    ns = pkg._NewtonStats()
    assert lib.tv_deblur_newton(None, None, 1e-3, 1e-2, None, 1e-10, 10, 1e-10, 100, ctypes.byref(ns),
                                None) == pkg.TVD_EINVAL
    assert b"tv_deblur_newton" in lib.tvd_last_error()


def test_stats_structures_match_the_header():
    """The ctypes mirrors of tvd_stats / tvd_newton_stats list the header's fields in order."""
    import re
    import paper_1011_5964_gb300 as pkg
    hdr = open(os.path.join(ROOT, "include", "tvd.h")).read()
    for cname, py in (("tvd_stats", pkg._Stats), ("tvd_newton_stats", pkg._NewtonStats),
                      ("tvd_batch_item", pkg._BatchItem), ("tvd_tune_report", pkg._TuneReport)):
        flat = re.sub(r"\[[^\]]*\]", "", re.sub(r"/\*.*?\*/", "", hdr, flags=re.S))
        body = re.search(r"typedef struct \{([^{}]*)\} " + cname + ";", flat).group(1)
        names = []
        for stmt in filter(str.strip, body.split(";")):
            parts = stmt.split(",")          # "double alpha, beta" declares two fields
            names += [re.findall(r"\w+", parts[0])[-1]] + [re.findall(r"\w+", q)[-1] for q in parts[1:]]
        assert names == [f[0] for f in py._fields_], (cname, names)


def test_tune_validation_and_constants(lib):
    """tvd_plan_tune refuses a NULL plan before touching the GPU; the binding's constants are the header's."""
    import ctypes
    import paper_1011_5964_gb300 as pkg
    rep = pkg._TuneReport()
    assert lib.tvd_plan_tune(None, 3, ctypes.byref(rep), None) == pkg.TVD_EINVAL
    assert b"tvd_plan_tune" in lib.tvd_last_error()
    assert lib.tvd_plan_gemm_tile(None) == 0
    hdr = open(HEADER).read()
    assert int(re.search(r"#define TVD_TUNE_MAX (\d+)", hdr).group(1)) == pkg.TUNE_MAX
    assert int(re.search(r"#define TVD_TUNE_SOLVES (\d+)", hdr).group(1)) == pkg.TUNE_SOLVES
