"""The C-ABI library builds, loads and exports every function include/wt.h
declares; argument checks that need no GPU.  CPU only (no compute calls)."""

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "wt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*int\s+(wt_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2406_00991_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_entry_points():
    names = declared_functions()
    for want in ("wt_create", "wt_poisson_solve", "wt_rk_stage", "wt_step", "wt_destroy",
                 "wt_apply_operator", "wt_precondition", "wt_set_state", "wt_get_state"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_wraps_every_declared_symbol():
    import paper_2406_00991_gb300 as w
    for name in declared_functions():
        assert hasattr(w, name) or name in ("wt_last_error",), name


def test_argument_checks_without_gpu():
    import paper_2406_00991_gb300 as w
    o = w.wt_default_options()
    assert (o.mode, o.restart, o.nu1, o.nu2, o.coarsest_max) == (w.WT_MIXED, 30, 2, 2, 64)
    # invalid sizes are rejected before any CUDA call
    st, h = w.wt_create(100, 1, 16, 1.0, 9.81, 0.0, np.ones(100))
    assert st == w.WT_EINVAL
    st, h = w.wt_create(64, 1, 40, 1.0, 9.81, 0.0, np.ones(64))
    assert st == w.WT_EINVAL
    st, h = w.wt_create(64, 1, 16, 1.0, 9.81, -1e-6, np.ones(64))
    assert st == w.WT_EINVAL
    code, msg = w.wt_last_error()
    assert code == w.WT_EINVAL and "nu" in msg
    assert w.wt_destroy(None) == w.WT_OK
    # the tuned-options file: a path, none, and an empty path (rejected)
    assert w.wt_autotune_cache("/nonexistent/dir/tuned.jsonl") == w.WT_OK
    assert w.wt_autotune_cache(None) == w.WT_OK
    assert w.wt_autotune_cache("") == w.WT_EINVAL


def test_product_path_has_no_oracle_import():
    pkg = os.path.join(ROOT, "paper_2406_00991_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
