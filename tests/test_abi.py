"""The C ABI: the built library exports every function include/wcl.h declares, and
the ctypes binding declares a signature for each (no GPU calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "wcl.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:[\w\*]+\s+)+\**(wcl_\w+)\s*\(", text, flags=re.M)))


def test_header_lists_the_boundary():
    names = header_functions()
    for required in ("wcl_create", "wcl_load_gauge", "wcl_apply_D", "wcl_apply_Mpc", "wcl_invert",
                     "wcl_invert_batch", "wcl_destroy", "wcl_precond_train", "wcl_precond_load"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2411_08461_gb300 import wcl

    lib = ctypes.CDLL(wcl.LIB_PATH)
    names = header_functions()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding declares every one of them
    assert sorted(set(names) - set(wcl.SIGNATURES)) == []


def test_host_only_calls_without_a_gpu():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2411_08461_gb300 import wcl

    lib = wcl.load_library()
    p = wcl.wcl_default_params()
    assert p.outer == 4 and p.tol == 1e-10 and p.gcr_nkrylov == 20  # double-float replacements, FP64 final
    assert lib.wcl_status_string(4) == b"not converged"
    tp = wcl.wcl_default_train_params()
    assert tp.epochs == 4 and tp.batch == 8
    # invalid dims are rejected before any device call
    h = ctypes.c_void_p()
    dims = (ctypes.c_int * 4)(3, 4, 4, 4)
    assert lib.wcl_create(ctypes.byref(h), dims, -1, 0, None) == 1
    assert b"even" in lib.wcl_last_error()
