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


def test_force_and_batched_multigrid_argument_checks_without_a_gpu():
    """The clover force and the batched multigrid cycle refuse null handles and pointers,
    and the cycle a right-hand-side count outside 1..12, before any device call."""
    import __graft_entry__

    __graft_entry__.build()
    from paper_2411_08461_gb300 import wcl

    lib = wcl.load_library()
    assert lib.wcl_clover_force(None, None, None, 1) == 1
    assert b"null" in lib.wcl_last_error()
    assert lib.wcl_mg_cycle_batched(None, None, None, 1) == 1
    assert lib.wcl_mg_cycle_batched(None, None, None, 13) == 1
    assert b"nrhs" in lib.wcl_last_error()
    assert lib.wcl_set_option(None, wcl.WCL_OPT_SLOPPY_UPDATES, 3) == 1


def test_gamma_and_kappa_helpers_without_a_gpu():
    """wcl_gamma reproduces the oracle's independently written Gamma(n) for all 16 n,
    and wcl_kappa_from_mass the isotropic kappa relation; both are host-only calls."""
    import numpy as np

    import __graft_entry__
    from oracle import gamma as G

    __graft_entry__.build()
    from paper_2411_08461_gb300 import wcl

    for n in range(16):
        np.testing.assert_array_equal(wcl.wcl_gamma(n), G.gamma(n))
    assert np.array_equal(wcl.wcl_gamma(15) @ wcl.wcl_gamma(4), G.GAMMA5 @ G.GAMMA[2])
    assert wcl.wcl_kappa_from_mass(0.0) == 0.125
    assert abs(wcl.wcl_kappa_from_mass(-0.2770) - 1 / (2 * 3.723)) < 1e-15
    for bad in (-4.0, -5.0, float("nan")):
        with pytest.raises(wcl.WclError):
            wcl.wcl_kappa_from_mass(bad)
    with pytest.raises(wcl.WclError):
        wcl.wcl_gamma(16)


def test_binding_argument_checks_without_a_gpu():
    """The binding's marshalling rejects what the ABI cannot take before any call:
    non-tensors, CPU tensors that are not page-locked, wrong dtype or size, non-contiguous
    views, malformed Gamma matrices and momentum triples."""
    import numpy as np
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2411_08461_gb300 import wcl

    with pytest.raises(TypeError):
        wcl._ptr(np.zeros(4), name="x")
    with pytest.raises(ValueError, match="CUDA device"):
        wcl._ptr(torch.zeros(4, dtype=torch.complex128), name="x")
    with pytest.raises(ValueError, match="pinned"):
        wcl._ptr(torch.zeros(4, dtype=torch.complex128), name="x", fermion=True)
    with pytest.raises(ValueError):
        wcl._gamma_arg(np.eye(3))
    buf, ptr = wcl._gamma_arg(1j * np.eye(4))
    assert buf.shape == (32,) and buf[1] == 1.0 and buf[0] == 0.0  # row-major (re, im) pairs
    assert wcl._gamma_arg(None) == (None, None)
    with pytest.raises(ValueError):
        wcl._mom_arg((1, 2))
    m = wcl._mom_arg((0, -1, 3))
    assert list(m) == [0, -1, 3]
    assert wcl._mom_arg(None) is None


def test_header_is_plain_c_and_links_from_c(tmp_path):
    """include/wcl.h is a C header (C99, -pedantic) and a C program links against
    libwcl.so and calls its host-only functions."""
    import shutil
    import subprocess

    import __graft_entry__

    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    __graft_entry__.build()
    from paper_2411_08461_gb300 import wcl

    inc = os.path.join(ROOT, "include")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only", "-x", "c",
                    os.path.join(inc, "wcl.h")], check=True)
    src = tmp_path / "user.c"
    src.write_text(
        '#include "wcl.h"\n'
        "#include <stdio.h>\n"
        "int main(void) {\n"
        "  wcl_solve_params p; double g[32]; double k = 0;\n"
        "  wcl_default_params(&p);\n"
        "  if (wcl_gamma(15, g) != WCL_OK || g[0] != 1.0 || g[2 * 15] != -1.0) return 1;\n"
        "  if (wcl_kappa_from_mass(0.0, &k) != WCL_OK || k != 0.125) return 2;\n"
        "  if (wcl_kappa_from_mass_aniso(0.0, 2.0, 1.0, &k) != WCL_OK || k != 0.2) return 3;\n"
        "  printf(\"%s\\n\", wcl_status_string(WCL_ERR_NOT_CONVERGED));\n"
        "  return p.solver == WCL_BICGSTAB ? 0 : 4;\n"
        "}\n")
    libdir = os.path.dirname(wcl.LIB_PATH)
    exe = tmp_path / "user"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", inc, str(src), "-L", libdir, "-lwcl",
                    f"-Wl,-rpath,{libdir}", "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out
    assert out.stdout.strip() == "not converged"
