"""The CUDA path against the stored fixture tests/golden/c1_apply_solve.txt (4^4,
point source): M b in FP64 and the solution of M x = b from the FP64 solver and from
the FP32 solver with reliable updates, at the source and its eight neighbours."""
import os

import numpy as np
import pytest

import workloads as W
from oracle import lattice as L

from _gpu import built, cuda, host

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
DIMS = (4, 4, 4, 4)


def _golden():
    import importlib.util

    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    vals = mod.read(os.path.join(HERE, "golden", "c1_apply_solve.txt"))
    pick = lambda field: np.array([[[vals[s + (field, sp, c)] for c in range(3)] for sp in range(4)] for s in mod.SITES])
    return mod.SITES, pick(0), pick(1)


def _at(full_qdp, sites):
    f = L.from_qdp(full_qdp, DIMS)
    return np.array([f[t, z, y, x] for x, y, z, t in sites])


@pytest.fixture(scope="module")
def ctx():
    pkg = built()
    c = pkg.Context(DIMS)
    c.wcl_load_gauge(cuda(W.gauge_links(DIMS, 0.2, 0)), 0.12, 1.0)
    yield pkg, c
    c.close()


def test_apply_matches_golden(ctx):
    pkg, c = ctx
    sites, mb_ref, _ = _golden()
    out = cuda(np.zeros_like(W.point_source(DIMS, 0, 0)))
    c.wcl_apply_D(out, cuda(W.point_source(DIMS, 0, 0)), "f64")
    got = _at(host(out), sites)
    assert np.linalg.norm(got - mb_ref) <= 1e-12 * np.linalg.norm(mb_ref)


@pytest.mark.parametrize("sloppy", ["f64", "f32"])
def test_solve_matches_golden(ctx, sloppy):
    pkg, c = ctx
    sites, _, x_ref = _golden()
    b = W.point_source(DIMS, 0, 0)
    x = cuda(np.zeros_like(b))
    prm = pkg.wcl_default_params(solver="bicgstab", sloppy=sloppy, tol=1e-12)
    _, info = c.wcl_invert(x, cuda(b), 1, prm)
    assert info[0]["status"] == 0 and info[0]["true_residual"] <= 1e-12, info
    got = _at(host(x), sites)
    assert np.linalg.norm(got - x_ref) <= 1e-10 * np.linalg.norm(x_ref)
