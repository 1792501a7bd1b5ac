"""The stored fixture tests/golden/c1_apply_solve.txt (written by make_golden.py from
the oracle) pinned to a library LU solve of the dense matrix built by the loop-based
definition in _dense_ref, and to the oracle as it stands (a change to the oracle's
arithmetic shows up here)."""
import os

import numpy as np

import workloads as W
from oracle import lattice as L

from _dense_ref import dense_matrix, site_index

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "c1_apply_solve.txt")
DIMS = (4, 4, 4, 4)


def _load():
    import importlib.util

    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod, mod.read(GOLDEN)


def _stored(vals, site, field):
    return np.array([[vals[site + (field, s, c)] for c in range(3)] for s in range(4)])


def test_golden_matches_dense_lu():
    mod, vals = _load()
    U = L.gauge_from_qdp(W.gauge_links(DIMS, 0.2, 0), DIMS)
    M = dense_matrix(U, DIMS, 0.12, 1.0)
    b = L.from_qdp(W.point_source(DIMS, 0, 0), DIMS)
    # the dense vector index is lexicographic in (t, z, y, x), then 3 * spin + colour
    bv = np.zeros(M.shape[0], dtype=np.complex128)
    bv[site_index((0, 0, 0, 0), DIMS) * 12] = 1.0
    assert np.array_equal(bv, b.ravel())
    mb = (M @ bv).reshape(-1, 4, 3)
    x = np.linalg.solve(M, bv).reshape(-1, 4, 3)
    for s in mod.SITES:
        i = site_index(s, DIMS)
        assert np.abs(_stored(vals, s, 0) - mb[i]).max() <= 1e-14, s
        assert np.abs(_stored(vals, s, 1) - x[i]).max() <= 1e-10 * np.abs(x).max(), s


def test_oracle_reproduces_golden():
    mod, vals = _load()
    for s, mb, x in mod.compute():
        assert np.abs(_stored(vals, s, 0) - mb).max() <= 1e-14, s
        assert np.abs(_stored(vals, s, 1) - x).max() <= 1e-11, s
