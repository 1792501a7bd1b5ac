"""GPU staggered operator (HISQ form, given fat and long links) and its even-odd CG solve
against the FP64 oracle (oracle/staggered.py): the whole-lattice operator in FP64 and
FP32 on lattices where the three-hop wraps around, both time boundaries, several
right-hand sides; the solve's true residual recomputed by the oracle and its solution
against the oracle's CG solution."""
import numpy as np
import pytest

import workloads as W
from oracle import staggered as S
from oracle import lattice as L

from _gpu import TOL, built, cuda, host, relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    return built()


def _links(dims, seed, scale):
    lx, ly, lz, lt = dims
    return scale * W.gaussian_complex((4, lt, lz, ly, lx, 3, 3), seed)


def _field(dims, seed):
    lx, ly, lz, lt = dims
    return W.gaussian_complex((lt, lz, ly, lx, 3), seed)


def _setup(pkg, dims, tb, mass, seed=0):
    V, Wl = _links(dims, 10 + seed, 0.3), _links(dims, 20 + seed, 0.05)
    ctx = pkg.Context(dims, t_boundary=tb)
    ctx.wcl_load_staggered(cuda(L.gauge_to_qdp(V, dims)), cuda(L.gauge_to_qdp(Wl, dims)), mass)
    return ctx, S.Staggered(V, Wl, mass, tb)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("tb", [-1, 1])
@pytest.mark.parametrize("dims", [(4, 4, 4, 6), (6, 4, 2, 8), (2, 2, 4, 4), (8, 6, 6, 4)])
def test_apply_parity(pkg, dims, tb, prec):
    ctx, op = _setup(pkg, dims, tb, 0.37)
    chis = [_field(dims, 30 + k) for k in range(3)]
    chis[1] *= 1e-6
    q = np.stack([L.to_qdp(c, dims) for c in chis])
    out = cuda(np.zeros_like(q))
    ctx.wcl_apply_staggered(out, cuda(q), prec, nrhs=3)
    got = host(out)
    for k in range(3):
        assert relerr(L.from_qdp(got[k], dims), op.M(chis[k])) <= TOL[prec], k
    ctx.close()


@pytest.mark.parametrize("sloppy", ["f64", "f32"])
def test_even_odd_cg_solve(pkg, sloppy):
    dims = (6, 4, 4, 8)
    ctx, op = _setup(pkg, dims, -1, 0.2, seed=3)
    bs = [_field(dims, 40 + k) for k in range(2)]
    q = np.stack([L.to_qdp(b, dims) for b in bs])
    x = cuda(np.zeros_like(q))
    _, info = ctx.wcl_invert_staggered(x, cuda(q), 2, pkg.wcl_default_params(sloppy=sloppy, tol=1e-10))
    xh = host(x)
    for k in range(2):
        xl = L.from_qdp(xh[k], dims)
        tr = np.linalg.norm(bs[k] - op.M(xl)) / np.linalg.norm(bs[k])
        assert tr <= 1e-10, (k, tr, info)
        assert abs(tr - info[k]["true_residual"]) <= 1e-3 * tr + 1e-15
        ref, _ = op.solve(bs[k], tol=1e-13)
        assert relerr(xl, ref) <= 1e-8
    ctx.close()


def test_staggered_errors(pkg):
    from paper_2411_08461_gb300.wcl import WclError

    dims = (4, 4, 4, 4)
    ctx = pkg.Context(dims)
    q = cuda(L.to_qdp(_field(dims, 50), dims))
    with pytest.raises(WclError) as e:  # no links loaded
        ctx.wcl_apply_staggered(cuda(np.zeros_like(host(q))), q)
    assert e.value.status == 9
    V = cuda(L.gauge_to_qdp(_links(dims, 51, 0.3), dims))
    with pytest.raises(WclError) as e:  # the even-odd solve needs m > 0
        ctx.wcl_load_staggered(V, V, 0.0)
    assert e.value.status == 1
    ctx.close()
