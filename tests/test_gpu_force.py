"""GPU clover fermion force (wcl_clover_force) against the FP64 oracle (oracle/force.py),
whose pins differentiate the action itself: Gaussian X on the even sites, with and without
the clover determinant term, on lattices with extent-2 axes (forward and backward
neighbours coincide), both time boundaries, and a lattice larger than a few tiles; an X
obtained from phi by the oracle's solve; the error statuses."""
import numpy as np
import pytest

import workloads as W
from oracle import dirac, force
from oracle import lattice as L

from _gpu import TOL, built, cuda, host, relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    return built()


def _even_qdp(dims, seed):
    f = W.gaussian_fermion(dims, seed)
    return np.ascontiguousarray(f[0])


def _gpu_force(pkg, dims, gauge, kappa, csw, x_even_qdp, logdet, tb=-1):
    ctx = pkg.Context(dims, t_boundary=tb)
    ctx.wcl_load_gauge(cuda(gauge), kappa, csw)
    out = cuda(np.zeros_like(gauge))
    ctx.wcl_clover_force(out, cuda(x_even_qdp), logdet)
    f = host(out)
    ctx.close()
    return f


def _oracle_force(dims, gauge, kappa, csw, x_even_qdp, logdet, tb=-1):
    op = dirac.from_qdp_problem(gauge, dims, kappa, csw, tb)
    full = np.zeros((2,) + x_even_qdp.shape, dtype=np.complex128)
    full[0] = x_even_qdp
    X = L.from_qdp(full, dims)
    F = force.clover_force(op, X, logdet)
    return L.gauge_to_qdp(F, dims)


@pytest.mark.parametrize("dims,tb", [((2, 2, 2, 2), -1), ((4, 2, 4, 2), 1), ((4, 4, 4, 4), -1), ((6, 4, 2, 8), -1),
                                     ((8, 8, 8, 16), -1)])
@pytest.mark.parametrize("logdet", [False, True])
def test_force_matches_oracle(pkg, dims, tb, logdet):
    gauge = W.gauge_links(dims, 0.3, 7)
    x = _even_qdp(dims, 8)
    got = _gpu_force(pkg, dims, gauge, 0.1235, 1.0, x, logdet, tb)
    want = _oracle_force(dims, gauge, 0.1235, 1.0, x, logdet, tb)
    assert relerr(got, want) <= TOL["f64"], relerr(got, want)
    # traceless anti-Hermitian per link
    m = got.reshape(-1, 3, 3)
    assert np.abs(m + np.conj(np.swapaxes(m, -1, -2))).max() <= 1e-13 * np.abs(m).max()


def test_force_of_a_solved_pseudofermion(pkg):
    """X = (M_hat^+ M_hat)^-1 phi from the oracle's dense solve, kappa 0.13, c_sw 1.5."""
    dims = (4, 4, 2, 4)
    gauge = W.gauge_links(dims, 0.3, 11)
    op = dirac.from_qdp_problem(gauge, dims, 0.13, 1.5)
    rng = np.random.default_rng(12)
    shp = op.even.shape[:4] + (4, 3)
    phi = (rng.standard_normal(shp) + 1j * rng.standard_normal(shp)) * op.even
    X = force.solve_normal(op, phi)
    x_even = np.ascontiguousarray(L.to_qdp(X, dims)[0])
    got = _gpu_force(pkg, dims, gauge, 0.13, 1.5, x_even, True)
    want = L.gauge_to_qdp(force.clover_force(op, X, True), dims)
    assert relerr(got, want) <= TOL["f64"]


def test_force_errors(pkg):
    from paper_2411_08461_gb300.wcl import WclError

    dims = (4, 4, 4, 4)
    gauge = W.gauge_links(dims, 0.3, 1)
    ctx = pkg.Context(dims)
    out = cuda(np.zeros_like(gauge))
    x = cuda(_even_qdp(dims, 2))
    with pytest.raises(WclError) as e:
        ctx.wcl_clover_force(out, x)
    assert e.value.status == 9  # WCL_ERR_NO_GAUGE
    ctx.wcl_load_gauge_aniso(cuda(gauge), 0.12, 2.0, 1.0, 1.0, 1.0)
    with pytest.raises(WclError) as e:
        ctx.wcl_clover_force(out, x)
    assert e.value.status == 1  # WCL_ERR_INVALID_ARG
    ctx.wcl_load_gauge(cuda(gauge), 0.12, 1.0)
    xb = _even_qdp(dims, 2)
    xb[0, 0, 0, 0, 0, 0] = np.nan
    with pytest.raises(WclError) as e:
        ctx.wcl_clover_force(out, cuda(xb))
    assert e.value.status == 6  # WCL_ERR_NONFINITE
    ctx.close()
