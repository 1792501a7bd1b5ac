"""GPU HISQ link smearing (wcl_hisq_smear) against the FP64 oracle (oracle/hisq.py): the
fat and long links on lattices with an L = 2 axis (where x + rho = x - rho) and L = 4
(the Naik link wraps around), with and without the Naik epsilon; then the staggered
solve on the GPU's smeared links, its true residual recomputed by the oracle on the
oracle's own links; and the error statuses."""
import numpy as np
import pytest

import workloads as W
from oracle import hisq as H
from oracle import lattice as L
from oracle import staggered as S

from _gpu import built, cuda, host, relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    return built()


def _smear(pkg, dims, gauge_qdp, eps):
    ctx = pkg.Context(dims)
    fat = cuda(np.zeros_like(gauge_qdp))
    lng = cuda(np.zeros_like(gauge_qdp))
    ctx.wcl_hisq_smear(fat, lng, cuda(gauge_qdp), eps)
    return ctx, fat, lng


@pytest.mark.parametrize("eps", [0.0, -0.1])
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 8), (2, 4, 4, 6), (8, 4, 6, 4)])
def test_smearing_matches_oracle(pkg, dims, eps):
    gauge = W.gauge_links(dims, 0.5, 3)
    ctx, fat, lng = _smear(pkg, dims, gauge, eps)
    ref_fat, ref_long = H.hisq_links(L.gauge_from_qdp(gauge, dims), eps)
    assert relerr(L.gauge_from_qdp(host(fat), dims), ref_fat) <= 1e-12
    assert relerr(L.gauge_from_qdp(host(lng), dims), ref_long) <= 1e-12
    ctx.close()


def test_smearing_rough_field(pkg):
    """Random SU(3) links (no smoothness): the first-level links are far from unitary, the
    projection does real work."""
    dims = (4, 4, 2, 4)
    lx, ly, lz, lt = dims
    thin = np.stack([W.random_su3(dims, 20 + mu) for mu in range(4)])  # (4, Lt, Lz, Ly, Lx, 3, 3)
    gauge = L.gauge_to_qdp(thin, dims)
    ctx, fat, lng = _smear(pkg, dims, gauge, 0.0)
    ref_fat, ref_long = H.hisq_links(thin)
    assert relerr(L.gauge_from_qdp(host(fat), dims), ref_fat) <= 1e-11
    assert relerr(L.gauge_from_qdp(host(lng), dims), ref_long) <= 1e-11
    ctx.close()


def test_smeared_staggered_solve(pkg):
    """Thin links -> HISQ links on the GPU -> the GPU's staggered CG; the oracle recomputes
    ||b - M x|| / ||b|| with its own smearing of the same thin links."""
    dims = (6, 4, 4, 8)
    lx, ly, lz, lt = dims
    gauge = W.gauge_links(dims, 0.4, 30)
    ctx, fat, lng = _smear(pkg, dims, gauge, 0.0)
    ctx.wcl_load_staggered(fat, lng, 0.1)
    b = W.gaussian_complex((lt, lz, ly, lx, 3), 31)
    x = cuda(np.zeros((1,) + L.to_qdp(b, dims).shape, dtype=np.complex128))
    _, info = ctx.wcl_invert_staggered(x, cuda(L.to_qdp(b, dims)[None]), 1, pkg.wcl_default_params(tol=1e-10))
    ref_fat, ref_long = H.hisq_links(L.gauge_from_qdp(gauge, dims))
    op = S.Staggered(ref_fat, ref_long, 0.1, -1)
    xl = L.from_qdp(host(x)[0], dims)
    tr = np.linalg.norm(b - op.M(xl)) / np.linalg.norm(b)
    assert tr <= 1e-10, (tr, info)
    ctx.close()


def test_smearing_errors(pkg):
    from paper_2411_08461_gb300.wcl import WclError

    dims = (4, 4, 4, 4)
    gauge = W.gauge_links(dims, 0.5, 40)
    ctx = pkg.Context(dims)
    out1, out2 = cuda(np.zeros_like(gauge)), cuda(np.zeros_like(gauge))
    bad = gauge.copy()
    bad[2, 1, 1, 0, 1, 1, 0, 0] = np.nan
    with pytest.raises(WclError) as e:
        ctx.wcl_hisq_smear(out1, out2, cuda(bad), 0.0)
    assert e.value.status == 6  # WCL_ERR_NONFINITE
    with pytest.raises(WclError) as e:  # zero links: the first level is zero, no U(3) projection
        ctx.wcl_hisq_smear(out1, out2, cuda(np.zeros_like(gauge)), 0.0)
    assert e.value.status == 7  # WCL_ERR_RECONSTRUCT
    ctx.wcl_hisq_smear(out1, out2, cuda(gauge), 0.0)  # the context is still usable
    ctx.close()
