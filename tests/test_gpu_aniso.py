"""The anisotropic form of Eq. 5 on the GPU (wcl_load_gauge_aniso) against the oracle's
anisotropic operator, with the parameters of the Sec. III.B example (xi_0 = 2.464,
nu = 0.95, c_sw^t = 0.91, c_sw^r = 1.07, kappa from m0 = 0.3): the full operator in
every precision, the Schur operator through the multi-RHS, staged and tensor-core
kernels, solves whose true residual the oracle recomputes, and the isotropic case."""
import numpy as np
import pytest

import workloads as W
from oracle import dirac
from oracle import lattice as L

from _gpu import TOL, built, cuda, host, relerr

pytestmark = pytest.mark.gpu

XI0, NU, CSW_T, CSW_R, M0 = 2.464, 0.95, 0.91, 1.07, 0.3
SHAPES = [(4, 4, 4, 8), (6, 4, 2, 6), (8, 8, 8, 16)]


@pytest.fixture(scope="module")
def pkg():
    return built()


def _setup(pkg, dims, seed=0, tb=-1):
    kappa = pkg.wcl_kappa_from_mass_aniso(M0, XI0, NU)
    assert kappa == pytest.approx(dirac.kappa_of_mass(M0, XI0, NU), rel=1e-15)
    gauge = W.gauge_links(dims, 0.3, seed)
    ctx = pkg.Context(dims, t_boundary=tb)
    ctx.wcl_load_gauge_aniso(cuda(gauge), kappa, XI0, NU, CSW_T, CSW_R)
    op = dirac.anisotropic(L.gauge_from_qdp(gauge, dims), kappa, XI0, NU, CSW_T, CSW_R, tb)
    return ctx, op, gauge


@pytest.mark.parametrize("prec", ["f64", "df64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("dims", SHAPES[:2])
@pytest.mark.parametrize("tb", [-1, 1])
def test_apply_D(pkg, dims, prec, tb):
    ctx, op, _ = _setup(pkg, dims, seed=1, tb=tb)
    psi = W.gaussian_fermion(dims, 2)
    out = cuda(np.zeros_like(psi))
    ctx.wcl_apply_D(out, cuda(psi), prec)
    assert relerr(host(out), dirac.apply_D_qdp(op, psi)) <= TOL[prec]
    ctx.close()


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
@pytest.mark.parametrize("dagger", [False, True])
@pytest.mark.parametrize("variant", ["tuned", "per_thread", "staged", "tensor_cores"])
def test_apply_Mpc_multi_rhs(pkg, prec, dagger, variant):
    from paper_2411_08461_gb300.wcl import (WCL_OPT_AUTOTUNE, WCL_OPT_SHARED_LINKS, WCL_OPT_STAGED_SPINORS,
                                            WCL_OPT_TENSOR_CORES)

    if variant == "tensor_cores" and prec != "f16":
        pytest.skip("the tensor-core kernel stores 16-bit fields")
    dims = SHAPES[2]
    ctx, op, _ = _setup(pkg, dims, seed=3)
    if variant != "tuned":
        ctx.wcl_set_option(WCL_OPT_AUTOTUNE, 0)
        ctx.wcl_set_option(WCL_OPT_SHARED_LINKS, 0 if variant == "per_thread" else 16)
        ctx.wcl_set_option(WCL_OPT_STAGED_SPINORS, int(variant == "staged"))
        ctx.wcl_set_option(WCL_OPT_TENSOR_CORES, int(variant == "tensor_cores"))
    nrhs = 8
    psi = W.gaussian_fermion(dims, 4, nrhs=nrhs)[:, 0].copy()
    out = cuda(np.zeros_like(psi))
    ctx.wcl_apply_Mpc(out, cuda(psi), prec, nrhs=nrhs, dagger=dagger)
    got = host(out)
    for k in range(nrhs):
        assert relerr(got[k], dirac.apply_Mhat_qdp(op, psi[k], dagger)) <= TOL[prec], (k, variant)
    ctx.close()


@pytest.mark.parametrize("solver,sloppy,tol", [("bicgstab", "f32", 1e-10), ("bicgstab", "f64", 1e-12),
                                               ("cgnr", "f64", 1e-10)])
def test_solve_true_residual(pkg, solver, sloppy, tol):
    dims = SHAPES[0]
    ctx, op, _ = _setup(pkg, dims, seed=5)
    b = np.stack([W.point_source(dims, s, c) for s in range(4) for c in range(3)])
    x = cuda(np.zeros_like(b))
    prm = pkg.wcl_default_params(solver=solver, sloppy=sloppy, tol=tol)
    _, info = ctx.wcl_invert(x, cuda(b), 12, prm)
    xh = host(x)
    for k in (0, 5, 11):
        assert info[k]["status"] == 0
        r = op.true_residual(L.from_qdp(xh[k], dims), L.from_qdp(b[k], dims))
        assert r <= tol, (k, r, info[k])
    ctx.close()


def test_isotropic_parameters_match_the_isotropic_loader(pkg):
    """xi0 = nu = 1 and c_sw^t = c_sw^r = c_sw give the same bits as wcl_load_gauge."""
    dims = SHAPES[1]
    gauge = cuda(W.gauge_links(dims, 0.3, 7))
    psi = cuda(W.gaussian_fermion(dims, 8))
    outs = []
    for aniso in (False, True):
        ctx = pkg.Context(dims)
        if aniso:
            ctx.wcl_load_gauge_aniso(gauge, 0.12, 1.0, 1.0, 1.3, 1.3)
        else:
            ctx.wcl_load_gauge(gauge, 0.12, 1.3)
        for prec in ("f64", "f32"):
            out = cuda(np.zeros_like(host(psi)))
            ctx.wcl_apply_D(out, psi, prec)
            outs.append(host(out))
        ctx.close()
    assert np.array_equal(outs[0], outs[2]) and np.array_equal(outs[1], outs[3])


def test_invalid_anisotropy(pkg):
    dims = SHAPES[0]
    ctx = pkg.Context(dims)
    gauge = cuda(W.gauge_links(dims, 0.3, 0))
    for bad in ((0.1, 0.0, 1.0, 1.0, 1.0), (0.1, 2.0, -1.0, 1.0, 1.0), (float("nan"), 2.0, 1.0, 1.0, 1.0)):
        with pytest.raises(pkg.WclError):
            ctx.wcl_load_gauge_aniso(gauge, *bad)
    with pytest.raises(pkg.WclError):
        pkg.wcl_kappa_from_mass_aniso(-5.0, 1.0, 1.0)
    ctx.close()
