"""Pins for the oracle's solvers: dense brute force and the free-field momentum-space propagator."""
import numpy as np
import pytest

import workloads as W
from oracle import dirac, solvers
from oracle import lattice as L
from oracle.gamma import GAMMA

from _dense_ref import dense_matrix


def _problem(dims, eps, seed, kappa, csw):
    U = L.gauge_from_qdp(W.gauge_links(dims, eps, seed), dims)
    return U, dirac.WilsonClover(U, kappa, csw)


@pytest.mark.parametrize("method", ["bicgstab", "cgnr"])
@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4)])
def test_even_odd_solve_matches_dense(dims, method):
    kappa, csw = 0.12, 1.0
    U, op = _problem(dims, 0.2, 0, kappa, csw)
    b = L.from_qdp(W.point_source(dims, 0, 0), dims)
    x, info = solvers.solve_even_odd(op, b, method=method, tol=1e-12)
    assert info["status"] == "ok"
    assert info["true_residual"] <= 1e-12
    M = dense_matrix(U, dims, kappa, csw)
    xd = np.linalg.solve(M, b.ravel())
    assert np.linalg.norm(x.ravel() - xd) <= 1e-10 * np.linalg.norm(xd)


def test_gcr_monotone_and_fgcr_with_preconditioner():
    dims = (4, 2, 2, 4)
    U, op = _problem(dims, 0.4, 4, 0.115, 1.0)
    b = L.from_qdp(W.gaussian_fermion(dims, 5), dims)
    res = []

    def A(v):
        return op.M(v)

    x, info = solvers.fgcr(A, b, tol=1e-11, nkrylov=8)
    assert info["status"] == "ok" and op.true_residual(x, b) < 2e-11
    # GCR residual never increases: rerun step by step and record ||r||
    for k in range(1, 30):
        xk, _ = solvers.fgcr(A, b, tol=0.0, maxiter=k, nkrylov=8)
        res.append(np.linalg.norm(b - A(xk)))
    assert all(r2 <= r1 * (1 + 1e-12) for r1, r2 in zip(res, res[1:]))
    # flexible variant with the clover inverse as preconditioner converges to the same x
    xp, infop = solvers.fgcr(A, b, precond=lambda r: dirac.apply_site_matrix(op.Ainv, r), tol=1e-11, nkrylov=8)
    assert infop["status"] == "ok"
    assert np.linalg.norm(xp - x) <= 1e-9 * np.linalg.norm(x)


def test_free_field_propagator_fft():
    """With unit links the solution is known in momentum space:
    M(p)^-1 = (a - i b.gamma)/(a^2 + b^2), a = 1 - 2 kappa sum cos p, b_mu = 2 kappa sin p_mu,
    with p_t shifted by pi/Lt for the antiperiodic time boundary."""
    dims = (4, 4, 2, 8)
    lx, ly, lz, lt = dims
    kappa = 0.124
    U = L.gauge_from_qdp(W.unit_gauge(dims), dims)
    op = dirac.WilsonClover(U, kappa, 1.0)
    b = L.from_qdp(W.gaussian_fermion(dims, 3), dims)
    t = np.arange(lt)[:, None, None, None, None, None]
    twist = np.exp(1j * np.pi * t / lt)
    bt = np.fft.fftn(b / twist, axes=(0, 1, 2, 3))
    kt, kz, ky, kx = np.meshgrid(np.fft.fftfreq(lt), np.fft.fftfreq(lz), np.fft.fftfreq(ly), np.fft.fftfreq(lx), indexing="ij")
    p = [2 * np.pi * kx, 2 * np.pi * ky, 2 * np.pi * kz, 2 * np.pi * kt + np.pi / lt]
    a = 1 - 2 * kappa * sum(np.cos(q) for q in p)
    bg = sum(2 * kappa * np.sin(p[m])[..., None, None] * GAMMA[m] for m in range(4))
    minv = (a[..., None, None] * np.eye(4) - 1j * bg) / (a ** 2 + sum((2 * kappa * np.sin(q)) ** 2 for q in p))[..., None, None]
    xf = np.fft.ifftn(np.einsum("...st,...tc->...sc", minv, bt), axes=(0, 1, 2, 3)) * twist
    x, info = solvers.solve_even_odd(op, b, tol=1e-12)
    assert info["true_residual"] <= 1e-12
    assert np.linalg.norm(x - xf) <= 1e-10 * np.linalg.norm(xf)
    assert op.true_residual(xf, b) < 1e-13
