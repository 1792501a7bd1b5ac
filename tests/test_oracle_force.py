"""Pins for the oracle's clover fermion force, oracle/force.py.

The force is the derivative of the action, so the pins differentiate the action
itself: central finite differences of S (dense solves) along random su(3) directions,
one term at a time (pseudofermion term, clover determinant term, both), on lattices with
extent-2 axes (forward and backward neighbours coincide) and without; the same along a
single link (catches a wrong site or offset that a sum over all links could average
away); gauge covariance; and the algebraic form of the result."""
import numpy as np
import pytest
from scipy.linalg import expm

import workloads as W
from oracle import dirac, force
from oracle import lattice as L


def _setup(dims, seed, kappa=0.12, csw=1.0, tb=-1):
    U = L.gauge_from_qdp(W.gauge_links(dims, 0.3, seed), dims)
    op = dirac.WilsonClover(U, kappa, csw, tb)
    rng = np.random.default_rng(seed + 100)
    shp = op.even.shape[:4] + (4, 3)
    phi = (rng.standard_normal(shp) + 1j * rng.standard_normal(shp)) * op.even
    return op, phi, rng


def _rotate(U, Q, e):
    out = np.empty_like(U)
    for idx in np.ndindex(U.shape[:5]):
        out[idx] = expm(e * Q[idx]) @ U[idx]
    return out


def _fd(op, phi, Q, logdet, eps=1e-4):
    def S(e):
        o = dirac.WilsonClover(_rotate(op.U, Q, e), op.kappa, op.csw, op.t_boundary)
        return force.action(o, phi, logdet)

    return (S(eps) - S(-eps)) / (2 * eps)


def _directional(F, Q):
    """<Q, F> = -sum Tr(Q F): the predicted dS/d eps."""
    return -float(np.real(np.einsum("...ab,...ba->...", Q, F).sum()))


def _su3_field(rng, shape):
    q = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return force.traceless_antihermitian(q)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 2, 4)])
@pytest.mark.parametrize("logdet", [False, True])
def test_force_is_the_derivative_of_the_action(dims, logdet):
    op, phi, rng = _setup(dims, 1)
    X = force.solve_normal(op, phi)
    F = force.clover_force(op, X, logdet)
    Q = _su3_field(rng, op.U.shape)
    fd = _fd(op, phi, Q, logdet)
    assert abs(_directional(F, Q) - fd) <= 2e-6 * abs(fd), (_directional(F, Q), fd)


def test_determinant_term_alone():
    """phi = 0: S = -2 sum_odd log det A, X = 0; the force is the determinant term's."""
    op, phi, rng = _setup((2, 2, 2, 4), 2, kappa=0.13, csw=1.3)
    phi = np.zeros_like(phi)
    F = force.clover_force(op, np.zeros_like(phi), True)
    Q = _su3_field(rng, op.U.shape)
    fd = _fd(op, phi, Q, True)
    assert abs(fd) > 1e-3
    assert abs(_directional(F, Q) - fd) <= 2e-6 * abs(fd)
    assert np.abs(force.clover_force(op, np.zeros_like(phi), False)).max() == 0.0


@pytest.mark.parametrize("tb", [-1, 1])
def test_single_link_variations(tb):
    """One link at a time, in every direction, at sites of both parities and on the time
    boundary."""
    dims = (2, 4, 2, 4)
    op, phi, rng = _setup(dims, 3, tb=tb)
    X = force.solve_normal(op, phi)
    F = force.clover_force(op, X, True)
    lx, ly, lz, lt = dims
    for mu, site in [(0, (0, 0, 0, 0)), (1, (3, 1, 2, 1)), (2, (1, 1, 3, 0)), (3, (3, 0, 1, 1)), (3, (0, 1, 0, 0))]:
        Q = np.zeros(op.U.shape, dtype=np.complex128)
        Q[(mu,) + site] = _su3_field(rng, (3, 3))
        fd = _fd(op, phi, Q, True)
        pred = _directional(F, Q)
        assert abs(pred - fd) <= 2e-6 * max(abs(fd), 1e-3), (mu, site, pred, fd)


def test_gauge_covariance():
    """U_mu(x) -> g(x) U_mu(x) g(x + mu)^+, phi -> g phi: F_mu(x) -> g(x) F_mu(x) g(x)^+."""
    dims = (4, 2, 2, 4)
    op, phi, rng = _setup(dims, 4)
    X = force.solve_normal(op, phi)
    F = force.clover_force(op, X, True)
    lx, ly, lz, lt = dims
    G = np.empty((lt, lz, ly, lx, 3, 3), dtype=np.complex128)
    for idx in np.ndindex(G.shape[:4]):
        G[idx] = expm(_su3_field(rng, (3, 3)))
    Ug = np.empty_like(op.U)
    for mu in range(4):
        Ug[mu] = np.einsum("...ab,...bc,...dc->...ad", G, op.U[mu], np.conj(L.fwd(G, mu)))
    phig = np.einsum("...ab,...sb->...sa", G, phi)
    opg = dirac.WilsonClover(Ug, op.kappa, op.csw, op.t_boundary)
    Fg = force.clover_force(opg, force.solve_normal(opg, phig), True)
    want = np.einsum("...ab,...bc,...dc->...ad", G[None], F, np.conj(G[None]))
    np.testing.assert_allclose(Fg, want, atol=1e-10 * np.abs(F).max())


def test_force_is_traceless_antihermitian():
    op, phi, _ = _setup((2, 2, 2, 2), 5)
    F = force.clover_force(op, force.solve_normal(op, phi), True)
    np.testing.assert_allclose(F, -np.conj(np.swapaxes(F, -1, -2)), atol=1e-13)
    np.testing.assert_allclose(np.trace(F, axis1=-2, axis2=-1), 0, atol=1e-13)
