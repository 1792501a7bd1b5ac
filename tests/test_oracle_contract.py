"""Pins for the oracle's propagator workflow (oracle/contract.py).

The dense inverse of the loop-built matrix in _dense_ref gives every point-to-point
propagator S(x; y) directly, so the correlators can be evaluated from the lines of
Eq. 1 and Eq. 3 / Eq. 4 as printed (sums over source points, the backward
propagator S(x0; x) taken from the inverse, no gamma_5-hermiticity) and compared with
the oracle's wall-source solves and Eq. 6 / Eq. 7 contractions."""
import numpy as np
import pytest

import workloads as W
from oracle import contract as C
from oracle import dirac
from oracle import gamma as G
from oracle import lattice as L

from _dense_ref import dense_matrix, site_index

DIMS = (4, 2, 4, 4)
KAPPA, CSW = 0.12, 1.0


def _coords(dims):
    lx, ly, lz, lt = dims
    return [(x, y, z, t) for t in range(lt) for z in range(lz) for y in range(ly) for x in range(lx)]


@pytest.fixture(scope="module")
def problem():
    U = L.gauge_from_qdp(W.gauge_links(DIMS, 0.4, 5), DIMS)
    op = dirac.WilsonClover(U, KAPPA, CSW)
    Minv = np.linalg.inv(dense_matrix(U, DIMS, KAPPA, CSW))
    return U, op, Minv


def _S(Minv, x, y):
    """12 x 12 block S(x; y) with compound (spin, colour) indices, 3 * spin + colour."""
    i, j = site_index(x, DIMS) * 12, site_index(y, DIMS) * 12
    return Minv[i:i + 12, j:j + 12]


def _p_dot(mom, c):
    lx, ly, lz, _ = DIMS
    return 2 * np.pi * (mom[0] * c[0] / lx + mom[1] * c[1] / ly + mom[2] * c[2] / lz)


def _g5_12():
    return np.kron(G.GAMMA5, np.eye(3))


def test_momentum_phase_plane_waves():
    """Plane waves of distinct integer modes are orthogonal over a timeslice, and a
    mode shifted by the lattice extent is the same wave."""
    lx, ly, lz, _ = DIMS
    modes = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 3), (3, 0, 2)]
    for n in modes:
        for m in modes:
            s = np.sum(C.momentum_phase(DIMS, n)[0] * np.conj(C.momentum_phase(DIMS, m)[0]))
            assert abs(s - (lx * ly * lz if n == m else 0)) < 1e-12
    np.testing.assert_allclose(C.momentum_phase(DIMS, (1 + lx, 1, 2 + lz)), C.momentum_phase(DIMS, (1, 1 - ly, 2)),
                               atol=1e-12)
    assert np.allclose(C.momentum_phase(DIMS, (0, 0, 0)), 1)


def test_propagator_layout_round_trip():
    x12 = np.random.default_rng(0).standard_normal((12, 2, 2, 2, 2, 4, 3)) + 0j
    S = C.fermions_to_propagator(x12)
    assert S[1, 0, 1, 0, 2, 3, 1, 2] == x12[3 * 3 + 2][1, 0, 1, 0, 2, 1]
    np.testing.assert_array_equal(C.propagator_to_fermions(S), x12)


def test_point_source_two_point_eq1_second_line(problem):
    """Point source at x0: the oracle's contraction of the forward propagator with
    itself equals Eq. 1's second line, Tr[S(x0; x) g5 S(x; x0) g5], with the backward
    propagator S(x0; x) read from the dense inverse."""
    U, op, Minv = problem
    x0, mom = (1, 1, 2, 1), (1, 0, 1)
    S = C.propagator(op, C.point_sources(DIMS, x0), tol=1e-13)
    Sp = S * np.exp(1j * _p_dot(mom, x0))
    got = C.two_point(S, Sp, mom)
    g5 = _g5_12()
    ref = np.zeros(DIMS[3], dtype=np.complex128)
    for x in _coords(DIMS):
        ref[x[3]] += np.exp(-1j * _p_dot(mom, x)) * np.exp(1j * _p_dot(mom, x0)) * np.trace(
            _S(Minv, x0, x) @ g5 @ _S(Minv, x, x0) @ g5)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-10 * np.abs(ref).max())


def test_wall_source_two_point_eq1_third_line(problem):
    """Wall sources (zero and nonzero momentum): Eq. 6 on the oracle's propagators
    equals the double sum over source points x0, x0' of Eq. 1's third line."""
    U, op, Minv = problem
    t0, mom = 1, (0, 0, 1)
    S0 = C.propagator(op, C.wall_sources(DIMS, t0), tol=1e-13)
    Sp = C.propagator(op, C.wall_sources(DIMS, t0, mom), tol=1e-13)
    got = C.two_point(S0, Sp, mom)
    wall = [c for c in _coords(DIMS) if c[3] == t0]
    ref = np.zeros(DIMS[3], dtype=np.complex128)
    for x in _coords(DIMS):
        s0 = sum(_S(Minv, x, y) for y in wall)  # sum over x0' (zero-momentum wall)
        sp = sum(np.exp(1j * _p_dot(mom, y)) * _S(Minv, x, y) for y in wall)
        ref[x[3]] += np.exp(-1j * _p_dot(mom, x)) * np.sum(np.conj(s0) * sp)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-10 * np.abs(ref).max())


def test_three_point_eq3_eq4(problem):
    """Sequential source, its twelve inversions and Eq. 7 on the oracle, against Eq. 4
    evaluated with the dense inverse (S(x1; x) g5 S_0(x) summed over the sink
    timeslice) contracted as in Eq. 3."""
    U, op, Minv = problem
    t0, t, mom = 0, 2, (1, 0, 1)
    S0 = C.propagator(op, C.wall_sources(DIMS, t0), tol=1e-13)
    Sp = C.propagator(op, C.wall_sources(DIMS, t0, mom), tol=1e-13)
    X = C.sequential_source(S0, t, mom)
    assert np.all(X[:t] == 0) and np.all(X[t + 1:] == 0)
    Sseq = C.propagator(op, C.propagator_to_fermions(X), tol=1e-13)
    got = C.three_point(Sseq, Sp)

    g5 = _g5_12()
    gins = np.kron(G.GAMMA5 @ G.GAMMA[2], np.eye(3))
    wall = [c for c in _coords(DIMS) if c[3] == t0]
    sink = [c for c in _coords(DIMS) if c[3] == t]
    s0 = {x: sum(_S(Minv, x, y) for y in wall) for x in sink}
    sp_wall = lambda x1: sum(np.exp(1j * _p_dot(mom, y)) * _S(Minv, x1, y) for y in wall)
    ref = np.zeros(DIMS[3], dtype=np.complex128)
    for x1 in _coords(DIMS):
        seq = sum(np.exp(-1j * _p_dot(mom, x)) * _S(Minv, x1, x) @ g5 @ s0[x] for x in sink)
        # Eq. 3: sum_{j,k,i,a,b} conj(seq)[j b, i a] (g5 g3)_{jk} S_p[k b, i a] = Tr[seq^+ G S_p]
        ref[x1[3]] += np.trace(seq.conj().T @ gins @ sp_wall(x1))
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-10 * np.abs(ref).max())


def test_point_two_point_gauge_invariant_and_positive(problem):
    """At zero momentum the point-source correlator is sum |S|^2: real, positive and
    unchanged by a random SU(3) gauge transformation of the links."""
    U, op, _ = problem
    x0 = (0, 1, 3, 2)
    c = C.two_point(*(2 * [C.propagator(op, C.point_sources(DIMS, x0), tol=1e-13)]), (0, 0, 0))
    omega = W.random_su3(DIMS, 11)
    Uo = np.empty_like(U)
    for mu in range(4):
        Uo[mu] = np.einsum("...ab,...bc,...dc->...ad", omega, U[mu], L.fwd(omega, mu).conj())
    So = C.propagator(dirac.WilsonClover(Uo, KAPPA, CSW), C.point_sources(DIMS, x0), tol=1e-13)
    co = C.two_point(So, So, (0, 0, 0))
    assert np.all(np.abs(c.imag) <= 1e-14 * np.abs(c)) and np.all(c.real > 0)
    np.testing.assert_allclose(co, c, rtol=1e-10)


def test_contract_gamma_structure():
    """Eq. 7's Gamma placement: for propagators that are spin matrices times a common
    colour-site factor, the contraction reduces to Tr[A_s^+ Gamma B_s] of the 4 x 4
    spin matrices; a transposed Gamma or a swapped spin axis changes the result."""
    rng = np.random.default_rng(4)
    As = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    Bs = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    f = rng.standard_normal((2, 2, 2, 2, 3, 3)) + 1j * rng.standard_normal((2, 2, 2, 2, 3, 3))
    A = np.einsum("ji,...ba->...jiba", As, f)
    B = np.einsum("ji,...ba->...jiba", Bs, f)
    colour = np.sum(np.abs(f) ** 2, axis=(-2, -1)).sum(axis=(1, 2, 3))
    for gm in [G.gamma(15) @ G.gamma(4)] + [G.gamma(n) for n in range(16)]:
        got = C.contract(A, B, gm)
        np.testing.assert_allclose(got, np.trace(As.conj().T @ gm @ Bs) * colour, rtol=1e-13)
        assert not np.allclose(got, np.trace(As.conj().T @ gm @ Bs.T) * colour)
        if not np.allclose(gm, gm.T):
            assert not np.allclose(got, np.trace(As.conj().T @ gm.T @ Bs) * colour)
