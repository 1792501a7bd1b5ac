"""Pins for the oracle's HISQ link smearing, oracle/hisq.py.

The abelian-flux test fixes every coefficient and path count of both smearing levels:
with links diag(e^{i phi}, e^{-i phi}, 1) carrying a constant flux B per plaquette in
the x-y plane only, every path of a link in that plane picks up the phase of the flux
it encloses, and the sums over paths have closed forms (derived in the test)."""
import numpy as np
import pytest

import workloads as W
from oracle import hisq as H
from oracle import lattice as L


def _eye(dims):
    lx, ly, lz, lt = dims
    return np.broadcast_to(np.eye(3), (4, lt, lz, ly, lx, 3, 3)).astype(np.complex128).copy()


def _thin(dims, eps, seed):
    return L.gauge_from_qdp(W.gauge_links(dims, eps, seed), dims)


@pytest.mark.parametrize("eps_naik", [0.0, -0.1])
def test_free_field(eps_naik):
    dims = (4, 4, 4, 6)
    one = _eye(dims)
    np.testing.assert_allclose(H.smear(one, H.FAT7), one, atol=1e-14)
    fat, long = H.hisq_links(one, eps_naik)
    np.testing.assert_allclose(fat, (9 + eps_naik) / 8 * one, atol=1e-14)
    np.testing.assert_allclose(long, -(1 + eps_naik) / 24 * one, atol=1e-14)


def test_commuting_constant_links():
    """Constant diagonal SU(3) links C_mu: every closed loop is 1, so each path equals C_mu
    and the smearing only rescales: fat7 gives C_mu, the projection keeps it, the second
    level gives 9/8 C_mu and the Naik link C_mu^3."""
    dims = (4, 6, 4, 4)
    th = np.array([[0.3, -0.7], [1.1, 0.2], [-0.4, 0.9], [0.5, 0.5]])
    C = np.stack([np.diag(np.exp(1j * np.array([a, b, -a - b]))) for a, b in th])
    U = np.broadcast_to(C[:, None, None, None, None], (4,) + tuple(dims[::-1]) + (3, 3)).copy()
    np.testing.assert_allclose(H.smear(U, H.FAT7), U, atol=1e-14)
    fat, long = H.hisq_links(U)
    np.testing.assert_allclose(fat, 9 / 8 * U, atol=1e-14)
    np.testing.assert_allclose(long, -1 / 24 * (U @ U @ U), atol=1e-14)


def _flux_links(dims, k):
    """U_y(x) = diag(e^{iBx}, e^{-iBx}, 1), B = 2 pi k / Lx, other links 1: every x-y
    plaquette is diag(e^{iB}, e^{-iB}, 1), all other plaquettes 1."""
    lx, ly, lz, lt = dims
    B = 2 * np.pi * k / lx
    U = _eye(dims)
    x = np.arange(lx)
    ph = np.stack([np.exp(1j * B * x), np.exp(-1j * B * x), np.ones(lx)], axis=-1)  # (Lx, 3)
    U[1] = ph[None, None, None, :, :, None] * np.eye(3)
    return U, np.array([B, -B, 0.0])


@pytest.mark.parametrize("k", [1, 2])
def test_abelian_flux_closed_form(k):
    """Links mu = x, y of the x-y plane: the one 3-staple pair in the plane encloses
    +-B (2 cos B), the other four are flat; of the 24 5-staples, 16 enclose +-B and 8 none;
    all 48 7-staples enclose +-B; the two in-plane Lepage staples enclose +-2B.  So
        fat7:   1/8 + (2 cos B + 4)/16 + (16 cos B + 8)/64 + 48 cos B / 384 = (1 + cos B)/2
        second: 5/8 + (2 cos B + 4)/16 + (16 cos B + 8)/64 + 48 cos B / 384
                - (2 cos 2B + 4)/16 = 3/4 + cos B / 2 - cos(2B) / 8
    per colour (B, -B, 0).  The fat7 links are positive multiples of U, so the U(3)
    projection returns U.  Links z, t: every path is flat (fat7 1, second level 9/8).
    Naik: N_y(x) = U_y(x)^3, N_x = 1."""
    dims = (6, 4, 4, 4)
    U, Bc = _flux_links(dims, k)
    V = H.smear(U, H.FAT7)
    f7 = (1 + np.cos(Bc)) / 2
    for mu in (0, 1):
        np.testing.assert_allclose(V[mu], U[mu] * f7[None, :], atol=1e-13)  # diag scale per colour
    for mu in (2, 3):
        np.testing.assert_allclose(V[mu], U[mu], atol=1e-13)
    Wp = H.u3_project(V)
    np.testing.assert_allclose(Wp, U, atol=1e-13)
    fat, long = H.hisq_links(U)
    f2 = 0.75 + np.cos(Bc) / 2 - np.cos(2 * Bc) / 8
    for mu in (0, 1):
        np.testing.assert_allclose(fat[mu], U[mu] * f2[None, :], atol=1e-13)
    for mu in (2, 3):
        np.testing.assert_allclose(fat[mu], 9 / 8 * U[mu], atol=1e-13)
    np.testing.assert_allclose(long[1], -1 / 24 * (U[1] @ U[1] @ U[1]), atol=1e-13)
    np.testing.assert_allclose(long[0], -1 / 24 * U[0], atol=1e-13)


def _gauge_rotate(U, om, hops):
    """U_mu(x) -> om(x) U_mu(x) om(x + hops mu)^+."""
    out = np.empty_like(U)
    for mu in range(4):
        out[mu] = om @ U[mu] @ np.conj(np.swapaxes(H._shift(om, mu, hops), -1, -2))
    return out


@pytest.mark.parametrize("coeffs", [H.FAT7, H.ASQ])
def test_smearing_gauge_covariance(coeffs):
    """Every path runs from x to x + mu, so the smeared link transforms like U_mu(x); a
    path with a wrong end point or orientation breaks this."""
    dims = (4, 4, 2, 6)
    U = _thin(dims, 0.5, 3)
    om = W.random_su3(dims, 4)
    np.testing.assert_allclose(H.smear(_gauge_rotate(U, om, 1), coeffs), _gauge_rotate(H.smear(U, coeffs), om, 1),
                               atol=1e-12)


def test_hisq_links_gauge_covariance():
    dims = (4, 2, 4, 6)
    U = _thin(dims, 0.5, 5)
    om = W.random_su3(dims, 6)
    fat, long = H.hisq_links(U, -0.05)
    fr, lr = H.hisq_links(_gauge_rotate(U, om, 1), -0.05)
    np.testing.assert_allclose(fr, _gauge_rotate(fat, om, 1), atol=1e-12)
    np.testing.assert_allclose(lr, _gauge_rotate(long, om, 3), atol=1e-12)


def test_u3_projection_is_the_polar_factor():
    """W = V (V^+ V)^(-1/2) is the unitary factor of the polar decomposition, which the
    SVD V = A S B^+ gives independently as A B^+; it is unitary, leaves a unitary V
    unchanged and ignores a positive scale."""
    dims = (2, 2, 2, 4)
    lx, ly, lz, lt = dims
    V = _thin(dims, 0.6, 7) + 0.4 * W.gaussian_complex((4, lt, lz, ly, lx, 3, 3), 8)
    Wp = H.u3_project(V)
    A, _, Bh = np.linalg.svd(V)
    np.testing.assert_allclose(Wp, A @ Bh, atol=1e-12)
    eye = np.broadcast_to(np.eye(3), Wp.shape)
    np.testing.assert_allclose(np.conj(np.swapaxes(Wp, -1, -2)) @ Wp, eye, atol=1e-13)
    U = _thin(dims, 0.6, 9)
    np.testing.assert_allclose(H.u3_project(U), U, atol=1e-13)
    np.testing.assert_allclose(H.u3_project(2.5 * V), Wp, atol=1e-13)


def test_naik_link_paths():
    """N_mu(x) is the product of the three links from x to x + 3 mu, checked site by site
    with explicit coordinates on a lattice where 3 mu wraps around (L = 4)."""
    dims = (4, 4, 2, 4)
    lx, ly, lz, lt = dims
    U = _thin(dims, 0.5, 10)
    N = H.naik(U)
    rng = np.random.default_rng(11)
    for _ in range(12):
        t, z, y, x = (int(rng.integers(n)) for n in (lt, lz, ly, lx))
        for mu in range(4):
            c = [x, y, z, t]
            prod = np.eye(3, dtype=complex)
            for _k in range(3):
                prod = prod @ U[mu][c[3], c[2], c[1], c[0]]
                c[mu] = (c[mu] + 1) % dims[mu]
            np.testing.assert_allclose(N[mu][t, z, y, x], prod, atol=1e-13)
