"""Pins for the oracle's staggered (HISQ-form) operator, oracle/staggered.py."""
import numpy as np
import pytest

import workloads as W
from oracle import lattice as L
from oracle import staggered as S


def _links(dims, seed, scale=1.0):
    """Generic (not unitary) link matrices: HISQ fat and long links are not SU(3)."""
    lx, ly, lz, lt = dims
    return scale * W.gaussian_complex((4, lt, lz, ly, lx, 3, 3), seed)


def _field(dims, seed):
    lx, ly, lz, lt = dims
    return W.gaussian_complex((lt, lz, ly, lx, 3), seed)


def test_anti_hermitian():
    dims = (4, 4, 4, 6)
    V, Wl = _links(dims, 1), _links(dims, 2, 0.1)
    phi, chi = _field(dims, 3), _field(dims, 4)
    for tb in (-1, 1):
        lhs = np.vdot(phi, S.dslash(V, Wl, chi, tb))
        rhs = -np.vdot(S.dslash(V, Wl, phi, tb), chi)
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)


@pytest.mark.parametrize("n", [(0, 0, 0, 0), (1, 2, 0, 1), (3, 1, 2, 2)])
def test_free_field_symbol(n):
    """Unit links scaled by c1 (one hop) and c3 (three hops): D^2 e^{ipx} =
    -sum_mu (2 c1 sin p_mu + 2 c3 sin 3 p_mu)^2 e^{ipx}, p_t twisted by the antiperiodic
    boundary."""
    dims = (8, 6, 6, 8)
    lx, ly, lz, lt = dims
    c1, c3 = 9.0 / 8.0, -1.0 / 24.0
    eye = np.broadcast_to(np.eye(3), (4, lt, lz, ly, lx, 3, 3)).astype(np.complex128)
    p = [2 * np.pi * n[0] / lx, 2 * np.pi * n[1] / ly, 2 * np.pi * n[2] / lz, (2 * np.pi * n[3] + np.pi) / lt]
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    u = np.array([1.0, 2.0 - 1j, 0.5j])
    chi = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))[..., None] * u
    d2 = S.dslash(c1 * eye, c3 * eye, S.dslash(c1 * eye, c3 * eye, chi))
    sym = -sum((2 * c1 * np.sin(q) + 2 * c3 * np.sin(3 * q)) ** 2 for q in p)
    np.testing.assert_allclose(d2, sym * chi, atol=1e-12)


def test_gauge_covariance():
    dims = (4, 4, 4, 4)
    V, Wl = _links(dims, 5), _links(dims, 6, 0.2)
    om = W.random_su3(dims, 7)
    Vo = np.einsum("...ab,m...bc,m...dc->m...ad", om, V, np.stack([S._shift(om, mu, 1) for mu in range(4)]).conj())
    Wo = np.einsum("...ab,m...bc,m...dc->m...ad", om, Wl, np.stack([S._shift(om, mu, 3) for mu in range(4)]).conj())
    chi = _field(dims, 8)
    rot = lambda f: np.einsum("...ab,...b->...a", om, f)
    np.testing.assert_allclose(S.dslash(Vo, Wo, rot(chi)), rot(S.dslash(V, Wl, chi)), atol=1e-12)


def _dense(V, Wl, dims, mass, tb):
    """Loop-built 3V x 3V matrix of M = 2m + D, site index ((t*Lz + z)*Ly + y)*Lx + x."""
    lx, ly, lz, lt = dims
    ext = (lx, ly, lz, lt)
    vol = lx * ly * lz * lt
    idx = lambda c: ((c[3] * lz + c[2]) * ly + c[1]) * lx + c[0]
    M = 2 * mass * np.eye(3 * vol, dtype=np.complex128)
    for t in range(lt):
        for z in range(lz):
            for y in range(ly):
                for x in range(lx):
                    c = (x, y, z, t)
                    eta = (1, (-1) ** x, (-1) ** (x + y), (-1) ** (x + y + z))
                    i = idx(c)
                    for mu in range(4):
                        for links, hop in ((V, 1), (Wl, 3)):
                            f = list(c)
                            f[mu] += hop
                            b = list(c)
                            b[mu] -= hop
                            sf = tb if (mu == 3 and (f[3] >= lt)) else 1
                            sb = tb if (mu == 3 and (b[3] < 0)) else 1
                            f = [f[k] % ext[k] for k in range(4)]
                            b = [b[k] % ext[k] for k in range(4)]
                            uf = links[mu][c[3], c[2], c[1], c[0]]
                            ub = links[mu][b[3], b[2], b[1], b[0]].conj().T
                            M[3 * i:3 * i + 3, 3 * idx(f):3 * idx(f) + 3] += eta[mu] * sf * uf
                            M[3 * i:3 * i + 3, 3 * idx(b):3 * idx(b) + 3] -= eta[mu] * sb * ub
    return M


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (4, 2, 4, 6)])
def test_dense_matrix_and_cg_solve(dims):
    V, Wl = _links(dims, 9, 0.5), _links(dims, 10, 0.1)
    mass = 0.2
    op = S.Staggered(V, Wl, mass)
    M = _dense(V, Wl, dims, mass, -1)
    chi = _field(dims, 11)
    np.testing.assert_allclose(op.M(chi).ravel(), M @ chi.ravel(), atol=1e-12)
    x, info = op.solve(chi, tol=1e-12)
    assert info["status"] == "ok"
    np.testing.assert_allclose(x.ravel(), np.linalg.solve(M, chi.ravel()), atol=1e-9)


def test_hops_change_parity():
    """Both the one- and three-site hops connect opposite parities (the even-odd form)."""
    dims = (4, 4, 4, 6)
    V, Wl = _links(dims, 12), _links(dims, 13)
    even = L.parity_mask(dims, 0)[..., None]
    chi = _field(dims, 14) * even
    out = S.dslash(V, Wl, chi)
    assert np.abs(out * even).max() == 0
