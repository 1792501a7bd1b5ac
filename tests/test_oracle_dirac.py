"""Pins for the oracle's Wilson-clover operator (Eq. 5, isotropic; Sec. II.A layouts).

Each test checks the oracle against something other than itself: a closed form,
an identity the operator must satisfy, or the loop-built dense matrix.
"""
import numpy as np
import pytest

import workloads as W
from oracle import dirac
from oracle import lattice as L
from oracle.gamma import GAMMA, GAMMA5, sigma

from _dense_ref import dense_matrix, parity_indices


def _rand_fermion(dims, seed):
    return L.from_qdp(W.gaussian_fermion(dims, seed), dims)


# --- layout ------------------------------------------------------------------

def test_qdp_roundtrip_and_parity():
    dims = (4, 2, 6, 4)
    q = W.gaussian_fermion(dims, 5)
    lex = L.from_qdp(q, dims)
    np.testing.assert_array_equal(L.to_qdp(lex, dims), q)
    # a point source at (x,y,z,t) = (3,1,2,1): parity 1, cb index ((1*6+2)*2+1)*2 + 1
    ps = W.point_source(dims, 2, 1, site=(3, 1, 2, 1))
    assert ps[1, 1, 2, 1, 1, 2, 1] == 1.0
    assert L.from_qdp(ps, dims)[1, 2, 1, 3, 2, 1] == 1.0


# --- free field: plane waves are eigenvectors with the closed-form symbol ------

@pytest.mark.parametrize("t_boundary", [-1, 1])
@pytest.mark.parametrize("n", [(0, 0, 0, 0), (1, 0, 2, 1), (1, 1, 1, 3)])
def test_free_field_plane_wave(n, t_boundary):
    dims = (4, 2, 6, 8)
    kappa, csw = 0.11, 1.3  # F = 0 on the free field, so the clover is the identity
    U = L.gauge_from_qdp(W.unit_gauge(dims), dims)
    op = dirac.WilsonClover(U, kappa, csw, t_boundary)
    lx, ly, lz, lt = dims
    p = [2 * np.pi * n[0] / lx, 2 * np.pi * n[1] / ly, 2 * np.pi * n[2] / lz,
         (2 * np.pi * n[3] + (np.pi if t_boundary == -1 else 0.0)) / lt]
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    rng = np.random.default_rng(1)
    u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    psi = phase[..., None, None] * u
    # M(p) = (1 - 2 kappa sum cos p) + 2 i kappa sum gamma_mu sin p_mu
    a = 1 - 2 * kappa * np.sum(np.cos(p))
    Mp = a * np.eye(4) + 2j * kappa * sum(GAMMA[m] * np.sin(p[m]) for m in range(4))
    expect = phase[..., None, None] * (Mp @ u)
    np.testing.assert_allclose(op.M(psi), expect, atol=1e-13)
    # eigenvalues a +- 2 i kappa sqrt(sum sin^2), each twice
    ev = np.linalg.eigvals(Mp)
    ev = ev[np.argsort(ev.imag)]
    b = 2 * kappa * np.sqrt(np.sum(np.sin(p) ** 2))
    np.testing.assert_allclose(ev, np.array([a - 1j * b] * 2 + [a + 1j * b] * 2), atol=1e-13)


# --- gamma5-hermiticity (Sec. III.A uses gamma5 S gamma5 = S^+) ------------------

def test_gamma5_hermiticity():
    dims = (4, 4, 2, 6)
    op = dirac.from_qdp_problem(W.gauge_links(dims, 0.5, 11), dims, 0.12, 1.7)
    phi, psi = _rand_fermion(dims, 1), _rand_fermion(dims, 2)
    lhs = np.vdot(phi, op.M(psi))
    rhs = np.vdot(dirac.gamma5(op.M(dirac.gamma5(phi))), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # the clover is Hermitian and commutes with gamma5
    np.testing.assert_allclose(op.A, np.conj(np.swapaxes(op.A, -1, -2)), atol=1e-15)
    g5 = np.kron(GAMMA5, np.eye(3))
    np.testing.assert_allclose(op.A @ g5, g5 @ op.A, atol=1e-15)
    # Schur operator: M_hat^+ = gamma5 M_hat gamma5
    xe, ye = phi * op.even, psi * op.even
    assert abs(np.vdot(xe, op.Mhat(ye)) - np.vdot(op.Mhat(xe, dagger=True), ye)) < 1e-12 * np.linalg.norm(xe) * np.linalg.norm(ye)


# --- gauge covariance --------------------------------------------------------

def _gauge_transform(U, omega):
    out = np.empty_like(U)
    for mu in range(4):
        out[mu] = np.einsum("...ab,...bc,...dc->...ad", omega, U[mu], L.fwd(omega, mu).conj())
    return out


def test_gauge_covariance():
    dims = (4, 2, 4, 4)
    U = L.gauge_from_qdp(W.gauge_links(dims, 0.6, 3), dims)
    omega = W.random_su3(dims, 9)
    Uo = _gauge_transform(U, omega)
    psi = _rand_fermion(dims, 4)
    op, opo = dirac.WilsonClover(U, 0.125, 1.1), dirac.WilsonClover(Uo, 0.125, 1.1)
    rot = lambda f: np.einsum("...ab,...sb->...sa", omega, f)
    np.testing.assert_allclose(opo.M(rot(psi)), rot(op.M(psi)), atol=1e-12)
    for mu, nu in dirac.PLANES:
        f, fo = dirac.field_strength(U, mu, nu), dirac.field_strength(Uo, mu, nu)
        np.testing.assert_allclose(fo, np.einsum("...ab,...bc,...dc->...ad", omega, f, omega.conj()), atol=1e-12)


# --- clover: abelian constant field closed form --------------------------------

@pytest.mark.parametrize("k", [1, 3])
def test_clover_abelian_constant_field(k):
    dims = (8, 4, 2, 4)
    lx = dims[0]
    B = 2 * np.pi * k / lx
    U = L.gauge_from_qdp(W.unit_gauge(dims), dims)
    x = np.arange(lx)[None, None, None, :]
    ph = np.exp(1j * B * x)
    U[1][..., 0, 0] = ph
    U[1][..., 1, 1] = ph
    U[1][..., 2, 2] = np.exp(-2j * B * x)
    # every xy plaquette is diag(e^{iB}, e^{iB}, e^{-2iB}); F_xy = (P - P^+)/2 minus trace/3
    d = np.array([np.sin(B), np.sin(B), -np.sin(2 * B)])
    d = d - d.sum() / 3
    Fxy = 1j * np.diag(d)
    for mu, nu in dirac.PLANES:
        f = dirac.field_strength(U, mu, nu)
        expect = Fxy if (mu, nu) == (0, 1) else np.zeros((3, 3))
        np.testing.assert_allclose(f, np.broadcast_to(expect, f.shape), atol=1e-14)
    kappa, csw = 0.13, 1.9
    A = dirac.clover_matrix(U, kappa, csw)
    expectA = np.eye(12) - kappa * csw * np.kron(sigma(0, 1), Fxy)
    np.testing.assert_allclose(A, np.broadcast_to(expectA, A.shape), atol=1e-14)


def test_clover_trivial_limits():
    dims = (4, 2, 2, 4)
    U = L.gauge_from_qdp(W.gauge_links(dims, 0.5, 2), dims)
    np.testing.assert_allclose(dirac.clover_matrix(U, 0.12, 0.0), np.broadcast_to(np.eye(12), (4, 2, 2, 4, 12, 12)), atol=0)
    U1 = L.gauge_from_qdp(W.unit_gauge(dims), dims)
    np.testing.assert_allclose(dirac.clover_matrix(U1, 0.12, 1.0), np.broadcast_to(np.eye(12), (4, 2, 2, 4, 12, 12)), atol=1e-15)


# --- dense brute force on 2^4 and a small 4^2 x 2^2 ----------------------------

@pytest.mark.parametrize("dims,t_boundary", [((2, 2, 2, 2), -1), ((4, 2, 2, 4), -1), ((2, 4, 2, 2), 1)])
def test_dense_matrix_matches(dims, t_boundary):
    Uq = W.gauge_links(dims, 0.7, 21)
    U = L.gauge_from_qdp(Uq, dims)
    kappa, csw = 0.12, 1.4
    op = dirac.WilsonClover(U, kappa, csw, t_boundary)
    M = dense_matrix(U, dims, kappa, csw, t_boundary)
    psi = _rand_fermion(dims, 7)
    np.testing.assert_allclose(op.M(psi).ravel(), M @ psi.ravel(), atol=1e-13)
    # Schur complement built from dense blocks vs the oracle's M_hat
    ie, io = parity_indices(dims, 0), parity_indices(dims, 1)
    Mee, Meo, Moe, Moo = M[np.ix_(ie, ie)], M[np.ix_(ie, io)], M[np.ix_(io, ie)], M[np.ix_(io, io)]
    Mhat = Mee - Meo @ np.linalg.solve(Moo, Moe)
    xe = psi * op.even
    np.testing.assert_allclose(op.Mhat(xe).ravel()[ie], Mhat @ xe.ravel()[ie], atol=1e-12)
    # dense solve of the full system vs Schur + BiCGStab, and the Schur source
    b = _rand_fermion(dims, 8)
    xs = np.linalg.solve(M, b.ravel())
    bhat = b.ravel()[ie] - Meo @ np.linalg.solve(Moo, b.ravel()[io])
    np.testing.assert_allclose(op.schur_source(b).ravel()[ie], bhat, atol=1e-12)
    xe_exact = np.linalg.solve(Mhat, bhat)
    np.testing.assert_allclose(xs[ie], xe_exact, atol=1e-11)
    full = np.zeros_like(psi).ravel()
    full[ie] = xe_exact
    np.testing.assert_allclose(op.reconstruct(full.reshape(psi.shape), b).ravel(), xs, atol=1e-11)


def test_site_by_site_evaluation_matches_whole_lattice():
    dims = (4, 2, 6, 4)
    gq = W.gauge_links(dims, 0.6, 17)
    psi_q = W.gaussian_fermion(dims, 18)
    op = dirac.from_qdp_problem(gq, dims, 0.127, 1.3)
    full = op.M(L.from_qdp(psi_q, dims))
    sites = [(0, 0, 0, 0), (3, 1, 5, 3), (1, 0, 2, 0), (2, 1, 0, 3)]
    vals = dirac.M_at_sites(gq, psi_q, dims, 0.127, 1.3, sites)
    for (x, y, z, t), v in zip(sites, vals):
        np.testing.assert_allclose(v, full[t, z, y, x], atol=1e-13)


@pytest.mark.parametrize("dagger", [False, True])
def test_site_by_site_schur_operator_matches_whole_lattice(dagger):
    """Mhat_at_sites (odd-site intermediates formed only where needed) equals the
    whole-lattice M_hat, including wrap-around sites and the antiperiodic t hop."""
    dims = (4, 2, 6, 4)
    gq = W.gauge_links(dims, 0.6, 19)
    xe = W.gaussian_fermion(dims, 20)[0]
    op = dirac.from_qdp_problem(gq, dims, 0.127, 1.3)
    full = np.zeros((2,) + xe.shape, dtype=np.complex128)
    full[0] = xe
    ref = op.Mhat(L.from_qdp(full, dims), dagger)
    sites = [(0, 0, 0, 0), (3, 1, 0, 0), (1, 0, 5, 0), (2, 1, 5, 2), (0, 1, 2, 3), (3, 0, 2, 3)]
    vals = dirac.Mhat_at_sites(gq, xe, dims, 0.127, 1.3, sites, dagger=dagger)
    for (x, y, z, t), v in zip(sites, vals):
        np.testing.assert_allclose(v, ref[t, z, y, x], atol=1e-13)


# --- slab-by-slab evaluation (oracle.residual) ----------------------------------

@pytest.mark.parametrize("dims,slab,t_boundary", [((4, 2, 6, 8), 3, -1), ((4, 2, 6, 8), 1, -1),
                                                  ((2, 4, 2, 6), 4, 1), ((4, 2, 2, 2), 1, -1)])
def test_slabwise_operator_matches_whole_lattice(dims, slab, t_boundary):
    """The slabs of oracle.residual put together equal WilsonClover.M: ragged last slab,
    one-timeslice slabs (halo rows on both sides are neighbours), Lt = 2 (both halo rows
    are the same timeslice), periodic and antiperiodic time."""
    from oracle import residual

    gq = W.gauge_links(dims, 0.6, 61)
    psi_q = W.gaussian_fermion(dims, 62)
    op = dirac.from_qdp_problem(gq, dims, 0.127, 1.3, t_boundary)
    full = op.M(L.from_qdp(psi_q, dims))
    got = np.concatenate([residual.M_slab(gq, psi_q, dims, 0.127, 1.3, t0, t1, t_boundary)
                          for t0, t1 in residual.slabs(dims[3], slab)])
    np.testing.assert_allclose(got, full, atol=1e-13)


def test_slabwise_anisotropic_operator_matches_whole_lattice():
    from oracle import residual

    dims = (4, 2, 2, 6)
    gq = W.gauge_links(dims, 0.6, 63)
    psi_q = W.gaussian_fermion(dims, 64)
    a = ANISO
    op = dirac.anisotropic(L.gauge_from_qdp(gq, dims), 0.11, a["xi0"], a["nu"], a["csw_t"], a["csw_r"])
    full = op.M(L.from_qdp(psi_q, dims))
    w = a["nu"] / a["xi0"]
    plane = [a["csw_t"] if nu == 3 else a["csw_r"] / a["xi0"] for _, nu in dirac.PLANES]
    got = np.concatenate([residual.M_slab(gq, psi_q, dims, 0.11, 0.0, t0, t1, -1, (w, w, w, 1.0), plane)
                          for t0, t1 in residual.slabs(dims[3], 4)])
    np.testing.assert_allclose(got, full, atol=1e-13)


@pytest.mark.parametrize("processes", [1, 2])
def test_slabwise_true_residuals(processes):
    """true_residuals equals the whole-array true_residual for several right-hand sides,
    serially and in a pool of spawned processes; b = M x gives zero."""
    from oracle import residual

    dims = (4, 4, 2, 6)
    gq = W.gauge_links(dims, 0.5, 65)
    op = dirac.from_qdp_problem(gq, dims, 0.12, 1.0)
    xs = W.gaussian_fermion(dims, 66, nrhs=3)
    bs = W.gaussian_fermion(dims, 67, nrhs=3)
    bs[2] = L.to_qdp(op.M(L.from_qdp(xs[2], dims)), dims)
    got = residual.true_residuals(gq, xs, bs, dims, 0.12, 1.0, slab=4, processes=processes)
    ref = [op.true_residual(L.from_qdp(x, dims), L.from_qdp(b, dims)) for x, b in zip(xs, bs)]
    np.testing.assert_allclose(got[:2], ref[:2], rtol=1e-12)
    assert got[2] <= 1e-14 and ref[2] <= 1e-14


# --- anisotropic form of Eq. 5 --------------------------------------------------

ANISO = dict(xi0=2.464, nu=0.95, csw_t=0.91, csw_r=1.07)  # the parameters of the Sec. III.B example


def test_anisotropic_reduces_to_isotropic():
    dims = (4, 2, 2, 4)
    U = L.gauge_from_qdp(W.gauge_links(dims, 0.5, 31), dims)
    psi = _rand_fermion(dims, 32)
    iso = dirac.WilsonClover(U, 0.12, 1.3)
    an = dirac.anisotropic(U, 0.12, 1.0, 1.0, 1.3, 1.3)
    np.testing.assert_allclose(an.M(psi), iso.M(psi), atol=1e-14)


@pytest.mark.parametrize("n", [(0, 0, 0, 0), (1, 0, 2, 1), (1, 1, 1, 3)])
def test_anisotropic_free_field_plane_wave(n):
    """Unit links: M e^{ipx} u = [1 - kappa sum_mu w_mu (2 cos p_mu - 2 i gamma_mu sin p_mu)] e^{ipx} u
    with w = nu/xi0 on the spatial directions and 1 on t."""
    dims = (4, 2, 6, 8)
    kappa = 0.09
    U = L.gauge_from_qdp(W.unit_gauge(dims), dims)
    op = dirac.anisotropic(U, kappa, **ANISO)
    lx, ly, lz, lt = dims
    p = [2 * np.pi * n[0] / lx, 2 * np.pi * n[1] / ly, 2 * np.pi * n[2] / lz, (2 * np.pi * n[3] + np.pi) / lt]
    w = [ANISO["nu"] / ANISO["xi0"]] * 3 + [1.0]
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    u = np.random.default_rng(3).standard_normal((4, 3)) + 0j
    Mp = (1 - 2 * kappa * sum(w[m] * np.cos(p[m]) for m in range(4))) * np.eye(4) + 2j * kappa * sum(
        w[m] * GAMMA[m] * np.sin(p[m]) for m in range(4))
    np.testing.assert_allclose(op.M(phase[..., None, None] * u), phase[..., None, None] * (Mp @ u), atol=1e-13)


def test_kappa_relation_massless_point():
    """kappa from m0 = 0 puts the free operator's zero-momentum mode at zero (periodic t)."""
    dims = (2, 2, 2, 4)
    U = L.gauge_from_qdp(W.unit_gauge(dims), dims)
    for xi0, nu in ((1.0, 1.0), (ANISO["xi0"], ANISO["nu"])):
        k0 = dirac.kappa_of_mass(0.0, xi0, nu)
        op = dirac.anisotropic(U, k0, xi0, nu, 1.0, 1.0, t_boundary=1)
        const = np.ones(op.dims[::-1] + (4, 3), dtype=np.complex128)
        assert np.abs(op.M(const)).max() < 1e-14
        m0 = 0.3
        k = dirac.kappa_of_mass(m0, xi0, nu)
        np.testing.assert_allclose(dirac.anisotropic(U, k, xi0, nu, 1.0, 1.0, 1).M(const), 2 * k * m0 * const,
                                   atol=1e-14)
    assert dirac.kappa_of_mass(0.0) == 0.125


@pytest.mark.parametrize("plane,coef_key", [((0, 1), "spatial"), ((0, 3), "temporal")])
def test_anisotropic_clover_abelian_field(plane, coef_key):
    """Constant abelian field in one plane: A = 1 - kappa c sigma (x) F with c = c_SW^r/xi0
    for a spatial plane and c_SW^t for a plane containing t."""
    mu, nu = plane
    dims = (8, 4, 2, 8)
    lmu = dims[mu]
    B = 2 * np.pi / lmu
    U = L.gauge_from_qdp(W.unit_gauge(dims), dims)
    coord = np.meshgrid(np.arange(dims[3]), np.arange(dims[2]), np.arange(dims[1]), np.arange(dims[0]),
                        indexing="ij")[3 - mu]
    U[nu][..., 0, 0] = np.exp(1j * B * coord)
    U[nu][..., 1, 1] = np.exp(1j * B * coord)
    U[nu][..., 2, 2] = np.exp(-2j * B * coord)
    d = np.array([np.sin(B), np.sin(B), -np.sin(2 * B)])
    F = 1j * np.diag(d - d.sum() / 3)
    kappa = 0.1
    op = dirac.anisotropic(U, kappa, **ANISO)
    c = ANISO["csw_r"] / ANISO["xi0"] if coef_key == "spatial" else ANISO["csw_t"]
    expect = np.eye(12) - kappa * c * np.kron(sigma(mu, nu), F)
    np.testing.assert_allclose(op.A, np.broadcast_to(expect, op.A.shape), atol=1e-14)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 2, 4)])
def test_anisotropic_dense_matrix_and_gamma5(dims):
    U = L.gauge_from_qdp(W.gauge_links(dims, 0.7, 33), dims)
    kappa = 0.1
    op = dirac.anisotropic(U, kappa, **ANISO)
    M = dense_matrix(U, dims, kappa, 0.0, -1, aniso=(ANISO["xi0"], ANISO["nu"], ANISO["csw_t"], ANISO["csw_r"]))
    psi, phi = _rand_fermion(dims, 34), _rand_fermion(dims, 35)
    np.testing.assert_allclose(op.M(psi).ravel(), M @ psi.ravel(), atol=1e-13)
    lhs = np.vdot(phi, op.M(psi))
    assert abs(lhs - np.vdot(dirac.gamma5(op.M(dirac.gamma5(phi))), psi)) < 1e-12 * abs(lhs)
