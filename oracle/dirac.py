"""Wilson-clover Dirac operator, kappa normalisation, isotropic form of Eq. 5.

Reading of Eq. 5 (Sec. III.B) with xi_0 = nu = 1 and c_SW^t = c_SW^r = c_sw,
multiplied through so that the operator is M = 2*kappa*a*M_phys:

    M = A - kappa * H
    H psi(s) = sum_mu [ eta+_mu(s) (1 - gamma_mu) U_mu(s)        psi(s + mu)
                      + eta-_mu(s) (1 + gamma_mu) U_mu(s - mu)^+ psi(s - mu) ]
    A(s)     = 1 - kappa * c_sw * sum_{mu<nu} sigma_{mu nu} (x) F_{mu nu}(s)

with sigma_{mu nu} = [gamma_mu, gamma_nu]/2 and F_{mu nu} the traceless
anti-Hermitian part of the clover-leaf sum Q_{mu nu} divided by 8.  eta is the
fermion time boundary (t_boundary = -1: antiperiodic, Sec. III.B); space is
periodic.  The clover uses the bare (periodic) links.

Even-odd (Sec. II.A, II.D: all fields are stored even-odd preconditioned):
    M_hat = A_ee - kappa^2 D_eo A_oo^-1 D_oe
    b_hat = b_e + kappa D_eo A_oo^-1 b_o
    x_o   = A_oo^-1 (b_o + kappa D_oe x_e)
where D_eo / D_oe are H restricted to (even out, odd in) / (odd out, even in).
Because H only couples nearest neighbours, H of a field supported on one
parity is supported on the other; the oracle therefore keeps whole-lattice
arrays and lets the parity of the support select D_eo or D_oe.

Anisotropic form (Eq. 5 with general xi_0, nu, c_SW^t, c_SW^r), through
``anisotropic``: the spatial hops carry nu/xi_0, the clover planes (i, 4) carry
c_SW^t and the planes (i, j) carry c_SW^r/xi_0, and kappa^-1 = 2 (m0 + 1 + 3 nu/xi_0)
(``kappa_of_mass``).  The isotropic operator is the case xi_0 = nu = 1,
c_SW^t = c_SW^r = c_sw.

Pins (tests/test_oracle_dirac.py): free-field plane waves (isotropic and
anisotropic), the massless point of the kappa relation, gamma_5-hermiticity,
gauge covariance, the abelian constant-field clover in a spatial and a temporal
plane, and a loop-built dense matrix on 2^4 and small anisotropic lattices.
"""
import numpy as np

from . import lattice as L
from .gamma import GAMMA, GAMMA5, ID4, sigma

PLANES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]


def _dag(u: np.ndarray) -> np.ndarray:
    return np.conj(np.swapaxes(u, -1, -2))


def _mul(a, b):
    return np.einsum("...ab,...bc->...ac", a, b)


def _colour(u, psi):
    """(U psi)_{s a} = sum_b U_ab psi_{s b} per site."""
    return np.einsum("...ab,...sb->...sa", u, psi)


def _spin(g, psi):
    """(g psi)_{s c} = sum_t g_st psi_{t c}."""
    return np.einsum("st,...tc->...sc", g, psi)


def hopping(U: np.ndarray, psi: np.ndarray, t_boundary: int = -1, dagger: bool = False,
            weights=None) -> np.ndarray:
    """H psi, or H^+ psi = gamma5 H gamma5 psi (projector signs swapped) when dagger is set.
    weights: optional factor per direction mu (the nu/xi_0 of Eq. 5's spatial hops)."""
    dims = L.dims_of(psi)
    out = np.zeros_like(psi)
    sgn = -1.0 if dagger else 1.0
    for mu in range(4):
        f = _colour(U[mu], L.fwd(psi, mu))
        b = _colour(_dag(L.bwd(U[mu], mu)), L.bwd(psi, mu))
        if mu == 3:
            f = f * L.time_boundary_sign(dims, t_boundary, True)[..., None, None]
            b = b * L.time_boundary_sign(dims, t_boundary, False)[..., None, None]
        term = _spin(ID4 - sgn * GAMMA[mu], f) + _spin(ID4 + sgn * GAMMA[mu], b)
        out += term if weights is None else weights[mu] * term
    return out


def clover_leaves(U: np.ndarray, mu: int, nu: int) -> np.ndarray:
    """Q_{mu nu}(s): the four plaquettes in the (mu, nu) plane that start and end at s,
    all with the orientation +mu, +nu, -mu, -nu (bare links, periodic)."""
    um, un = U[mu], U[nu]
    f, b = L.fwd, L.bwd
    leaf1 = _mul(_mul(um, f(un, mu)), _mul(_dag(f(um, nu)), _dag(un)))
    leaf2 = _mul(_mul(un, _dag(f(b(um, mu), nu))), _mul(_dag(b(un, mu)), b(um, mu)))
    leaf3 = _mul(_mul(_dag(b(um, mu)), _dag(b(b(un, mu), nu))), _mul(b(b(um, mu), nu), b(un, nu)))
    leaf4 = _mul(_mul(_dag(b(un, nu)), b(um, nu)), _mul(f(b(un, nu), mu), _dag(um)))
    return leaf1 + leaf2 + leaf3 + leaf4


def field_strength(U: np.ndarray, mu: int, nu: int) -> np.ndarray:
    """F_{mu nu} = (Q - Q^+)/8 minus its trace/3: traceless anti-Hermitian, per site (3x3)."""
    q = clover_leaves(U, mu, nu)
    f = (q - _dag(q)) / 8.0
    tr = np.trace(f, axis1=-2, axis2=-1)
    return f - tr[..., None, None] / 3.0 * np.eye(3)


def clover_matrix(U: np.ndarray, kappa: float, csw: float, plane_csw=None) -> np.ndarray:
    """A(s) = 1 - kappa c_sw sum_{mu<nu} sigma_{mu nu} (x) F_{mu nu}(s), as 12x12 per site.

    Row/column index is 3*spin + colour.  plane_csw: optional coefficient per plane
    of PLANES replacing c_sw (Eq. 5's c_SW^t on (i, 4), c_SW^r/xi_0 on (i, j)).
    """
    site_shape = U.shape[1:5]
    if plane_csw is not None:
        a = np.zeros(site_shape + (12, 12), dtype=np.complex128)
        for (mu, nu), c in zip(PLANES, plane_csw):
            fmn = field_strength(U, mu, nu)
            a += c * np.einsum("st,...ab->...satb", sigma(mu, nu), fmn).reshape(site_shape + (12, 12))
        return np.eye(12) - kappa * a
    a = np.zeros(site_shape + (12, 12), dtype=np.complex128)
    for mu, nu in PLANES:
        fmn = field_strength(U, mu, nu)
        a += np.einsum("st,...ab->...satb", sigma(mu, nu), fmn).reshape(site_shape + (12, 12))
    return np.eye(12) - kappa * csw * a


def apply_site_matrix(a: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """(A psi)(s) with A a 12x12 matrix per site acting on (spin, colour)."""
    shp = psi.shape
    v = psi.reshape(shp[:4] + (12,))
    return np.einsum("...ij,...j->...i", a, v).reshape(shp)


def gamma5(psi: np.ndarray) -> np.ndarray:
    return _spin(GAMMA5, psi)


class WilsonClover:
    """The operator M = A - kappa H of one gauge field, with its even-odd pieces."""

    def __init__(self, U: np.ndarray, kappa: float, csw: float, t_boundary: int = -1, hop_weights=None,
                 plane_csw=None):
        self.U = U
        self.kappa = float(kappa)
        self.csw = float(csw)
        self.t_boundary = int(t_boundary)
        self.hop_weights = hop_weights
        self.dims = (U.shape[4], U.shape[3], U.shape[2], U.shape[1])
        self.A = clover_matrix(U, kappa, csw, plane_csw)
        self.Ainv = np.linalg.inv(self.A)
        self.even = L.parity_mask(self.dims, 0)[..., None, None]
        self.odd = ~self.even

    # full operator ---------------------------------------------------------
    def H(self, psi, dagger=False):
        return hopping(self.U, psi, self.t_boundary, dagger, self.hop_weights)

    def M(self, psi):
        """M psi = A psi - kappa H psi on the whole lattice."""
        return apply_site_matrix(self.A, psi) - self.kappa * self.H(psi)

    def Mdag(self, psi):
        """M^+ = gamma5 M gamma5 (A is Hermitian and commutes with gamma5)."""
        return gamma5(self.M(gamma5(psi)))

    # even-odd --------------------------------------------------------------
    def Mhat(self, xe, dagger=False):
        """M_hat x_e = A_ee x_e - kappa^2 D_eo A_oo^-1 D_oe x_e (x_e supported on even sites)."""
        xe = xe * self.even
        t = apply_site_matrix(self.Ainv, self.H(xe, dagger))
        return (apply_site_matrix(self.A, xe) - self.kappa ** 2 * self.H(t, dagger)) * self.even

    def schur_source(self, b):
        """b_hat = b_e + kappa D_eo A_oo^-1 b_o."""
        t = apply_site_matrix(self.Ainv, b * self.odd)
        return (b + self.kappa * self.H(t)) * self.even

    def reconstruct(self, xe, b):
        """Full solution x = x_e + A_oo^-1 (b_o + kappa D_oe x_e)."""
        xe = xe * self.even
        xo = apply_site_matrix(self.Ainv, (b + self.kappa * self.H(xe)) * self.odd) * self.odd
        return xe + xo

    def true_residual(self, x, b) -> float:
        """||b - M x||_2 / ||b||_2 over the whole lattice: the relative true residual of the full system."""
        return float(np.linalg.norm(b - self.M(x)) / np.linalg.norm(b))


def anisotropic(U, kappa, xi0, nu, csw_t, csw_r, t_boundary=-1) -> WilsonClover:
    """Eq. 5 with anisotropy: 2 kappa a_t M = 1 - kappa [gamma_4 W_4 + (nu/xi_0) sum_i gamma_i W_i
    + c_SW^t sum_i sigma_{i4} F_{i4} + (c_SW^r/xi_0) sum_{i<j} sigma_{ij} F_{ij}], with the
    hopping read as for the isotropic operator (Wilson r = 1 projectors)."""
    w = nu / xi0
    plane_csw = [csw_t if nu_ == 3 else csw_r / xi0 for _, nu_ in PLANES]
    return WilsonClover(U, kappa, 0.0, t_boundary, hop_weights=(w, w, w, 1.0), plane_csw=plane_csw)


def kappa_of_mass(m0, xi0=1.0, nu=1.0):
    """kappa^-1 = 2 (m0 + 1 + 3 nu/xi_0), the relation stated under Eq. 5."""
    return 1.0 / (2.0 * (m0 + 1.0 + 3.0 * nu / xi0))


# QDP-layout conveniences used by the tests -------------------------------------

def from_qdp_problem(gauge_qdp, dims, kappa, csw, t_boundary=-1) -> WilsonClover:
    return WilsonClover(L.gauge_from_qdp(gauge_qdp, dims), kappa, csw, t_boundary)


def apply_D_qdp(op: WilsonClover, psi_qdp):
    return L.to_qdp(op.M(L.from_qdp(psi_qdp, op.dims)), op.dims)


def apply_Mhat_qdp(op: WilsonClover, psi_even_qdp, dagger=False):
    """M_hat on the even half [Lt][Lz][Ly][Lx/2][4][3] of a QDP field."""
    full = np.zeros((2,) + psi_even_qdp.shape, dtype=np.complex128)
    full[0] = psi_even_qdp
    y = op.Mhat(L.from_qdp(full, op.dims), dagger)
    return L.to_qdp(y, op.dims)[0]


# Site-by-site evaluation for lattices too large for whole-array evaluation -------

def _qdp_link(gauge_qdp, dims, mu, c):
    lx, ly, lz, lt = dims
    x, y, z, t = (c[0] % lx, c[1] % ly, c[2] % lz, c[3] % lt)
    p = (x + y + z + t) % 2
    return gauge_qdp[mu, p, t, z, y, x // 2]


def _qdp_psi(psi_qdp, dims, c):
    lx, ly, lz, lt = dims
    x, y, z, t = (c[0] % lx, c[1] % ly, c[2] % lz, c[3] % lt)
    return psi_qdp[(x + y + z + t) % 2, t, z, y, x // 2]


def _hop_at(gauge_qdp, field, dims, s, t_boundary):
    """(H psi)(s) at one site; field(c) returns the spinor [4][3] at coordinates c."""
    lt = dims[3]
    hop = np.zeros((4, 3), dtype=np.complex128)
    for mu in range(4):
        cf, cb = list(s), list(s)
        cf[mu] += 1
        cb[mu] -= 1
        ef = t_boundary if (mu == 3 and s[3] == lt - 1) else 1.0
        eb = t_boundary if (mu == 3 and s[3] == 0) else 1.0
        uf = _qdp_link(gauge_qdp, dims, mu, s)
        ub = _qdp_link(gauge_qdp, dims, mu, cb).conj().T
        hop += ef * (ID4 - GAMMA[mu]) @ (field(tuple(cf)) @ uf.T)
        hop += eb * (ID4 + GAMMA[mu]) @ (field(tuple(cb)) @ ub.T)
    return hop


def _clover_at(gauge_qdp, dims, s, kappa, csw):
    """A(s) as a 12x12 matrix (index 3 spin + colour) from the four leaves at s."""
    a = np.eye(12, dtype=np.complex128)
    for mu, nu in PLANES:
        def link(d, dm, dn):
            c = list(s)
            c[mu] += dm
            c[nu] += dn
            return _qdp_link(gauge_qdp, dims, d, c)
        q = (link(mu, 0, 0) @ link(nu, 1, 0) @ link(mu, 0, 1).conj().T @ link(nu, 0, 0).conj().T
             + link(nu, 0, 0) @ link(mu, -1, 1).conj().T @ link(nu, -1, 0).conj().T @ link(mu, -1, 0)
             + link(mu, -1, 0).conj().T @ link(nu, -1, -1).conj().T @ link(mu, -1, -1) @ link(nu, 0, -1)
             + link(nu, 0, -1).conj().T @ link(mu, 0, -1) @ link(nu, 1, -1) @ link(mu, 0, 0).conj().T)
        f = (q - q.conj().T) / 8.0
        f = f - np.trace(f) / 3.0 * np.eye(3)
        a -= kappa * csw * np.kron(sigma(mu, nu), f)
    return a


def M_at_sites(gauge_qdp, psi_qdp, dims, kappa, csw, sites, t_boundary=-1):
    """(M psi)(s) for each s = (x, y, z, t) in `sites`, read straight from QDP arrays.

    Same definition as WilsonClover.M (Eq. 5: hopping term with the time-boundary
    sign, clover term from the four leaves), evaluated one site at a time so that
    it works on lattices of any size.  Pinned against WilsonClover.M.
    """
    out = []
    for s in sites:
        s = tuple(int(v) for v in s)
        hop = _hop_at(gauge_qdp, lambda c: _qdp_psi(psi_qdp, dims, c), dims, s, t_boundary)
        a = _clover_at(gauge_qdp, dims, s, kappa, csw)
        out.append((a @ _qdp_psi(psi_qdp, dims, s).reshape(12)).reshape(4, 3) - kappa * hop)
    return np.array(out)


def Mhat_at_sites(gauge_qdp, psi_even_qdp, dims, kappa, csw, sites, dagger=False, t_boundary=-1):
    """(M_hat x_e)(s) for even sites s: A(s) x(s) - kappa^2 (D_eo A_oo^-1 D_oe x)(s),
    the even-odd Schur complement of Eq. 5's operator on the even sublattice (§II.A
    layout), one site at a time; M_hat^+ = gamma5 M_hat gamma5.  The odd-site
    vectors A^-1 (D x)(n) are formed only at the neighbours of the sampled sites.
    Pinned against WilsonClover.Mhat."""
    lx, ly, lz, lt = dims
    g5 = np.diag([1.0, 1.0, -1.0, -1.0]).astype(np.complex128)

    def x_at(c):
        x, y, z, t = (c[0] % lx, c[1] % ly, c[2] % lz, c[3] % lt)
        if (x + y + z + t) % 2:
            return np.zeros((4, 3), dtype=np.complex128)
        v = psi_even_qdp[t, z, y, x // 2]
        return g5 @ v if dagger else v

    cache = {}

    def y_at(c):
        key = (c[0] % lx, c[1] % ly, c[2] % lz, c[3] % lt)
        if key not in cache:
            hop = _hop_at(gauge_qdp, x_at, dims, key, t_boundary)
            a = _clover_at(gauge_qdp, dims, key, kappa, csw)
            cache[key] = np.linalg.solve(a, hop.reshape(12)).reshape(4, 3)
        return cache[key]

    out = []
    for s in sites:
        s = tuple(int(v) for v in s)
        assert sum(s) % 2 == 0, "M_hat lives on the even sites"
        a = _clover_at(gauge_qdp, dims, s, kappa, csw)
        val = (a @ x_at(s).reshape(12)).reshape(4, 3) - kappa * kappa * _hop_at(gauge_qdp, y_at, dims, s, t_boundary)
        out.append(g5 @ val if dagger else val)
    return np.array(out)
