"""Fermion force of the two-flavour even-odd clover action (the HMC force of Sec. IV).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. IV states that the paper provides the clover fermion forces used by its HMC
(1- and 2-flavour clover actions) without printing them.  The readings taken here
(listed in the design notes):

* Two flavours, even-odd preconditioned (Sec. II.A, II.D):
      det(M^+ M) = det(A_oo)^2 det(M_hat^+ M_hat),
  so with a pseudofermion phi on the even sites
      S(U) = phi^+ (M_hat^+ M_hat)^-1 phi  -  2 sum_{x odd} log det A(x).
  The second term (``include_logdet``) is the clover determinant of the odd sites.
* The force F_mu(x) is the gradient of S in su(3) for a left variation of one link:
  for U_mu(x) -> exp(eps Q) U_mu(x), Q traceless anti-Hermitian,
      dS/d eps = <Q, F_mu(x)> = -Tr(Q F_mu(x)),
  which makes F_mu(x) = -TA(U_mu(x) G_mu(x)) where dS = Re sum Tr(dU G) and
  TA(M) = (M - M^+)/2 - Tr((M - M^+)/2)/3 (traceless anti-Hermitian part).

Derivation (X = (M_hat^+ M_hat)^-1 phi, Y = M_hat X on the even sites):
      dS_pf = -2 Re Y^+ dM_hat X
  with dM_hat = dA_ee - kappa^2 (dD_eo A^-1 D_oe - D_eo A^-1 dA_oo A^-1 D_oe + D_eo A^-1 dD_oe).
  With Z = A_oo^-1 D_oe X and W = A_oo^-1 (H^+ Y)_odd (odd sites):
      dS_pf = 2 kappa^2 Re[Y^+ dH Z + W^+ dH X] - 2 Re[Y^+ dA X]_even - 2 kappa^2 Re[W^+ dA Z]_odd
      dS_det = -2 sum_odd Tr(A^-1 dA).
  The hopping variation gives, per link, the spin-traced outer products of
  A = Y (+) W and B = Z (+) X (even (+) odd); the clover variation goes through
  dA = -kappa c_sw sum_{mu<nu} sigma_{mu nu} (x) dF_{mu nu} and the four leaves of
  every Q_{mu nu}: each link of a leaf is varied in turn (product rule).

The pins (tests/test_oracle_force.py) compare this analytic force with central
finite differences of S itself, computed by dense solves on small lattices, per
term, and check gauge covariance.
"""
import numpy as np

from . import lattice as L
from .dirac import PLANES, WilsonClover, _dag, _mul, apply_site_matrix, hopping
from .gamma import GAMMA, ID4, sigma


def traceless_antihermitian(m: np.ndarray) -> np.ndarray:
    """TA(M) = (M - M^+)/2 minus its trace/3, per site (last two axes 3x3)."""
    a = 0.5 * (m - _dag(m))
    tr = np.trace(a, axis1=-2, axis2=-1)
    return a - tr[..., None, None] / 3.0 * np.eye(3)


# ---------------------------------------------------------------------------
# The action, for finite differences

def schur_matrix(op: WilsonClover) -> np.ndarray:
    """M_hat as a dense matrix on the even sites (columns: unit vectors)."""
    even = op.even[..., 0, 0]
    idx = np.argwhere(even)
    n = len(idx) * 12
    m = np.zeros((n, n), dtype=np.complex128)
    shape = op.even.shape[:4] + (4, 3)
    for k in range(n):
        e = np.zeros(shape, dtype=np.complex128)
        site = tuple(idx[k // 12])
        e[site + divmod(k % 12, 3)] = 1.0
        y = op.Mhat(e)
        m[:, k] = y[even].reshape(-1)
    return m


def action(op: WilsonClover, phi: np.ndarray, include_logdet: bool = True) -> float:
    """S = phi^+ (M_hat^+ M_hat)^-1 phi - 2 sum_odd log det A (phi on the even sites)."""
    even = op.even[..., 0, 0]
    m = schur_matrix(op)
    p = phi[even].reshape(-1)
    x = np.linalg.solve(m.conj().T @ m, p)
    s = float(np.real(np.vdot(p, x)))
    if include_logdet:
        odd = op.odd[..., 0, 0]
        _, logdet = np.linalg.slogdet(op.A[odd])
        s -= 2.0 * float(np.sum(logdet))
    return s


def solve_normal(op: WilsonClover, phi: np.ndarray) -> np.ndarray:
    """X = (M_hat^+ M_hat)^-1 phi on the even sites (dense solve)."""
    even = op.even[..., 0, 0]
    m = schur_matrix(op)
    x = np.linalg.solve(m.conj().T @ m, phi[even].reshape(-1))
    out = np.zeros_like(phi)
    out[even] = x.reshape(-1, 4, 3)
    return out


# ---------------------------------------------------------------------------
# The analytic force

def _outer_trace(g: np.ndarray, b: np.ndarray, a: np.ndarray) -> np.ndarray:
    """C_{cd}(s) = sum_{alpha beta} g_{alpha beta} b_{beta c}(s) conj(a_{alpha d}(s)): Tr_spin[g b a^+]."""
    return np.einsum("ab,...bc,...ad->...cd", g, b, np.conj(a))


def hopping_variation(U: np.ndarray, a: np.ndarray, b: np.ndarray, t_boundary: int) -> np.ndarray:
    """G_mu(s) with Re sum Tr(dU G) = Re a^+ dH b (H of the hopping term, both parities):
    G_mu(s) = eta(s) { Tr_s[(1 - g_mu) b(s+mu) a(s)^+] + Tr_s[(1 + g_mu) b(s) a(s+mu)^+]^+ }."""
    dims = L.dims_of(a)
    g = np.zeros(U.shape, dtype=np.complex128)
    for mu in range(4):
        fwd_term = _outer_trace(ID4 - GAMMA[mu], L.fwd(b, mu), a)
        bwd_term = _dag(_outer_trace(ID4 + GAMMA[mu], b, L.fwd(a, mu)))
        t = fwd_term + bwd_term
        if mu == 3:
            t = t * L.time_boundary_sign(dims, t_boundary, True)[..., None, None]
        g[mu] = t
    return g


# The four leaves of Q_{mu nu}(s) as in dirac.clover_leaves: factors (direction
# index 0 = mu / 1 = nu, daggered, site offset (in mu, in nu) of the link).
LEAVES = (
    ((0, False, (0, 0)), (1, False, (1, 0)), (0, True, (0, 1)), (1, True, (0, 0))),
    ((1, False, (0, 0)), (0, True, (-1, 1)), (1, True, (-1, 0)), (0, False, (-1, 0))),
    ((0, True, (-1, 0)), (1, True, (-1, -1)), (0, False, (-1, -1)), (1, False, (0, -1))),
    ((1, True, (0, -1)), (0, False, (0, -1)), (1, False, (1, -1)), (0, True, (0, 0))),
)


def _shift(field: np.ndarray, mu: int, nu: int, off) -> np.ndarray:
    """g(s) = f(s + off[0] mu_hat + off[1] nu_hat)."""
    out = field
    for d, k in ((mu, off[0]), (nu, off[1])):
        for _ in range(abs(k)):
            out = L.fwd(out, d) if k > 0 else L.bwd(out, d)
    return out


def clover_variation(U: np.ndarray, omega: dict) -> np.ndarray:
    """G_mu(y) with Re sum Tr(dU G) = Re sum_s sum_{mu<nu} Tr(dQ_{mu nu}(s) omega_{mu nu}(s)).

    Every leaf is a product f1 f2 f3 f4 of shifted (and possibly daggered) links; varying
    factor j gives Re Tr(df_j R_j) with R_j = f_{j+1} .. f_4 omega f_1 .. f_{j-1}, which is
    credited to the link's own site (R_j shifted back), daggered when f_j is a U^+."""
    g = np.zeros(U.shape, dtype=np.complex128)
    eye = np.broadcast_to(np.eye(3, dtype=np.complex128), U.shape[1:])
    for (mu, nu) in PLANES:
        om = omega[(mu, nu)]
        for leaf in LEAVES:
            facs = []
            for d, dag, off in leaf:
                u = _shift(U[(mu, nu)[d]], mu, nu, off)
                facs.append(_dag(u) if dag else u)
            for j, (d, dag, off) in enumerate(leaf):
                after = eye
                for k in range(j + 1, 4):
                    after = _mul(after, facs[k])
                before = eye
                for k in range(j):
                    before = _mul(before, facs[k])
                rj = _mul(_mul(after, om), before)
                if dag:
                    rj = _dag(rj)
                g[(mu, nu)[d]] += _shift(rj, mu, nu, (-off[0], -off[1]))
    return g


def sigma_trace(a: np.ndarray, b: np.ndarray) -> dict:
    """Lambda_{mu nu}(s) = Tr_spin[sigma_{mu nu} b(s) a(s)^+] (colour 3x3) per plane."""
    return {pl: _outer_trace(sigma(*pl), b, a) for pl in PLANES}


def logdet_trace(ainv: np.ndarray) -> dict:
    """Lambda^det_{mu nu}(s)_{ba} = sum_{alpha beta} sigma_{alpha beta} (A^-1)_{(beta b),(alpha a)}."""
    ai = ainv.reshape(ainv.shape[:4] + (4, 3, 4, 3))
    return {pl: np.einsum("ab,...bcad->...cd", sigma(*pl), ai) for pl in PLANES}


def clover_force(op: WilsonClover, X: np.ndarray, include_logdet: bool = True) -> np.ndarray:
    """F_mu(x) (traceless anti-Hermitian, shape (4, Lt, Lz, Ly, Lx, 3, 3)) of S at the
    current links, given X = (M_hat^+ M_hat)^-1 phi on the even sites."""
    if op.hop_weights is not None:
        raise ValueError("the force is defined for the isotropic operator")
    k, csw = op.kappa, op.csw
    X = X * op.even
    Y = op.Mhat(X)
    Z = apply_site_matrix(op.Ainv, op.H(X)) * op.odd
    W = apply_site_matrix(op.Ainv, hopping(op.U, Y, op.t_boundary, dagger=True)) * op.odd
    # hopping term: 2 kappa^2 Re[Y^+ dH Z + W^+ dH X] = 2 kappa^2 Re[A^+ dH B]
    g = 2.0 * k * k * hopping_variation(op.U, Y + W, Z + X, op.t_boundary)
    # clover term: 2 kappa c_sw Re sum Tr(dF_{mu nu} Xi_{mu nu}), Xi from the even pair
    # (Y, X), the odd pair kappa^2 (W, Z) and the odd determinant term
    lam_e = sigma_trace(Y, X)
    lam_o = sigma_trace(W, Z)
    lam_d = logdet_trace(op.Ainv) if include_logdet else None
    even = op.even[..., 0, 0][..., None, None]
    odd = op.odd[..., 0, 0][..., None, None]
    omega = {}
    for pl in PLANES:
        xi = lam_e[pl] * even + k * k * lam_o[pl] * odd
        if include_logdet:
            xi = xi + lam_d[pl] * odd
        tr = np.trace(xi, axis1=-2, axis2=-1)
        xi0 = xi - tr[..., None, None] / 3.0 * np.eye(3)
        # Re Tr(dF Xi) = Re Tr((dQ - dQ^+)/8 Xi0) = Re Tr(dQ (Xi0 - Xi0^+))/8
        omega[pl] = (xi0 - _dag(xi0)) * (2.0 * k * csw / 8.0)
    g = g + clover_variation(op.U, omega)
    return -traceless_antihermitian(_mul(op.U, g))
