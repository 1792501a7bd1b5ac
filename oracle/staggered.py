"""Staggered fermion operator of the HISQ action on given smeared links (Sec. II.A:
MILC staggered phase convention; Sec. II.E: CG is the default solver for HISQ).

TEST INFRASTRUCTURE ONLY (see the package docstring).  The operator takes the two
link fields the HISQ smearing produces -- the fat links V (one-hop) and the long links
W (three-hop, Naik coefficient included) -- as inputs; the smearing itself (fat7,
U(3) projection, second level) is oracle/hisq.py.

    M chi = 2 m chi + D chi
    D chi(x) = sum_mu eta_mu(x) [ V_mu(x) chi(x + mu) - V_mu(x - mu)^+ chi(x - mu)
                                + W_mu(x) chi(x + 3mu) - W_mu(x - 3mu)^+ chi(x - 3mu) ]

with the MILC phases eta_x = 1, eta_y = (-1)^x, eta_z = (-1)^(x+y),
eta_t = (-1)^(x+y+z), and the fermion time boundary sign on every hop that crosses
t = Lt - 1 -> 0.  D is anti-Hermitian, so M^+ M = 4 m^2 - D^2.

Fields are colour vectors (Lt, Lz, Ly, Lx, 3); links (4, Lt, Lz, Ly, Lx, 3, 3).
Pins (tests/test_oracle_staggered.py): anti-Hermiticity, the free-field symbol of
D^2, gauge covariance, a loop-built dense matrix, and a CG solve against it.
"""
import numpy as np

from . import lattice as L
from . import solvers


def milc_phases(dims):
    """eta_mu(x) for mu = x, y, z, t: shape (4, Lt, Lz, Ly, Lx)."""
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    return np.stack([np.ones_like(x), (-1.0) ** x, (-1.0) ** (x + y), (-1.0) ** (x + y + z)]).astype(float)


def _shift(f, mu, n):
    """g(x) = f(x + n mu_hat), periodic."""
    return np.roll(f, -n, axis=L.AXIS[mu])


def _tb_sign(dims, t_boundary, n):
    """Sign of a t hop of n sites (n > 0 forward, n < 0 backward) from each site."""
    lt = dims[3]
    t = np.arange(lt)[:, None, None, None]
    crosses = (t + n >= lt) | (t + n < 0)
    return np.where(crosses, float(t_boundary), 1.0) * np.ones(dims[::-1])


def _colour(u, chi):
    return np.einsum("...ab,...b->...a", u, chi)


def _dag(u):
    return np.conj(np.swapaxes(u, -1, -2))


def dslash(V, W, chi, t_boundary=-1):
    dims = (chi.shape[3], chi.shape[2], chi.shape[1], chi.shape[0])
    eta = milc_phases(dims)
    out = np.zeros_like(chi)
    for mu in range(4):
        terms = 0
        for links, n in ((V, 1), (W, 3)):
            f = _colour(links[mu], _shift(chi, mu, n))
            b = _colour(_dag(_shift(links[mu], mu, -n)), _shift(chi, mu, -n))
            if mu == 3:
                f = f * _tb_sign(dims, t_boundary, n)[..., None]
                b = b * _tb_sign(dims, t_boundary, -n)[..., None]
            terms = terms + f - b
        out += eta[mu][..., None] * terms
    return out


class Staggered:
    """M = 2 m + D on given fat links V and long links W."""

    def __init__(self, V, W, mass, t_boundary=-1):
        self.V, self.W, self.mass, self.t_boundary = V, W, float(mass), int(t_boundary)

    def D(self, chi):
        return dslash(self.V, self.W, chi, self.t_boundary)

    def M(self, chi):
        return 2 * self.mass * chi + self.D(chi)

    def Mdag(self, chi):
        return 2 * self.mass * chi - self.D(chi)

    def solve(self, b, tol=1e-12, maxiter=10000):
        """CG on M^+ M x = M^+ b (Sec. II.E: CG is the HISQ default)."""
        return solvers.cgnr(self.M, self.Mdag, b, tol=tol, maxiter=maxiter)
