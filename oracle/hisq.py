"""HISQ link smearing: the fat and long links of the staggered operator (staggered.py)
built from the thin gauge links.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. II.A names the highly improved staggered quark (HISQ) process of Follana et al.
(hep-lat/0610092) in the MILC convention: a first fattening step, a U(3) projection of
its result (MILC; Chroma projects to SU(3)), and a second fattening step with the Naik
term.  The paper prints neither the paths nor the coefficients.  The readings taken
here (listed in the design notes):

* A smearing with coefficients (c1, c3, c5, c7, cL) replaces each link by
      c1 U_mu(x) + c3 sum S3 + c5 sum S5 + c7 sum S7 + cL sum SL,
  where a "staple" carries a mu-directed object F one step along a signed direction
  +-rho perpendicular to mu and back:
      staple(+rho, F)(x) = U_rho(x) F(x + rho) U_rho(x + mu)^+
      staple(-rho, F)(x) = U_rho(x - rho)^+ F(x - rho) U_rho(x - rho + mu),
  S3 = staple(r, U_mu) over the 6 signed r, S5 = staple(r, staple(s, U_mu)) over the
  24 ordered pairs of signed directions on different axes, S7 = staple(r, staple(s,
  staple(n, U_mu))) over the 48 ordered triples on three different axes, and the
  Lepage term SL = staple(r, staple(r, U_mu)) over the 6 signed r (straight 5-link).
* First level: the fat7 smearing, prod_{rho != mu} (1 + delta_rho^2 / 4) expanded:
  (c1, c3, c5, c7, cL) = (1/8, 1/16, 1/64, 1/384, 0); U = 1 gives 1.
* U(3) projection: W = V (V^+ V)^(-1/2), the unitary polar factor of V.
* Second level on W: the same paths with (5/8, 1/16, 1/64, 1/384, -1/16), which adds
  the Lepage term and makes the free one-hop coefficient 9/8; the Naik link
  N_mu(x) = W_mu(x) W_mu(x + mu) W_mu(x + 2 mu) enters with -(1 + eps)/24, and the fat
  link gains eps/8 W_mu(x), so that the free derivative keeps 9/8 + eps/8 - 3 (1 + eps)/24
  = 1 (eps = 0 for light quarks).
* The smearing uses the bare gauge links (periodic); the fermion time-boundary sign
  and the MILC phases are the operator's (staggered.py), not the links'.

Links are arrays (4, Lt, Lz, Ly, Lx, 3, 3).  Pins (tests/test_oracle_hisq.py): the free
field, constant commuting links, a constant abelian flux in one plane (closed forms
for both levels and the Naik link, which fix every coefficient and path count), gauge
covariance, and the projection against the SVD polar factor.
"""
import numpy as np

from . import lattice as L

FAT7 = (1 / 8, 1 / 16, 1 / 64, 1 / 384, 0.0)
ASQ = (5 / 8, 1 / 16, 1 / 64, 1 / 384, -1 / 16)


def _shift(f, mu, n):
    """g(x) = f(x + n mu_hat), periodic."""
    return np.roll(f, -n, axis=L.AXIS[mu])


def _dag(u):
    return np.conj(np.swapaxes(u, -1, -2))


def staple(U, mu, rho, sign, F):
    """The mu-directed field F carried one step along sign * rho and back."""
    if sign > 0:
        return U[rho] @ _shift(F, rho, 1) @ _dag(_shift(U[rho], mu, 1))
    back = _shift(U[rho], rho, -1)  # U_rho(x - rho)
    return _dag(back) @ _shift(F, rho, -1) @ _shift(back, mu, 1)


def smear(U, coeffs):
    """Each link replaced by the weighted sum of its paths (module docstring)."""
    c1, c3, c5, c7, cl = coeffs
    out = np.empty_like(U)
    for mu in range(4):
        perp = [r for r in range(4) if r != mu]
        acc = c1 * U[mu]
        for rho in perp:
            for s in (1, -1):
                acc = acc + c3 * staple(U, mu, rho, s, U[mu])
                for sig in perp:
                    if sig == rho:
                        continue
                    nu = [r for r in perp if r not in (rho, sig)][0]
                    for s2 in (1, -1):
                        acc = acc + c5 * staple(U, mu, rho, s, staple(U, mu, sig, s2, U[mu]))
                        for s3 in (1, -1):
                            inner = staple(U, mu, sig, s2, staple(U, mu, nu, s3, U[mu]))
                            acc = acc + c7 * staple(U, mu, rho, s, inner)
                if cl != 0.0:
                    acc = acc + cl * staple(U, mu, rho, s, staple(U, mu, rho, s, U[mu]))
        out[mu] = acc
    return out


def u3_project(V):
    """W = V (V^+ V)^(-1/2) link by link, from the eigen-decomposition of V^+ V."""
    Q = _dag(V) @ V
    lam, E = np.linalg.eigh(Q)
    if np.any(lam <= 0):
        raise ValueError("u3_project: singular link")
    inv_sqrt = (E * (1.0 / np.sqrt(lam))[..., None, :]) @ _dag(E)
    return V @ inv_sqrt


def naik(W):
    """N_mu(x) = W_mu(x) W_mu(x + mu) W_mu(x + 2 mu)."""
    out = np.empty_like(W)
    for mu in range(4):
        out[mu] = W[mu] @ _shift(W[mu], mu, 1) @ _shift(W[mu], mu, 2)
    return out


def hisq_links(U, eps_naik=0.0):
    """(fat, long) links of the HISQ staggered operator from thin links U."""
    V = smear(U, FAT7)
    W = u3_project(V)
    fat = smear(W, ASQ) + (eps_naik / 8.0) * W
    long = -(1.0 + eps_naik) / 24.0 * naik(W)
    return fat, long
