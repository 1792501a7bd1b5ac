"""Dirac matrices in the DeGrand-Rossi (chiral) basis, Chroma convention (Sec. II.A).

The paper names the basis but does not print the matrices; the table below is
the standard DeGrand-Rossi one.  Pinned by the Clifford algebra, hermiticity
and gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(1, 1, -1, -1) (the basis is
chiral, Sec. II.A), and by the QDP index convention of ``gamma(n)`` that the
example script relies on (Listing 1 and Eq. 7: gamma(15) @ gamma(4) is
gamma_5 gamma_3).
"""
import numpy as np

_i = 1j

#: gamma_mu for mu = 0..3 <-> x, y, z, t (gamma_1 .. gamma_4 of the paper).
GAMMA = np.array(
    [
        [[0, 0, 0, _i], [0, 0, _i, 0], [0, -_i, 0, 0], [-_i, 0, 0, 0]],
        [[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]],
        [[0, 0, _i, 0], [0, 0, 0, -_i], [-_i, 0, 0, 0], [0, _i, 0, 0]],
        [[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]],
    ],
    dtype=np.complex128,
)

ID4 = np.eye(4, dtype=np.complex128)

#: gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]


def gamma(n: int) -> np.ndarray:
    """QDP Gamma(n) = gamma_1^b0 gamma_2^b1 gamma_3^b2 gamma_4^b3, b_k the bits of n."""
    g = ID4.copy()
    for k in range(4):
        if (n >> k) & 1:
            g = g @ GAMMA[k]
    return g


def sigma(mu: int, nu: int) -> np.ndarray:
    """sigma_{mu nu} = (1/2)[gamma_mu, gamma_nu]  (anti-Hermitian reading of Eq. 5)."""
    return 0.5 * (GAMMA[mu] @ GAMMA[nu] - GAMMA[nu] @ GAMMA[mu])
