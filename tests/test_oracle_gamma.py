"""Pins for the oracle's Dirac matrices (Sec. II.A: DeGrand-Rossi basis, QDP Gamma(n))."""
import itertools

import numpy as np
import pytest

from oracle.gamma import GAMMA, GAMMA5, ID4, gamma, sigma


def test_hermitian_and_clifford():
    for mu, nu in itertools.product(range(4), repeat=2):
        anti = GAMMA[mu] @ GAMMA[nu] + GAMMA[nu] @ GAMMA[mu]
        np.testing.assert_allclose(anti, 2.0 * (mu == nu) * ID4, atol=0)
    for g in GAMMA:
        np.testing.assert_allclose(g, g.conj().T, atol=0)


def test_chiral_basis_gamma5():
    # Sec. II.A: the DeGrand-Rossi basis is a chiral basis, gamma5 diagonal.
    np.testing.assert_allclose(GAMMA5, np.diag([1, 1, -1, -1]), atol=0)
    for g in GAMMA:
        np.testing.assert_allclose(GAMMA5 @ g, -g @ GAMMA5, atol=0)


def test_projectors_rank_two():
    for g in GAMMA:
        for s in (+1, -1):
            p = 0.5 * (ID4 + s * g)
            np.testing.assert_allclose(p @ p, p, atol=1e-15)
            assert np.linalg.matrix_rank(p) == 2


def test_qdp_gamma_index():
    # Listing 1 uses gamma(15) for gamma5 and gamma(15) @ gamma(4) for gamma5 gamma3 (Eq. 7).
    np.testing.assert_allclose(gamma(15), GAMMA5, atol=0)
    np.testing.assert_allclose(gamma(15) @ gamma(4), GAMMA5 @ GAMMA[2], atol=0)
    np.testing.assert_allclose(gamma(8), GAMMA[3], atol=0)
    np.testing.assert_allclose(gamma(0), ID4, atol=0)


@pytest.mark.parametrize("mu,nu", [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)])
def test_sigma_block_diagonal_antihermitian(mu, nu):
    s = sigma(mu, nu)
    np.testing.assert_allclose(s, -s.conj().T, atol=0)
    np.testing.assert_allclose(s @ GAMMA5, GAMMA5 @ s, atol=0)
    # commuting with gamma5 = diag(1,1,-1,-1): no coupling between spins {0,1} and {2,3}
    assert np.all(s[:2, 2:] == 0) and np.all(s[2:, :2] == 0)
