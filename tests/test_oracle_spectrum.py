"""Pin for oracle/spectrum.py: inverse iteration against numpy's SVD of the dense Schur
matrix built from the loop-based definition in _dense_ref."""
import numpy as np
import pytest

import workloads as W
from oracle import dirac, spectrum
from oracle import lattice as L

from _dense_ref import dense_matrix, parity_indices


@pytest.mark.parametrize("dims,kappa", [((2, 2, 2, 2), 0.12), ((4, 2, 2, 4), 0.124)])
def test_smallest_singular_value_matches_dense_svd(dims, kappa):
    U = L.gauge_from_qdp(W.gauge_links(dims, 0.3, 4), dims)
    op = dirac.WilsonClover(U, kappa, 1.0)
    M = dense_matrix(U, dims, kappa, 1.0)
    ie, io = parity_indices(dims, 0), parity_indices(dims, 1)
    Mhat = M[np.ix_(ie, ie)] - M[np.ix_(ie, io)] @ np.linalg.solve(M[np.ix_(io, io)], M[np.ix_(io, ie)])
    exact = np.linalg.svd(Mhat, compute_uv=False).min()
    x0 = L.from_qdp(W.gaussian_fermion(dims, 5), dims) * op.even
    n = len(ie)
    est, k = spectrum.smallest_singular_value(op.Mhat, lambda v: op.Mhat(v, dagger=True), x0, steps=n)
    assert est == pytest.approx(exact, rel=1e-8), (est, exact, k)
    # fewer steps give an upper bound
    est_short, _ = spectrum.smallest_singular_value(op.Mhat, lambda v: op.Mhat(v, dagger=True), x0, steps=n // 8)
    assert est_short >= exact * (1 - 1e-10)
