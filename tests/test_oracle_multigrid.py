"""Pins for the oracle's aggregation multigrid (oracle/multigrid.py)."""
import numpy as np
import pytest

import workloads as W
from oracle import dirac, multigrid as MG, solvers
from oracle import lattice as L
from oracle.gamma import GAMMA5


def _op(dims, kappa, csw=1.0, eps=0.3, seed=0):
    return dirac.WilsonClover(L.gauge_from_qdp(W.gauge_links(dims, eps, seed), dims), kappa, csw)


def _starts(dims, n, seed):
    return [L.from_qdp(W.gaussian_fermion(dims, seed + k), dims) for k in range(n)]


def test_prolongator_orthonormal_and_chiral():
    dims, block, nv = (4, 4, 2, 4), (2, 2, 2, 2), 6
    P = MG.Prolongator(_starts(dims, nv, 10), block)
    assert P.coarse_shape == (2, 1, 2, 2, 2, nv)
    c = W.gaussian_complex(P.coarse_shape, 1)
    np.testing.assert_allclose(P.restrict(P.prolong(c)), c, atol=1e-13)  # P^+ P = 1
    # P maps each coarse chirality into the matching gamma_5 eigenspace
    cp = c.copy()
    cp[..., 1, :] = 0
    f = P.prolong(cp)
    np.testing.assert_allclose(np.einsum("st,...tc->...sc", GAMMA5, f), f, atol=1e-13)
    # and P P^+ is an orthogonal projector onto the span of the null vectors
    v = _starts(dims, 1, 30)[0]
    pv = P.prolong(P.restrict(v))
    np.testing.assert_allclose(P.prolong(P.restrict(pv)), pv, atol=1e-12)
    assert abs(solvers.dot(v - pv, pv)) < 1e-10 * solvers.norm2(v)


def test_coarse_operator_inherits_gamma5_hermiticity():
    """A_c = P^+ M P with a chirality-preserving P satisfies A_c^+ = G5 A_c G5, G5 = diag(1, -1)
    on the coarse chirality index."""
    dims, block, nv = (4, 4, 4, 4), (2, 2, 2, 2), 4
    op = _op(dims, 0.12)
    top = MG.setup(op.M, (4, 4, 4, 4, 4, 3), [block], [nv], [_starts(dims, nv, 40)], relax_steps=5)
    g5c = lambda c: c * np.array([1.0, -1.0])[:, None]
    x = W.gaussian_complex(top.P.coarse_shape, 2)
    y = W.gaussian_complex(top.P.coarse_shape, 3)
    lhs = solvers.dot(x, top.Ac(y))
    rhs = solvers.dot(g5c(top.Ac(g5c(x))), y)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_null_vectors_are_near_kernel():
    dims = (4, 4, 4, 4)
    op = _op(dims, 0.124)
    s = _starts(dims, 3, 50)
    vs = MG.null_vectors(op.M, s, 30)
    for v0, v in zip(s, vs):
        ratio0 = np.sqrt(solvers.norm2(op.M(v0)) / solvers.norm2(v0))
        ratio = np.sqrt(solvers.norm2(op.M(v)))
        assert ratio < 0.3 * ratio0


def test_full_span_cycle_is_exact():
    """N_v equal to every degree of freedom of a block-chirality makes P unitary; with an
    exact coarse solve one cycle inverts M and FGCR stops after one iteration."""
    dims, block = (2, 2, 2, 2), (2, 2, 2, 2)
    nv = 16 * 6
    op = _op(dims, 0.12, eps=0.5, seed=3)
    starts = [W.gaussian_complex((2, 2, 2, 2, 4, 3), 100 + k) for k in range(nv)]
    top = MG.setup(op.M, (2, 2, 2, 2, 4, 3), [block], [nv], [starts], relax_steps=0, pre=1, post=1,
                   coarse_tol=1e-14, coarse_maxiter=2000, coarse_nkrylov=400)
    b = L.from_qdp(W.gaussian_fermion(dims, 7), dims)
    x, info = MG.solve(op.M, b, top, tol=1e-11)
    assert info["iters"] == 1
    assert op.true_residual(x, b) < 1e-11


@pytest.mark.parametrize("levels", [1, 2])
def test_multigrid_cuts_iterations(levels):
    """Near the critical kappa, FGCR with the two- or three-level cycle needs far fewer
    outer iterations than plain GCR(20), and reaches the requested true residual."""
    dims = (8, 8, 8, 8)
    op = _op(dims, 0.1255, eps=0.3, seed=5)
    b = L.from_qdp(W.point_source(dims, 0, 0), dims)
    tol = 1e-8
    _, plain = solvers.fgcr(op.M, b, tol=tol, maxiter=2000, nkrylov=20)
    blocks = [(2, 2, 2, 2)] * levels
    nvs = [8] * levels
    starts = [_starts(dims, 8, 200)]
    if levels == 2:
        starts.append([W.gaussian_complex((4, 4, 4, 4, 2, 8), 300 + k) for k in range(8)])
    top = MG.setup(op.M, (8, 8, 8, 8, 4, 3), blocks, nvs, starts, relax_steps=20)
    x, info = MG.solve(op.M, b, top, tol=tol)
    assert op.true_residual(x, b) <= tol * 1.01
    assert info["iters"] * 4 <= plain["iters"], (info["iters"], plain["iters"])


def test_coarse_stencil_equals_galerkin_product():
    """The nine-point coarse stencil read off column by column reproduces P^+ M P on
    random coarse vectors, and its blocks inherit gamma_5-hermiticity:
    Yb_mu(x + mu) = G5 Yf_mu(x)^+ G5 and X = G5 X^+ G5."""
    dims, block, nv = (6, 6, 6, 6), (2, 2, 2, 2), 2
    op = _op(dims, 0.12, seed=8)
    top = MG.setup(op.M, (6, 6, 6, 6, 4, 3), [block], [nv], [_starts(dims, nv, 60)], relax_steps=3)
    X, Yf, Yb = MG.coarse_stencil(op.M, top.P)
    for seed in (1, 2):
        c = W.gaussian_complex(top.P.coarse_shape, seed)
        np.testing.assert_allclose(MG.apply_stencil(X, Yf, Yb, c), top.Ac(c), atol=1e-12)
    g5 = np.diag([1.0] * nv + [-1.0] * nv)
    np.testing.assert_allclose(X, g5 @ np.conj(np.swapaxes(X, -1, -2)) @ g5, atol=1e-13)
    for mu in range(4):
        shifted = np.roll(Yb[mu], -1, axis=3 - mu)  # Yb_mu(x + mu) stored at x
        np.testing.assert_allclose(shifted, g5 @ np.conj(np.swapaxes(Yf[mu], -1, -2)) @ g5, atol=1e-13)


@pytest.mark.parametrize("aniso", [False, True])
def test_coarse_stencil_from_links(aniso):
    """The local construction from links, clover and P(x) equals the stencil read off
    the Galerkin product (isotropic and anisotropic operators, antiperiodic t)."""
    dims, block, nv = (6, 6, 6, 6), (2, 2, 2, 2), 2
    U = L.gauge_from_qdp(W.gauge_links(dims, 0.4, 9), dims)
    op = dirac.anisotropic(U, 0.1, 2.0, 0.9, 0.8, 1.1) if aniso else dirac.WilsonClover(U, 0.12, 1.2)
    top = MG.setup(op.M, (6, 6, 6, 6, 4, 3), [block], [nv], [_starts(dims, nv, 70)], relax_steps=3)
    ref = MG.coarse_stencil(op.M, top.P)
    got = MG.coarse_stencil_from_links(op, top.P)
    for a, b in zip(got, ref):
        np.testing.assert_allclose(a, b, atol=1e-12)
