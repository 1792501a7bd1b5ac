"""Pins for the oracle's parallel-transport network (learned preconditioner)."""
import numpy as np
import pytest

import workloads as W
from oracle import dirac, ptc
from oracle import lattice as L
from oracle.gamma import GAMMA


def _field(dims, seed, n=None):
    q = W.gaussian_fermion(dims, seed)
    return L.from_qdp(q, dims)


def test_transport_adjoint():
    dims = (4, 2, 2, 4)
    U = L.gauge_from_qdp(W.gauge_links(dims, 0.8, 1), dims)
    phi, psi = _field(dims, 2), _field(dims, 3)
    for s in range(ptc.NSHIFT):
        lhs = np.vdot(phi, ptc.transport(U, psi, s))
        rhs = np.vdot(ptc.transport_adjoint(U, phi, s), psi)
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_layer_reproduces_wilson_operator():
    """A single 1->1 layer with W_0 = 1, W_{+mu} = -kappa(1-gamma_mu), W_{-mu} = -kappa(1+gamma_mu)
    is the c_sw = 0 Wilson operator 1 - kappa H (pinned separately against closed forms)."""
    dims = (4, 4, 2, 4)
    U = L.gauge_from_qdp(W.gauge_links(dims, 0.5, 6), dims)
    kappa = 0.12
    Wt = np.zeros((1, 1, 9, 4, 4), dtype=np.complex128)
    Wt[0, 0, 0] = np.eye(4)
    for mu in range(4):
        Wt[0, 0, 1 + 2 * mu] = -kappa * (np.eye(4) - GAMMA[mu])
        Wt[0, 0, 2 + 2 * mu] = -kappa * (np.eye(4) + GAMMA[mu])
    psi = _field(dims, 7)
    out = ptc.layer_forward(U, Wt, psi[None])[0]
    np.testing.assert_allclose(out, dirac.WilsonClover(U, kappa, 0.0).M(psi), atol=1e-13)


def test_layer_gauge_covariance():
    dims = (4, 2, 4, 2)
    U = L.gauge_from_qdp(W.gauge_links(dims, 0.7, 2), dims)
    om = W.random_su3(dims, 5)
    Uo = np.empty_like(U)
    for mu in range(4):
        Uo[mu] = np.einsum("...ab,...bc,...dc->...ad", om, U[mu], L.fwd(om, mu).conj())
    ws = ptc.init_weights((2, 3), seed=1, scale=0.3)
    x = np.stack([_field(dims, 8), _field(dims, 9)])
    rot = lambda f: np.einsum("...ab,...sb->...sa", om, f)
    lhs = ptc.layer_forward(Uo, ws[0], np.stack([rot(c) for c in x]))
    rhs = np.stack([rot(c) for c in ptc.layer_forward(U, ws[0], x)])
    np.testing.assert_allclose(lhs, rhs, atol=1e-12)


@pytest.mark.parametrize("layer", [0, 1, 3])
def test_gradient_finite_differences(layer):
    dims = (2, 2, 2, 4)
    U = L.gauge_from_qdp(W.gauge_links(dims, 0.6, 3), dims)
    ws = ptc.init_weights(ptc.DEFAULT_CHANNELS, seed=2, scale=0.2)
    rs = [_field(dims, 10), _field(dims, 11)]
    es = [_field(dims, 12), _field(dims, 13)]
    _, grads = ptc.loss_and_grad(U, ws, rs, es)
    rng = np.random.default_rng(layer)
    h = 1e-6
    for _ in range(4):
        idx = tuple(rng.integers(0, n) for n in ws[layer].shape)
        for part, unit in (("re", 1.0), ("im", 1j)):
            wp = [w.copy() for w in ws]
            wm = [w.copy() for w in ws]
            wp[layer][idx] += h * unit
            wm[layer][idx] -= h * unit
            fd = (ptc.loss_and_grad(U, wp, rs, es)[0] - ptc.loss_and_grad(U, wm, rs, es)[0]) / (2 * h)
            an = grads[layer][idx].real if part == "re" else grads[layer][idx].imag
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (idx, part, fd, an)


def test_masked_loss_gradient_finite_differences():
    """Loss restricted to even sites (the even-odd preconditioner's objective)."""
    dims = (2, 2, 2, 4)
    U = L.gauge_from_qdp(W.gauge_links(dims, 0.6, 8), dims)
    ws = ptc.init_weights(ptc.DEFAULT_CHANNELS, seed=4, scale=0.2)
    even = L.parity_mask(dims, 0)
    rs = [_field(dims, 40) * even[..., None, None]]
    es = [_field(dims, 41) * even[..., None, None]]
    _, grads = ptc.loss_and_grad(U, ws, rs, es, mask=even)
    h = 1e-6
    for layer, idx in [(0, (1, 0, 3, 2, 1)), (2, (3, 1, 8, 0, 3)), (3, (0, 2, 0, 1, 1))]:
        for unit, part in ((1.0, "re"), (1j, "im")):
            wp = [w.copy() for w in ws]
            wm = [w.copy() for w in ws]
            wp[layer][idx] += h * unit
            wm[layer][idx] -= h * unit
            fd = (ptc.loss_and_grad(U, wp, rs, es, mask=even)[0] - ptc.loss_and_grad(U, wm, rs, es, mask=even)[0]) / (2 * h)
            an = grads[layer][idx].real if part == "re" else grads[layer][idx].imag
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))


def test_input_gradient_finite_differences():
    dims = (2, 2, 2, 4)
    U = L.gauge_from_qdp(W.gauge_links(dims, 0.6, 4), dims)
    ws = ptc.init_weights((2, 3), seed=3, scale=0.3)
    x = np.stack([_field(dims, 20), _field(dims, 21)])
    target = ptc.layer_forward(U, ws[0], x) * 0.5 + 0.1
    loss = lambda xx: float(np.sum(np.abs(ptc.layer_forward(U, ws[0], xx) - target) ** 2))
    g_out = 2 * (ptc.layer_forward(U, ws[0], x) - target)
    _, gx = ptc.layer_backward(U, ws[0], x, g_out)
    h = 1e-6
    rng = np.random.default_rng(0)
    for _ in range(6):
        idx = tuple(rng.integers(0, n) for n in x.shape)
        for unit, part in ((1.0, "re"), (1j, "im")):
            xp, xm = x.copy(), x.copy()
            xp[idx] += h * unit
            xm[idx] -= h * unit
            fd = (loss(xp) - loss(xm)) / (2 * h)
            an = gx[idx].real if part == "re" else gx[idx].imag
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))


def test_adam_reduces_loss():
    dims = (2, 2, 2, 4)
    U = L.gauge_from_qdp(W.gauge_links(dims, 0.3, 5), dims)
    op = dirac.WilsonClover(U, 0.12, 1.0)
    es = [_field(dims, 30 + k) for k in range(3)]
    rs = [op.M(e) for e in es]
    ws = ptc.init_weights(ptc.DEFAULT_CHANNELS, seed=0)
    l0, g = ptc.loss_and_grad(U, ws, rs, es)
    state = {}
    for _ in range(30):
        ws = ptc.adam_step(ws, g, state, lr=1e-2)
        l1, g = ptc.loss_and_grad(U, ws, rs, es)
    assert l1 < 0.5 * l0


def test_adam_two_steps_closed_form():
    """Two Adam steps on L = sum |W|^2 (G = dL/dRe W + i dL/dIm W = 2 W) from W = 1 + 2i,
    written out from the update rule with bias correction (Kingma & Ba 2015, Algorithm 1)
    on the real and imaginary parts separately:
      step 1: m = (1-b1) g, v = (1-b2) g^2, m/(1-b1) = g, v/(1-b2) = g^2,
              W1 = W0 - lr g / (|g| + eps)
      step 2: m = b1 (1-b1) g1 + (1-b1) g2, v = b2 (1-b2) g1^2 + (1-b2) g2^2,
              W2 = W1 - lr (m / (1-b1^2)) / (sqrt(v / (1-b2^2)) + eps)."""
    lr, b1, b2, eps = 0.1, 0.9, 0.999, 1e-8
    w0 = np.array([1.0 + 2.0j])
    state = {}
    w1 = ptc.adam_step([w0], [2 * w0], state, lr=lr, b1=b1, b2=b2, eps=eps)[0]
    # step 1 by hand: g = (2, 4)
    e1 = (1.0 - 0.1 * 2.0 / (2.0 + 1e-8)) + 1j * (2.0 - 0.1 * 4.0 / (4.0 + 1e-8))
    assert abs(w1[0] - e1) <= 1e-15
    w2 = ptc.adam_step([w1], [2 * w1], state, lr=lr, b1=b1, b2=b2, eps=eps)[0]
    # step 2 by hand: g1 = (2, 4), g2 = 2 * w1 = (1.8, 3.8) up to the eps terms
    g2r, g2i = 2 * e1.real, 2 * e1.imag
    mr = (0.9 * 0.1 * 2.0 + 0.1 * g2r) / (1 - 0.81)
    mi = (0.9 * 0.1 * 4.0 + 0.1 * g2i) / (1 - 0.81)
    vr = (0.999 * 0.001 * 4.0 + 0.001 * g2r ** 2) / (1 - 0.998001)
    vi = (0.999 * 0.001 * 16.0 + 0.001 * g2i ** 2) / (1 - 0.998001)
    e2 = (e1.real - 0.1 * mr / (np.sqrt(vr) + 1e-8)) + 1j * (e1.imag - 0.1 * mi / (np.sqrt(vi) + 1e-8))
    assert abs(w2[0] - e2) <= 1e-14
    # the numbers themselves: first step moves each part by lr, the second by about lr
    assert abs(w1[0] - (0.9 + 1.9j)) <= 1e-8
    assert abs(w2[0] - (0.800412 + 1.800166j)) <= 1e-6
