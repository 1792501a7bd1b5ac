"""Gauge-covariant parallel-transport convolution (PTC) network, FP64 oracle.

The paper itself has no learned component; this module defines the learned
preconditioner for flexible GCR as a linear stack of PTC layers
(gauge-equivariant layers in the style of Lehner and Wettig, 2023):

    out_{c'}(x) = sum_{c, s} W[c', c, s] (T_s in_c)(x)

for shifts s in {0, +x, -x, +y, -y, +z, -z, +t, -t} (index 0, then 1+2mu for
+mu and 2+2mu for -mu), with W[c', c, s] a complex 4x4 matrix on spin and the
parallel transports

    T_0 psi(x)   = psi(x)
    T_+mu psi(x) = eta+ U_mu(x) psi(x + mu)
    T_-mu psi(x) = eta- U_mu(x - mu)^+ psi(x - mu)

(eta: the fermion time boundary, as in the Dirac operator).  Because every
term moves colour with a link, a layer commutes with gauge transformations, so
the weights do not depend on the gauge configuration.  Default architecture:
channels 1 -> 4 -> 4 -> 4 -> 1, no nonlinearity.

Training objective: L = (1/B) sum_b ||N(r_b) - e_b||^2 / ||e_b||^2.

Gradients use G = dL/dRe + i dL/dIm for every complex variable:
    G_W[c',c,s]  = sum_x G_out[c'](x) (T_s in_c)(x)^+      (spin x spin, colour summed)
    G_in[c]      = sum_{c',s} T_s^+ (W[c',c,s]^+ G_out[c']),   T_{+mu}^+ = T_{-mu}.

Pins (tests/test_oracle_ptc.py): gauge covariance of a layer, adjointness
<phi, T_s psi> = <T_s^+ phi, psi>, central finite differences of the loss.
"""
import numpy as np

from . import lattice as L

NSHIFT = 9
DEFAULT_CHANNELS = (1, 4, 4, 4, 1)


def _dag(u):
    return np.conj(np.swapaxes(u, -1, -2))


def transport(U, psi, s, t_boundary=-1):
    """T_s psi for one field (Lt, Lz, Ly, Lx, 4, 3)."""
    if s == 0:
        return psi.copy()
    mu, back = (s - 1) // 2, (s - 1) % 2 == 1
    dims = L.dims_of(psi)
    if not back:
        out = np.einsum("...ab,...sb->...sa", U[mu], L.fwd(psi, mu))
    else:
        out = np.einsum("...ab,...sb->...sa", _dag(L.bwd(U[mu], mu)), L.bwd(psi, mu))
    if mu == 3:
        out = out * L.time_boundary_sign(dims, t_boundary, not back)[..., None, None]
    return out


def transport_adjoint(U, psi, s, t_boundary=-1):
    """T_s^+ psi: the adjoint of +mu is -mu and vice versa."""
    if s == 0:
        return psi.copy()
    return transport(U, psi, s + 1 if (s - 1) % 2 == 0 else s - 1, t_boundary)


def layer_forward(U, W, x, t_boundary=-1):
    """x: (Cin, Lt, Lz, Ly, Lx, 4, 3); W: (Cout, Cin, 9, 4, 4) -> (Cout, ...)."""
    cout, cin = W.shape[:2]
    out = np.zeros((cout,) + x.shape[1:], dtype=np.complex128)
    for c in range(cin):
        for s in range(NSHIFT):
            ts = transport(U, x[c], s, t_boundary)
            out += np.einsum("oab,...bc->o...ac", W[:, c, s], ts)
    return out


def layer_backward(U, W, x, g_out, t_boundary=-1):
    """Return (G_W, G_x) for one layer given G_out (Cout, ...)."""
    cout, cin = W.shape[:2]
    gW = np.zeros_like(W)
    gx = np.zeros_like(x)
    for c in range(cin):
        for s in range(NSHIFT):
            ts = transport(U, x[c], s, t_boundary)
            go = g_out.reshape(cout, -1, 4, 3)
            gW[:, c, s] = np.einsum("oxac,xbc->oab", go, ts.reshape(-1, 4, 3).conj())
            back = np.einsum("oba,o...bc->...ac", W[:, c, s].conj(), g_out)
            gx[c] += transport_adjoint(U, back, s, t_boundary)
    return gW, gx


def init_weights(channels=DEFAULT_CHANNELS, seed=0, scale=None):
    """Random complex weights, N(0, scale^2) in real and imaginary parts."""
    rng = np.random.default_rng(seed)
    ws = []
    for cin, cout in zip(channels[:-1], channels[1:]):
        sc = scale if scale is not None else 0.1 / np.sqrt(cin * NSHIFT)
        w = sc * (rng.standard_normal((cout, cin, NSHIFT, 4, 4)) + 1j * rng.standard_normal((cout, cin, NSHIFT, 4, 4)))
        ws.append(w)
    return ws


def forward(U, weights, r, t_boundary=-1):
    """N(r) for one field r (Lt, Lz, Ly, Lx, 4, 3); returns (output, activations)."""
    acts = [r[None]]
    for W in weights:
        acts.append(layer_forward(U, W, acts[-1], t_boundary))
    return acts[-1][0], acts


def loss_and_grad(U, weights, rs, es, t_boundary=-1, mask=None):
    """Relative squared error averaged over the batch, and G_W for every layer.

    With a site mask (boolean (Lt, Lz, Ly, Lx)), only the masked sites of the
    output enter the loss: the even-odd form of the preconditioner, whose input
    is an even-parity field and whose even output approximates M_hat^-1 r.
    """
    nb = len(rs)
    total = 0.0
    grads = [np.zeros_like(W) for W in weights]
    m = 1.0 if mask is None else mask[..., None, None]
    for r, e in zip(rs, es):
        out, acts = forward(U, weights, r, t_boundary)
        e = e * m
        en = float(np.vdot(e, e).real)
        diff = (out - e) * m
        total += float(np.vdot(diff, diff).real) / en / nb
        g = (2.0 / en / nb) * diff[None]
        for li in range(len(weights) - 1, -1, -1):
            gW, g = layer_backward(U, weights[li], acts[li], g, t_boundary)
            grads[li] += gW
    return total, grads


def adam_step(weights, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """Adam on the real and imaginary parts separately (G = dL/dRe + i dL/dIm)."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    out = []
    for i, (W, g) in enumerate(zip(weights, grads)):
        gr = np.stack([g.real, g.imag])
        m = state.setdefault(("m", i), np.zeros_like(gr))
        v = state.setdefault(("v", i), np.zeros_like(gr))
        m[:] = b1 * m + (1 - b1) * gr
        v[:] = b2 * v + (1 - b2) * gr * gr
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        upd = lr * mh / (np.sqrt(vh) + eps)
        out.append(W - (upd[0] + 1j * upd[1]))
    return out
