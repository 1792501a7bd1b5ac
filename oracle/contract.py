"""Propagator workflow around the solve: wall and momentum sources, the sequential
source and the meson two- and three-point contractions (§III.A, §III.B).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Arrays are lexicographic like the rest of the oracle:

    propagator  (Lt, Lz, Ly, Lx, 4, 4, 3, 3)   [sink spin, source spin, sink colour, source colour]
    fermion     (Lt, Lz, Ly, Lx, 4, 3)

The propagator axis order is the sink-source spin, sink-source colour order of §II.A.
Source column (s0, c0) of a propagator is the solution for the source with spin s0 and
colour c0: S[..., s, s0, c, c0] = x_{3 s0 + c0}[..., s, c].

Readings of the paper taken here:

* Momentum phase.  Eq. 1 and Eq. 2 carry exp(-i p.x) at the sink and exp(+i p.x0) at
  the source, and in §III.B the momentum source is filled with the same phase array
  whose conjugate multiplies the sink.  The source of the momentum propagator is
  therefore exp(+i p.x0) on the wall, S_p(x) = sum_x0 exp(+i p.x0) S(x; x0); the
  definition printed after Eq. 2 has the opposite sign, which would make the
  correlator carry no definite momentum.  p = 2 pi n / L per spatial axis, n integer.
* Eq. 6 and Eq. 7 contract conj(A)[j, i, b, a] Gamma[j, k] B[k, i, b, a] summed over
  every spin and colour index and over the sites of each timeslice, with the phase
  exp(-i p.x) of the sink site.
* The sequential source (the unnumbered equation after Eq. 7, built from Eq. 4) is
  X[i, k, a, b] = exp(-i p.x) gamma_5[i, j] S_0[j, k, a, b] on the sink timeslice and
  zero elsewhere.
"""
import numpy as np

from . import gamma as G
from . import solvers


def _spatial_coords(dims):
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    return x, y, z, t


def momentum_phase(dims, mom):
    """exp(+i p.x), p_k = 2 pi n_k / L_k for the three spatial axes, on every site
    (shape (Lt, Lz, Ly, Lx)).  Pinned by the plane-wave orthogonality sum and the
    point-source correlator identity of the tests."""
    lx, ly, lz, lt = dims
    x, y, z, _ = _spatial_coords(dims)
    arg = 2 * np.pi * (mom[0] * x / lx + mom[1] * y / ly + mom[2] * z / lz)
    return np.exp(1j * arg)


def wall_sources(dims, t0, mom=(0, 0, 0)):
    """The twelve spin-colour wall sources on timeslice t0 (§III.B): field 3 s + c is
    the momentum phase in spin s and colour c on timeslice t0 and zero elsewhere.
    Shape (12, Lt, Lz, Ly, Lx, 4, 3)."""
    lx, ly, lz, lt = dims
    ph = momentum_phase(dims, mom)
    out = np.zeros((12, lt, lz, ly, lx, 4, 3), dtype=np.complex128)
    for s in range(4):
        for c in range(3):
            out[3 * s + c, t0, :, :, :, s, c] = ph[t0]
    return out


def point_sources(dims, site):
    """The twelve spin-colour unit sources at one site (x, y, z, t)."""
    lx, ly, lz, lt = dims
    x, y, z, t = site
    out = np.zeros((12, lt, lz, ly, lx, 4, 3), dtype=np.complex128)
    for s in range(4):
        for c in range(3):
            out[3 * s + c, t, z, y, x, s, c] = 1.0
    return out


def fermions_to_propagator(x12):
    """(12, ..., 4, 3) solutions, source k = 3 s0 + c0 -> (..., 4, 4, 3, 3)."""
    sh = x12.shape[1:-2]
    prop = np.zeros(sh + (4, 4, 3, 3), dtype=np.complex128)
    for s0 in range(4):
        for c0 in range(3):
            prop[..., :, s0, :, c0] = x12[3 * s0 + c0]
    return prop


def propagator_to_fermions(prop):
    return np.stack([prop[..., :, s0, :, c0] for s0 in range(4) for c0 in range(3)])


def propagator(op, sources12, tol=1e-12):
    """Solve M x = b for each of the twelve sources with the oracle's even-odd BiCGStab
    and assemble the propagator (§III.B: twelve inversions per propagator)."""
    xs = []
    for b in sources12:
        x, info = solvers.solve_even_odd(op, b, tol=tol)
        if info["status"] != "ok":
            raise RuntimeError(f"oracle solve did not converge: {info}")
        xs.append(x)
    return fermions_to_propagator(np.stack(xs))


def sequential_source(S, t, mom=(0, 0, 0), gamma=None):
    """X[x, i, k, a, b] = exp(-i p.x) sum_j Gamma[i, j] S[x, j, k, a, b] on timeslice t,
    zero elsewhere (Eq. 4 and the sequential-source equation of §III.B; Gamma =
    gamma_5 when not given).  Pinned against a dense-inverse construction of Eq. 4."""
    gm = G.GAMMA5 if gamma is None else gamma
    dims = (S.shape[3], S.shape[2], S.shape[1], S.shape[0])
    ph = np.conj(momentum_phase(dims, mom))
    X = np.zeros_like(S)
    for i in range(4):
        for j in range(4):
            if gm[i, j] != 0:
                X[t, :, :, :, i] += gm[i, j] * S[t, :, :, :, j]
    X[t] *= ph[t][..., None, None, None, None]
    return X


def contract(A, B, gamma=None, mom=(0, 0, 0)):
    """C(t) = sum over the sites x of timeslice t of exp(-i p.x) times
    sum_{i,j,k,a,b} conj(A[x, j, i, b, a]) Gamma[j, k] B[x, k, i, b, a]  (Eq. 6, Eq. 7;
    Gamma = 1 when not given).  Returns Lt complex values.  Pinned against the
    dense-inverse forms of Eq. 1 (both lines) and Eq. 3 and by gauge invariance."""
    gm = np.eye(4) if gamma is None else gamma
    dims = (A.shape[3], A.shape[2], A.shape[1], A.shape[0])
    ph = np.conj(momentum_phase(dims, mom))
    # GB[x, j, i, b, a] = sum_k Gamma[j, k] B[x, k, i, b, a]
    GB = np.zeros_like(B)
    for j in range(4):
        for k in range(4):
            if gm[j, k] != 0:
                GB[..., j, :, :, :] += gm[j, k] * B[..., k, :, :, :]
    per_site = np.sum(np.conj(A) * GB, axis=(4, 5, 6, 7))
    return np.sum(ph * per_site, axis=(1, 2, 3))


def two_point(S0, Sp, mom):
    """Pion two-point function from the zero- and p-momentum wall propagators (Eq. 6)."""
    return contract(S0, Sp, None, mom)


def three_point(Sseq, Sp):
    """Vector-current three-point function, Gamma = gamma_5 gamma_3 (Eq. 7)."""
    return contract(Sseq, Sp, G.GAMMA5 @ G.GAMMA[2], (0, 0, 0))
