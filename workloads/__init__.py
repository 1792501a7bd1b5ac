"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and bench.py.

This module draws random numbers and lays them out in the QDP checkerboard
("cb2") convention of the paper (Sec. II.A):

    gauge    [Nd=4][2][Lt][Lz][Ly][Lx/2][Nc][Nc]   complex128, row-column colour
    fermion  [2][Lt][Lz][Ly][Lx/2][Ns][Nc]         complex128

It holds none of the Dirac-operator or solver arithmetic: the only
computation here is the synthetic gauge-link recipe
U = exp(i*eps*sum_a r_a*lambda_a/2) with r_a ~ N(0,1), which is how the
benchmark workloads are defined, and plain index permutations into cb2 order.
Both the CPU oracle and the CUDA path receive the arrays built here.

Random draws use numpy's PCG64 (``numpy.random.default_rng(seed)``).  Gauge
generators r are drawn with shape (Lt, Lz, Ly, Lx, 4, 8), i.e. lexicographic
site order with x fastest, then reordered to cb2.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "GELL_MANN",
    "lex_to_cb2_index",
    "sites_to_cb2",
    "gauge_links",
    "unit_gauge",
    "gaussian_fermion",
    "z2_fermion",
    "point_source",
    "random_su3",
]


def _gell_mann() -> np.ndarray:
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1] = -1j
    lam[1][1, 0] = 1j
    lam[2][0, 0] = 1
    lam[2][1, 1] = -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2] = -1j
    lam[4][2, 0] = 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2] = -1j
    lam[6][2, 1] = 1j
    lam[7][0, 0] = lam[7][1, 1] = 1 / np.sqrt(3)
    lam[7][2, 2] = -2 / np.sqrt(3)
    return lam


#: The eight Gell-Mann matrices, normalised so that Tr(l_a l_b) = 2 delta_ab.
GELL_MANN = _gell_mann()


def _check_dims(dims) -> tuple[int, int, int, int]:
    lx, ly, lz, lt = (int(d) for d in dims)
    if min(lx, ly, lz, lt) < 2 or lx % 2:
        raise ValueError(f"lattice dims {dims}: every extent >= 2 and Lx even")
    return lx, ly, lz, lt


def lex_to_cb2_index(dims):
    """Return (parity, cb) integer arrays of shape (Lt, Lz, Ly, Lx).

    parity = (x+y+z+t) mod 2 and cb = ((t*Lz+z)*Ly+y)*(Lx/2) + x//2 (Sec. II.A).
    """
    lx, ly, lz, lt = _check_dims(dims)
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    parity = (x + y + z + t) % 2
    cb = ((t * lz + z) * ly + y) * (lx // 2) + x // 2
    return parity, cb


def sites_to_cb2(field_lex: np.ndarray, dims) -> np.ndarray:
    """Permute a field with leading site axes (Lt, Lz, Ly, Lx) into (2, Lt, Lz, Ly, Lx/2)."""
    lx, ly, lz, lt = _check_dims(dims)
    parity, cb = lex_to_cb2_index(dims)
    tail = field_lex.shape[4:]
    out = np.empty((2, lt * lz * ly * (lx // 2)) + tail, dtype=field_lex.dtype)
    flat = field_lex.reshape((-1,) + tail)
    out[parity.ravel(), cb.ravel()] = flat
    return out.reshape((2, lt, lz, ly, lx // 2) + tail)


def _su3_from_generators(r: np.ndarray, eps: float) -> np.ndarray:
    """U = exp(i eps H), H = sum_a r_a lambda_a / 2, via the eigendecomposition of H."""
    h = np.einsum("...a,aij->...ij", r, GELL_MANN) * 0.5
    w, v = np.linalg.eigh(h)
    return np.einsum("...ij,...j,...kj->...ik", v, np.exp(1j * eps * w), v.conj())


def gauge_links(dims, eps: float, seed: int) -> np.ndarray:
    """Synthetic gauge field U_mu(s) = exp(i eps sum_a r_a lambda_a/2), r_a ~ N(0,1).

    Returns the QDP cb2 array [4][2][Lt][Lz][Ly][Lx/2][3][3] complex128.
    """
    lx, ly, lz, lt = _check_dims(dims)
    rng = np.random.default_rng(seed)
    r = rng.standard_normal((lt, lz, ly, lx, 4, 8))
    u = _su3_from_generators(r, eps)  # (Lt,Lz,Ly,Lx,4,3,3)
    u = np.moveaxis(u, 4, 0)  # (4,Lt,Lz,Ly,Lx,3,3)
    return np.ascontiguousarray(np.stack([sites_to_cb2(u[mu], dims) for mu in range(4)]))


def unit_gauge(dims) -> np.ndarray:
    """Free field: every link the 3x3 identity, QDP cb2 layout."""
    lx, ly, lz, lt = _check_dims(dims)
    u = np.zeros((4, 2, lt, lz, ly, lx // 2, 3, 3), dtype=np.complex128)
    u[..., 0, 0] = u[..., 1, 1] = u[..., 2, 2] = 1
    return u


def gaussian_fermion(dims, seed: int, nrhs: int | None = None) -> np.ndarray:
    """Gaussian spinor field, re and im ~ N(0,1), drawn in lexicographic order."""
    lx, ly, lz, lt = _check_dims(dims)
    rng = np.random.default_rng(seed)
    n = 1 if nrhs is None else nrhs
    out = []
    for _ in range(n):
        z = rng.standard_normal((lt, lz, ly, lx, 4, 3, 2))
        out.append(sites_to_cb2(z[..., 0] + 1j * z[..., 1], dims))
    out = np.stack(out)
    return out[0] if nrhs is None else out


def z2_fermion(dims, seed: int, nrhs: int | None = None) -> np.ndarray:
    """Z2 noise: every complex component (+-1 +- i)/sqrt(2)."""
    lx, ly, lz, lt = _check_dims(dims)
    rng = np.random.default_rng(seed)
    n = 1 if nrhs is None else nrhs
    out = []
    for _ in range(n):
        s = rng.integers(0, 2, size=(lt, lz, ly, lx, 4, 3, 2)) * 2 - 1
        out.append(sites_to_cb2((s[..., 0] + 1j * s[..., 1]) / np.sqrt(2.0), dims))
    out = np.stack(out)
    return out[0] if nrhs is None else out


def point_source(dims, spin: int, colour: int, site=(0, 0, 0, 0)) -> np.ndarray:
    """Unit point source at site (x,y,z,t), given spin and colour, QDP cb2 layout."""
    lx, ly, lz, lt = _check_dims(dims)
    x, y, z, t = site
    out = np.zeros((2, lt, lz, ly, lx // 2, 4, 3), dtype=np.complex128)
    p = (x + y + z + t) % 2
    out[p, t, z, y, x // 2, spin, colour] = 1.0
    return out


def random_su3(dims, seed: int) -> np.ndarray:
    """Haar-ish random SU(3) matrix per site (for gauge transformations), lexicographic (Lt,Lz,Ly,Lx,3,3)."""
    lx, ly, lz, lt = _check_dims(dims)
    rng = np.random.default_rng(seed)
    r = rng.standard_normal((lt, lz, ly, lx, 8))
    return _su3_from_generators(r, 2.0)



def ptc_weights(channels, seed: int, scale: float, nshift: int = 9) -> list[np.ndarray]:
    """Random complex weights of a PTC network with the given channel counts: one
    array [c_out][c_in][nshift][4][4] per layer, real and imaginary parts N(0, scale^2)."""
    rng = np.random.default_rng(seed)
    ws = []
    for cin, cout in zip(channels[:-1], channels[1:]):
        shape = (cout, cin, nshift, 4, 4)
        ws.append(scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)))
    return ws


def gaussian_propagator(dims, seed: int) -> np.ndarray:
    """Gaussian propagator-shaped field, re and im ~ N(0,1), drawn in lexicographic
    order; QDP layout [2][Lt][Lz][Ly][Lx/2][4][4][3][3]."""
    lx, ly, lz, lt = _check_dims(dims)
    z = np.random.default_rng(seed).standard_normal((lt, lz, ly, lx, 4, 4, 3, 3, 2))
    return sites_to_cb2(z[..., 0] + 1j * z[..., 1], dims)


def gaussian_propagator_runs(dims, t: int, seed: int) -> np.ndarray:
    """Gaussian data for the two storage runs of timeslice t of a QDP propagator (the
    sites of parity 0, then of parity 1, each in [Lz][Ly][Lx/2] order): shape
    [2][Lz][Ly][Lx/2][4][4][3][3]."""
    lx, ly, lz, lt = _check_dims(dims)
    z = np.random.default_rng([seed, t]).standard_normal((2, lz, ly, lx // 2, 4, 4, 3, 3, 2))
    return z[..., 0] + 1j * z[..., 1]


def gaussian_complex(shape, seed: int) -> np.ndarray:
    """Complex Gaussian array of any shape (re, im ~ N(0,1)), e.g. the random starts of a
    coarse level's null-space vectors."""
    z = np.random.default_rng(seed).standard_normal(tuple(shape) + (2,))
    return z[..., 0] + 1j * z[..., 1]
