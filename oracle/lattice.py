"""Lattice layouts and nearest-neighbour shifts for the oracle (Sec. II.A).

Oracle arrays are lexicographic with leading site axes (Lt, Lz, Ly, Lx):

    fermion  (Lt, Lz, Ly, Lx, 4, 3)
    gauge    (4, Lt, Lz, Ly, Lx, 3, 3)    U[mu][s] is the link s -> s + mu_hat

The boundary format is the QDP cb2 layout [2][Lt][Lz][Ly][Lx/2][...]: parity
p = (x+y+z+t) mod 2 first, then the checkerboarded site index
cb = ((t*Lz + z)*Ly + y)*(Lx/2) + x//2.  The conversion below is written
independently of the generator module (site loop over lexicographic coordinates).

Direction mu = 0, 1, 2, 3 is x, y, z, t; in the (Lt, Lz, Ly, Lx) arrays that is
array axis 3, 2, 1, 0.
"""
import numpy as np

AXIS = (3, 2, 1, 0)


def dims_of(field: np.ndarray):
    lt, lz, ly, lx = field.shape[:4]
    return (lx, ly, lz, lt)


def _cb_coords(dims):
    lx, ly, lz, lt = dims
    t = np.arange(lt)[:, None, None, None]
    z = np.arange(lz)[None, :, None, None]
    y = np.arange(ly)[None, None, :, None]
    x = np.arange(lx)[None, None, None, :]
    p = (x + y + z + t) % 2
    xh = x // 2
    p, t, z, y, xh = np.broadcast_arrays(p, t, z, y, xh)
    return p, t, z, y, xh


def from_qdp(qdp: np.ndarray, dims) -> np.ndarray:
    """QDP cb2 field [2][Lt][Lz][Ly][Lx/2][...] -> lexicographic (Lt, Lz, Ly, Lx, ...)."""
    p, t, z, y, xh = _cb_coords(dims)
    return np.ascontiguousarray(qdp[p, t, z, y, xh])


def to_qdp(lex: np.ndarray, dims) -> np.ndarray:
    """Lexicographic (Lt, Lz, Ly, Lx, ...) -> QDP cb2 [2][Lt][Lz][Ly][Lx/2][...]."""
    lx, ly, lz, lt = dims
    p, t, z, y, xh = _cb_coords(dims)
    out = np.zeros((2, lt, lz, ly, lx // 2) + lex.shape[4:], dtype=lex.dtype)
    out[p, t, z, y, xh] = lex
    return out


def gauge_from_qdp(qdp: np.ndarray, dims) -> np.ndarray:
    """QDP gauge [4][2][Lt][Lz][Ly][Lx/2][3][3] -> (4, Lt, Lz, Ly, Lx, 3, 3)."""
    return np.stack([from_qdp(qdp[mu], dims) for mu in range(4)])


def gauge_to_qdp(lex: np.ndarray, dims) -> np.ndarray:
    return np.stack([to_qdp(lex[mu], dims) for mu in range(4)])


def parity_mask(dims, parity: int) -> np.ndarray:
    """Boolean (Lt, Lz, Ly, Lx) mask of sites with (x+y+z+t) mod 2 == parity."""
    p = _cb_coords(dims)[0]
    return p == parity


def fwd(field: np.ndarray, mu: int) -> np.ndarray:
    """g(s) = f(s + mu_hat), periodic wrap; site axes must lead (or follow a leading mu axis)."""
    return np.roll(field, -1, axis=AXIS[mu])


def bwd(field: np.ndarray, mu: int) -> np.ndarray:
    """g(s) = f(s - mu_hat), periodic wrap."""
    return np.roll(field, +1, axis=AXIS[mu])


def time_boundary_sign(dims, t_boundary: int, forward: bool) -> np.ndarray:
    """eta(s) per site for the mu = t hop (Sec. III.B: t_boundary = -1 is antiperiodic).

    Forward hops from t = Lt-1 and backward hops from t = 0 cross the boundary
    and pick up the factor t_boundary; every other hop has eta = 1.
    """
    lx, ly, lz, lt = dims
    eta = np.ones((lt, 1, 1, 1))
    eta[lt - 1 if forward else 0] = t_boundary
    return eta
