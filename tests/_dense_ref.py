"""A second, loop-based definition of the Wilson-clover matrix for tiny lattices.

Written site by site with integer coordinate arithmetic (no array rolls, no
einsum over the lattice) so that it shares no indexing code with the
vectorised oracle.  Used only to pin the oracle on 2^4 and 4^4 lattices:
the dense matrix M (12V x 12V) with vector index ((t*Lz+z)*Ly+y)*Lx+x)*12 + 3*spin + colour.
"""
import numpy as np

from oracle.gamma import GAMMA


def _coords(dims):
    lx, ly, lz, lt = dims
    for t in range(lt):
        for z in range(lz):
            for y in range(ly):
                for x in range(lx):
                    yield (x, y, z, t)


def site_index(c, dims):
    lx, ly, lz, lt = dims
    x, y, z, t = c
    return ((t * lz + z) * ly + y) * lx + x


def step(c, mu, d, dims):
    c = list(c)
    c[mu] = (c[mu] + d) % dims[mu]
    return tuple(c)


def link(U, c, mu):
    """U[mu] in lexicographic oracle layout (Lt, Lz, Ly, Lx, 3, 3) at coordinate c=(x,y,z,t)."""
    x, y, z, t = c
    return U[mu][t, z, y, x]


def leaf_sum(U, c, mu, nu, dims):
    """Sum of the four plaquettes in the (mu, nu) plane through site c, walked one link at a time."""
    def walk(path):
        m = np.eye(3, dtype=np.complex128)
        cur = c
        for direction, sign in path:
            if sign > 0:
                m = m @ link(U, cur, direction)
                cur = step(cur, direction, +1, dims)
            else:
                prev = step(cur, direction, -1, dims)
                m = m @ link(U, prev, direction).conj().T
                cur = prev
        assert cur == c
        return m

    return (walk([(mu, 1), (nu, 1), (mu, -1), (nu, -1)])
            + walk([(nu, 1), (mu, -1), (nu, -1), (mu, 1)])
            + walk([(mu, -1), (nu, -1), (mu, 1), (nu, 1)])
            + walk([(nu, -1), (mu, 1), (nu, 1), (mu, -1)]))


def dense_matrix(U, dims, kappa, csw, t_boundary=-1, aniso=None):
    """Eq. 5; aniso = (xi0, nu, csw_t, csw_r) gives the anisotropic form: spatial hops
    times nu/xi0, clover planes containing t times csw_t, purely spatial planes times
    csw_r/xi0 (csw unused)."""
    lx, ly, lz, lt = dims
    V = lx * ly * lz * lt
    M = np.zeros((12 * V, 12 * V), dtype=np.complex128)
    one = np.eye(4)
    for c in _coords(dims):
        i = site_index(c, dims)
        # clover block
        a = np.eye(12, dtype=np.complex128)
        for mu in range(4):
            for nu in range(mu + 1, 4):
                q = leaf_sum(U, c, mu, nu, dims)
                f = (q - q.conj().T) / 8.0
                f = f - np.trace(f) / 3.0 * np.eye(3)
                sig = 0.5 * (GAMMA[mu] @ GAMMA[nu] - GAMMA[nu] @ GAMMA[mu])
                if aniso is None:
                    coef = csw
                else:
                    coef = aniso[2] if nu == 3 else aniso[3] / aniso[0]
                a -= kappa * coef * np.kron(sig, f)
        M[12 * i:12 * i + 12, 12 * i:12 * i + 12] += a
        # hopping: forward and backward in every direction
        for mu in range(4):
            cf = step(c, mu, +1, dims)
            cb = step(c, mu, -1, dims)
            sf = t_boundary if (mu == 3 and c[3] == lt - 1) else 1.0
            sb = t_boundary if (mu == 3 and c[3] == 0) else 1.0
            if aniso is not None and mu < 3:
                sf, sb = sf * aniso[1] / aniso[0], sb * aniso[1] / aniso[0]
            jf, jb = site_index(cf, dims), site_index(cb, dims)
            M[12 * i:12 * i + 12, 12 * jf:12 * jf + 12] += -kappa * sf * np.kron(one - GAMMA[mu], link(U, c, mu))
            M[12 * i:12 * i + 12, 12 * jb:12 * jb + 12] += -kappa * sb * np.kron(one + GAMMA[mu], link(U, cb, mu).conj().T)
    return M


def parity_indices(dims, parity):
    idx = []
    for c in _coords(dims):
        if sum(c) % 2 == parity:
            i = site_index(c, dims)
            idx.extend(range(12 * i, 12 * i + 12))
    return np.array(idx)
