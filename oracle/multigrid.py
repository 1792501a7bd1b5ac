"""Adaptive aggregation multigrid preconditioner for the Wilson-clover operator, the
solver the paper enables by passing a block size per level (Sec. II.E: the multigrid
parameters follow QUDA's test example with the geometric block size left open; Sec.
III.B: two levels, each projecting a 2^4 sublattice onto one coarse site).

TEST INFRASTRUCTURE ONLY (see the package docstring).  The paper names the method
without its steps; the reading taken here is the standard aggregation-based one:

* null space: N_v vectors from random starts (passed in) relaxed towards the
  near-kernel of the operator by minimal-residual steps on A x = 0;
* prolongator P: per block of sites and per chirality (gamma_5 = diag(1, 1, -1, -1)
  on the fine level, the first coarse index on coarser ones), the restrictions of the
  null vectors orthonormalised (QR): P^+ P = 1, and P commutes with gamma_5;
* coarse operator A_c = P^+ A P (Galerkin), applied as that product;
* preconditioner (one cycle): minimal-residual pre-smoothing from zero, coarse
  correction P A_c^-1 P^+ r with the coarse system solved by flexible GCR to a
  relative tolerance (recursively preconditioned by the next level: a K-cycle), then
  minimal-residual post-smoothing;
* outer solver: flexible GCR (oracle.solvers.fgcr) with this preconditioner.

Vectors of a level are arrays with the four site axes (Lt, Lz, Ly, Lx) first and the
level's internal axes after: (4, 3) spin-colour on the fine level, (2, N_v) chirality
and vector index on a coarse one.

The coarse operator is also available as the nine-point stencil a GPU kernel would
apply (coarse_stencil / apply_stencil), read off the Galerkin product column by
column, and built locally from the links, the clover and P(x)
(coarse_stencil_from_links), the construction a GPU kernel would run.

Pins (tests/test_oracle_multigrid.py): orthonormality and chirality of P, the
gamma_5-hermiticity the coarse operator and its stencil blocks inherit, the stencil
against the Galerkin product, exactness when the null space spans each block, and
the iteration reduction against plain GCR.
"""
import numpy as np

from . import solvers


def chirality_halves(internal_shape):
    """Index tuples into the internal axes selecting chirality +1 and -1."""
    if internal_shape == (4, 3):
        return (np.s_[0:2, :], np.s_[2:4, :])
    return (np.s_[0:1, :], np.s_[1:2, :])


def _blocked(v, block):
    """(Lt, Lz, Ly, Lx, ...) -> (Ct, Cz, Cy, Cx, bt, bz, by, bx, ...) with block = (bx, by, bz, bt)."""
    lt, lz, ly, lx = v.shape[:4]
    bx, by, bz, bt = block
    tail = v.shape[4:]
    w = v.reshape((lt // bt, bt, lz // bz, bz, ly // by, by, lx // bx, bx) + tail)
    return w.transpose((0, 2, 4, 6, 1, 3, 5, 7) + tuple(range(8, 8 + len(tail))))


def _unblocked(w, block):
    ct, cz, cy, cx, bt, bz, by, bx = w.shape[:8]
    tail = w.shape[8:]
    v = w.transpose((0, 4, 1, 5, 2, 6, 3, 7) + tuple(range(8, 8 + len(tail))))
    return v.reshape((ct * bt, cz * bz, cy * by, cx * bx) + tail)


class Prolongator:
    """P for one level: per coarse site and chirality an orthonormal basis (dof x N_v) of
    the block-chirality restrictions of the null vectors."""

    def __init__(self, vectors, block):
        self.block = tuple(block)
        self.nv = len(vectors)
        self.internal = vectors[0].shape[4:]
        self.halves = chirality_halves(self.internal)
        fine_sites = vectors[0].shape[:4]
        lt, lz, ly, lx = fine_sites
        bx, by, bz, bt = self.block
        if lx % bx or ly % by or lz % bz or lt % bt:
            raise ValueError("block size must divide the lattice")
        self.coarse_sites = (lt // bt, lz // bz, ly // by, lx // bx)
        self.fine_shape = vectors[0].shape
        self.basis = []  # per chirality: (Ct, Cz, Cy, Cx, dof, N_v)
        for h in self.halves:
            cols = []
            for v in vectors:
                w = _blocked(v, self.block)
                part = w[(Ellipsis,) + h]  # (..., block sites..., half internal)
                cols.append(part.reshape(self.coarse_sites + (-1,)))
            m = np.stack(cols, axis=-1)  # (C..., dof, N_v)
            if m.shape[-2] < self.nv:
                raise ValueError("more null vectors than block-chirality degrees of freedom")
            q, _ = np.linalg.qr(m)
            self.basis.append(q)
        self.coarse_shape = self.coarse_sites + (2, self.nv)

    def restrict(self, v):
        """P^+ v: fine vector -> coarse vector (Ct, Cz, Cy, Cx, 2, N_v)."""
        w = _blocked(v, self.block)
        out = np.zeros(self.coarse_shape, dtype=np.complex128)
        for chi, h in enumerate(self.halves):
            part = w[(Ellipsis,) + h].reshape(self.coarse_sites + (-1,))
            out[..., chi, :] = np.einsum("...dn,...d->...n", np.conj(self.basis[chi]), part)
        return out

    def prolong(self, c):
        """P c: coarse vector -> fine vector."""
        w = np.zeros(_blocked(np.zeros(self.fine_shape, dtype=np.complex128), self.block).shape,
                     dtype=np.complex128)
        for chi, h in enumerate(self.halves):
            part = np.einsum("...dn,...n->...d", self.basis[chi], c[..., chi, :])
            w[(Ellipsis,) + h] = part.reshape(w[(Ellipsis,) + h].shape)
        return _unblocked(w, self.block)


def minres_relax(A, b, steps, x0=None):
    """`steps` minimal-residual steps on A x = b: r = b - A x, alpha = <A r, r>/<A r, A r>,
    x += alpha r.  With b = 0 this damps every component except the near-kernel."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A(x) if x0 is not None else b.copy()
    for _ in range(steps):
        ar = A(r)
        den = solvers.norm2(ar)
        if den == 0.0:
            break
        alpha = solvers.dot(ar, r) / den
        x = x + alpha * r
        r = r - alpha * ar
    return x


def null_vectors(A, starts, steps):
    """Relax each random start towards A x = 0 and normalise it."""
    out = []
    zero = np.zeros_like(starts[0])
    for s in starts:
        v = minres_relax(A, zero, steps, x0=s)
        out.append(v / np.sqrt(solvers.norm2(v)))
    return out


class Level:
    """One level of the hierarchy: its operator, prolongator to the next coarser level,
    the coarse operator P^+ A P and (recursively) the next level."""

    def __init__(self, A, P, coarse=None, pre=2, post=2, coarse_tol=0.1, coarse_maxiter=50, coarse_nkrylov=8):
        self.A, self.P, self.coarse = A, P, coarse
        self.pre, self.post = pre, post
        self.coarse_tol, self.coarse_maxiter, self.coarse_nkrylov = coarse_tol, coarse_maxiter, coarse_nkrylov
        self.stats = {"coarse_iters": 0, "cycles": 0}

    def Ac(self, c):
        """Galerkin coarse operator P^+ A P."""
        return self.P.restrict(self.A(self.P.prolong(c)))

    def cycle(self, r):
        """One preconditioner application e ~ A^-1 r."""
        self.stats["cycles"] += 1
        e = minres_relax(self.A, r, self.pre)
        r1 = r - self.A(e)
        rc = self.P.restrict(r1)
        pc = self.coarse.cycle if self.coarse is not None else None
        ec, info = solvers.fgcr(self.Ac, rc, precond=pc, tol=self.coarse_tol, maxiter=self.coarse_maxiter,
                                nkrylov=self.coarse_nkrylov)
        self.stats["coarse_iters"] += info["iters"]
        e = e + self.P.prolong(ec)
        if self.post:
            e = minres_relax(self.A, r, self.post, x0=e)
        return e


def setup(A, fine_shape, blocks, nvs, starts_per_level, relax_steps=20, **level_kw):
    """Build the hierarchy.  blocks: block size per level (fine first); nvs: N_v per
    level; starts_per_level: for each level, N_v random starts shaped like that level's
    vectors (random numbers are inputs, drawn by the caller)."""
    ops = [A]
    prolongators = []
    shape = fine_shape
    for lvl, (block, nv) in enumerate(zip(blocks, nvs)):
        starts = starts_per_level[lvl]
        assert len(starts) == nv and starts[0].shape == shape
        vecs = null_vectors(ops[-1], starts, relax_steps)
        P = Prolongator(vecs, block)
        prolongators.append(P)
        Aprev = ops[-1]
        ops.append(lambda c, P=P, Aprev=Aprev: P.restrict(Aprev(P.prolong(c))))
        shape = P.coarse_shape
    level = None
    for lvl in reversed(range(len(blocks))):
        level = Level(ops[lvl], prolongators[lvl], coarse=level, **level_kw)
    return level


def solve(A, b, top, tol=1e-10, maxiter=500, nkrylov=20):
    """Flexible GCR on A x = b preconditioned by one multigrid cycle per iteration."""
    return solvers.fgcr(A, b, precond=top.cycle, tol=tol, maxiter=maxiter, nkrylov=nkrylov)


def coarse_stencil(A, P):
    """The coarse operator P^+ A P of a nearest-neighbour fine operator as a nine-point
    stencil on the coarse lattice: (A_c c)(x) = X(x) c(x) + sum_mu [Yf_mu(x) c(x + mu)
    + Yb_mu(x) c(x - mu)], every block (2 N_v) x (2 N_v).  Read off column by column:
    A_c applied to the unit coarse vector of site y and component j has X(y)[:, j] at y,
    Yf_mu(y - mu)[:, j] at y - mu and Yb_mu(y + mu)[:, j] at y + mu.  Needs every coarse
    extent >= 3 so that y + mu and y - mu are different sites.  Returns (X, Yf, Yb) with
    X: (Ct, Cz, Cy, Cx, n, n), Yf, Yb: (4, Ct, Cz, Cy, Cx, n, n), n = 2 N_v."""
    ct, cz, cy, cx = P.coarse_sites
    if min(ct, cz, cy, cx) < 3:
        raise ValueError("coarse extents must be at least 3")
    nv = P.nv
    n = 2 * nv
    X = np.zeros(P.coarse_sites + (n, n), dtype=np.complex128)
    Yf = np.zeros((4,) + X.shape, dtype=np.complex128)
    Yb = np.zeros_like(Yf)
    ext = (cx, cy, cz, ct)  # direction mu = 0..3 is x, y, z, t
    for site in np.ndindex(*P.coarse_sites):  # (t, z, y, x)
        for j in range(n):
            e = np.zeros(P.coarse_shape, dtype=np.complex128)
            e[site + (j // nv, j % nv)] = 1.0
            col = P.restrict(A(P.prolong(e))).reshape(P.coarse_sites + (n,))
            X[site][:, j] = col[site]
            for mu in range(4):
                ax = 3 - mu
                dn = list(site)
                dn[ax] = (dn[ax] - 1) % ext[mu]
                up = list(site)
                up[ax] = (up[ax] + 1) % ext[mu]
                Yf[mu][tuple(dn)][:, j] = col[tuple(dn)]
                Yb[mu][tuple(up)][:, j] = col[tuple(up)]
    return X, Yf, Yb


def apply_stencil(X, Yf, Yb, c):
    """(A_c c)(x) from the nine-point stencil of coarse_stencil."""
    shape = c.shape
    sites = shape[:4]
    v = c.reshape(sites + (-1,))
    out = np.einsum("...ij,...j->...i", X, v)
    for mu in range(4):
        ax = 3 - mu
        out += np.einsum("...ij,...j->...i", Yf[mu], np.roll(v, -1, axis=ax))
        out += np.einsum("...ij,...j->...i", Yb[mu], np.roll(v, +1, axis=ax))
    return out.reshape(shape)


def fine_prolongator(P):
    """P(x) per fine site: (Lt, Lz, Ly, Lx, 12, 2 N_v) on the fine level (blocks are
    disjoint, so prolonging the unit vector of component j on every coarse site at once
    gives column j of every site's block)."""
    n = 2 * P.nv
    cols = []
    for j in range(n):
        e = np.zeros(P.coarse_shape, dtype=np.complex128)
        e[..., j // P.nv, j % P.nv] = 1.0
        cols.append(P.prolong(e).reshape(P.fine_shape[:4] + (-1,)))
    return np.stack(cols, axis=-1)


def coarse_stencil_from_links(op, P):
    """The nine-point coarse stencil built directly from the fine links and clover of a
    WilsonClover operator -- the local form a GPU kernel evaluates:
    X(c) = sum_{x in c} P(x)^+ A(x) P(x) + the hops that stay inside block c, and
    Yf_mu(c) (Yb_mu(c)) = the hops from block c across its upper (lower) face in mu,
    -kappa w_mu eta P(x)^+ (1 -/+ gamma_mu) U P(x +/- mu)."""
    from .gamma import GAMMA, ID4
    from . import lattice as L

    pf = fine_prolongator(P)
    n = pf.shape[-1]
    dims = op.dims
    lt, lz, ly, lx = dims[3], dims[2], dims[1], dims[0]
    bx, by, bz, bt = P.block
    bsz = (bx, by, bz, bt)
    w = op.hop_weights if op.hop_weights is not None else (1.0, 1.0, 1.0, 1.0)

    def to_coarse(field):  # (Lt, Lz, Ly, Lx, n, n) summed over each block
        return _blocked(field, P.block).sum(axis=(4, 5, 6, 7))

    pdag = np.conj(np.swapaxes(pf, -1, -2))
    X_fine = pdag @ op.A @ pf
    X = to_coarse(X_fine)
    Yf = np.zeros((4,) + X.shape, dtype=np.complex128)
    Yb = np.zeros_like(Yf)
    coord = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    for mu in range(4):
        ax = 3 - mu
        sf = L.time_boundary_sign(dims, op.t_boundary, True) if mu == 3 else np.ones((lt, lz, ly, lx))
        sb = L.time_boundary_sign(dims, op.t_boundary, False) if mu == 3 else np.ones((lt, lz, ly, lx))
        u = op.U[mu]
        ub = np.conj(np.swapaxes(L.bwd(u, mu), -1, -2))  # U_mu(x - mu)^+
        hf = np.einsum("st,...ab->...satb", ID4 - GAMMA[mu], u).reshape(u.shape[:4] + (12, 12))
        hb = np.einsum("st,...ab->...satb", ID4 + GAMMA[mu], ub).reshape(u.shape[:4] + (12, 12))
        fwd_term = (-op.kappa * w[mu]) * sf[..., None, None] * (pdag @ hf @ L.fwd(pf, mu))
        bwd_term = (-op.kappa * w[mu]) * sb[..., None, None] * (pdag @ hb @ L.bwd(pf, mu))
        upper = (coord[ax] % bsz[mu]) == bsz[mu] - 1  # x + mu leaves the block
        lower = (coord[ax] % bsz[mu]) == 0             # x - mu leaves the block
        X += to_coarse(np.where(upper[..., None, None], 0, fwd_term) + np.where(lower[..., None, None], 0, bwd_term))
        Yf[mu] = to_coarse(np.where(upper[..., None, None], fwd_term, 0))
        Yb[mu] = to_coarse(np.where(lower[..., None, None], bwd_term, 0))
    return X, Yf, Yb
