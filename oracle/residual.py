"""The relative true residual ||b - M x|| / ||b|| of the whole-lattice operator of Eq. 5,
evaluated one slab of timeslices at a time, for lattices where the whole-array oracle
would not fit in memory or time (32^3x64 with 12 right-hand sides).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and by the CPU-baseline leg of
``bench.py``; the CUDA library never calls it.

Definition.  M = A - kappa H exactly as ``oracle.dirac.WilsonClover.M`` (Eq. 5,
isotropic or anisotropic through per-direction hop weights and per-plane clover
coefficients).  M psi on timeslices [t0, t1) depends only on the links and the field
on [t0 - 1, t1]: a hop reaches one timeslice away, and so does every clover leaf
(Sec. III.B's clover term).  So the slab is cut out of the QDP arrays (Sec. II.A)
together with one halo timeslice on each side (periodic wrap in t), the whole-array
definitions ``dirac.hopping`` and ``dirac.clover_matrix`` are applied to it, and only
the interior timeslices are kept: the halo rows are the only ones the cyclic shifts
of the slab array get wrong.

The fermion time boundary (eta of Eq. 5, t_boundary = -1 antiperiodic) is applied by
multiplying the t links on the last global timeslice by t_boundary for the hopping
term only: the forward hop from t = Lt - 1 uses U_t(Lt - 1) and the backward hop into
t = 0 uses U_t(Lt - 1)^+, each exactly once, and t_boundary is real.  The clover term
uses the bare links, as the whole-array oracle does.

Pins (tests/test_oracle_dirac.py): the slabs put together equal WilsonClover.M on
small lattices for every slab size (ragged last slab, slabs of one timeslice, Lt = 2),
both time boundaries and the anisotropic weights; the residual equals the whole-array
``true_residual``.
"""
from __future__ import annotations

import os

import numpy as np

from . import dirac


def lex_timeslices(qdp: np.ndarray, dims, ts) -> np.ndarray:
    """Lexicographic (T, Lz, Ly, Lx, ...) field on the global timeslices ts, read from a
    QDP cb2 array [2][Lt][Lz][Ly][Lx/2][...]; parity uses the global t."""
    lx, ly, lz, _ = dims
    t = np.asarray(ts)[:, None, None, None]
    z = np.arange(lz)[None, :, None, None]
    y = np.arange(ly)[None, None, :, None]
    x = np.arange(lx)[None, None, None, :]
    p = (x + y + z + t) % 2
    return np.ascontiguousarray(qdp[p, t, z, y, x // 2])


def slab_links(gauge_qdp: np.ndarray, dims, t0: int, t1: int):
    """Bare links on timeslices t0 - 1 .. t1 (wrapped), (4, T + 2, Lz, Ly, Lx, 3, 3),
    and the global timeslice of each slab row."""
    lt = dims[3]
    ts = [(t0 - 1 + k) % lt for k in range(t1 - t0 + 2)]
    U = np.stack([lex_timeslices(gauge_qdp[mu], dims, ts) for mu in range(4)])
    return U, ts


def slab_operator(gauge_qdp: np.ndarray, dims, kappa, csw, t0, t1, t_boundary=-1, hop_weights=None,
                  plane_csw=None):
    """The pieces of M on the slab [t0, t1) with its halo: (U with the boundary sign
    folded into the t links of t = Lt - 1, A on every slab row, global timeslices)."""
    U, ts = slab_links(gauge_qdp, dims, t0, t1)
    A = dirac.clover_matrix(U, kappa, csw, plane_csw)
    Uh = U.copy()
    for k, t in enumerate(ts):
        if t == dims[3] - 1:
            Uh[3, k] *= t_boundary
    return Uh, A, ts


def M_slab(gauge_qdp, psi_qdp, dims, kappa, csw, t0, t1, t_boundary=-1, hop_weights=None, plane_csw=None,
           pieces=None):
    """(M psi) on timeslices [t0, t1), lexicographic (t1 - t0, Lz, Ly, Lx, 4, 3)."""
    Uh, A, ts = pieces if pieces is not None else slab_operator(
        gauge_qdp, dims, kappa, csw, t0, t1, t_boundary, hop_weights, plane_csw)
    psi = lex_timeslices(psi_qdp, dims, ts)
    # the sign is in the links: the slab array itself has no time boundary
    m = dirac.apply_site_matrix(A, psi) - kappa * dirac.hopping(Uh, psi, +1, False, hop_weights)
    return m[1:-1]


def residual_slab(gauge_qdp, x_qdp, b_qdp, dims, kappa, csw, t0, t1, t_boundary=-1, hop_weights=None,
                  plane_csw=None):
    """Per right-hand side (||b - M x||^2, ||b||^2) restricted to timeslices [t0, t1);
    x_qdp and b_qdp are [nrhs][2][Lt][Lz][Ly][Lx/2][4][3]."""
    pieces = slab_operator(gauge_qdp, dims, kappa, csw, t0, t1, t_boundary, hop_weights, plane_csw)
    ts = list(range(t0, t1))
    r2 = np.zeros(len(x_qdp))
    b2 = np.zeros(len(x_qdp))
    for k in range(len(x_qdp)):
        mx = M_slab(gauge_qdp, x_qdp[k], dims, kappa, csw, t0, t1, t_boundary, hop_weights, plane_csw, pieces)
        b = lex_timeslices(b_qdp[k], dims, ts)
        r2[k] = float(np.vdot(b - mx, b - mx).real)
        b2[k] = float(np.vdot(b, b).real)
    return r2, b2


def slabs(lt: int, size: int):
    return [(t0, min(lt, t0 + size)) for t0 in range(0, lt, size)]


# --- process-parallel evaluation over slabs (shared-memory inputs) --------------

_SHARED = {}


def _attach(spec):
    from multiprocessing import shared_memory

    out = {}
    for name, (shm_name, shape, dtype) in spec.items():
        shm = shared_memory.SharedMemory(name=shm_name)
        _SHARED[name] = shm  # keep the mapping alive in this worker
        out[name] = np.ndarray(shape, dtype=dtype, buffer=shm.buf)
    return out


def _worker(args):
    spec, dims, kappa, csw, t0, t1, t_boundary, hop_weights, plane_csw = args
    a = _attach(spec)
    return residual_slab(a["gauge"], a["x"], a["b"], dims, kappa, csw, t0, t1, t_boundary, hop_weights, plane_csw)


def true_residuals(gauge_qdp, x_qdp, b_qdp, dims, kappa, csw, t_boundary=-1, hop_weights=None, plane_csw=None,
                   slab=4, processes=None):
    """||b_k - M x_k|| / ||b_k|| for every right-hand side k, in FP64, over the whole
    lattice, one slab of `slab` timeslices per task.  processes > 1 runs the slabs in a
    pool of spawned processes (safe after CUDA has been initialised in the caller)
    reading the inputs from shared memory; processes = 1 runs them here."""
    x_qdp = np.asarray(x_qdp)
    b_qdp = np.asarray(b_qdp)
    if x_qdp.ndim == 7:
        x_qdp, b_qdp = x_qdp[None], b_qdp[None]
    nrhs = len(x_qdp)
    parts = slabs(dims[3], slab)
    if processes is None:
        processes = min(len(parts), os.cpu_count() or 1, 16)
    r2 = np.zeros(nrhs)
    b2 = np.zeros(nrhs)
    if processes <= 1:
        for t0, t1 in parts:
            a, b = residual_slab(gauge_qdp, x_qdp, b_qdp, dims, kappa, csw, t0, t1, t_boundary, hop_weights,
                                 plane_csw)
            r2 += a
            b2 += b
    else:
        import multiprocessing as mp
        from multiprocessing import shared_memory

        blocks = []
        spec = {}
        try:
            for name, arr in (("gauge", gauge_qdp), ("x", x_qdp), ("b", b_qdp)):
                arr = np.ascontiguousarray(arr, dtype=np.complex128)
                shm = shared_memory.SharedMemory(create=True, size=max(1, arr.nbytes))
                blocks.append(shm)
                np.ndarray(arr.shape, dtype=arr.dtype, buffer=shm.buf)[...] = arr
                spec[name] = (shm.name, arr.shape, arr.dtype.str)
            saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
            os.environ["OMP_NUM_THREADS"] = os.environ["OPENBLAS_NUM_THREADS"] = "1"
            try:
                with mp.get_context("spawn").Pool(processes) as pool:
                    res = pool.map(_worker, [(spec, tuple(dims), kappa, csw, t0, t1, t_boundary, hop_weights,
                                              plane_csw) for t0, t1 in parts], chunksize=1)
            finally:
                for k, v in saved.items():
                    if v is None:
                        os.environ.pop(k, None)
                    else:
                        os.environ[k] = v
            for a, b in res:
                r2 += a
                b2 += b
        finally:
            for shm in blocks:
                shm.close()
                shm.unlink()
    return np.sqrt(r2 / np.where(b2 > 0, b2, 1.0))
