"""FP64 CPU oracle for the even-odd Wilson-clover propagator solve.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
never calls it, and it shares no code with the CUDA path: the two meet only in
the seeded arrays of the ``workloads`` module.

The oracle is a plain, slow, direct transcription of the definitions:

* ``gamma``   -- DeGrand-Rossi Dirac matrices and the QDP Gamma(n) index (Sec. II.A).
* ``lattice`` -- lexicographic <-> QDP cb2 layouts and nearest-neighbour shifts (Sec. II.A).
* ``dirac``   -- hopping term, clover term and the kappa-normalised operator
                 M = A - kappa*H of Eq. 5 (isotropic), its even-odd Schur complement and
                 the true residual.
* ``solvers`` -- BiCGStab and CG on the normal equations (Sec. II.E, the defaults for
                 Wilson/clover), and flexible GCR.
* ``ptc``     -- the gauge-covariant parallel-transport network used as a learned
                 preconditioner, forward and analytic backward.
* ``contract``-- wall and momentum sources, the sequential source and the meson two-
                 and three-point contractions around the solve (Sec. III.A, III.B).
* ``spectrum`` -- the smallest singular value of the Schur operator (Lanczos on
                 M_hat^+ M_hat), to tell a well-posed workload from a near-singular draw.
* ``staggered``- the staggered operator of the HISQ action on given fat and long links
                 (MILC phases), and its CG solve (Sec. II.A, II.E).
* ``hisq``    -- the HISQ link smearing that makes those fat and long links from the thin
                 links: fat7, U(3) projection, the second level with the Lepage and Naik
                 terms (Sec. II.A).
* ``multigrid``- aggregation multigrid preconditioner (null space, block prolongator,
                 Galerkin coarse operator, K-cycle) for flexible GCR (Sec. II.E, III.B).
* ``residual`` -- the true residual ||b - M x|| / ||b|| of Eq. 5's operator evaluated one
                 slab of timeslices at a time (optionally in spawned processes), for
                 lattices too large for the whole-array evaluation.
* ``force``   -- the HMC fermion force of the two-flavour even-odd clover action (with
                 the odd-site clover determinant) and the action itself (Sec. IV).

Everything is complex128 and operates on whole-lattice arrays in
lexicographic order (Lt, Lz, Ly, Lx, ...), converting to and from the QDP
layout at the edges.  Which pins check each function is stated in its
docstring; functions without a pin say "parity unpinned".
"""
from . import gamma, lattice, dirac, solvers, ptc, contract, multigrid, spectrum, staggered, hisq, residual, force  # noqa: F401
