"""Writes the stored expected values of tests/golden/ from the FP64 oracle only.

c1_apply_solve.txt: the 4^4 workload (links exp(i 0.2 sum r_a lambda_a / 2), seed 0,
kappa 0.12, c_sw 1.0, antiperiodic time, point source at site 0, spin 0, colour 0):
(M b) on the 9 sites that touch the source (the source and its 8 neighbours) and the
solution x of M x = b at the same sites, solved by the oracle's even-odd BiCGStab to
1e-13.  The operator is the isotropic reading of Eq. 5 (kappa normalisation); b is one
spin-colour column of a point-source propagator (§III.A).

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle import dirac, solvers  # noqa: E402
from oracle import lattice as L  # noqa: E402

DIMS = (4, 4, 4, 4)
SITES = [(0, 0, 0, 0), (1, 0, 0, 0), (3, 0, 0, 0), (0, 1, 0, 0), (0, 3, 0, 0), (0, 0, 1, 0), (0, 0, 3, 0),
         (0, 0, 0, 1), (0, 0, 0, 3)]


def compute():
    gauge = W.gauge_links(DIMS, 0.2, 0)
    op = dirac.from_qdp_problem(gauge, DIMS, 0.12, 1.0)
    b = L.from_qdp(W.point_source(DIMS, 0, 0), DIMS)
    mb = op.M(b)
    x, _ = solvers.solve_even_odd(op, b, tol=1e-13)
    return [(s, mb[s[3], s[2], s[1], s[0]], x[s[3], s[2], s[1], s[0]]) for s in SITES]


def write(path):
    with open(path, "w") as f:
        f.write("# 4^4, eps 0.2, seed 0, kappa 0.12, c_sw 1, t_boundary -1, b = point source (0,0,0,0) spin 0 colour 0\n")
        f.write("# columns: x y z t field spin colour re im   (field 0: M b, 1: x with M x = b)\n")
        for s, mb, x in compute():
            for fi, v in ((0, mb), (1, x)):
                for sp in range(4):
                    for c in range(3):
                        z = v[sp, c]
                        f.write(f"{s[0]} {s[1]} {s[2]} {s[3]} {fi} {sp} {c} {z.real:.17e} {z.imag:.17e}\n")


def read(path):
    out = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        x, y, z, t, fi, sp, c, re, im = line.split()
        out[(int(x), int(y), int(z), int(t), int(fi), int(sp), int(c))] = complex(float(re), float(im))
    return out


if __name__ == "__main__":
    write(os.path.join(HERE, "c1_apply_solve.txt"))
