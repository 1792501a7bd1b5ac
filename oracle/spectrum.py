"""Smallest singular value of the Schur operator, to tell a well-posed workload from a
near-singular draw (the critical kappa of the synthetic fields is not known; free
fields have kappa_c = 1/8).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Lanczos on the Hermitian
positive operator N = A^+ A with full reorthogonalisation: the smallest eigenvalue of
the tridiagonal matrix after k steps is an upper bound on sigma_min(A)^2 that reaches
it once k covers the low spectrum (the low spectra of small lattices are too
clustered for plain inverse iteration).  Pinned against numpy's SVD of dense Schur
matrices (tests/test_oracle_spectrum.py).

    python -m oracle.spectrum     # the 8^3x16 record: sigma_min(M_hat) at the benchmark kappas
"""
import numpy as np

from . import solvers


def smallest_singular_value(A, Adag, x0, steps=100):
    """Lanczos on N = A^+ A from x0, every new vector orthogonalised twice against all
    previous ones; returns (sqrt of the smallest Ritz value, steps taken)."""
    N = lambda v: Adag(A(v))
    q = x0 / np.sqrt(solvers.norm2(x0))
    basis = [q]
    alphas, betas = [], []
    beta_prev, q_prev = 0.0, None
    for _ in range(steps):
        w = N(q)
        alpha = solvers.dot(q, w).real
        w = w - alpha * q - (beta_prev * q_prev if q_prev is not None else 0.0)
        for _pass in range(2):
            for b in basis:
                w = w - solvers.dot(b, w) * b
        alphas.append(alpha)
        beta = np.sqrt(solvers.norm2(w))
        if beta <= 1e-12 * abs(alpha):
            break
        betas.append(beta)
        q_prev, q, beta_prev = q, w / beta, beta
        basis.append(q)
    k = len(alphas)
    t = np.diag(alphas) + np.diag(betas[:k - 1], 1) + np.diag(betas[:k - 1], -1)
    lam = np.linalg.eigvalsh(t).min()
    return float(np.sqrt(max(lam, 0.0))), k


def _record():
    import workloads as W
    from . import dirac
    from . import lattice as L

    dims = (8, 8, 8, 16)
    gauge = W.gauge_links(dims, 0.3, 0)
    x0 = L.from_qdp(W.gaussian_fermion(dims, 1), dims)
    for kappa in (0.1235, 0.124):
        op = dirac.from_qdp_problem(gauge, dims, kappa, 1.0)
        xe = x0 * op.even
        for steps in (100, 200):
            s, k = smallest_singular_value(op.Mhat, lambda v: op.Mhat(v, dagger=True), xe, steps=steps)
            print(f"8^3x16 eps 0.3 seed 0 kappa {kappa} c_sw 1: sigma_min(M_hat) <= {s:.4e} ({k} Lanczos steps)")


if __name__ == "__main__":
    _record()
