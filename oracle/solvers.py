"""Krylov solvers for the oracle (Sec. II.E: BiCGStab is the default for
Wilson/clover, CG for the normal equations), plus flexible GCR.

Inner product <a, b> = sum conj(a) * b over every component.  All solvers take
the operator as a callable on whole-lattice arrays and return (x, info) with
info = {"iters", "residual" (the recurrence residual, relative to ||b||),
"status"}.  None of them is tuned: they are the textbook recurrences.

Pins: the 2^4 / 4^4 dense solves (numpy.linalg.solve) and the free-field
momentum-space propagator in tests/test_oracle_solvers.py.
"""
import numpy as np


def dot(a, b) -> complex:
    return complex(np.vdot(a, b))


def norm2(a) -> float:
    return float(np.vdot(a, a).real)


def bicgstab(A, b, x0=None, tol=1e-12, maxiter=10000, breakdown_eps=1e-300):
    """BiCGStab (van der Vorst 1992) for A x = b; stop when ||r|| <= tol ||b||.

    r = b - A x, r_hat = r, rho = alpha = omega = 1, v = p = 0, then per iteration
    rho' = <r_hat, r>, beta = (rho'/rho)(alpha/omega), p = r + beta (p - omega v),
    v = A p, alpha = rho'/<r_hat, v>, s = r - alpha v, t = A s,
    omega = <t, s>/<t, t>, x += alpha p + omega s, r = s - omega t.
    """
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A(x) if x0 is not None else b.copy()
    bnorm = np.sqrt(norm2(b))
    if bnorm == 0.0:
        return x, {"iters": 0, "residual": 0.0, "status": "ok"}
    rhat = r.copy()
    rho = alpha = omega = 1.0 + 0j
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    it = 0
    rn = np.sqrt(norm2(r))
    while rn > tol * bnorm and it < maxiter:
        rho_new = dot(rhat, r)
        if abs(rho_new) < breakdown_eps:
            return x, {"iters": it, "residual": rn / bnorm, "status": "breakdown"}
        beta = (rho_new / rho) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = A(p)
        alpha = rho_new / dot(rhat, v)
        s = r - alpha * v
        t = A(s)
        tt = norm2(t)
        if tt < breakdown_eps:
            x = x + alpha * p
            r = s
            it += 1
            rn = np.sqrt(norm2(r))
            break
        omega = dot(t, s) / tt
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho = rho_new
        it += 1
        rn = np.sqrt(norm2(r))
    status = "ok" if rn <= tol * bnorm else "not_converged"
    return x, {"iters": it, "residual": rn / bnorm, "status": status}


def cgnr(A, Adag, b, x0=None, tol=1e-12, maxiter=10000):
    """CG on the normal equations A^+ A x = A^+ b; stop on the true-system
    recurrence residual ||b - A x|| <= tol ||b|| (not on the normal residual)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A(x) if x0 is not None else b.copy()
    bnorm = np.sqrt(norm2(b))
    if bnorm == 0.0:
        return x, {"iters": 0, "residual": 0.0, "status": "ok"}
    z = Adag(r)  # normal-equation residual
    p = z.copy()
    zz = norm2(z)
    it = 0
    rn = np.sqrt(norm2(r))
    while rn > tol * bnorm and it < maxiter:
        q = A(p)
        alpha = zz / norm2(q)
        x = x + alpha * p
        r = r - alpha * q
        z = Adag(r)
        zz_new = norm2(z)
        p = z + (zz_new / zz) * p
        zz = zz_new
        it += 1
        rn = np.sqrt(norm2(r))
    status = "ok" if rn <= tol * bnorm else "not_converged"
    return x, {"iters": it, "residual": rn / bnorm, "status": status}


def fgcr(A, b, precond=None, x0=None, tol=1e-12, maxiter=10000, nkrylov=20):
    """Flexible GCR (restarted after nkrylov directions).

    Per step k: z_k = N(r), w_k = A z_k; w_k is orthogonalised against
    w_0..w_{k-1} by modified Gram-Schmidt (z_k gets the same combination) and
    normalised; then alpha = <w_k, r>, x += alpha z_k, r -= alpha w_k.
    With N the identity this is GCR, whose residual norm never increases.
    """
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A(x) if x0 is not None else b.copy()
    bnorm = np.sqrt(norm2(b))
    if bnorm == 0.0:
        return x, {"iters": 0, "residual": 0.0, "status": "ok"}
    it = 0
    rn = np.sqrt(norm2(r))
    zs, ws = [], []
    while rn > tol * bnorm and it < maxiter:
        if len(ws) == nkrylov:
            zs, ws = [], []
        z = r.copy() if precond is None else precond(r)
        w = A(z)
        for zj, wj in zip(zs, ws):
            beta = dot(wj, w)
            w = w - beta * wj
            z = z - beta * zj
        wn = np.sqrt(norm2(w))
        if wn == 0.0:
            return x, {"iters": it, "residual": rn / bnorm, "status": "breakdown"}
        w, z = w / wn, z / wn
        alpha = dot(w, r)
        x = x + alpha * z
        r = r - alpha * w
        zs.append(z)
        ws.append(w)
        it += 1
        rn = np.sqrt(norm2(r))
    status = "ok" if rn <= tol * bnorm else "not_converged"
    return x, {"iters": it, "residual": rn / bnorm, "status": status}


def solve_even_odd(op, b, method="bicgstab", tol=1e-12, maxiter=10000):
    """Solve M x = b through the Schur complement: M_hat x_e = b_hat, then reconstruct
    x_o.  The inner stopping tolerance is scaled so that the full-system relative
    residual (equal to the Schur residual in exact arithmetic) meets tol."""
    bhat = op.schur_source(b)
    scale = np.sqrt(norm2(b)) / max(np.sqrt(norm2(bhat)), 1e-300)
    inner_tol = tol * scale
    if method == "bicgstab":
        xe, info = bicgstab(op.Mhat, bhat, tol=inner_tol, maxiter=maxiter)
    elif method == "cgnr":
        xe, info = cgnr(op.Mhat, lambda v: op.Mhat(v, dagger=True), bhat, tol=inner_tol, maxiter=maxiter)
    else:
        raise ValueError(method)
    x = op.reconstruct(xe, b)
    info["true_residual"] = op.true_residual(x, b)
    return x, info
