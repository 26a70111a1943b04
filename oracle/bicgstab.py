"""Right-preconditioned BiCGStab, the paper's Krylov method (Sec. 3: BiCGStab
with L^-1 -- source iteration -- or the multigrid cycle as preconditioner).

Oracle (test infrastructure only).

The iteration is van der Vorst's stabilised bi-conjugate gradient method
with the preconditioner applied on the right: with the shadow residual r^
fixed to the initial residual, each step forms a search direction p from
the residual and the previous direction, takes the BiCG step along M^-1 p,
then a minimal-residual step along M^-1 s.  Stop criterion of Sec. 5.1,
||b - A x|| / ||b|| < tol on the true residual (the recursive residual
decides when to check it).  Zero initial guess unless given.
"""
import numpy as np


def bicgstab(apply_A, b, apply_M, tol, maxit=1000, x0=None):
    """Returns (x, iterations, history of recursive relres, true relres)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    hist = []
    if bnorm == 0.0:
        return np.zeros_like(b), 0, hist, 0.0
    r = b - apply_A(x)
    if np.linalg.norm(r) / bnorm < tol:
        return x, 0, hist, np.linalg.norm(r) / bnorm
    rhat = r.copy()
    rho_old = alpha = omega = 1.0
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    its = 0
    while its < maxit:
        its += 1
        rho = np.vdot(rhat, r)
        if rho == 0.0:
            break
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        ph = apply_M(p)
        v = apply_A(ph)
        alpha = rho / np.vdot(rhat, v)
        s = r - alpha * v
        if np.linalg.norm(s) / bnorm < tol:
            x = x + alpha * ph
            hist.append(np.linalg.norm(s) / bnorm)
            break
        sh = apply_M(s)
        t = apply_A(sh)
        omega = np.vdot(t, s) / np.vdot(t, t)
        x = x + alpha * ph + omega * sh
        r = s - omega * t
        rho_old = rho
        hist.append(np.linalg.norm(r) / bnorm)
        if hist[-1] < tol:
            break
    rel = np.linalg.norm(b - apply_A(x)) / bnorm
    return x, its, hist, rel
