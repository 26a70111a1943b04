"""Right-preconditioned restarted GMRES(m) with classical Gram-Schmidt applied
twice (CGS2) and Givens rotations.

Oracle (test infrastructure only).

The paper's Krylov method is BiCGStab with L^-1 or the multigrid cycle as
preconditioner (Sec. 3); the stop criterion is ||r|| / ||b|| < tol with r the
residual and b the right-hand side (Sec. 5.1).  The reading taken here is
GMRES(m), right-preconditioned, zero initial guess unless given, Euclidean norm
of the coefficient vector, convergence declared on the true residual.  The
preconditioned directions z_j = M^-1 v_j are stored and the update is
x += sum_j y_j z_j, which is the flexible form and equals x += M^-1 V y for a
fixed linear M.
"""
import numpy as np


def gmres(apply_A, b, apply_M, tol, restart=20, maxit=1000, x0=None):
    """Returns (x, iterations, history of estimated relres, true relres)."""
    b = np.asarray(b)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    hist = []
    if bnorm == 0.0:
        return np.zeros_like(b), 0, hist, 0.0
    its = 0
    m = restart
    while True:
        r = b - apply_A(x)
        beta = np.linalg.norm(r)
        rel = beta / bnorm
        if rel < tol or its >= maxit:
            return x, its, hist, rel
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        j_done = 0
        for j in range(m):
            z = apply_M(V[j])
            w = apply_A(z)
            Vm = np.stack([v.reshape(-1) for v in V])      # [j+1, n]
            wv = w.reshape(-1)
            h = Vm @ wv
            wv = wv - Vm.T @ h
            h2 = Vm @ wv
            wv = wv - Vm.T @ h2
            h = h + h2
            hn = np.linalg.norm(wv)
            H[:j + 1, j] = h
            H[j + 1, j] = hn
            Z.append(z)
            # previous rotations
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_done = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) / bnorm < tol or its >= maxit or hn == 0.0:
                break
            V.append((wv / hn).reshape(b.shape))
        k = j_done
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        for i in range(k):
            x = x + y[i] * Z[i]
