"""Angular multigrid: transfers, smoother, V-cycle and coarse solver (Sec. 4).

Oracle (test infrastructure only).

Paper passages followed
-----------------------
* Fig. lmg: the recursive linear V-cycle LMG(phi_l, f_l, l): pre-smooth,
  residual r_l = f_l - A_l phi_l, f_{l-1} = R r_l, phi_{l-1} = 0, recurse,
  phi_l += P phi_{l-1}, post-smooth; the coarsest level is handled by the
  coarse solver.
* Sec. 4.1: nested meshes T_l, P by Galerkin projection (exact), R = P^T,
  smoother = source iteration L_l phi^{k+1} = S_l phi^k + f_l, coarse
  operators by direct re-discretisation (DCA).
* Sec. 4.2: coarse solver = block Gauss-Seidel over (cell, patch) blocks in
  the sweep order; each block solve keeps every unknown outside (j, q) at its
  latest value and includes the self-scatter; the scatter source is the
  moment form; 10 such sweeps.
* Sec. 4.3: the preconditioner uses a reduced scatter order N_r.

Readings
--------
* A k-level cycle uses the angular meshes T_L ... T_{L-k+1}; the scatter order
  of level k is Nr[k] (Nr[0] is the finest level's, normally the full N).
* Coarse Gauss-Seidel order: sweep directions in index order, cells in the
  direction's upwind order, the direction's patches in index order inside a
  cell.
"""
import numpy as np

from . import angular
from .transport import Transport


class Hierarchy:
    def __init__(self, prob, paths=None):
        mg = prob["mg"]
        if paths is None:
            paths = angular.uniform_paths(prob["level"])
        L = angular.max_level(paths)
        self.levels = []
        self.P = []
        k = mg["nlevels"]
        meshes = [angular.AngularMesh(angular.coarsen_paths(paths, L - i), prob["basis"])
                  for i in range(k)]
        for i in range(k):
            self.levels.append(Transport(prob, meshes[i], mg["Nr"][i]))
        for i in range(k - 1):
            self.P.append(angular.prolongation(meshes[i], meshes[i + 1]))
        self.nu_pre = mg["nu_pre"]
        self.nu_post = mg["nu_post"]
        self.coarse_sweeps = mg["coarse_sweeps"]

    def restrict(self, r, k):
        """f_{k+1} = P^T r_k (R = P^T)."""
        return r @ self.P[k]

    def prolong(self, x, k):
        """P x_{k+1} on the finer level k."""
        return x @ self.P[k].T

    def smooth(self, phi, f, k, nu):
        T = self.levels[k]
        for _ in range(nu):
            phi = T.sweep(T.scatter(phi) + f)
        return phi

    def vcycle(self, f, k=0, phi=None):
        T = self.levels[k]
        if phi is None:
            phi = np.zeros_like(f)
        if k == len(self.levels) - 1:
            return coarse_gs(T, f, phi, self.coarse_sweeps)
        phi = self.smooth(phi, f, k, self.nu_pre)
        r = f - T.apply_A(phi)
        fc = self.restrict(r, k)
        phic = self.vcycle(fc, k + 1, None)
        phi = phi + self.prolong(phic, k)
        phi = self.smooth(phi, f, k, self.nu_post)
        return phi


def coarse_gs(T, f, phi, nsweeps):
    """Block Gauss-Seidel over (cell, patch) blocks with self-scatter included
    in the block solve and the other blocks' scatter through the moment form
    sum_{p != q} X_q diag(f_n) X_p^T phi_p (Sec. 4.2)."""
    s, a = T.s, T.a
    fb = T.to_blocks(f)
    xb = T.to_blocks(phi).copy()
    Sfs = [T.angular_scatter_matrix(m) for m in range(T.nshape)]
    N = T.cell.N
    for _ in range(nsweeps):
        for d in range(T.ndir):
            qs = T.patches_of(d)
            for c in T.sweep_order(d):
                for q in qs:
                    rhs = fb[c, q].copy()
                    for fc in range(2 * T.dim):
                        nb = T.neighbour(c, fc)
                        if nb >= 0 and not T.outflow[fc, q]:
                            rhs -= T.U[fc, q] @ xb[nb, q]
                    # scatter from all other patches of the cell (latest values)
                    xc = xb[c].reshape(T.P, s, a)
                    Sf = Sfs[T.fid[c]]
                    src = np.zeros((s, a))
                    for p in range(T.P):
                        if p == q:
                            continue
                        Sqp = Sf[q * a:(q + 1) * a, p * a:(p + 1) * a]
                        src += N @ xc[p] @ Sqp.T
                    rhs += T.sigma_s[c] * src.reshape(-1)
                    Sqq = Sf[q * a:(q + 1) * a, q * a:(q + 1) * a]
                    Amat = T.block(c, q) - T.sigma_s[c] * np.kron(N, Sqq)
                    xb[c, q] = np.linalg.solve(Amat, rhs)
    return T.from_blocks(xb)
