"""Adjoint transport and the gradients of a detector response.

Oracle (test infrastructure only: imported by tests/, smoke() and bench.py's
CPU leg).  Plain FP64 NumPy, written from the discrete problem of
Eq. complete and Sec. 4.2.

Definitions
-----------
* Response: R = g^T psi with A psi = f and g the source of an isotropic
  emission density 4 pi * weight[c] (so g^T psi = sum_c weight[c] int_cell
  phi_s dV, the flux integral over the cells with weight 1).
* Adjoint: A^T lam = g; then for any parameter p of A (f does not depend on
  the cross sections or the Legendre moments)
      dR/dp = -lam^T (dA/dp) psi.
  With A = L - S, L's collision block sigma_t(c) kron(N, M_q) and S's cell
  block sigma_s(c) kron(N, S_f), S_f = X diag(f_n) X^T:
      dR/dsigma_t[c] = -sum_q lam_cq^T kron(N, M_q) psi_cq
      dR/dsigma_s[c] = +lam_c^T kron(N, S_f) psi_c
      dR/df_n        = +sum_c sigma_s(c) lam_c^T kron(N, X_n X_n^T) psi_c
  where X_n are the 2n+1 columns of X of degree n; with several materials
  (moment shapes) the sum over c runs over the cells of each material.

Reading (pinned in tests/test_oracle_adjoint.py against the plain transpose)
-------------------------------------------------------------------------
L^T is the same DG operator with every direction reversed: A^xi_q -> -A^xi_q
and the upwind side of every face flipped.  On a Q1 cell, integration by
parts gives V_xi + V_xi^T = Fown_high - Fown_low, so the transposed diagonal
streaming block of one sign equals the streaming block of the other sign
with -A^xi; the face mass matrices and M_q are symmetric, so the transposed
upwind couplings are the reversed-direction couplings with -A^xi; S is
symmetric.  `ReversedMesh` applies that reversal to an angular mesh.
"""
import numpy as np

from . import harmonics
from .transport import Transport


class ReversedMesh:
    """An angular mesh with every direction Omega replaced by -Omega in the
    streaming terms: A^xi and int Omega Psi negated, the sign of each Omega
    component and the octant bits flipped.  Basis, mass matrices, weights and
    the harmonics moments are those of the forward mesh."""

    def __init__(self, am):
        self._am = am
        self.P = am.P
        self.a = am.a
        self.A = -am.A
        self.Aw = -am.Aw
        self.signs = -am.signs
        self.octant = am.octant ^ 7
        self.M = am.M
        self.w = am.w
        # patch q covers -D_q: vertices negated, same basis
        self.verts = -am.verts
        self.basis = am.basis

    def X(self, N):
        return self._am.X(N)


def response_problem(prob, weight):
    """The problem whose source is the adjoint source g: isotropic emission
    4 pi * weight per cell, vacuum boundaries."""
    q = dict(prob)
    q["q"] = 4.0 * np.pi * np.asarray(weight, dtype=np.float64)
    q["boundary"] = [(0, 0.0)] * (2 * prob["dim"])
    return q


def adjoint_transport(prob, amesh, weight, Nscat=None):
    """Transport operators of the adjoint problem (reversed directions) with
    the adjoint source g as its source."""
    return Transport(response_problem(prob, weight), ReversedMesh(amesh), Nscat)


def response(T, psi, weight):
    """R = sum_c weight[c] int_cell phi_s dV for the solution psi of T."""
    phis = T.scalar_flux(psi).reshape(T.C, T.s)
    return float(np.sum(np.asarray(weight)[:, None] * phis * T.cell.mu[None, :]))


def dense_solve(T, rhs):
    """Direct solve of (L - S) x = rhs (tiny meshes only)."""
    A = T.dense_L() - T.dense_S()
    return np.linalg.solve(A, rhs.reshape(-1)).reshape(T.nsdof, T.nadof)


def gradients(T, psi, lam):
    """(dR/dsigma_t [C], dR/dsigma_s [C], dR/df_n [N+1], or [materials][N+1]
    with several moment shapes) from the forward solution psi and the adjoint
    solution lam (definitions in the module docstring), cell by cell."""
    s = T.s
    N = T.cell.N
    pb = T.to_blocks(psi)
    lb = T.to_blocks(lam)
    dsigt = np.zeros(T.C)
    for c in range(T.C):
        for q in range(T.P):
            dsigt[c] -= lb[c, q] @ T.B[q] @ pb[c, q]
    Sfs = [T.angular_scatter_matrix(m) for m in range(T.nshape)]
    deg = harmonics.degree_of_index(T.Nscat)
    dsigs = np.zeros(T.C)
    dfn = np.zeros((T.nshape, T.Nscat + 1))
    for c in range(T.C):
        psi_c = psi[c * s:(c + 1) * s]
        lam_c = lam[c * s:(c + 1) * s]
        # kron(N, S_f) acting on the cell block with index (l, j): N psi_c S_f^T
        dsigs[c] = np.sum(lam_c * (N @ psi_c @ Sfs[T.fid[c]].T))
        for n in range(T.Nscat + 1):
            Xn = T.X[:, deg == n]
            dfn[T.fid[c], n] += T.sigma_s[c] * np.sum(lam_c * (N @ psi_c @ (Xn @ Xn.T)))
    return dsigt, dsigs, (dfn[0] if T.nshape == 1 else dfn)
