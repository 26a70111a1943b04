"""Discrete transport operators of the space-angle DG scheme.

Oracle (test infrastructure only).  Vectors use the layout psi[Nsdof, Nadof]
with sdof = cell*s + l (spatial node l of cell `cell`) and adof = q*a + m
(angular function m of patch q), the expansion of Eq. Expansion.

Paper passages followed
-----------------------
* Eq. complete and the shorthands below it (Sec. 2.3): per cell j and patch q,
      sum_f Upsilon_{[f,j,q]} - sum_xi V_xi (x) A^xi_q phi + Sigma N (x) M_q phi = Q.
* Sec. 3: L phi = S phi + f; the sweep visits, per S2 ordinate (octant), the
  cells in upwind order and solves each (cell, patch) block.
* Sec. 4.2: the Legendre scatter source through flux moments,
      Q_{[j,q]lm} = sum_{p,d,i} N_li sum_{n,o} sigma_{s,n} X_{[p]d,no} X_{[q]m,no} phi_{[j,p]}^{id}.

Readings
--------
* The collision coefficient of L is sigma_t (Eq. LBE); S carries the whole
  Legendre in-scatter including n = 0, sigma_{s,n} = sigma_s(cell) * f_n,
  with one moment shape f_n per material (`mat_id` maps cells to materials;
  one shape for every cell without it).
* Faces of an axis-aligned box are normal to a coordinate axis and a patch
  never crosses a coordinate plane, so Omega.n has one sign on a patch and the
  face flux is the exact upwind value: the own trace on outflow faces, the
  neighbour's trace (or the boundary data) on inflow faces.
* In 2D the mesh is a slab infinite and uniform in z: Omega_z never streams,
  and the patches of the two octants that differ only in the z sign share one
  sweep direction (4 sweep directions, direction d = 2*bx + by).
* The isotropic source q is a scalar emission density: Q(r, Omega) = q/(4 pi).
* An isotropic inflow of angular flux psi_b on a boundary face adds
  -psi_b int_face Phi_l int_{D_q} (Omega.n) Psi_m to f for inflow patches.
* A normally incident pencil beam (Sec. 5.4: Dirac boundary data taken in the
  DG weak form) of strength S on a face with outward normal n is
  psi_b = S delta(Omega - Omega_b), Omega_b = -n, uniform over the face.  Its
  inflow term is -S int_face Phi_l (Omega_b.n) Psi_m(Omega_b) for a patch
  holding Omega_b.  Omega_b is a vertex of k patches (k = 4: the octahedron
  vertex keeps a right angle in each of the 4 octants around it at every
  level), and the Dirac mass is split equally, 1/k to each; this is the limit
  of a uniform inflow over a shrinking cap around Omega_b, each of whose
  quarters lies in one of those patches.
* A beam of general direction over part of a face (Sec. 5.4's cube with a
  boundary source on a square of its face): psi_b = S delta(Omega - Omega_b)
  on the range, zero on the rest of the face; its inflow term is
  -S (Omega_b.n) int_{face & range} Phi_l Psi_m(Omega_b) share_q, with the
  share of patch q the fraction of an infinitesimal cap around Omega_b that
  lies in it (1 inside, 1/2 on an edge, interior angle / 2 pi at a vertex).
"""
import itertools

import numpy as np

from . import angular, harmonics
from .spatial import Q1Cell


def _vertex_angle(A, B, C):
    """Interior angle at vertex A of the spherical triangle ABC: the angle
    between the great circles AB and AC at A."""
    tb = B - (B @ A) * A
    tc = C - (C @ A) * A
    return np.arctan2(np.linalg.norm(np.cross(tb, tc)), tb @ tc)


def beam_weights(amesh, omega_b):
    """wb[P, a]: Psi_[q]m(omega_b) times the share of the Dirac mass that
    patch q receives, zero elsewhere.  A patch holds omega_b iff omega_b is a
    non-negative combination of its vertices.  The share is the fraction of an
    infinitesimal cap around omega_b that lies in the patch: 1 inside it, 1/2
    on an edge (a great circle halves the cap), and at a vertex the patch's
    interior angle there over 2 pi (1/4 at a vertex of the octahedron, where
    four right angles meet)."""
    wb = np.zeros((amesh.P, amesh.a))
    for q in range(amesh.P):
        V = amesh.verts[q]
        lam = np.linalg.solve(V.T, omega_b)
        if lam.min() < -1e-12:
            continue
        zero = np.abs(lam) <= 1e-12 * np.abs(lam).max()
        nz = int(zero.sum())
        if nz == 0:
            share = 1.0
        elif nz == 1:
            share = 0.5
        else:
            i = int(np.argmax(~zero))            # omega_b is vertex i
            share = _vertex_angle(V[i], V[(i + 1) % 3], V[(i + 2) % 3]) / (2.0 * np.pi)
        wb[q] = share * angular.basis_eval(V, amesh.octant[q], amesh.basis, omega_b)
    return wb


class Transport:
    """Operators L, S, A = L - S, the sweep L^-1, the source f and the scalar
    flux on one angular mesh with scatter truncated at order Nscat."""

    def __init__(self, prob, amesh, Nscat=None):
        self.prob = prob
        self.dim = prob["dim"]
        self.ncell = tuple(prob["ncell"])
        d = self.dim
        nc = list(self.ncell) + [1] * (3 - d)
        self.nx, self.ny, self.nz = nc
        self.C = self.nx * self.ny * self.nz
        h = [(prob["hi"][e] - prob["lo"][e]) / self.ncell[e] for e in range(d)]
        self.cell = Q1Cell(h)
        self.s = self.cell.s
        self.am = amesh
        self.P = amesh.P
        self.a = amesh.a
        self.nsdof = self.C * self.s
        self.nadof = self.P * self.a
        self.sigma_t = np.asarray(prob["sigma_t"], dtype=np.float64)
        self.sigma_s = np.asarray(prob["sigma_s"], dtype=np.float64)
        N = prob["N"] if Nscat is None else Nscat
        self.Nscat = N
        # moment shapes: one row f_n per material of mat_id (one for all
        # cells without it); sigma_{s,n}(c) = sigma_s(c) f_{mat_id(c), n}
        ftab = np.atleast_2d(np.asarray(prob["fmom"], dtype=np.float64))
        nkeep = min(N, prob["N"]) + 1
        fm = np.zeros((ftab.shape[0], N + 1))
        fm[:, :nkeep] = ftab[:, :nkeep]
        mid = prob.get("mat_id")
        self.fid = (np.zeros(self.C, dtype=np.int64) if mid is None
                    else np.asarray(mid, dtype=np.int64))
        self.nshape = fm.shape[0]
        self.fmom_tab = fm
        self.fmom = fm[0]
        # --- angular scatter matrices S_f = X diag(f_n) X^T (Sec. 4.2) ---
        self.X = amesh.X(N).reshape(self.nadof, harmonics.nmoments(N))
        self.Ftab = fm[:, harmonics.degree_of_index(N)]   # [shapes, nmom]
        self.Fdiag = self.Ftab[0]
        # --- per-patch blocks of L ---
        s, a = self.s, self.a
        nf = 2 * d
        self.Afq = np.zeros((nf, self.P, a, a))
        self.outflow = np.zeros((nf, self.P), dtype=bool)
        for f in range(nf):
            xi, side = divmod(f, 2)
            sgn = 2.0 * side - 1.0
            self.Afq[f] = sgn * amesh.A[:, xi]
            self.outflow[f] = amesh.signs[:, xi] * sgn > 0
        self.K0 = np.zeros((self.P, s * a, s * a))
        self.B = np.zeros((self.P, s * a, s * a))
        self.U = np.zeros((nf, self.P, s * a, s * a))
        for q in range(self.P):
            K = np.zeros((s * a, s * a))
            for f in range(nf):
                if self.outflow[f, q]:
                    K += np.kron(self.cell.Fown[f], self.Afq[f, q])
                else:
                    self.U[f, q] = np.kron(self.cell.Fnb[f], self.Afq[f, q])
            for xi in range(d):
                K -= np.kron(self.cell.V[xi], amesh.A[q, xi])
            self.K0[q] = K
            self.B[q] = np.kron(self.cell.N, amesh.M[q])
        # sweep directions
        if d == 2:
            self.ndir = 4
            self.pdir = np.array([2 * ((o >> 2) & 1) + ((o >> 1) & 1) for o in amesh.octant])
        else:
            self.ndir = 8
            self.pdir = amesh.octant.copy()

    # ------------------------------------------------------------------ helpers
    def cell_index(self, ix, iy, iz=0):
        return ix + self.nx * (iy + self.ny * iz)

    def cell_coords(self, c):
        return c % self.nx, (c // self.nx) % self.ny, c // (self.nx * self.ny)

    def neighbour(self, c, f):
        """Neighbour across face f, or -1 on the domain boundary."""
        xi, side = divmod(f, 2)
        idx = list(self.cell_coords(c))
        idx[xi] += 1 if side == 1 else -1
        n = [self.nx, self.ny, self.nz][xi]
        if idx[xi] < 0 or idx[xi] >= n:
            return -1
        return self.cell_index(*idx)

    def to_blocks(self, x):
        """[Nsdof, Nadof] -> [C, P, s*a] with block index l*a + m."""
        return (x.reshape(self.C, self.s, self.P, self.a)
                .transpose(0, 2, 1, 3).reshape(self.C, self.P, self.s * self.a))

    def from_blocks(self, xb):
        return (xb.reshape(self.C, self.P, self.s, self.a)
                .transpose(0, 2, 1, 3).reshape(self.nsdof, self.nadof))

    def direction_signs(self, d):
        if self.dim == 2:
            return (1 - 2 * ((d >> 1) & 1), 1 - 2 * (d & 1), 1)
        return (1 - 2 * ((d >> 2) & 1), 1 - 2 * ((d >> 1) & 1), 1 - 2 * (d & 1))

    def sweep_order(self, d):
        """Cells in an upwind (topological) order for sweep direction d."""
        sx, sy, sz = self.direction_signs(d)
        xs = range(self.nx) if sx > 0 else range(self.nx - 1, -1, -1)
        ys = range(self.ny) if sy > 0 else range(self.ny - 1, -1, -1)
        zs = range(self.nz) if sz > 0 else range(self.nz - 1, -1, -1)
        return [self.cell_index(ix, iy, iz) for iz in zs for iy in ys for ix in xs]

    def patches_of(self, d):
        return np.nonzero(self.pdir == d)[0]

    def block(self, c, q):
        """Diagonal block of L for cell c and patch(es) q."""
        return self.K0[q] + self.sigma_t[c] * self.B[q]

    # ---------------------------------------------------------------- operators
    def apply_L(self, x, cells=None):
        """y = L x (Eq. complete, left-hand side, with upwind face fluxes).
        With `cells`, only the rows of those cells are computed (others 0)."""
        xb = self.to_blocks(x)
        yb = np.zeros_like(xb)
        for c in (range(self.C) if cells is None else cells):
            Kc = self.block(c, slice(None))
            yb[c] = np.einsum("qij,qj->qi", Kc, xb[c])
            for f in range(2 * self.dim):
                nb = self.neighbour(c, f)
                if nb < 0:
                    continue
                yb[c] += np.einsum("qij,qj->qi", self.U[f], xb[nb])
        return self.from_blocks(yb)

    def scatter(self, x, cells=None):
        """y = S x through the flux moments of Sec. 4.2.  S couples only the
        rows of one cell, so with `cells` only those cells' rows are computed
        (x may then hold just those rows, cell by cell, [len(cells)*s, Nadof])."""
        N = self.cell.N
        if cells is not None:
            y = np.empty_like(x)
            for i, c in enumerate(cells):
                rows = slice(i * self.s, (i + 1) * self.s)
                Phi = x[rows] @ self.X
                y[rows] = self.sigma_s[c] * (N @ ((Phi * self.Ftab[self.fid[c]]) @ self.X.T))
            return y
        Phi = x @ self.X                       # [Nsdof, Nmom] moments
        # sum_{n,o} f_n X_q Phi with each cell's moment shape
        Frow = np.repeat(self.Ftab[self.fid], self.s, axis=0)
        Yang = (Phi * Frow) @ self.X.T
        y = np.empty_like(x)
        for c in range(self.C):
            rows = slice(c * self.s, (c + 1) * self.s)
            y[rows] = self.sigma_s[c] * (N @ Yang[rows])
        return y

    def apply_A(self, x):
        return self.apply_L(x) - self.scatter(x)

    def sweep(self, b, patches=None):
        """psi = L^-1 b: per direction, cells in upwind order, all patches of
        the direction solved block by block (Sec. 3).  L couples a patch only
        to itself, so with `patches` only those columns are swept (others 0)."""
        bb = self.to_blocks(b)
        psi = np.zeros_like(bb)
        for d in range(self.ndir):
            qs = self.patches_of(d)
            if patches is not None:
                qs = np.array([q for q in qs if q in set(patches)], dtype=np.int64)
            if len(qs) == 0:
                continue
            for c in self.sweep_order(d):
                rhs = bb[c, qs].copy()
                for f in range(2 * self.dim):
                    nb = self.neighbour(c, f)
                    if nb < 0:
                        continue
                    # inflow faces only carry a coupling block
                    rhs -= np.einsum("qij,qj->qi", self.U[f, qs], psi[nb, qs])
                psi[c, qs] = np.linalg.solve(self.block(c, qs), rhs[..., None])[..., 0]
        return self.from_blocks(psi)

    def source(self):
        """f: isotropic volumetric source plus boundary inflow data."""
        s, a = self.s, self.a
        fb = np.zeros((self.C, self.P, s, a))
        q = np.asarray(self.prob["q"], dtype=np.float64)
        mu = self.cell.mu
        for c in range(self.C):
            fb[c] = (q[c] / (4.0 * np.pi)) * mu[None, :, None] * self.am.w[:, None, :]
        for f, (kind, val) in enumerate(self.prob["boundary"]):
            if kind == 0:
                continue
            if kind not in (1, 2, 3):
                raise ValueError("oracle supports vacuum, isotropic inflow and the beams")
            xi, side = divmod(f, 2)
            sgn = 2.0 * side - 1.0
            inflow = ~self.outflow[f]
            if kind == 3:
                self._general_beam(fb, f, val)
                continue
            if kind == 2:
                n = np.zeros(3)
                n[xi] = sgn
                omega_b = -n
                wb = beam_weights(self.am, omega_b)       # Psi_m(Omega_b) / k
                assert not wb[~inflow].any()
                term = -val * (omega_b @ n) * self.cell.mf[f][None, :, None] * wb[:, None, :]
                for c in range(self.C):
                    if self.neighbour(c, f) < 0:
                        fb[c] += term
                continue
            ndotpsi = sgn * self.am.Aw[:, xi, :]          # int (Omega.n) Psi_m
            for c in range(self.C):
                if self.neighbour(c, f) >= 0:
                    continue
                term = -val * self.cell.mf[f][None, :, None] * ndotpsi[:, None, :]
                fb[c][inflow] += term[inflow]
        return fb.transpose(0, 2, 1, 3).reshape(self.nsdof, self.nadof)

    def _general_beam(self, fb, f, val):
        """Beam psi_b = S delta(Omega - Omega_b) over the part of face f whose
        tangential coordinates (axes in increasing order) lie in
        [u0, u1] (x [v0, v1] in 3D), val = (S, Omega_b[3], u0, u1, v0, v1):
        the inflow term -S (Omega_b.n) int_{face cell & range} Phi_l
        Psi_m(Omega_b) share_q (beam_weights), Omega_b normalised and
        pointing into the domain."""
        S = float(val[0])
        om = np.asarray(val[1:4], dtype=np.float64)
        om = om / np.linalg.norm(om)
        rng = [(float(val[4]), float(val[5])), (float(val[6]), float(val[7]))]
        xi, side = divmod(f, 2)
        n = np.zeros(3)
        n[xi] = 2.0 * side - 1.0
        if om @ n >= 0.0:
            raise ValueError("the beam must point into the domain")
        wb = beam_weights(self.am, om)
        others = [e for e in range(self.dim) if e != xi]
        h = self.cell.h
        for c in range(self.C):
            if self.neighbour(c, f) >= 0:
                continue
            ic = self.cell_coords(c)
            a, b = [], []
            for j, e in enumerate(others):
                x0 = self.prob["lo"][e] + ic[e] * h[e]
                lo_, hi_ = max(x0, rng[j][0]), min(x0 + h[e], rng[j][1])
                a.append(lo_ - x0)
                b.append(max(hi_, lo_) - x0)
            if any(bb <= aa for aa, bb in zip(a, b)):
                continue
            I = self.cell.face_integral(f, a, b)
            fb[c] += -S * (om @ n) * I[None, :, None] * wb[:, None, :]

    def scalar_flux(self, psi):
        """phi_s[Nsdof] = sum_{q,d} psi * int Psi_{[q]d} (n = 0 moment)."""
        return psi @ self.am.w.reshape(-1)

    # ------------------------------------------------------- dense assembly
    def dense_L(self):
        n = self.nsdof * self.nadof
        Ld = np.zeros((n, n))
        s, a = self.s, self.a

        def gidx(c, q):
            ls = np.arange(s)
            ms = np.arange(a)
            return ((c * s + ls)[:, None] * self.nadof + q * a + ms[None, :]).reshape(-1)

        for c in range(self.C):
            for q in range(self.P):
                r = gidx(c, q)
                Ld[np.ix_(r, r)] += self.block(c, q)
                for f in range(2 * self.dim):
                    nb = self.neighbour(c, f)
                    if nb >= 0 and not self.outflow[f, q]:
                        Ld[np.ix_(r, gidx(nb, q))] += self.U[f, q]
        return Ld

    def dense_S(self):
        Sfs = [self.angular_scatter_matrix(m) for m in range(self.nshape)]
        blocks = []
        for c in range(self.C):
            blocks.append(self.sigma_s[c] * np.kron(self.cell.N, Sfs[self.fid[c]]))
        n = self.nsdof * self.nadof
        Sd = np.zeros((n, n))
        m = self.s * self.nadof
        for c in range(self.C):
            Sd[c * m:(c + 1) * m, c * m:(c + 1) * m] = blocks[c]
        return Sd

    def angular_scatter_matrix(self, shape=0):
        """S_f = X diag(f_n) X^T over the angular DOFs (unit sigma_s) for the
        moment shape of material `shape`."""
        return (self.X * self.Ftab[shape]) @ self.X.T
