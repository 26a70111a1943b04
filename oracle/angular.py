"""Angular discretisation: spherical patch hierarchy, Const/Lin bases, patch
quadrature, the angular matrices and the nested-mesh prolongation.

Oracle (test infrastructure only).

Paper passages followed
-----------------------
* Sec. 2.1: the coordinate planes cut the sphere into 8 octants (level 0); a
  patch is refined by halving its edges and joining the new points by great
  circles, giving 4 daughters.
* Sec. 2.2: Const = 1 on the patch; Lin = three nodal functions obtained by
  projecting the Lagrange functions of the flat triangle whose vertices are the
  patch vertices projected onto the octahedron |x|+|y|+|z| = 1.
* Sec. 2.3: M_{[q]md} = int Psi_m Psi_d, A^xi_{[q]md} = int Omega_xi Psi_m Psi_d.
* Sec. 4.2 (definition of X): X_{[q]m,n,o} = int Psi_m Y_{n,o}.
* Sec. 4.1: nested meshes T_l; prolongation by Galerkin projection, exact for
  the nested spaces; restriction R = P^T.
* Sec. 5.4: anisotropic refinement bands 0.97 / 0.9 / 0.8 / 0.6 about an axis.

Readings (where the paper is silent)
------------------------------------
* The edge midpoint is normalize(a + b).  Children of (a, b, c) are
  (a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca).  Octant o has sign bits
  (bx, by, bz) = ((o>>2)&1, (o>>1)&1, o&1), bit 1 meaning negative, and vertices
  (sx e_x, sy e_y, sz e_z).  Patches are ordered depth first.
* The projection onto the octahedron is the central (gnomonic) one,
  x = Omega / |Omega|_1, so great circles map to straight lines and the Lin
  functions are barycentric coordinates of x in the flat triangle.
* Anisotropic rule: the target level of an element is set by the largest
  Omega.axis over its three vertices; an element is split while its level is
  below its target.
* Integrals over a patch use the gnomonic map onto the flat triangle with
  dOmega = h |x|^-3 dA, h = 1/sqrt(3), and a Duffy-collapsed Gauss-Legendre
  product rule on the triangle.
"""
import numpy as np

from . import harmonics

H_PLANE = 1.0 / np.sqrt(3.0)


# ----------------------------------------------------------------------------
# patch hierarchy
# ----------------------------------------------------------------------------
def octant_signs(o):
    """Sign vector (sx, sy, sz) of octant o (bit 1 = negative)."""
    return np.array([1.0 - 2.0 * ((o >> 2) & 1),
                     1.0 - 2.0 * ((o >> 1) & 1),
                     1.0 - 2.0 * (o & 1)])


def octant_vertices(o):
    s = octant_signs(o)
    return np.diag(s)  # rows: s_x e_x, s_y e_y, s_z e_z


def _unit(v):
    return v / np.linalg.norm(v)


def child_vertices(verts, c):
    """Vertices of daughter c (0..3) of the spherical triangle verts[3,3]."""
    a, b, cc = verts
    ab = _unit(a + b)
    bc = _unit(b + cc)
    ca = _unit(cc + a)
    return np.array([(a, ab, ca), (ab, b, bc), (ca, bc, cc), (ab, bc, ca)][c])


def path_vertices(path):
    """Vertices of the patch reached by path = (octant, c1, c2, ...)."""
    v = octant_vertices(path[0])
    for c in path[1:]:
        v = child_vertices(v, c)
    return v


def uniform_paths(level):
    """Depth-first list of the 8*4^level patch paths of the uniform mesh."""
    out = []

    def rec(path):
        if len(path) - 1 == level:
            out.append(tuple(path))
            return
        for c in range(4):
            rec(path + [c])

    for o in range(8):
        rec([o])
    return out


def aniso_target(verts, axis, lmax):
    """Target level of an element from the refinement bands of Sec. 5.4."""
    m = max(float(np.dot(v, axis)) for v in verts)
    if m > 0.97:
        t = lmax
    elif m > 0.9:
        t = lmax - 1
    elif m > 0.8:
        t = lmax - 2
    elif m > 0.6:
        t = lmax - 3
    else:
        t = lmax - 4
    return max(t, 0)


def aniso_paths(lmax, axis=(0.0, 0.0, 1.0)):
    """Depth-first leaf paths of the anisotropically refined mesh."""
    axis = _unit(np.asarray(axis, dtype=np.float64))
    out = []

    def rec(path, verts):
        lev = len(path) - 1
        if lev < aniso_target(verts, axis, lmax):
            for c in range(4):
                rec(path + [c], child_vertices(verts, c))
        else:
            out.append(tuple(path))

    for o in range(8):
        rec([o], octant_vertices(o))
    return out


def coarsen_paths(paths, level):
    """Mesh T_level of a nested series: every leaf deeper than `level` is
    replaced by its ancestor at `level` (Sec. 4.1)."""
    seen = []
    last = None
    for p in paths:
        q = p[:level + 1]
        if q != last:
            seen.append(q)
            last = q
    return seen


def max_level(paths):
    return max(len(p) - 1 for p in paths)


# ----------------------------------------------------------------------------
# bases
# ----------------------------------------------------------------------------
def flat_vertices(verts):
    """Patch vertices projected onto the octahedron (rows)."""
    return verts / np.sum(np.abs(verts), axis=1, keepdims=True)


def basis_eval(verts, octant, basis, omega):
    """Psi_d(omega) for omega[..., 3] inside the patch; returns [..., a]."""
    omega = np.asarray(omega, dtype=np.float64)
    if basis == "const":
        return np.ones(omega.shape[:-1] + (1,))
    s = octant_signs(octant)
    U = flat_vertices(verts).T          # columns u_k
    x = omega / (omega @ s)[..., None]  # central projection onto s.x = 1
    lam = np.linalg.solve(U, x.reshape(-1, 3).T).T
    return lam.reshape(omega.shape[:-1] + (3,))


def nbasis(basis):
    return 1 if basis == "const" else 3


# ----------------------------------------------------------------------------
# quadrature on a spherical patch
# ----------------------------------------------------------------------------
def patch_quadrature(verts, order):
    """Nodes (unit vectors) and weights integrating over the spherical patch."""
    g, wg = np.polynomial.legendre.leggauss(order)
    t = 0.5 * (g + 1.0)
    wt = 0.5 * wg
    u = flat_vertices(verts)
    e1 = u[1] - u[0]
    e2 = u[2] - u[1]
    twoA = np.linalg.norm(np.cross(e1, e2))
    xi, eta = np.meshgrid(t, t, indexing="ij")
    wxi, weta = np.meshgrid(wt, wt, indexing="ij")
    xi = xi.ravel()
    eta = eta.ravel()
    w = (wxi * weta).ravel() * xi * twoA
    x = u[0][None, :] + xi[:, None] * (e1[None, :] + eta[:, None] * e2[None, :])
    r = np.linalg.norm(x, axis=1)
    omega = x / r[:, None]
    w = w * H_PLANE / r ** 3
    return omega, w


def default_order(level, N):
    """Gauss order per direction for a patch of the given level when the
    integrand carries harmonics up to degree N (generous for the oracle)."""
    return 22 + int(np.ceil(1.6 * N / (2 ** level)))


# ----------------------------------------------------------------------------
# tables
# ----------------------------------------------------------------------------
class AngularMesh:
    """A mesh of patches with its basis and per-patch tables.

    Attributes: paths, verts[P,3,3], octant[P], level[P], a (DOF per patch),
    w[P,a] (int Psi), M[P,a,a], A[P,3,a,a] (xi = x, y, z).
    """

    def __init__(self, paths, basis):
        self.paths = list(paths)
        self.basis = basis
        self.a = nbasis(basis)
        self.P = len(self.paths)
        self.verts = np.array([path_vertices(p) for p in self.paths])
        self.octant = np.array([p[0] for p in self.paths], dtype=np.int64)
        self.level = np.array([len(p) - 1 for p in self.paths], dtype=np.int64)
        a = self.a
        self.w = np.zeros((self.P, a))
        self.M = np.zeros((self.P, a, a))
        self.A = np.zeros((self.P, 3, a, a))
        self.Aw = np.zeros((self.P, 3, a))   # int Omega_xi Psi_m
        for q in range(self.P):
            om, wq = patch_quadrature(self.verts[q], default_order(self.level[q], 4))
            psi = basis_eval(self.verts[q], self.octant[q], basis, om)
            self.w[q] = wq @ psi
            self.M[q] = np.einsum("k,km,kd->md", wq, psi, psi)
            for xi in range(3):
                self.A[q, xi] = np.einsum("k,k,km,kd->md", wq, om[:, xi], psi, psi)
                self.Aw[q, xi] = np.einsum("k,k,km->m", wq, om[:, xi], psi)
        self.signs = np.array([octant_signs(o) for o in self.octant])

    @property
    def nadof(self):
        return self.P * self.a

    def X(self, N):
        """X[P, a, (N+1)^2] = int_{D_q} Psi_m Y_{n,o} (Sec. 4.2)."""
        out = np.zeros((self.P, self.a, harmonics.nmoments(N)))
        for q in range(self.P):
            om, wq = patch_quadrature(self.verts[q], default_order(self.level[q], N))
            psi = basis_eval(self.verts[q], self.octant[q], self.basis, om)
            Y = harmonics.real_sph_harm(N, om)
            out[q] = np.einsum("k,km,kn->mn", wq, psi, Y)
        return out


def prolongation(fine, coarse):
    """Dense P[nadof_f, nadof_c] between nested meshes (Sec. 4.1).

    The coarse function restricted to a fine patch is represented exactly in
    the fine basis; for the nodal Lin basis its fine coefficients are its
    values at the fine patch vertices."""
    P = np.zeros((fine.nadof, coarse.nadof))
    index = {p: i for i, p in enumerate(coarse.paths)}
    for f, path in enumerate(fine.paths):
        c = None
        for k in range(len(path), 0, -1):
            if path[:k] in index:
                c = index[path[:k]]
                break
        assert c is not None, "meshes are not nested"
        if fine.basis == "const":
            P[f, c] = 1.0
        else:
            vals = basis_eval(coarse.verts[c], coarse.octant[c], "lin", fine.verts[f])
            # vals[k, d] = Psi_{c,d}(fine vertex k)
            P[f * 3:(f + 1) * 3, c * 3:(c + 1) * 3] = vals
    return P
