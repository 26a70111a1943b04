"""Pins of the oracle's angular discretisation against closed forms, the
paper's printed mesh sizes and exact invariants (CPU only)."""
import os

import numpy as np
import pytest

from oracle import angular

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _vos_area(v):
    """Van Oosterom-Strackee solid angle of a spherical triangle."""
    a, b, c = v
    num = abs(np.dot(a, np.cross(b, c)))
    den = 1.0 + np.dot(a, b) + np.dot(b, c) + np.dot(c, a)
    return 2.0 * np.arctan2(num, den)


@pytest.mark.parametrize("level", [0, 1, 2, 3])
def test_uniform_counts_and_areas(level):
    paths = angular.uniform_paths(level)
    assert len(paths) == 8 * 4 ** level           # Sec. 2.1: 4 daughters per split
    am = angular.AngularMesh(paths, "const")
    assert abs(am.w.sum() - 4 * np.pi) < 1e-12
    for q in range(am.P):
        assert abs(am.w[q, 0] - _vos_area(am.verts[q])) < 1e-13


def test_aniso_counts_match_paper():
    rows = [l.split() for l in open(os.path.join(GOLD, "aniso_counts.txt"))
            if l.strip() and not l.startswith("#")]
    for lmax, cnt in rows:
        assert len(angular.aniso_paths(int(lmax))) == int(cnt)


def test_aniso_axis_rotation_invariant():
    # refining about +x gives the same count as about +z (octahedral symmetry)
    for lmax in (2, 4):
        assert len(angular.aniso_paths(lmax, (1, 0, 0))) == len(angular.aniso_paths(lmax))


def test_aniso_areas_cover_sphere():
    am = angular.AngularMesh(angular.aniso_paths(4), "const")
    assert abs(am.w.sum() - 4 * np.pi) < 1e-12


def _interior_points(v, rng, n=7):
    lam = rng.dirichlet([1, 1, 1], size=n)
    x = lam @ v
    return x / np.linalg.norm(x, axis=1, keepdims=True)


def test_lin_nodal_and_partition_of_unity():
    rng = np.random.default_rng(0)
    am = angular.AngularMesh(angular.uniform_paths(2), "lin")
    for q in range(0, am.P, 5):
        vals = angular.basis_eval(am.verts[q], am.octant[q], "lin", am.verts[q])
        assert np.abs(vals - np.eye(3)).max() < 1e-14          # Psi_d(Omega_d') = delta
        pts = _interior_points(am.verts[q], rng)
        psi = angular.basis_eval(am.verts[q], am.octant[q], "lin", pts)
        assert np.abs(psi.sum(axis=1) - 1).max() < 1e-14
        assert psi.min() > 0


def test_lin_is_linear_on_flat_triangle():
    # Psi_d(Omega) * (s.Omega) must be a linear function of Omega (it is the
    # barycentric coordinate of the central projection)
    rng = np.random.default_rng(1)
    am = angular.AngularMesh(angular.uniform_paths(1), "lin")
    q = 11
    pts = _interior_points(am.verts[q], rng, 20)
    psi = angular.basis_eval(am.verts[q], am.octant[q], "lin", pts)
    s = am.signs[q]
    lin = psi * (pts @ s)[:, None]
    coef, res, *_ = np.linalg.lstsq(pts, lin, rcond=None)
    assert np.abs(pts @ coef - lin).max() < 1e-14


@pytest.mark.parametrize("basis", ["lin", "const"])
def test_quadrature_moments_of_sphere(basis):
    # int Omega_x^2 = 4 pi / 3, int Omega_x Omega_y = 0, int Omega_z^4 = 4 pi / 5
    tot = np.zeros(3)
    for p in angular.uniform_paths(1):
        v = angular.path_vertices(p)
        om, w = angular.patch_quadrature(v, 16)
        tot += [w @ om[:, 0] ** 2, w @ (om[:, 0] * om[:, 1]), w @ om[:, 2] ** 4]
    assert abs(tot[0] - 4 * np.pi / 3) < 1e-13
    assert abs(tot[1]) < 1e-14
    assert abs(tot[2] - 4 * np.pi / 5) < 1e-13


def test_angular_tables_invariants():
    am = angular.AngularMesh(angular.uniform_paths(2), "lin")
    for q in range(am.P):
        assert np.allclose(am.M[q], am.M[q].T, atol=1e-16)
        assert np.linalg.eigvalsh(am.M[q]).min() > 0
        for xi in range(3):
            assert np.allclose(am.A[q, xi], am.A[q, xi].T, atol=1e-16)
            # sign of Omega_xi is fixed on a patch: A^xi is definite
            ev = np.linalg.eigvalsh(am.signs[q, xi] * am.A[q, xi])
            assert ev.min() > 0
    # int over the sphere of Omega_xi Psi Psi summed with partition of unity = 0
    for xi in range(3):
        assert abs(am.A[:, xi].sum()) < 1e-13
        assert abs(am.Aw[:, xi].sum()) < 1e-13
    # sum_d M_md = int Psi_m = w_m
    assert np.abs(am.M.sum(axis=2) - am.w).max() < 1e-15


@pytest.mark.parametrize("path", [(0,), (3, 2), (5, 1, 3)])
def test_quadrature_converged(path):
    v = angular.path_vertices(path)
    lev = len(path) - 1
    om, w = angular.patch_quadrature(v, angular.default_order(lev, 0))
    assert abs(w.sum() - _vos_area(v)) < 1e-14
    for N in (8, 16):
        o1, w1 = angular.patch_quadrature(v, angular.default_order(lev, N))
        o2, w2 = angular.patch_quadrature(v, angular.default_order(lev, N) + 10)
        from oracle import harmonics
        X1 = w1 @ harmonics.real_sph_harm(N, o1)
        X2 = w2 @ harmonics.real_sph_harm(N, o2)
        assert np.abs(X1 - X2).max() < 1e-14


@pytest.mark.parametrize("basis", ["lin", "const"])
def test_prolongation_exact_and_galerkin(basis):
    fine = angular.AngularMesh(angular.uniform_paths(2), basis)
    coarse = angular.AngularMesh(angular.uniform_paths(1), basis)
    P = angular.prolongation(fine, coarse)
    assert np.abs(P @ np.ones(coarse.nadof) - 1).max() < 1e-15   # P 1 = 1
    a = fine.a
    Mf = np.zeros((fine.nadof, fine.nadof))
    Mc = np.zeros((coarse.nadof, coarse.nadof))
    for q in range(fine.P):
        Mf[q * a:(q + 1) * a, q * a:(q + 1) * a] = fine.M[q]
    for q in range(coarse.P):
        Mc[q * a:(q + 1) * a, q * a:(q + 1) * a] = coarse.M[q]
    assert np.abs(P.T @ Mf @ P - Mc).max() < 1e-14                # P^T M_f P = M_c
    # integrals preserved: w_f^T P = w_c
    assert np.abs(fine.w.reshape(-1) @ P - coarse.w.reshape(-1)).max() < 1e-14
    if basis == "lin":
        # pointwise: a coarse function equals its prolongation inside each fine patch
        rng = np.random.default_rng(3)
        c = rng.standard_normal(coarse.nadof)
        fvec = P @ c
        for f in range(0, fine.P, 7):
            pts = _interior_points(fine.verts[f], rng, 5)
            pc = coarse.paths.index(fine.paths[f][:2])
            vc = angular.basis_eval(coarse.verts[pc], coarse.octant[pc], "lin", pts) @ c[pc * 3:pc * 3 + 3]
            vf = angular.basis_eval(fine.verts[f], fine.octant[f], "lin", pts) @ fvec[f * 3:f * 3 + 3]
            assert np.abs(vc - vf).max() < 1e-14


def test_aniso_hierarchy_nested():
    paths = angular.aniso_paths(3)
    L = angular.max_level(paths)
    prev = None
    for l in range(L, -1, -1):
        T = angular.coarsen_paths(paths, l)
        m = angular.AngularMesh(T, "lin")
        assert abs(m.w.sum() - 4 * np.pi) < 1e-12
        if prev is not None:
            P = angular.prolongation(prev, m)
            assert np.abs(P @ np.ones(m.nadof) - 1).max() < 1e-15
        prev = m
