"""Pins of the oracle with one Legendre moment shape per material (mat_id,
f[nmat][N+1]; Sec. 4.2 with sigma_{s,n} depending on the cell's material):
the moment-form scatter against the assembled per-cell S and LAPACK, the
single-shape problem as a special case, the infinite-medium closed form
(only the n = 0 moment acts on an isotropic flux), the zeroth-moment sum
rule per cell, the Gauss-Seidel fixed point and the adjoint gradients per
material against central finite differences (CPU)."""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint, angular, gmres, harmonics, multigrid, transport


def _T(prob, level=None, Nscat=None):
    level = prob["level"] if level is None else level
    am = angular.AngularMesh(angular.uniform_paths(level), prob["basis"])
    return transport.Transport(prob, am, Nscat)


@pytest.mark.parametrize("dim,nc,level", [(2, (3, 3), 1), (3, (2, 2, 2), 0)])
def test_two_shape_solution_matches_dense_lu(dim, nc, level):
    prob = W.two_shape_problem(dim, nc, level, 5, 81)
    assert 0 < prob["mat_id"].sum() < prob["mat_id"].size
    T = _T(prob)
    f = T.source()
    A = T.dense_L() - T.dense_S()
    xr = np.linalg.solve(A, f.reshape(-1)).reshape(f.shape)
    x, its, _, rel = gmres.gmres(T.apply_A, f, T.sweep, 1e-13, 20, 400)
    assert rel < 1e-13
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) < 1e-11
    # the moment-form scatter is the assembled per-cell S
    v = W.random_vector((T.nsdof, T.nadof), 82)
    Sv = (T.dense_S() @ v.reshape(-1)).reshape(v.shape)
    assert np.abs(T.scatter(v) - Sv).max() < 1e-13 * np.abs(Sv).max()


def test_equal_shapes_reduce_to_the_single_shape_problem():
    prob = W.two_shape_problem(2, (3, 2), 1, 6, 83)
    g = 0.7
    prob["fmom"] = np.stack([W.hg_moments(g, 6), W.hg_moments(g, 6)])
    one = dict(prob)
    one.pop("mat_id")
    one["fmom"] = W.hg_moments(g, 6)
    T2, T1 = _T(prob), _T(one)
    v = W.random_vector((T1.nsdof, T1.nadof), 84)
    assert np.abs(T2.scatter(v) - T1.scatter(v)).max() < 1e-14 * np.abs(T1.scatter(v)).max()
    assert np.abs(T2.dense_S() - T1.dense_S()).max() == 0.0


def test_different_shapes_change_the_scatter_of_an_anisotropic_flux():
    prob = W.two_shape_problem(2, (3, 2), 1, 6, 85)
    one = dict(prob)
    one.pop("mat_id")
    one["fmom"] = prob["fmom"][0]
    T2, T1 = _T(prob), _T(one)
    v = W.random_vector((T1.nsdof, T1.nadof), 86)
    d = np.abs(T2.scatter(v) - T1.scatter(v)).reshape(T1.C, -1).max(axis=1)
    m = prob["mat_id"]
    assert d[m == 0].max() < 1e-14 * np.abs(v).max()
    assert d[m == 1].min() > 1e-5 * np.abs(v).max()


def test_infinite_medium_closed_form_with_two_shapes():
    """Isotropic inflow psi_inf = Q/(sigma_t - sigma_s) on every face of a
    medium whose cells carry different moment shapes: the constant psi_inf
    is still the exact solution, because only the n = 0 moment (f_0 = 1 for
    every material) acts on an isotropic flux."""
    nc = (3, 4)
    C = 12
    st, ss, q = 2.5, 2.0, 1.0
    psi_inf = q / (4 * np.pi) / (st - ss)
    mat = np.array([0, 1] * 6)
    fm = np.stack([W.hg_moments(0.9, 6), W.hg_moments(-0.3, 6)])
    prob = W.problem(2, nc, np.full(C, st), np.full(C, ss), 6, fm, np.full(C, q), 1,
                     boundary=[(1, psi_inf)] * 4, mat_id=mat)
    T = _T(prob)
    x, _, _, rel = gmres.gmres(T.apply_A, T.source(), T.sweep, 1e-13, 20, 400)
    assert rel < 1e-13
    assert np.abs(x - psi_inf).max() < 1e-10 * psi_inf


def test_zeroth_moment_sum_rule_per_cell():
    prob = W.two_shape_problem(2, (2, 2), 1, 8, 87)
    T = _T(prob)
    for m in range(T.nshape):
        Sf = T.angular_scatter_matrix(m)
        w = T.am.w.reshape(-1)
        assert np.abs(Sf.sum(axis=0) - w).max() < 1e-12


def test_coarse_gs_fixed_point_with_two_shapes():
    prob = W.two_shape_problem(2, (3, 3), 1, 6, 88)
    T = _T(prob, Nscat=4)
    f = T.source()
    A = T.dense_L() - T.dense_S()
    xr = np.linalg.solve(A, f.reshape(-1)).reshape(f.shape)
    x1 = multigrid.coarse_gs(T, f, xr, 1)
    assert np.linalg.norm(x1 - xr) / np.linalg.norm(xr) < 1e-13


def test_adjoint_gradients_per_material_match_finite_differences():
    prob = W.two_shape_problem(2, (3, 2), 1, 4, 89)
    weight = np.zeros(6)
    weight[[0, 4]] = 1.0
    am = angular.AngularMesh(angular.uniform_paths(1), "lin")
    T = transport.Transport(prob, am)
    psi = adjoint.dense_solve(T, T.source())
    Ta = adjoint.adjoint_transport(prob, am, weight)
    lam = adjoint.dense_solve(Ta, Ta.source())
    _, _, dfn = adjoint.gradients(T, psi, lam)
    assert dfn.shape == (2, 5)

    def R(fm):
        p = dict(prob)
        p["fmom"] = fm
        Tp = transport.Transport(p, am)
        return adjoint.response(Tp, adjoint.dense_solve(Tp, Tp.source()), weight)
    h = 1e-5
    for m in range(2):
        for n in (1, 3):
            fp = prob["fmom"].copy()
            fm_ = prob["fmom"].copy()
            fp[m, n] += h
            fm_[m, n] -= h
            fd = (R(fp) - R(fm_)) / (2 * h)
            assert abs(fd - dfn[m, n]) < 1e-6 * np.abs(dfn).max(), (m, n)
