"""Pins of the oracle's transport operators, scatter, sweep, multigrid and
GMRES against dense LU, closed-form solutions and conservation laws (CPU)."""
import numpy as np
import pytest
import scipy.special as sp

import workloads as W
from oracle import angular, gmres, harmonics, multigrid, transport


def _T(prob, level=None, basis=None, Nscat=None):
    level = prob["level"] if level is None else level
    basis = prob["basis"] if basis is None else basis
    am = angular.AngularMesh(angular.uniform_paths(level), basis)
    return transport.Transport(prob, am, Nscat)


CASES = [
    (2, (3, 2), 0, "lin"),
    (2, (2, 3), 1, "const"),
    (2, (3, 3), 1, "lin"),
    (3, (2, 2, 2), 0, "lin"),
    (3, (2, 1, 2), 0, "const"),
]


@pytest.mark.parametrize("dim,nc,level,basis", CASES)
def test_sweep_is_exact_inverse_of_L(dim, nc, level, basis):
    prob = W.random_problem(dim, nc, level, 4, 11, basis=basis)
    T = _T(prob)
    b = W.random_vector((T.nsdof, T.nadof), 3)
    x = T.sweep(b)
    Ld = T.dense_L()
    xr = np.linalg.solve(Ld, b.reshape(-1)).reshape(b.shape)
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) < 1e-13
    # apply_L is the matrix-free form of the same L
    assert np.linalg.norm(T.apply_L(x) - b) / np.linalg.norm(b) < 1e-13


@pytest.mark.parametrize("dim,nc,level,basis", CASES)
def test_gmres_matches_dense_lu(dim, nc, level, basis):
    prob = W.random_problem(dim, nc, level, 4, 12, basis=basis, inflow=0.3)
    T = _T(prob)
    f = T.source()
    A = T.dense_L() - T.dense_S()
    xr = np.linalg.solve(A, f.reshape(-1)).reshape(f.shape)
    x, its, hist, rel = gmres.gmres(T.apply_A, f, T.sweep, 1e-13, 20, 400)
    assert rel < 1e-13
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) < 1e-11


@pytest.mark.parametrize("dim,nc,basis", [(2, (3, 2), "lin"), (2, (2, 2), "const"),
                                          (3, (2, 2, 1), "lin")])
def test_infinite_medium_closed_form(dim, nc, basis):
    """Inflow psi_inf = Q/(sigma_t - sigma_s) on every face: the exact solution
    is the constant psi_inf, which lies in the DG space, so the discrete
    solution equals it and the scalar flux is q/(sigma_t - sigma_s)."""
    C = int(np.prod(nc))
    st, ss, q = 2.5, 2.0, 1.0
    psi_inf = q / (4 * np.pi) / (st - ss)
    prob = W.problem(dim, nc, np.full(C, st), np.full(C, ss), 6, W.hg_moments(0.8, 6),
                     np.full(C, q), 1 if dim == 2 else 0, basis=basis,
                     boundary=[(1, psi_inf)] * (2 * dim))
    T = _T(prob)
    x, its, _, rel = gmres.gmres(T.apply_A, T.source(), T.sweep, 1e-13, 20, 400)
    assert np.abs(x - psi_inf).max() / psi_inf < 1e-11
    assert np.abs(T.scalar_flux(x) - q / (st - ss)).max() < 1e-10


def _balance_terms(T, psi):
    """outflow - inflow leakage, absorption and source of the solution."""
    s, a = T.s, T.a
    leak = 0.0
    for c in range(T.C):
        for f in range(2 * T.dim):
            if T.neighbour(c, f) >= 0:
                continue
            xi, side = divmod(f, 2)
            sgn = 2.0 * side - 1.0
            blk = psi[c * s:(c + 1) * s].reshape(s, T.P, a)
            for q in range(T.P):
                if T.outflow[f, q]:
                    leak += T.cell.mf[f] @ blk[:, q, :] @ (sgn * T.am.Aw[q, xi])
    phis = T.scalar_flux(psi)
    absn = sum((T.sigma_t[c] - T.sigma_s[c]) * (T.cell.mu @ phis[c * s:(c + 1) * s])
               for c in range(T.C))
    src = sum(T.prob["q"][c] * np.prod(T.cell.h) for c in range(T.C))
    return leak, absn, src


@pytest.mark.parametrize("dim,nc,level", [(2, (4, 3), 1), (3, (2, 2, 2), 0)])
def test_particle_balance(dim, nc, level):
    prob = W.random_problem(dim, nc, level, 6, 13)
    T = _T(prob)
    x, its, _, rel = gmres.gmres(T.apply_A, T.source(), T.sweep, 1e-13, 20, 400)
    leak, absn, src = _balance_terms(T, x)
    assert abs(leak + absn - src) / src < 1e-11
    assert leak > 0 and absn > 0


def test_scatter_matrix_symmetric_psd_sum_rule():
    prob = W.random_problem(2, (2, 2), 1, 8, 14, g=0.9)
    T = _T(prob)
    Sf = T.angular_scatter_matrix()
    assert np.abs(Sf - Sf.T).max() < 1e-15
    assert np.linalg.eigvalsh(Sf).min() > -1e-14
    # zeroth-moment sum rule: sum over test functions = f_0 * int Psi
    assert np.abs(Sf.sum(axis=0) - T.am.w.reshape(-1)).max() < 1e-14


def test_scatter_order_zero_is_isotropic():
    prob = W.random_problem(2, (2, 2), 1, 8, 15)
    T = _T(prob, Nscat=0)
    w = T.am.w.reshape(-1)
    assert np.abs(T.angular_scatter_matrix() - np.outer(w, w) / (4 * np.pi)).max() < 1e-15


def test_scatter_matrix_equals_legendre_double_integral():
    """S_f[(q,m),(p,d)] = sum_n f_n (2n+1)/(4pi) int int Psi_qm Psi_pd P_n(Omega.Omega'),
    the kernel written with Legendre polynomials (no harmonics involved)."""
    N = 4
    prob = W.random_problem(2, (1, 1), 0, N, 16, g=0.7)
    T = _T(prob)
    am = T.am
    nodes = []
    for q in range(am.P):
        om, w = angular.patch_quadrature(am.verts[q], 24)
        psi = angular.basis_eval(am.verts[q], am.octant[q], "lin", om)
        nodes.append((om, w, psi))
    S = np.zeros((am.nadof, am.nadof))
    f = prob["fmom"]
    for q in range(am.P):
        oq, wq, pq = nodes[q]
        for p in range(am.P):
            op, wp, pp = nodes[p]
            mu = oq @ op.T
            K = sum(f[n] * (2 * n + 1) / (4 * np.pi) * sp.eval_legendre(n, mu) for n in range(N + 1))
            S[q * 3:q * 3 + 3, p * 3:p * 3 + 3] = (pq * wq[:, None]).T @ K @ (pp * wp[:, None])
    assert np.abs(S - T.angular_scatter_matrix()).max() < 1e-13


def test_pure_absorber_converges_in_one_iteration():
    prob = W.random_problem(2, (3, 3), 1, 4, 17)
    prob["sigma_s"] = np.zeros_like(prob["sigma_s"])
    T = _T(prob)
    x, its, _, rel = gmres.gmres(T.apply_A, T.source(), T.sweep, 1e-12, 20, 50)
    assert its == 1 and rel < 1e-12


def test_2d_z_mirror_symmetry():
    prob = W.random_problem(2, (3, 2), 1, 6, 18)
    T = _T(prob)
    x, *_ = gmres.gmres(T.apply_A, T.source(), T.sweep, 1e-13, 20, 400)
    # octants o and o^1 differ only in the z sign; patches keep their local order
    per = T.P // 8
    mirror = np.array([((q // per) ^ 1) * per + q % per for q in range(T.P)])
    xb = x.reshape(T.nsdof, T.P, T.a)
    assert np.abs(xb - xb[:, mirror]).max() < 1e-12 * np.abs(xb).max()


def test_multigrid_preconditioned_solution_and_fewer_iterations():
    prob = W.random_problem(2, (4, 4), 2, 8, 19, g=0.9)
    prob["mg"] = dict(nlevels=3, Nr=[8, 4, 4], nu_pre=1, nu_post=1, coarse_sweeps=10)
    H = multigrid.Hierarchy(prob)
    T = H.levels[0]
    f = T.source()
    xs, its_s, *_ = gmres.gmres(T.apply_A, f, T.sweep, 1e-11, 20, 400)
    xm, its_m, _, rel = gmres.gmres(T.apply_A, f, lambda v: H.vcycle(v), 1e-11, 20, 400)
    assert rel < 1e-11
    assert np.linalg.norm(xm - xs) / np.linalg.norm(xs) < 1e-9
    assert its_m < its_s


def test_vcycle_is_linear():
    prob = W.random_problem(2, (3, 3), 2, 6, 20)
    prob["mg"] = dict(nlevels=3, Nr=[6, 3, 2], nu_pre=1, nu_post=1, coarse_sweeps=3)
    H = multigrid.Hierarchy(prob)
    T = H.levels[0]
    f1 = W.random_vector((T.nsdof, T.nadof), 21)
    f2 = W.random_vector((T.nsdof, T.nadof), 22)
    lhs = H.vcycle(2.0 * f1 - 0.5 * f2)
    rhs = 2.0 * H.vcycle(f1) - 0.5 * H.vcycle(f2)
    assert np.linalg.norm(lhs - rhs) / np.linalg.norm(rhs) < 1e-12


def test_coarse_gs_fixed_point_and_convergence():
    prob = W.random_problem(2, (3, 3), 1, 6, 23, g=0.9)
    T = _T(prob, Nscat=4)
    f = T.source()
    A = T.dense_L() - T.dense_S()
    xr = np.linalg.solve(A, f.reshape(-1)).reshape(f.shape)
    # the exact solution is a fixed point of a Gauss-Seidel sweep
    x1 = multigrid.coarse_gs(T, f, xr, 1)
    assert np.linalg.norm(x1 - xr) / np.linalg.norm(xr) < 1e-13
    # and the sweeps converge to it from zero
    x = multigrid.coarse_gs(T, f, np.zeros_like(f), 25)
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) < 1e-9


def test_coarse_gs_block_equation_holds():
    """After one GS sweep from x0, every block (c, q) satisfies its local
    equation with newer values for blocks visited before it and older values
    for blocks visited after it (the definition of Gauss-Seidel)."""
    prob = W.random_problem(2, (2, 2), 0, 4, 24)
    T = _T(prob)
    f = W.random_vector((T.nsdof, T.nadof), 25)
    x0 = W.random_vector((T.nsdof, T.nadof), 26)
    x1 = multigrid.coarse_gs(T, f, x0, 1)
    A = T.dense_L() - T.dense_S()
    # visiting order
    order = []
    for d in range(T.ndir):
        for c in T.sweep_order(d):
            for q in T.patches_of(d):
                order.append((c, q))
    s, a = T.s, T.a

    def gidx(c, q):
        return ((c * s + np.arange(s))[:, None] * T.nadof + q * a + np.arange(a)[None, :]).reshape(-1)

    pos = {blk: i for i, blk in enumerate(order)}
    newer = np.zeros(T.nsdof * T.nadof, dtype=bool)
    for blk, i in pos.items():
        pass
    v0 = x0.reshape(-1)
    v1 = x1.reshape(-1)
    fv = f.reshape(-1)
    for k, (c, q) in enumerate(order):
        r = gidx(c, q)
        mix = v0.copy()
        for (c2, q2) in order[:k + 1]:
            g = gidx(c2, q2)
            mix[g] = v1[g]
        res = fv[r] - A[r] @ mix
        assert np.abs(res).max() < 1e-12 * (1 + np.abs(fv).max())


def test_scatter_on_a_subset_of_cells_equals_the_full_scatter():
    prob = W.random_problem(2, (3, 2), 1, 5, 27)
    T = _T(prob)
    x = W.random_vector((T.nsdof, T.nadof), 28)
    full = T.scatter(x)
    cells = [4, 1]
    rows = np.concatenate([np.arange(c * T.s, (c + 1) * T.s) for c in cells])
    part = T.scatter(x[rows], cells=cells)
    assert np.abs(part - full[rows]).max() < 1e-13 * np.abs(full).max()
