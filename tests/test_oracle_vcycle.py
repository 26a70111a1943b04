"""Pins of the oracle's linear V-cycle (Fig. lmg, Sec. 4.1) against the cycle's
algebra written with dense matrices that the pins assemble themselves (CPU).

The V-cycle of Fig. lmg is a linear map f -> M f.  Its error propagator is
fixed by the figure: nu_pre source iterations (error map E_s = I - L^-1 A =
L^-1 S), the coarse-grid correction with the re-discretised coarse operator
(error map I - P A_c^-1 P^T A, where R = P^T and the coarsest level is solved
by Gauss-Seidel sweeps that converge to A_c^-1), then nu_post source
iterations:

    I - M A = E_s^nu_post (I - P A_c^-1 P^T A) E_s^nu_pre.

Every dense matrix below is assembled from the problem alone (the angular
mesh coarsened to each level, that level's scatter order N_r, dense L and S,
the prolongation P) and solved by LAPACK; none comes from the hierarchy whose
cycle is checked.  So a dropped smoothing step, a restriction of f instead of
the residual, or the fine scatter order on the coarse level (A_c built with N
instead of N_r) breaks one of these identities
(tests/test_oracle_pins_catch_mistakes.py plants each of them).
"""
import numpy as np
import pytest

import workloads as W
from oracle import angular, multigrid, transport


def _hierarchy(nu_pre, nu_post, Nr, sweeps, ratio=0.5, nc=(3, 2), level=1, seed=41):
    prob = W.random_problem(2, nc, level, Nr[0], seed, g=0.8)
    prob["sigma_s"] = ratio * prob["sigma_t"]
    prob["mg"] = dict(nlevels=len(Nr), Nr=list(Nr), nu_pre=nu_pre, nu_post=nu_post,
                      coarse_sweeps=sweeps)
    return prob, multigrid.Hierarchy(prob)


def _dense(T):
    L = T.dense_L()
    return L, L - T.dense_S()


def _mesh(prob, k):
    """Angular mesh of level k of the cycle (k = 0 the finest): the problem's
    uniform mesh coarsened k times (Sec. 4.1)."""
    paths = angular.uniform_paths(prob["level"])
    return angular.AngularMesh(angular.coarsen_paths(paths, prob["level"] - k), prob["basis"])


def _level(prob, k):
    """Operators of level k built from the problem: its mesh and N_r[k]."""
    return transport.Transport(prob, _mesh(prob, k), prob["mg"]["Nr"][k])


def _kron_P(prob, k, nsdof):
    """Prolongation of level k+1 to level k on flattened vectors: x @ P^T per
    spatial row, i.e. kron(I_nsdof, P)."""
    return np.kron(np.eye(nsdof), angular.prolongation(_mesh(prob, k), _mesh(prob, k + 1)))


def _two_grid_error_map(prob, nu_pre, nu_post):
    T0, T1 = _level(prob, 0), _level(prob, 1)
    L0, A0 = _dense(T0)
    _, A1 = _dense(T1)
    n = A0.shape[0]
    I = np.eye(n)
    Es = I - np.linalg.solve(L0, A0)             # source iteration: L^-1 S
    P = _kron_P(prob, 0, T0.nsdof)
    CGC = I - P @ np.linalg.solve(A1, P.T @ A0)  # exact coarse-grid correction
    return (np.linalg.matrix_power(Es, nu_post) @ CGC @ np.linalg.matrix_power(Es, nu_pre),
            A0)


def _coarse_gs_converged(prob, sweeps):
    """The coarsest-level Gauss-Seidel with `sweeps` sweeps has converged to
    A_c^-1 (checked against LAPACK on a random right-hand side)."""
    Tc = _level(prob, len(prob["mg"]["Nr"]) - 1)
    _, Ac = _dense(Tc)
    fc = W.random_vector((Tc.nsdof, Tc.nadof), 44)
    xr = np.linalg.solve(Ac, fc.reshape(-1))
    xg = multigrid.coarse_gs(Tc, fc, np.zeros_like(fc), sweeps).reshape(-1)
    return np.linalg.norm(xg - xr) / np.linalg.norm(xr)


@pytest.mark.parametrize("nu_pre,nu_post,Nr", [(1, 1, (6, 3)), (1, 0, (6, 2)), (2, 1, (5, 3))])
def test_two_grid_error_propagator(nu_pre, nu_post, Nr):
    """I - M A equals E_s^nu_post (I - P A_c^-1 P^T A) E_s^nu_pre on random
    vectors, with A_c the coarse level re-discretised at order N_r (Fig. lmg,
    Sec. 4.1, Sec. 4.3)."""
    sweeps = 60
    prob, H = _hierarchy(nu_pre, nu_post, Nr, sweeps)
    assert _coarse_gs_converged(prob, sweeps) < 1e-13
    E, A0 = _two_grid_error_map(prob, nu_pre, nu_post)
    T0 = _level(prob, 0)
    for seed in (45, 46):
        v = W.random_vector((T0.nsdof, T0.nadof), seed)
        Av = (A0 @ v.reshape(-1)).reshape(v.shape)
        lhs = v - H.vcycle(Av)
        rhs = (E @ v.reshape(-1)).reshape(v.shape)
        assert np.linalg.norm(lhs - rhs) / np.linalg.norm(v) < 1e-11


def test_pure_absorber_cycle_is_exact():
    """sigma_s = 0: one pre-smoothing step is L^-1 f = A^-1 f, the residual
    vanishes, the coarse correction of a zero residual is zero, and the
    post-smoothing step keeps A^-1 f (Fig. lmg)."""
    prob, H = _hierarchy(1, 1, (4, 2, 2), 10, ratio=0.0, level=2, nc=(2, 2))
    T0 = _level(prob, 0)
    _, A0 = _dense(T0)
    f = W.random_vector((T0.nsdof, T0.nadof), 47)
    x = np.linalg.solve(A0, f.reshape(-1)).reshape(f.shape)
    y = H.vcycle(f)
    assert np.linalg.norm(y - x) / np.linalg.norm(x) < 1e-12


def test_cycle_without_smoothing_is_coarse_correction():
    """nu_pre = nu_post = 0: the cycle is P A_c^-1 P^T f (restriction of the
    right-hand side, coarse solve, prolongation; Fig. lmg)."""
    sweeps = 60
    prob, H = _hierarchy(0, 0, (6, 3), sweeps)
    assert _coarse_gs_converged(prob, sweeps) < 1e-13
    T0, T1 = _level(prob, 0), _level(prob, 1)
    _, A1 = _dense(T1)
    P = _kron_P(prob, 0, T0.nsdof)
    f = W.random_vector((T0.nsdof, T0.nadof), 48)
    expect = P @ np.linalg.solve(A1, P.T @ f.reshape(-1))
    y = H.vcycle(f).reshape(-1)
    assert np.linalg.norm(y - expect) / np.linalg.norm(expect) < 1e-11


def test_three_level_recursion():
    """A three-level cycle applies the level-1 cycle as its coarse solve:
    I - M A = E_s (I - P M_1 P^T A) E_s, with M_1 the two-level cycle of
    levels 1-2 (itself pinned by the two-grid identity), so the recursion
    passes the restricted residual, not f, and prolongs into the smoothed
    iterate (Fig. lmg)."""
    prob, H = _hierarchy(1, 1, (6, 3, 2), 60, level=2, nc=(2, 2))
    T0 = _level(prob, 0)
    L0, A0 = _dense(T0)
    n = A0.shape[0]
    Es = np.eye(n) - np.linalg.solve(L0, A0)
    P = _kron_P(prob, 0, T0.nsdof)
    v = W.random_vector((T0.nsdof, T0.nadof), 49)
    Av = A0 @ v.reshape(-1)
    # error map applied to v with the coarse solve replaced by the level-1 cycle
    e1 = Es @ v.reshape(-1)
    T1 = _level(prob, 1)
    rc = (P.T @ (A0 @ e1)).reshape(T1.nsdof, T1.nadof)
    e2 = e1 - P @ H.vcycle(rc, k=1).reshape(-1)
    expect = Es @ e2
    lhs = v.reshape(-1) - H.vcycle(Av.reshape(v.shape)).reshape(-1)
    assert np.linalg.norm(lhs - expect) / np.linalg.norm(v) < 1e-11
