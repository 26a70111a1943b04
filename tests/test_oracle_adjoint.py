"""Pins of the oracle's adjoint (oracle/adjoint.py) against the plain
definitions: the transpose of the assembled operator, the adjoint identity
<g, A^-1 f> = <A^-T g, f>, and central finite differences of the detector
response with respect to per-cell sigma_t, sigma_s and the Legendre moments."""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint, angular, transport

CASES = [
    (2, (3, 2), 1, "lin"),
    (2, (2, 3), 1, "const"),
    (3, (2, 2, 2), 0, "lin"),
]


def _setup(dim, nc, level, basis, N=3, seed=11):
    prob = W.random_problem(dim, nc, level, N, seed, basis=basis, g=0.7)
    am = angular.AngularMesh(angular.uniform_paths(level), basis)
    return prob, am


@pytest.mark.parametrize("dim,nc,level,basis", CASES)
def test_reversed_direction_operator_is_the_transpose(dim, nc, level, basis):
    prob, am = _setup(dim, nc, level, basis)
    T = transport.Transport(prob, am)
    Ta = transport.Transport(prob, adjoint.ReversedMesh(am))
    L = T.dense_L()
    La = Ta.dense_L()
    assert np.abs(La - L.T).max() < 1e-13 * np.abs(L).max()
    # the reversal changes L: the test is not vacuous
    assert np.abs(La - L).max() > 1e-3 * np.abs(L).max()
    S = T.dense_S()
    assert np.abs(Ta.dense_S() - S).max() < 1e-14 * np.abs(S).max()


@pytest.mark.parametrize("dim,nc,level,basis", CASES)
def test_reversed_direction_sweep_inverts_the_transpose(dim, nc, level, basis):
    """The sweep of the reversed-direction operators (every direction swept
    in its own upwind order) is the exact inverse of L^T, checked against
    LAPACK on the assembled transpose of the forward L."""
    prob, am = _setup(dim, nc, level, basis)
    T = transport.Transport(prob, am)
    Ta = transport.Transport(prob, adjoint.ReversedMesh(am))
    b = W.random_vector((T.nsdof, T.nadof), 5)
    x = Ta.sweep(b)
    xr = np.linalg.solve(T.dense_L().T, b.reshape(-1)).reshape(b.shape)
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) < 1e-12


@pytest.mark.parametrize("dim,nc,level,basis", CASES)
def test_adjoint_identity(dim, nc, level, basis):
    prob, am = _setup(dim, nc, level, basis)
    T = transport.Transport(prob, am)
    rng = np.random.default_rng(3)
    weight = (rng.uniform(size=T.C) < 0.5).astype(float)
    weight[0] = 1.0
    Ta = adjoint.adjoint_transport(prob, am, weight)
    f = T.source()
    psi = adjoint.dense_solve(T, f)
    g = Ta.source()
    lam = adjoint.dense_solve(Ta, g)
    R = adjoint.response(T, psi, weight)
    assert abs(np.sum(g * psi) - R) < 1e-12 * abs(R)
    assert abs(np.sum(lam * f) - R) < 1e-10 * abs(R)
    # lam solves the transposed system of the forward operator
    A = T.dense_L() - T.dense_S()
    assert np.abs(A.T @ lam.reshape(-1) - g.reshape(-1)).max() < 1e-10 * np.abs(g).max()


def _response(prob, am, weight):
    T = transport.Transport(prob, am)
    return adjoint.response(T, adjoint.dense_solve(T, T.source()), weight)


@pytest.mark.parametrize("dim,nc,level,basis", [CASES[0], CASES[2]])
def test_gradients_match_central_differences(dim, nc, level, basis):
    prob, am = _setup(dim, nc, level, basis)
    T = transport.Transport(prob, am)
    C = T.C
    weight = np.zeros(C)
    weight[-1] = 1.0
    weight[C // 2] = 1.0
    Ta = adjoint.adjoint_transport(prob, am, weight)
    psi = adjoint.dense_solve(T, T.source())
    lam = adjoint.dense_solve(Ta, Ta.source())
    dsigt, dsigs, dfn = adjoint.gradients(T, psi, lam)

    def fd(key, idx):
        p = {k: (np.array(v, dtype=float) if k in ("sigma_t", "sigma_s", "fmom") else v)
             for k, v in prob.items()}
        h = 1e-5 * max(1.0, abs(p[key][idx]))
        p[key][idx] += h
        rp = _response(p, am, weight)
        p[key][idx] -= 2 * h
        rm = _response(p, am, weight)
        return (rp - rm) / (2 * h)

    scale_t = np.abs(dsigt).max()
    for c in (0, C // 2, C - 1):
        assert abs(fd("sigma_t", c) - dsigt[c]) < 1e-6 * scale_t, c
        assert abs(fd("sigma_s", c) - dsigs[c]) < 1e-6 * scale_t, c
    for n in (1, 2, 3):
        assert abs(fd("fmom", n) - dfn[n]) < 1e-6 * np.abs(dfn).max(), n
    # physics: more absorption lowers the response, more scatter raises it
    assert dsigt.sum() < 0 and dsigs.sum() > 0
