"""Pins of the oracle's BiCGStab (oracle/bicgstab.py): a plain linear system
against LAPACK, and the transport system with the sweep and with the
multigrid cycle as preconditioner against the dense LU solution."""
import numpy as np
import pytest

import workloads as W
from oracle import angular, bicgstab, multigrid, transport


def test_unpreconditioned_matches_lapack():
    rng = np.random.default_rng(5)
    n = 60
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) * 0.4  # nonsymmetric, well conditioned
    b = rng.standard_normal(n)
    x, its, hist, rel = bicgstab.bicgstab(lambda v: A @ v, b, lambda v: v, 1e-13, 500)
    assert rel < 1e-12
    assert np.linalg.norm(x - np.linalg.solve(A, b)) / np.linalg.norm(b) < 1e-11
    assert its < n


@pytest.mark.parametrize("dim,nc,level,basis", [(2, (3, 2), 1, "lin"), (2, (2, 3), 1, "const"),
                                                (3, (2, 2, 2), 0, "lin")])
def test_sweep_preconditioned_matches_dense_lu(dim, nc, level, basis):
    prob = W.random_problem(dim, nc, level, 4, 13, basis=basis, inflow=0.3)
    T = transport.Transport(prob, angular.AngularMesh(angular.uniform_paths(level), basis))
    f = T.source()
    xr = np.linalg.solve(T.dense_L() - T.dense_S(), f.reshape(-1)).reshape(f.shape)
    x, its, hist, rel = bicgstab.bicgstab(T.apply_A, f, T.sweep, 1e-13, 400)
    assert rel < 1e-12
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) < 1e-10


def test_multigrid_preconditioned_matches_dense_lu():
    prob = W.random_problem(2, (3, 2), 2, 6, 14, g=0.85)
    prob["mg"] = dict(nlevels=3, Nr=[6, 4, 3], nu_pre=1, nu_post=1, coarse_sweeps=4)
    H = multigrid.Hierarchy(prob)
    T = H.levels[0]
    f = T.source()
    xr = np.linalg.solve(T.dense_L() - T.dense_S(), f.reshape(-1)).reshape(f.shape)
    x, its, _, rel = bicgstab.bicgstab(T.apply_A, f, H.vcycle, 1e-13, 400)
    assert rel < 1e-12
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) < 1e-10
