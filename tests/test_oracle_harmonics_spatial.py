"""Pins of the oracle's spherical harmonics (against scipy and the addition
theorem), its Q1 spatial matrices (against closed forms) and the HG moment
input (against numerical integration of the phase function). CPU only."""
import numpy as np
import pytest
import scipy.special as sp
from scipy import integrate

import workloads as W
from oracle import angular, harmonics
from oracle.spatial import Q1Cell


def _unit_vectors(n, seed):
    v = np.random.default_rng(seed).standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def test_real_harmonics_match_scipy():
    N = 12
    om = _unit_vectors(40, 0)
    Y = harmonics.real_sph_harm(N, om)
    theta = np.arccos(om[:, 2])
    phi = np.arctan2(om[:, 1], om[:, 0])
    for n in range(N + 1):
        for o in range(-n, n + 1):
            m = abs(o)
            c = sp.sph_harm_y(n, m, theta, phi)   # Condon-Shortley phase included
            if o == 0:
                ref = c.real
            elif o > 0:
                ref = np.sqrt(2) * (-1) ** m * c.real
            else:
                ref = np.sqrt(2) * (-1) ** m * c.imag
            assert np.abs(Y[:, n * n + n + o] - ref).max() < 1e-12, (n, o)


def test_addition_theorem():
    N = 64
    a = _unit_vectors(5, 1)
    b = _unit_vectors(5, 2)
    Ya = harmonics.real_sph_harm(N, a)
    Yb = harmonics.real_sph_harm(N, b)
    deg = harmonics.degree_of_index(N)
    for n in (0, 1, 5, 17, 40, 64):
        sel = deg == n
        lhs = np.sum(Ya[:, sel] * Yb[:, sel], axis=1)
        rhs = (2 * n + 1) / (4 * np.pi) * sp.eval_legendre(n, np.sum(a * b, axis=1))
        assert np.abs(lhs - rhs).max() < 1e-11 * (2 * n + 1)


def test_orthonormal_under_patch_quadrature():
    N = 8
    G = np.zeros((harmonics.nmoments(N),) * 2)
    for p in angular.uniform_paths(1):
        v = angular.path_vertices(p)
        om, w = angular.patch_quadrature(v, angular.default_order(1, 2 * N))
        Y = harmonics.real_sph_harm(N, om)
        G += (Y * w[:, None]).T @ Y
    assert np.abs(G - np.eye(len(G))).max() < 1e-13


@pytest.mark.parametrize("g", [0.5, 0.8, 0.95])
def test_hg_moments_are_legendre_moments(g):
    # 2 pi int p_HG(mu) P_n(mu) dmu = g^n with the normalised HG phase function
    def p_hg(mu):
        return (1 - g * g) / (4 * np.pi * (1 + g * g - 2 * g * mu) ** 1.5)
    f = W.hg_moments(g, 8)
    for n in range(9):
        val, _ = integrate.quad(lambda mu: 2 * np.pi * p_hg(mu) * sp.eval_legendre(n, mu),
                                -1, 1, epsabs=1e-13, epsrel=1e-13, limit=400)
        assert abs(val - f[n]) < 1e-10


@pytest.mark.parametrize("alpha,N", [(1.0, 4), (0.5, 12), (2.0, 24)])
def test_fp_equivalent_moments(alpha, N):
    # the momentum-transfer cross section sigma_{s,0} - sigma_{s,1} equals
    # alpha (Sec. 5: a transport cross section of 1 means alpha = 1); the
    # expansion vanishes at n = N, and sigma_{s,0} - sigma_{s,n} grows with
    # the Laplace-Beltrami eigenvalues n(n+1), checked on a harmonic: the
    # surface Laplacian of P_n(mu) is -n(n+1) P_n(mu)
    s0, f = W.fp_moments(alpha, N)
    sn = s0 * f
    assert abs((sn[0] - sn[1]) - alpha) < 1e-12 * max(1.0, s0)
    assert abs(sn[N]) < 1e-12 * s0 and abs(f[0] - 1.0) < 1e-15
    import sympy
    x = sympy.symbols("x")
    mu = [sympy.Rational(k, 10) for k in (-9, -4, 0, 3, 8)]
    for n in range(N + 1):
        # (1 - x^2) P'' - 2 x P' is the surface Laplacian of a zonal function
        # (exact rational arithmetic)
        p = sympy.legendre(n, x)
        lap = (1 - x ** 2) * sympy.diff(p, x, 2) - 2 * x * sympy.diff(p, x)
        lam = sn[0] - sn[n]
        for m in mu:
            v = float(0.5 * alpha * lap.subs(x, m)) + lam * float(p.subs(x, m))
            assert abs(v) < 1e-9 * max(1.0, lam)


def _m1(h):
    return h / 6.0 * np.array([[2.0, 1.0], [1.0, 2.0]])


G1 = np.array([[-0.5, -0.5], [0.5, 0.5]])    # int l_l' l_i


def test_q1_2d_closed_forms():
    hx, hy = 0.3, 0.7
    c = Q1Cell([hx, hy])
    # node i = a + 2b  ->  N = kron(m1y, m1x) in (b, a) ordering
    assert np.abs(c.N - np.kron(_m1(hy), _m1(hx))).max() < 1e-15
    assert np.abs(c.V[0] - np.kron(_m1(hy), G1)).max() < 1e-15
    assert np.abs(c.V[1] - np.kron(G1, _m1(hx))).max() < 1e-15
    e0 = np.diag([1.0, 0.0])
    e1 = np.diag([0.0, 1.0])
    ex01 = np.array([[0.0, 1.0], [0.0, 0.0]])   # own node a=0 meets neighbour node a=1
    ex10 = ex01.T
    # faces: f = 2*axis + side
    assert np.abs(c.Fown[0] - np.kron(_m1(hy), e0)).max() < 1e-15
    assert np.abs(c.Fown[1] - np.kron(_m1(hy), e1)).max() < 1e-15
    assert np.abs(c.Fown[3] - np.kron(e1, _m1(hx))).max() < 1e-15
    assert np.abs(c.Fnb[0] - np.kron(_m1(hy), ex01)).max() < 1e-15
    assert np.abs(c.Fnb[1] - np.kron(_m1(hy), ex10)).max() < 1e-15
    assert np.abs(c.Fnb[2] - np.kron(ex01, _m1(hx))).max() < 1e-15
    assert np.abs(c.mu - hx * hy / 4).max() < 1e-16
    assert np.abs(c.mf[1] - np.array([0, hy / 2, 0, hy / 2])).max() < 1e-16


def test_q1_3d_closed_forms():
    h = [0.2, 0.5, 0.9]
    c = Q1Cell(h)
    M = [_m1(x) for x in h]
    assert np.abs(c.N - np.kron(M[2], np.kron(M[1], M[0]))).max() < 1e-15
    assert np.abs(c.V[0] - np.kron(M[2], np.kron(M[1], G1))).max() < 1e-15
    assert np.abs(c.V[1] - np.kron(M[2], np.kron(G1, M[0]))).max() < 1e-15
    assert np.abs(c.V[2] - np.kron(G1, np.kron(M[1], M[0]))).max() < 1e-15
    e1 = np.diag([0.0, 1.0])
    assert np.abs(c.Fown[5] - np.kron(e1, np.kron(M[1], M[0]))).max() < 1e-15
    assert abs(c.mu.sum() - np.prod(h)) < 1e-15
