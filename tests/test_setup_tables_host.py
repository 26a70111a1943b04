"""The library's host set-up tables against the oracle's (CPU): the library's
set-up source (csrc/setup.cpp) is compiled with a test-only shim
(tests/setup_tables_shim.cpp) and its angular meshes (uniform and
band-refined), angular matrices, harmonics moments (through the scatter
matrix S_f = X diag(f_n) X^T, which does not depend on the harmonics' axis
convention), prolongations, Q1 element matrices, block inverse and
pencil-beam weights are compared with the oracle's independent construction
of the same objects."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import workloads as W
from oracle import angular, harmonics
from oracle.spatial import Q1Cell

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2010_04559_gb300", "csrc")
D = ctypes.POINTER(ctypes.c_double)


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("shim") / "libsetupshim.so")
    cmd = ["g++", "-std=c++17", "-O2", "-shared", "-fPIC", "-I", CSRC,
           "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "setup_tables_shim.cpp"),
           os.path.join(CSRC, "setup.cpp"), "-o", out, "-lpthread"]
    subprocess.run(cmd, check=True, capture_output=True)
    lib = ctypes.CDLL(out)
    lib.shim_paths.restype = ctypes.c_int
    lib.shim_mesh.restype = ctypes.c_int
    lib.shim_invert.restype = ctypes.c_int
    return lib


def _p(a):
    return a.ctypes.data_as(D)


def _axis(ax):
    return (ctypes.c_double * 3)(*ax)


MESHES = [(0, 0, None), (1, 0, None), (2, 0, None), (3, 1, (0.0, 0.0, 1.0)),
          (3, 1, (1.0, 0.0, 0.0))]
MESH_IDS = ["uniform0", "uniform1", "uniform2", "aniso3z", "aniso3x"]


def _oracle_paths(level, aniso, axis):
    return angular.aniso_paths(level, axis) if aniso else angular.uniform_paths(level)


def _lib_paths(shim, level, aniso, axis):
    ax = _axis(axis or (0.0, 0.0, 1.0))
    P = shim.shim_paths(level, aniso, ax, None, 0)
    buf = np.zeros((P, 8), dtype=np.uint8)
    shim.shim_paths(level, aniso, ax, buf.ctypes.data_as(ctypes.c_void_p), P)
    return [tuple(int(v) for v in row if v != 255) for row in buf]


@pytest.mark.parametrize("level,aniso,axis", MESHES, ids=MESH_IDS)
def test_patch_hierarchy_is_the_oracles(shim, level, aniso, axis):
    """Same patches in the same depth-first order (uniform and band-refined)."""
    assert _lib_paths(shim, level, aniso, axis) == _oracle_paths(level, aniso, axis)


@pytest.mark.parametrize("basis", ["lin", "const"])
@pytest.mark.parametrize("level,aniso,axis", MESHES, ids=MESH_IDS)
def test_angular_matrices_are_the_oracles(shim, level, aniso, axis, basis):
    """w = int Psi, M = int Psi Psi, A^xi = int Omega_xi Psi Psi and
    Aw = int Omega_xi Psi per patch (Sec. 2.3), each side with its own
    quadrature."""
    am = angular.AngularMesh(_oracle_paths(level, aniso, axis), basis)
    P, a = am.P, am.a
    w, M = np.zeros((P, a)), np.zeros((P, a, a))
    A, Aw = np.zeros((P, 3, a, a)), np.zeros((P, 3, a))
    n = shim.shim_mesh(level, aniso, _axis(axis or (0.0, 0.0, 1.0)), 1 if basis == "lin" else 0,
                       _p(w), _p(M), _p(A), _p(Aw))
    assert n == P
    for lib, orc in ((w, am.w), (M, am.M), (A, am.A), (Aw, am.Aw)):
        assert np.abs(lib - orc).max() < 1e-13 * max(1.0, np.abs(orc).max())


@pytest.mark.parametrize("level,aniso,axis,N", [(1, 0, None, 8), (2, 0, None, 16),
                                                (3, 1, (0.0, 0.0, 1.0), 12), (0, 0, None, 0)],
                         ids=["uniform1-N8", "uniform2-N16", "aniso3z-N12", "uniform0-N0"])
@pytest.mark.parametrize("basis", ["lin", "const"])
def test_harmonics_moments_give_the_oracles_scatter_matrix(shim, level, aniso, axis, N, basis):
    """S_f = X diag(f_n) X^T from the library's X (polar axis e_x) against the
    oracle's (polar axis e_z): equal by the addition theorem (Sec. 4.2)."""
    am = angular.AngularMesh(_oracle_paths(level, aniso, axis), basis)
    nm = harmonics.nmoments(N)
    Xl = np.zeros((am.nadof, nm))
    shim.shim_xtable(level, aniso, _axis(axis or (0.0, 0.0, 1.0)), 1 if basis == "lin" else 0,
                     N, _p(Xl))
    Xo = am.X(N).reshape(am.nadof, nm)
    f = W.hg_moments(0.85, N)[harmonics.degree_of_index(N)]
    Sl = (Xl * f) @ Xl.T
    So = (Xo * f) @ Xo.T
    assert np.abs(Sl - So).max() < 1e-13 * np.abs(So).max()
    # the zeroth moment is the integral of each basis function
    assert np.abs(Xl[:, 0] * np.sqrt(4 * np.pi) - am.w.reshape(-1)).max() < 1e-13


@pytest.mark.parametrize("basis", ["lin", "const"])
@pytest.mark.parametrize("level,aniso,axis,coarse", [(2, 0, None, 1), (2, 0, None, 0),
                                                     (3, 1, (1.0, 0.0, 0.0), 2)],
                         ids=["uniform2-to-1", "uniform2-to-0", "aniso3x-to-2"])
def test_prolongation_is_the_oracles(shim, level, aniso, axis, coarse, basis):
    paths = _oracle_paths(level, aniso, axis)
    fine = angular.AngularMesh(paths, basis)
    crs = angular.AngularMesh(angular.coarsen_paths(paths, coarse), basis)
    P = np.zeros((fine.nadof, crs.nadof))
    shim.shim_prolongation(level, aniso, _axis(axis or (0.0, 0.0, 1.0)),
                           1 if basis == "lin" else 0, coarse, _p(P))
    assert np.abs(P - angular.prolongation(fine, crs)).max() < 1e-14


@pytest.mark.parametrize("dim,h", [(2, (0.3, 0.7)), (3, (0.2, 0.5, 0.9))])
def test_q1_matrices_are_the_oracles(shim, dim, h):
    """The library's closed forms against the oracle's Gauss-rule integrals."""
    c = Q1Cell(list(h))
    s = 2 ** dim
    N, V = np.zeros((s, s)), np.zeros((dim, s, s))
    Fo, Fn = np.zeros((2 * dim, s, s)), np.zeros((2 * dim, s, s))
    mu, mf = np.zeros(s), np.zeros((2 * dim, s))
    hh = (ctypes.c_double * 3)(*(list(h) + [1.0] * (3 - dim)))
    shim.shim_q1(dim, hh, _p(N), _p(V), _p(Fo), _p(Fn), _p(mu), _p(mf))
    for lib, orc in ((N, c.N), (V, c.V), (Fo, c.Fown), (Fn, c.Fnb), (mu, c.mu), (mf, c.mf)):
        assert np.abs(lib - orc).max() < 1e-15


@pytest.mark.parametrize("dim,h", [(2, (0.3, 0.7)), (3, (0.2, 0.5, 0.9))])
def test_q1_face_mass_is_the_oracles_face_integral(shim, dim, h):
    """facemass[xi][j'][j]: the integral over a face normal to xi of the
    products of the face's nodal functions (j', j: nodes of the face, the bit
    of axis xi inserted), which the kernels use for the upwind coupling."""
    c = Q1Cell(list(h))
    hs = 2 ** (dim - 1)
    fm = np.zeros((dim, hs, hs))
    shim.shim_q1_facemass(dim, (ctypes.c_double * 3)(*(list(h) + [1.0] * (3 - dim))), _p(fm))

    def face_node(j, axis, bit):
        lo = j & ((1 << axis) - 1)
        return lo | (bit << axis) | ((j >> axis) << (axis + 1))
    for xi in range(dim):
        for jp in range(hs):
            for j in range(hs):
                own = c.Fown[2 * xi][face_node(jp, xi, 0), face_node(j, xi, 0)]
                nb = c.Fnb[2 * xi][face_node(jp, xi, 0), face_node(j, xi, 1)]
                assert abs(fm[xi, jp, j] - own) < 1e-15 and abs(fm[xi, jp, j] - nb) < 1e-15


@pytest.mark.parametrize("lmax", [4, 5, 6])
def test_band_refined_hierarchies_up_to_the_papers_largest(shim, lmax):
    """The library's band-refined meshes about z for l_max = 4, 5, 6 (the
    paper's 128, 440 and 1388 patches) equal the oracle's path for path."""
    assert _lib_paths(shim, lmax, 1, (0.0, 0.0, 1.0)) == angular.aniso_paths(lmax)


def test_block_inverse_is_lapacks(shim):
    rng = np.random.default_rng(7)
    for n in (1, 3, 12, 24, 48):
        A = rng.standard_normal((n, n)) + n * np.eye(n)
        Ai = np.zeros((n, n))
        assert shim.shim_invert(n, _p(np.ascontiguousarray(A)), _p(Ai)) == 1
        assert np.abs(Ai - np.linalg.inv(A)).max() < 1e-13 * np.abs(np.linalg.inv(A)).max()
    Z = np.zeros((4, 4))
    assert shim.shim_invert(4, _p(Z), _p(np.zeros((4, 4)))) == 0     # singular: refused


def _beam_directions():
    import test_oracle_beam as PB
    out = [("normal+x", np.array([1.0, 0.0, 0.0])), ("normal-z", np.array([0.0, 0.0, -1.0]))]
    for name, e in PB._general_directions():
        out.append((name, e / np.linalg.norm(e)))
    out.append(("inside-other-octant", np.array([-0.3, 0.5, -0.8]) / np.linalg.norm([0.3, 0.5, 0.8])))
    return out


@pytest.mark.parametrize("basis", ["lin", "const"])
@pytest.mark.parametrize("level,aniso,axis", [(2, 0, None), (3, 1, (1.0, 0.0, 0.0))],
                         ids=["uniform2", "aniso3x"])
def test_beam_weights_are_the_oracles(shim, level, aniso, axis, basis):
    """The library's pencil-beam weights (shares of the Dirac mass times
    Psi at the beam direction) against the oracle's, for directions at an
    octahedron vertex, inside a patch, on an edge and at vertices of unequal
    angles (Sec. 5.4 reading)."""
    from oracle import transport
    am = angular.AngularMesh(_oracle_paths(level, aniso, axis), basis)
    shim.shim_beam.restype = ctypes.c_double
    for name, e in _beam_directions():
        out = np.zeros(am.nadof)
        total = shim.shim_beam(level, aniso, _axis(axis or (0.0, 0.0, 1.0)),
                               1 if basis == "lin" else 0, _p(np.ascontiguousarray(e)), _p(out))
        ref = transport.beam_weights(am, e).reshape(-1)
        assert abs(total - 1.0) < 1e-12, name
        assert np.abs(out - ref).max() < 1e-13, name
