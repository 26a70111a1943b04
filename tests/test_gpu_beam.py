"""GPU parity of the pencil-beam boundary source (Sec. 5.4): the source vector
against the oracle on uniform and band-refined angular meshes, 2D and 3D, the
forward and adjoint contexts; the FP64 and mixed solves of a beam problem
against the oracle's; and the forward-peaked beam workload (sigma_t = 5,
sigma_s = 4.95, HG g = 0.98) at reduced size, mixed against FP64."""
import numpy as np
import pytest

import workloads as W
from oracle import angular, gmres, multigrid, transport

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_04559_gb300 import build
    build.build()


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _beam(dim, nc, level, faces, N=4, g=0.8, basis="lin", ss=0.8, q=0.0, seed=71):
    rng = np.random.default_rng(seed)
    C = int(np.prod(nc))
    st = 1.0 + rng.random(C)
    bnd = [(0, 0.0)] * (2 * dim)
    for f, S in faces:
        bnd[f] = (2, S)
    return W.problem(dim, nc, st, ss * st, N, W.hg_moments(g, N), np.full(C, q), level,
                     basis=basis, boundary=bnd)


SRC = [
    (2, (5, 4), 1, "lin", [(0, 1.0)], None),
    (2, (3, 6), 2, "const", [(1, 0.7), (2, 1.3)], None),
    (3, (3, 2, 4), 1, "lin", [(5, 2.0), (0, 0.5)], None),
    (2, (4, 3), None, "lin", [(0, 1.0)], ((1.0, 0.0, 0.0), 3)),
    (3, (2, 3, 2), None, "lin", [(4, 1.0), (3, 0.4)], ((0.0, 0.0, 1.0), 3)),
]


@pytest.mark.parametrize("dim,nc,level,basis,faces,aniso", SRC)
def test_beam_source_matches_oracle(dim, nc, level, basis, faces, aniso):
    from paper_2010_04559_gb300 import context_from_problem
    prob = _beam(dim, nc, level if level is not None else 0, faces, basis=basis, q=0.3)
    paths = (angular.uniform_paths(level) if aniso is None
             else angular.aniso_paths(aniso[1], aniso[0]))
    T = transport.Transport(prob, angular.AngularMesh(paths, basis))
    ctx = context_from_problem(prob, device=0, aniso=aniso)
    assert ctx.amgt_query_sizes(0) == (T.nsdof, T.nadof)
    ref = T.source()
    for td, tol in ((torch.float64, 1e-14), (torch.float32, 1e-7)):
        f = torch.empty((T.nsdof, T.nadof), device="cuda", dtype=td)
        ctx.amgt_op_source(0, f)
        torch.cuda.synchronize()
        assert _rel(f.double().cpu().numpy(), ref) < tol
    ctx.close()


def test_beam_on_an_adjoint_context_uses_the_reversed_directions():
    """An adjoint context holds the operator with every direction reversed:
    its patch q covers -D_q, so a beam there is the oracle's beam on the
    mirrored face of the reversed mesh."""
    from oracle import adjoint as oadj
    from paper_2010_04559_gb300 import context_from_problem
    prob = _beam(2, (4, 5), 1, [(0, 1.0)], q=0.0)
    am = angular.AngularMesh(angular.uniform_paths(1), "lin")
    Ta = transport.Transport(prob, oadj.ReversedMesh(am))
    ctx = context_from_problem(prob, device=0)
    ctx.amgt_set_adjoint(1)
    f = torch.empty((Ta.nsdof, Ta.nadof), device="cuda", dtype=torch.float64)
    ctx.amgt_op_source(0, f)
    torch.cuda.synchronize()
    assert _rel(f.cpu().numpy(), Ta.source()) < 1e-14
    ctx.close()


def _mg(prob, nlevels, Nr):
    prob["mg"] = dict(nlevels=nlevels, Nr=Nr, nu_pre=1, nu_post=1, coarse_sweeps=10)
    return prob


@pytest.mark.parametrize("mode", ["f64", "mixed"])
def test_beam_solve_matches_oracle(mode):
    from paper_2010_04559_gb300 import (AMGT_MODE_F64, AMGT_MODE_MIXED, AMGT_PREC_MG,
                                        context_from_problem)
    prob = _mg(_beam(2, (9, 7), 2, [(0, 1.0)], N=8, g=0.9, ss=0.95), 3, [8, 4, 4])
    H = multigrid.Hierarchy(prob)
    T = H.levels[0]
    xo, _, _, rel = gmres.gmres(T.apply_A, T.source(), lambda v: H.vcycle(v), 1e-13, 20, 1000)
    assert rel < 1e-13
    ctx = context_from_problem(prob, device=0)
    md = AMGT_MODE_F64 if mode == "f64" else AMGT_MODE_MIXED
    tol = 1e-13 if mode == "f64" else 1e-11
    psi, phi, st, _ = ctx.amgt_solve(tol=tol, precond=AMGT_PREC_MG, mode=md)
    assert st.relres < tol
    assert _rel(psi, xo) < (1e-10 if mode == "f64" else 1e-6)
    assert _rel(phi, T.scalar_flux(xo)) < (1e-10 if mode == "f64" else 1e-6)
    ctx.close()


def test_beam_solve_on_a_band_refined_mesh_matches_oracle():
    """Beam along +x on the mesh refined about +x by the Sec. 5.4 bands
    (l_max = 3), 3-level multigrid over its coarsened meshes."""
    from paper_2010_04559_gb300 import AMGT_MODE_F64, AMGT_PREC_MG, context_from_problem
    prob = _mg(_beam(2, (6, 5), 0, [(0, 1.0)], N=6, g=0.9, ss=0.9), 3, [6, 3, 3])
    paths = angular.aniso_paths(3, (1.0, 0.0, 0.0))
    H = multigrid.Hierarchy(prob, paths)
    T = H.levels[0]
    xo, _, _, rel = gmres.gmres(T.apply_A, T.source(), lambda v: H.vcycle(v), 1e-13, 20, 1000)
    ctx = context_from_problem(prob, device=0, aniso=((1.0, 0.0, 0.0), 3))
    assert ctx.amgt_query_sizes(0) == (T.nsdof, T.nadof)
    psi, phi, st, _ = ctx.amgt_solve(tol=1e-13, precond=AMGT_PREC_MG, mode=AMGT_MODE_F64)
    assert st.relres < 1e-13
    assert _rel(psi, xo) < 1e-10
    ctx.close()


def test_forward_peaked_beam_workload_reduced_mixed_vs_fp64():
    """The beam workload (sigma_t = 5, sigma_s = 4.95, HG g = 0.98, beam over
    the low-x edge, 4-level multigrid) at 48^2 cells, level 3, order 24: the
    mixed solve to 1e-8 agrees with the FP64 solve to 1e-6, both balance the
    incident current, and the flux is mirror-symmetric about y = 1/2."""
    from paper_2010_04559_gb300 import (AMGT_MODE_F64, AMGT_MODE_MIXED, AMGT_PREC_MG,
                                        context_from_problem)
    n = 48
    prob = W.config5_beam(n=n, level=3, N=24, nlevels=4, Nr=8)
    ctx = context_from_problem(prob, device=0)
    p64, f64, st64, _ = ctx.amgt_solve(tol=1e-11, precond=AMGT_PREC_MG, mode=AMGT_MODE_F64)
    p32, f32, st32, _ = ctx.amgt_solve(tol=1e-8, precond=AMGT_PREC_MG, mode=AMGT_MODE_MIXED)
    assert st64.relres < 1e-11 and st32.relres < 1e-8
    assert _rel(p32, p64) < 1e-6
    # cell integrals of the scalar flux: symmetric about the beam's mid-line
    mu = np.full(4, 0.25 / n ** 2)
    avg = (f64.reshape(n * n, 4) @ mu).reshape(n, n)
    assert np.abs(avg - avg[::-1]).max() < 1e-9 * np.abs(avg).max()
    ctx.close()


def test_forward_peaked_beam_workload_full_size_mixed():
    """The full beam workload: 256^2 cells, uniform level 4 (2048 patches,
    6144 angular DOF), HG g = 0.98 at order 64, 4-level multigrid with coarse
    order 12 -- 1.61e9 unknowns.  The mixed solve reaches 1e-8 (FP64 true
    residual); the scalar flux is mirror-symmetric about y = 1/2 and larger
    at the beam edge than at the far edge."""
    from paper_2010_04559_gb300 import AMGT_MODE_MIXED, AMGT_PREC_MG, context_from_problem
    n = 256
    prob = W.config5_beam()
    stream = torch.cuda.Stream()
    ctx = context_from_problem(prob, device=0, stream=stream.cuda_stream)
    ns, na = ctx.amgt_query_sizes(0)
    assert (ns, na) == (4 * n * n, 6144)
    psi = torch.empty((ns, na), device="cuda", dtype=torch.float64)
    phi = torch.empty(ns, device="cuda", dtype=torch.float64)
    with torch.cuda.stream(stream):
        _, _, st, _ = ctx.amgt_solve(tol=1e-8, restart=8, precond=AMGT_PREC_MG,
                                     mode=AMGT_MODE_MIXED, psi=psi, phi=phi, device_ptrs=True)
    torch.cuda.synchronize()
    ctx.close()
    del psi
    assert st.relres < 1e-8
    avg = phi.cpu().numpy().reshape(n * n, 4).sum(axis=1).reshape(n, n)
    assert np.abs(avg - avg[::-1]).max() < 1e-7 * np.abs(avg).max()
    assert avg[:, 0].mean() > avg[:, -1].mean() > 0


# ------------------------------------------------ beams of any direction, part of a face
def _gbeam(dim, nc, level, faces, N=4, g=0.8, basis="lin", ss=0.8, q=0.0, seed=73):
    """faces: (face, (S, Omega_b[3], u0, u1, v0, v1)) for kind-3 beams."""
    rng = np.random.default_rng(seed)
    C = int(np.prod(nc))
    st = 1.0 + rng.random(C)
    bnd = [(0, 0.0)] * (2 * dim)
    for f, val in faces:
        bnd[f] = (3, tuple(val))
    return W.problem(dim, nc, st, ss * st, N, W.hg_moments(g, N), np.full(C, q), level,
                     basis=basis, boundary=bnd)


GSRC = [
    # inside a patch, cutting cells at both ends of the range
    (2, (5, 7), 1, "lin", [(0, (1.0, 0.8, 0.35, 0.2, 0.23, 0.61, 0, 0))], None),
    # on an edge of the patches (the x-y great circle), high-y face
    (2, (6, 4), 2, "const", [(3, (0.7, 0.3, -1.0, 0.0, 0.1, 0.95, 0, 0))], None),
    # at a level-1 vertex (six patches, unequal angles), 3D, two beams
    (3, (4, 3, 3), 2, "lin", [(4, (1.0, 0.0, 1.0, 1.0, 0.3, 0.7, 0.15, 0.52)),
                              (1, (0.5, -1.0, 0.2, 0.3, 0.0, 1.0, 0.0, 1.0))], None),
    # the cube's boundary source of Sec. 5.4: along +z on a central square of
    # the low-z face, z-pole band-refined mesh
    (3, (4, 4, 3), None, "lin", [(4, (1.0, 0.0, 0.0, 1.0, 0.375, 0.625, 0.375, 0.625))],
     ((0.0, 0.0, 1.0), 3)),
]


@pytest.mark.parametrize("dim,nc,level,basis,faces,aniso", GSRC,
                         ids=["inside", "edge", "vertex3d", "zpole-square"])
def test_general_beam_source_matches_oracle(dim, nc, level, basis, faces, aniso):
    from paper_2010_04559_gb300 import context_from_problem
    prob = _gbeam(dim, nc, level if level is not None else 0, faces, basis=basis, q=0.2)
    paths = (angular.uniform_paths(level) if aniso is None
             else angular.aniso_paths(aniso[1], aniso[0]))
    T = transport.Transport(prob, angular.AngularMesh(paths, basis))
    ctx = context_from_problem(prob, device=0, aniso=aniso)
    assert ctx.amgt_query_sizes(0) == (T.nsdof, T.nadof)
    ref = T.source()
    for td, tol in ((torch.float64, 1e-13), (torch.float32, 1e-6)):
        f = torch.empty((T.nsdof, T.nadof), device="cuda", dtype=td)
        ctx.amgt_op_source(0, f)
        torch.cuda.synchronize()
        assert _rel(f.double().cpu().numpy(), ref) < tol
    ctx.close()


def test_general_beam_arguments_are_checked():
    from paper_2010_04559_gb300 import AMGT_ERR_ARG, AmgtError, context_from_problem
    prob = _beam(2, (3, 3), 1, [(0, 1.0)])
    ctx = context_from_problem(prob, device=0)
    for val in ((1.0, -1.0, 0.0, 0.0, 0.0, 1.0, 0, 0),     # outward on the low-x face
                (1.0, 0.0, 0.0, 0.0, 0.0, 1.0, 0, 0),      # zero direction
                (1.0, 1.0, 0.0, 0.0, 0.6, 0.4, 0, 0),      # empty range
                (1.0, 1.0, np.nan, 0.0, 0.0, 1.0, 0, 0)):  # not finite
        with pytest.raises(AmgtError) as e:
            ctx.amgt_set_boundary(0, 3, val)
        assert e.value.code == AMGT_ERR_ARG
    ctx.close()


@pytest.mark.parametrize("mode", ["f64", "mixed"])
def test_cube_partial_face_beam_solve_on_a_zpole_mesh_matches_oracle(mode):
    """Sec. 5.4's second test problem, reduced: a cube with a pencil beam
    along +z entering through the square 0.375 < x, y < 0.625 of its low-z
    face, the angular mesh refined about the z pole (l_max = 3, bands of
    Sec. 5.4), 3-level multigrid over its coarsened meshes; FP64 and mixed
    solves against the oracle's."""
    from paper_2010_04559_gb300 import (AMGT_MODE_F64, AMGT_MODE_MIXED, AMGT_PREC_MG,
                                        context_from_problem)
    beam = (1.0, 0.0, 0.0, 1.0, 0.375, 0.625, 0.375, 0.625)
    prob = _mg(_gbeam(3, (4, 4, 4), 0, [(4, beam)], N=6, g=0.9, ss=0.9), 3, [6, 3, 3])
    paths = angular.aniso_paths(3, (0.0, 0.0, 1.0))
    H = multigrid.Hierarchy(prob, paths)
    T = H.levels[0]
    xo, _, _, rel = gmres.gmres(T.apply_A, T.source(), lambda v: H.vcycle(v), 1e-13, 20, 1000)
    assert rel < 1e-13
    ctx = context_from_problem(prob, device=0, aniso=((0.0, 0.0, 1.0), 3))
    md = AMGT_MODE_F64 if mode == "f64" else AMGT_MODE_MIXED
    tol = 1e-13 if mode == "f64" else 1e-11
    psi, phi, st, _ = ctx.amgt_solve(tol=tol, precond=AMGT_PREC_MG, mode=md)
    assert st.relres < tol
    assert _rel(psi, xo) < (1e-10 if mode == "f64" else 1e-6)
    assert _rel(phi, T.scalar_flux(xo)) < (1e-10 if mode == "f64" else 1e-6)
    ctx.close()
