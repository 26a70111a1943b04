"""Degenerate cases of the method on the GPU against the oracle: a zero
right-hand side in every solve mode (psi = 0 is the exact solution),
isotropic scattering (N = 0: one moment per node, S_f = w w^T / (4 pi)), and
meshes one cell wide or one cell high in 2D and 3D (sweeps with no x or no y
neighbour, one row of cells for the row-pipelined Gauss-Seidel, wavefronts
one cell long)."""
import numpy as np
import pytest

import workloads as W
from oracle import gmres, multigrid

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
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _ctx(prob):
    from paper_2010_04559_gb300 import context_from_problem
    return context_from_problem(prob, device=0)


def _dev(x, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def _host(t):
    torch.cuda.synchronize()
    return t.detach().double().cpu().numpy()


def _mg(prob, Nr, sweeps=4):
    prob["mg"] = dict(nlevels=len(Nr), Nr=list(Nr), nu_pre=1, nu_post=1, coarse_sweeps=sweeps)
    return prob


def _modes(mode, precond):
    from paper_2010_04559_gb300 import (AMGT_MODE_F64, AMGT_MODE_MIXED, AMGT_PREC_MG,
                                        AMGT_PREC_SWEEP)
    return ((AMGT_MODE_F64 if mode == "f64" else AMGT_MODE_MIXED),
            (AMGT_PREC_SWEEP if precond == "sweep" else AMGT_PREC_MG))


@pytest.mark.parametrize("precond", ["sweep", "mg"])
@pytest.mark.parametrize("krylov", [0, 1], ids=["gmres", "bicgstab"])
@pytest.mark.parametrize("mode", ["f64", "mixed"])
def test_zero_right_hand_side_in_every_mode(mode, krylov, precond):
    """q = 0 and vacuum boundaries: every mode returns psi = 0 with status
    OK, no iteration and relres 0, also from a non-zero initial guess."""
    prob = _mg(W.random_problem(2, (5, 4), 2, 4, 71), [4, 2])
    prob["q"] = np.zeros_like(prob["q"])
    ctx = _ctx(prob)
    md, pc = _modes(mode, precond)
    psi, phi, st, rc = ctx.amgt_solve(tol=1e-10, precond=pc, mode=md, krylov=krylov)
    assert rc == 0 and st.iterations == 0 and st.relres == 0.0
    assert not psi.any() and not phi.any()
    x0 = W.random_vector(psi.shape, 72)
    psi, phi, st, rc = ctx.amgt_solve(tol=1e-10, precond=pc, mode=md, krylov=krylov, x0=x0)
    assert rc == 0 and st.iterations == 0 and not psi.any() and not phi.any()
    ctx.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_isotropic_scattering_operators(dtype):
    """N = 0 on every level: the scatter (also in BF16 on the tensor cores),
    A, the smoother, the coarse Gauss-Seidel and a V-cycle against the
    oracle."""
    prob = _mg(W.random_problem(2, (6, 5), 2, 0, 73), [0, 0, 0], sweeps=3)
    H = multigrid.Hierarchy(prob)
    T0, Tc = H.levels[0], H.levels[-1]
    ctx = _ctx(prob)
    td = torch.float64 if dtype == "f64" else torch.float32
    tol = 1e-12 if dtype == "f64" else 2e-5
    x = W.random_vector((T0.nsdof, T0.nadof), 74)
    y = torch.empty((T0.nsdof, T0.nadof), device="cuda", dtype=td)
    ctx.amgt_op_scatter(0, _dev(x, td), y)
    assert _rel(_host(y), T0.scatter(x)) < tol
    ctx.amgt_op_apply_A(0, _dev(x, td), y)
    assert _rel(_host(y), T0.apply_A(x)) < tol
    if dtype == "f32":
        yb = torch.empty_like(y)
        ctx.amgt_op_scatter(0, _dev(x, td), yb, tc=True)
        assert _rel(_host(yb), T0.scatter(x)) < 1e-2
    f = W.random_vector((T0.nsdof, T0.nadof), 75)
    phi0 = W.random_vector((T0.nsdof, T0.nadof), 76)
    ph = _dev(phi0, td)
    ctx.amgt_op_smooth(0, 2, _dev(f, td), ph)
    assert _rel(_host(ph), H.smooth(phi0, f, 0, 2)) < tol
    fc = W.random_vector((Tc.nsdof, Tc.nadof), 77)
    pc0 = W.random_vector((Tc.nsdof, Tc.nadof), 78)
    pc = _dev(pc0, td)
    ctx.amgt_op_coarse_gs(3, _dev(fc, td), pc)
    assert _rel(_host(pc), multigrid.coarse_gs(Tc, fc, pc0, 3)) < tol * 10
    out = torch.empty_like(ph)
    ctx.amgt_op_vcycle(_dev(f, td), out)
    assert _rel(_host(out), H.vcycle(f)) < tol * 10
    ctx.close()


@pytest.mark.parametrize("mode", ["f64", "mixed"])
def test_isotropic_scattering_solve(mode):
    """N = 0 with isotropic inflow: the multigrid-preconditioned solve
    against the oracle's GMRES solution."""
    prob = _mg(W.random_problem(2, (8, 7), 2, 0, 79, inflow=0.2), [0, 0, 0], sweeps=10)
    T = multigrid.Hierarchy(prob).levels[0]
    xo, _, _, rel = gmres.gmres(T.apply_A, T.source(), T.sweep, 1e-13, 20, 1000)
    assert rel < 1e-13
    ctx = _ctx(prob)
    md, pc = _modes(mode, "mg")
    psi, phi, st, rc = ctx.amgt_solve(tol=1e-12, precond=pc, mode=md, inner_tol=1e-4)
    assert st.relres < 1e-12
    assert _rel(psi, xo) < (1e-10 if mode == "f64" else 1e-6)
    assert _rel(phi, T.scalar_flux(xo)) < (1e-10 if mode == "f64" else 1e-6)
    ctx.close()


THIN = [(2, (1, 9), 2), (2, (9, 1), 2), (2, (1, 1), 2), (3, (1, 1, 6), 1), (3, (5, 1, 1), 1),
        (3, (1, 4, 1), 1)]
THIN_IDS = [f"{d}d-{'x'.join(map(str, n))}" for d, n, _ in THIN]


@pytest.mark.parametrize("dim,nc,level", THIN, ids=THIN_IDS)
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_one_cell_wide_meshes(dim, nc, level, dtype):
    """Every sweep kernel of the dimension, L x, the coarse Gauss-Seidel and
    a V-cycle against the oracle on meshes one cell wide, with inflow on
    every face."""
    from paper_2010_04559_gb300 import AMGT_TUNE_SWEEP_KERNEL
    prob = _mg(W.random_problem(dim, nc, level, 4, 80, inflow=0.3), [4, 2])
    H = multigrid.Hierarchy(prob)
    T0, Tc = H.levels[0], H.levels[-1]
    ctx = _ctx(prob)
    td = torch.float64 if dtype == "f64" else torch.float32
    tol = 1e-12 if dtype == "f64" else 2e-5
    b = W.random_vector((T0.nsdof, T0.nadof), 81)
    ref = T0.sweep(b)
    y = torch.empty((T0.nsdof, T0.nadof), device="cuda", dtype=td)
    for kernel in (1, 2):
        ctx.amgt_set_tuning(AMGT_TUNE_SWEEP_KERNEL, kernel)
        ctx.amgt_op_sweep(0, _dev(b, td), y)
        ctx.amgt_sync()
        assert _rel(_host(y), ref) < tol, kernel
    ctx.amgt_set_tuning(AMGT_TUNE_SWEEP_KERNEL, 0)
    ctx.amgt_op_apply_L(0, _dev(b, td), y)
    assert _rel(_host(y), T0.apply_L(b)) < tol
    fc = W.random_vector((Tc.nsdof, Tc.nadof), 82)
    pc0 = W.random_vector((Tc.nsdof, Tc.nadof), 83)
    pc = _dev(pc0, td)
    ctx.amgt_op_coarse_gs(3, _dev(fc, td), pc)
    ctx.amgt_sync()
    assert _rel(_host(pc), multigrid.coarse_gs(Tc, fc, pc0, 3)) < tol * 10
    out = torch.empty_like(y)
    ctx.amgt_op_vcycle(_dev(b, td), out)
    assert _rel(_host(out), H.vcycle(b)) < tol * 10
    ctx.close()


@pytest.mark.parametrize("dim,nc", [(2, (1, 12)), (2, (12, 1)), (3, (1, 1, 7))],
                         ids=["2d-1x12", "2d-12x1", "3d-1x1x7"])
def test_one_cell_wide_solve(dim, nc):
    """FP64 and mixed multigrid-preconditioned solves on one-cell-wide meshes
    against the oracle's solution."""
    from paper_2010_04559_gb300 import AMGT_MODE_F64, AMGT_MODE_MIXED, AMGT_PREC_MG
    level = 2 if dim == 2 else 1
    prob = _mg(W.random_problem(dim, nc, level, 4, 84, inflow=0.2), [4, 2], sweeps=10)
    T = multigrid.Hierarchy(prob).levels[0]
    xo, _, _, rel = gmres.gmres(T.apply_A, T.source(), T.sweep, 1e-13, 20, 1000)
    ctx = _ctx(prob)
    psi, _, st, _ = ctx.amgt_solve(tol=1e-12, precond=AMGT_PREC_MG, mode=AMGT_MODE_F64)
    assert st.relres < 1e-12 and _rel(psi, xo) < 1e-10
    psi, _, st, _ = ctx.amgt_solve(tol=1e-12, precond=AMGT_PREC_MG, mode=AMGT_MODE_MIXED,
                                   inner_tol=1e-4)
    assert st.relres < 1e-12 and _rel(psi, xo) < 1e-6
    ctx.close()


@pytest.mark.parametrize("krylov", [0, 1], ids=["gmres", "bicgstab"])
@pytest.mark.parametrize("mode", ["f64", "mixed"])
def test_converged_initial_guess_returns_at_once(mode, krylov):
    """An initial guess that already meets the tolerance (the oracle's
    solution to 1e-13) is returned unchanged after one residual, with no
    iteration."""
    prob = _mg(W.random_problem(2, (6, 5), 1, 4, 85, inflow=0.3), [4, 2], sweeps=10)
    T = multigrid.Hierarchy(prob).levels[0]
    xo, _, _, rel = gmres.gmres(T.apply_A, T.source(), T.sweep, 1e-13, 20, 1000)
    assert rel < 1e-13
    ctx = _ctx(prob)
    md, pc = _modes(mode, "mg")
    psi, _, st, rc = ctx.amgt_solve(tol=1e-9, precond=pc, mode=md, krylov=krylov, x0=xo)
    assert rc == 0 and st.iterations == 0 and st.relres < 1e-9
    assert np.array_equal(psi, xo)
    ctx.close()


@pytest.mark.parametrize("m", [1, 2, 3])
def test_short_gmres_restarts(m):
    """GMRES(m) with m = 1, 2, 3 (one- to three-column Hessenberg systems,
    a restart after every few directions) reaches the oracle's solution."""
    from paper_2010_04559_gb300 import AMGT_MODE_F64, AMGT_PREC_SWEEP
    prob = W.random_problem(2, (5, 4), 1, 4, 86, inflow=0.2)
    T = multigrid.Hierarchy(_mg(dict(prob), [4])).levels[0]
    xo, _, _, rel = gmres.gmres(T.apply_A, T.source(), T.sweep, 1e-13, 20, 1000)
    ctx = _ctx(prob)
    psi, _, st, rc = ctx.amgt_solve(tol=1e-12, restart=m, maxit=5000, precond=AMGT_PREC_SWEEP,
                                    mode=AMGT_MODE_F64)
    assert st.relres < 1e-12 and _rel(psi, xo) < 1e-10
    assert st.outer_iterations >= st.iterations // m
    ctx.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_one_level_hierarchy(dtype):
    """nlevels = 1: the cycle is the coarse Gauss-Seidel on the finest mesh
    at the full order, from zero (Fig. lmg at its coarsest level); the
    multigrid-preconditioned FP64 solve reaches the oracle's solution."""
    from paper_2010_04559_gb300 import AMGT_MODE_F64, AMGT_PREC_MG
    prob = _mg(W.random_problem(2, (6, 5), 1, 4, 87, inflow=0.2), [4], sweeps=3)
    H = multigrid.Hierarchy(prob)
    T = H.levels[0]
    ctx = _ctx(prob)
    td = torch.float64 if dtype == "f64" else torch.float32
    tol = 1e-11 if dtype == "f64" else 2e-4
    f = W.random_vector((T.nsdof, T.nadof), 88)
    out = torch.empty((T.nsdof, T.nadof), device="cuda", dtype=td)
    ctx.amgt_op_vcycle(_dev(f, td), out)
    assert _rel(_host(out), H.vcycle(f)) < tol
    if dtype == "f64":
        xo, _, _, rel = gmres.gmres(T.apply_A, T.source(), T.sweep, 1e-13, 20, 1000)
        psi, _, st, _ = ctx.amgt_solve(tol=1e-12, precond=AMGT_PREC_MG, mode=AMGT_MODE_F64)
        assert st.relres < 1e-12 and _rel(psi, xo) < 1e-10
    ctx.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_zero_coarse_sweeps(dtype):
    """coarse_sweeps = 0: the coarse Gauss-Seidel leaves phi as it is and the
    cycle has no coarse correction (smoothing only), as in the oracle."""
    prob = _mg(W.random_problem(2, (6, 5), 2, 6, 89), [6, 3], sweeps=0)
    H = multigrid.Hierarchy(prob)
    T0, Tc = H.levels[0], H.levels[-1]
    ctx = _ctx(prob)
    td = torch.float64 if dtype == "f64" else torch.float32
    tol = 1e-11 if dtype == "f64" else 2e-4
    pc0 = W.random_vector((Tc.nsdof, Tc.nadof), 90)
    pc = _dev(pc0, td)
    ctx.amgt_op_coarse_gs(0, _dev(W.random_vector((Tc.nsdof, Tc.nadof), 91), td), pc)
    assert np.array_equal(_host(pc), _host(_dev(pc0, td)))
    f = W.random_vector((T0.nsdof, T0.nadof), 92)
    out = torch.empty((T0.nsdof, T0.nadof), device="cuda", dtype=td)
    ctx.amgt_op_vcycle(_dev(f, td), out)
    assert _rel(_host(out), H.vcycle(f)) < tol
    ctx.close()


@pytest.mark.parametrize("mode", ["f64", "mixed"])
def test_warm_start_in_place(mode):
    """x0 = psi on the device (resuming a solve in place): a solved psi is
    kept as it is with no iteration, and a solve to a tighter tolerance from
    it reaches the oracle's solution."""
    prob = _mg(W.random_problem(2, (6, 5), 1, 4, 93, inflow=0.3), [4, 2], sweeps=10)
    T = multigrid.Hierarchy(prob).levels[0]
    xo, _, _, _ = gmres.gmres(T.apply_A, T.source(), T.sweep, 1e-13, 20, 1000)
    ctx = _ctx(prob)
    md, pc = _modes(mode, "mg")
    ns, na = ctx.amgt_query_sizes(0)
    psi = torch.empty((ns, na), device="cuda", dtype=torch.float64)
    _, _, st, _ = ctx.amgt_solve(tol=1e-6, precond=pc, mode=md, psi=psi, device_ptrs=True)
    first = _host(psi).copy()
    _, _, st, rc = ctx.amgt_solve(tol=1e-6, precond=pc, mode=md, x0=psi, psi=psi,
                                  device_ptrs=True)
    assert rc == 0 and st.iterations == 0 and np.array_equal(_host(psi), first)
    tight = 1e-13 if mode == "f64" else 1e-12
    _, _, st, _ = ctx.amgt_solve(tol=tight, precond=pc, mode=md, x0=psi, psi=psi,
                                 device_ptrs=True, inner_tol=1e-4)
    assert st.relres < tight
    assert _rel(_host(psi), xo) < (1e-10 if mode == "f64" else 1e-6)
    ctx.close()
