"""GPU parity of every hot-path operator against the FP64 CPU oracle, through
the C ABI (include/amgt.h) on seeded inputs.

Tolerances (relative L2 over the compared entries):
  FP64 operators            1e-12  (deterministic linear maps; rounding only)
  FP64 solves               1e-10  (both sides solved to relres 1e-13)
  FP32 operators            2e-5   (unit roundoff 6e-8 times sum lengths <= a few 1e3)
  BF16 tensor-core scatter  1e-2   (inputs rounded to 8-bit mantissas, FP32 sums)
  FP16 three-product scatter 2e-5 (hi + lo parts keep ~22 bits, FP32 sums)
  mixed-precision solve     1e-6   (after FP64 iterative refinement to relres 1e-12)
"""
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


def _oracle(prob, level=None, Nscat=None):
    lev = prob["level"] if level is None else level
    am = angular.AngularMesh(angular.uniform_paths(lev), prob["basis"])
    return transport.Transport(prob, am, Nscat)


# (dim, ncell, level, basis): spans several wavefront levels, ragged sizes,
# Const and Lin, 2D and 3D
CASES = [
    (2, (7, 5), 1, "lin"),
    (2, (9, 4), 2, "const"),
    (2, (4, 6), 0, "lin"),
    (3, (3, 4, 2), 1, "lin"),
    (3, (2, 3, 3), 0, "const"),
]
IDS = [f"{d}d-{'x'.join(map(str, n))}-l{l}-{b}" for d, n, l, b in CASES]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_L_apply_with_many_patches(dtype):
    """L x and (L - S) x at angular level 3 (512 Lin patches: grid-stride
    items over many patch blocks per cell), per-cell cross sections and
    inflow, against the oracle."""
    prob = W.random_problem(2, (6, 5), 3, 4, 33, inflow=0.4)
    T = _oracle(prob)
    ctx = _ctx(prob)
    td = torch.float64 if dtype == "f64" else torch.float32
    tol = 1e-12 if dtype == "f64" else 2e-5
    x = W.random_vector((T.nsdof, T.nadof), 34)
    xd = _dev(x, td)
    y = torch.empty_like(xd)
    ctx.amgt_op_apply_L(0, xd, y)
    assert _rel(_host(y), T.apply_L(x)) < tol
    ctx.amgt_op_apply_A(0, xd, y)
    assert _rel(_host(y), T.apply_A(x)) < tol
    ctx.close()


@pytest.mark.parametrize("dim,nc,level,basis", CASES, ids=IDS)
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_transport_operators(dim, nc, level, basis, dtype):
    prob = W.random_problem(dim, nc, level, 6, 31, basis=basis, inflow=0.4)
    T = _oracle(prob)
    ctx = _ctx(prob)
    td = torch.float64 if dtype == "f64" else torch.float32
    tol = 1e-12 if dtype == "f64" else 2e-5
    x = W.random_vector((T.nsdof, T.nadof), 32)
    xd = _dev(x, td)
    y = torch.empty_like(xd)
    # sweep L^-1
    ctx.amgt_op_sweep(0, xd, y)
    assert _rel(_host(y), T.sweep(x)) < tol
    # L x
    ctx.amgt_op_apply_L(0, xd, y)
    assert _rel(_host(y), T.apply_L(x)) < tol
    # S x
    ctx.amgt_op_scatter(0, xd, y)
    assert _rel(_host(y), T.scatter(x)) < tol
    # (L - S) x
    ctx.amgt_op_apply_A(0, xd, y)
    assert _rel(_host(y), T.apply_A(x)) < tol
    # source f
    f = torch.empty_like(xd)
    ctx.amgt_op_source(0, f)
    assert _rel(_host(f), T.source()) < tol
    # scalar flux
    ph = torch.empty(T.nsdof, device="cuda", dtype=td)
    ctx.amgt_op_scalar_flux(0, xd, ph)
    assert _rel(_host(ph), T.scalar_flux(x)) < tol
    ctx.close()


def _mg_problem(dim, nc, level, basis, nlev, Nr, sweeps=4, seed=41):
    prob = W.random_problem(dim, nc, level, 8, seed, basis=basis, g=0.85)
    prob["mg"] = dict(nlevels=nlev, Nr=Nr, nu_pre=1, nu_post=1, coarse_sweeps=sweeps)
    if nc == (12, 10):
        # two materials in 4x4-cell tiles (the layout the shared-memory tables serve)
        mat = np.array([((ix // 4) + (iy // 4)) % 2 for iy in range(10) for ix in range(12)])
        prob["sigma_t"] = np.where(mat == 0, 1.0, 6.0)
        prob["sigma_s"] = np.where(mat == 0, 0.5, 5.7)
    return prob


MG_CASES = [
    (2, (6, 5), 2, "lin", 3, [8, 4, 3]),
    (2, (12, 10), 2, "lin", 3, [8, 5, 4]),
    (2, (5, 7), 2, "const", 2, [8, 5]),
    (3, (3, 2, 3), 1, "lin", 2, [8, 4]),
]
MG_IDS = [f"{d}d-{'x'.join(map(str, n))}-l{l}-{b}-{k}lev" for d, n, l, b, k, _ in MG_CASES]


@pytest.mark.parametrize("dim,nc,level,basis,nlev,Nr", MG_CASES, ids=MG_IDS)
@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("gs_kernel", [1, 2, 3, 4, 5, 6],
                         ids=["gs-per-patch", "gs-warp", "gs-group", "gs-grid", "gs-tc", "gs-rows"])
def test_multigrid_operators(dim, nc, level, basis, nlev, Nr, dtype, gs_kernel):
    prob = _mg_problem(dim, nc, level, basis, nlev, Nr)
    H = multigrid.Hierarchy(prob)
    ctx = _ctx(prob)
    ctx.amgt_set_tuning(1, gs_kernel)
    td = torch.float64 if dtype == "f64" else torch.float32
    tol = 1e-12 if dtype == "f64" else 2e-5
    T0, T1 = H.levels[0], H.levels[1]
    # level sizes agree
    assert ctx.amgt_query_sizes(0) == (T0.nsdof, T0.nadof)
    assert ctx.amgt_query_sizes(1) == (T1.nsdof, T1.nadof)
    r = W.random_vector((T0.nsdof, T0.nadof), 42)
    rc = torch.empty((T1.nsdof, T1.nadof), device="cuda", dtype=td)
    ctx.amgt_op_restrict(0, _dev(r, td), rc)
    assert _rel(_host(rc), H.restrict(r, 0)) < tol
    xc = W.random_vector((T1.nsdof, T1.nadof), 43)
    xf = _dev(r, td)
    ctx.amgt_op_prolong(0, _dev(xc, td), xf)
    assert _rel(_host(xf), r + H.prolong(xc, 0)) < tol
    # coarse-level scatter with the reduced order
    y1 = torch.empty_like(rc)
    ctx.amgt_op_scatter(1, _dev(xc, td), y1)
    assert _rel(_host(y1), T1.scatter(xc)) < tol
    # smoother
    f = W.random_vector((T0.nsdof, T0.nadof), 44)
    phi0 = W.random_vector((T0.nsdof, T0.nadof), 45)
    ph = _dev(phi0, td)
    ctx.amgt_op_smooth(0, 2, _dev(f, td), ph)
    assert _rel(_host(ph), H.smooth(phi0, f, 0, 2)) < tol
    # coarse Gauss-Seidel on the coarsest level
    Tc = H.levels[-1]
    fc = W.random_vector((Tc.nsdof, Tc.nadof), 46)
    pc0 = W.random_vector((Tc.nsdof, Tc.nadof), 47)
    pc = _dev(pc0, td)
    ctx.amgt_op_coarse_gs(3, _dev(fc, td), pc)
    assert _rel(_host(pc), multigrid.coarse_gs(Tc, fc, pc0, 3)) < tol * 10
    # one V-cycle
    out = torch.empty_like(ph)
    ctx.amgt_op_vcycle(_dev(f, td), out)
    assert _rel(_host(out), H.vcycle(f)) < tol * 10
    ctx.close()


@pytest.mark.parametrize("nu", [(1, 1), (2, 1), (3, 0)], ids=["V11", "V21", "V30"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_vcycle_smoothing_counts(nu, dtype):
    """One V-cycle against the oracle with one, two and three pre-smoothing
    sweeps: the residual after pre-smoothing is formed as S phi + f - t with
    t the last sweep's right-hand side (the sweep inverts L), which must
    equal the oracle's f - A phi."""
    prob = _mg_problem(2, (6, 5), 2, "lin", 3, [8, 4, 3])
    prob["mg"]["nu_pre"], prob["mg"]["nu_post"] = nu
    H = multigrid.Hierarchy(prob)
    ctx = _ctx(prob)
    td = torch.float64 if dtype == "f64" else torch.float32
    tol = 1e-11 if dtype == "f64" else 2e-4
    T0 = H.levels[0]
    f = W.random_vector((T0.nsdof, T0.nadof), 48)
    out = torch.empty((T0.nsdof, T0.nadof), device="cuda", dtype=td)
    ctx.amgt_op_vcycle(_dev(f, td), out)
    assert _rel(_host(out), H.vcycle(f)) < tol
    ctx.close()


@pytest.mark.parametrize("precond", ["sweep", "mg"])
def test_fp64_solve_matches_oracle(precond):
    from paper_2010_04559_gb300 import AMGT_MODE_F64, AMGT_PREC_MG, AMGT_PREC_SWEEP
    prob = _mg_problem(2, (8, 7), 2, "lin", 3, [8, 4, 4], sweeps=10, seed=51)
    prob["boundary"] = [(1, 0.3), (0, 0.0), (1, 0.1), (0, 0.0)]
    H = multigrid.Hierarchy(prob)
    T = H.levels[0]
    f = T.source()
    xo, its, _, rel = gmres.gmres(T.apply_A, f, T.sweep, 1e-13, 20, 1000)
    ctx = _ctx(prob)
    pc = AMGT_PREC_SWEEP if precond == "sweep" else AMGT_PREC_MG
    psi, phi, st, rc = ctx.amgt_solve(tol=1e-13, restart=20, maxit=1000, precond=pc,
                                      mode=AMGT_MODE_F64)
    assert st.relres < 1e-13
    assert _rel(psi, xo) < 1e-10
    assert _rel(phi, T.scalar_flux(xo)) < 1e-10
    if precond == "mg":
        _, its_mg, _, _ = gmres.gmres(T.apply_A, f, lambda v: H.vcycle(v), 1e-13, 20, 1000)
        # same preconditioner and same GMRES: iteration counts agree closely
        assert abs(st.iterations - its_mg) <= 1
    ctx.close()


def test_mixed_solve_matches_oracle():
    from paper_2010_04559_gb300 import AMGT_MODE_MIXED, AMGT_PREC_MG
    prob = _mg_problem(2, (8, 8), 2, "lin", 3, [8, 4, 4], sweeps=10, seed=52)
    H = multigrid.Hierarchy(prob)
    T = H.levels[0]
    xo, *_ = gmres.gmres(T.apply_A, T.source(), T.sweep, 1e-13, 20, 1000)
    ctx = _ctx(prob)
    psi, phi, st, rc = ctx.amgt_solve(tol=1e-12, restart=20, maxit=1000, precond=AMGT_PREC_MG,
                                      mode=AMGT_MODE_MIXED, inner_tol=1e-4)
    assert st.relres < 1e-12
    assert _rel(psi, xo) < 1e-6
    ctx.close()


def test_fp64_coarse_solve_in_the_fp32_cycle():
    """AMGT_TUNE_COARSE_F64: the FP32 V-cycle with its coarsest Gauss-Seidel
    solve in FP64 against the oracle's cycle, and the mixed solve with it
    against the oracle's solution."""
    from paper_2010_04559_gb300 import AMGT_MODE_MIXED, AMGT_PREC_MG, AMGT_TUNE_COARSE_F64
    prob = _mg_problem(2, (8, 8), 2, "lin", 3, [8, 4, 4], sweeps=10, seed=53)
    H = multigrid.Hierarchy(prob)
    T = H.levels[0]
    ctx = _ctx(prob)
    ctx.amgt_set_tuning(AMGT_TUNE_COARSE_F64, 1)
    f = W.random_vector((T.nsdof, T.nadof), 54)
    out = torch.empty((T.nsdof, T.nadof), device="cuda", dtype=torch.float32)
    ctx.amgt_op_vcycle(_dev(f, torch.float32), out)
    assert _rel(_host(out), H.vcycle(f)) < 2e-4
    xo, *_ = gmres.gmres(T.apply_A, T.source(), T.sweep, 1e-13, 20, 1000)
    psi, phi, st, rc = ctx.amgt_solve(tol=1e-12, restart=20, maxit=1000, precond=AMGT_PREC_MG,
                                      mode=AMGT_MODE_MIXED, inner_tol=1e-4)
    assert st.relres < 1e-12
    assert _rel(psi, xo) < 1e-6
    ctx.close()


def test_config1_square16_fp64_gmres20():
    """The 16x16 / level-1 / HG g = 0.8 order-8 problem, FP64 GMRES(20) to 1e-8,
    sweep preconditioner; compared with the oracle solved to 1e-12."""
    from paper_2010_04559_gb300 import AMGT_MODE_F64, AMGT_PREC_SWEEP
    prob = W.config1_square16()
    T = _oracle(prob)
    xo, *_ = gmres.gmres(T.apply_A, T.source(), T.sweep, 1e-12, 20, 2000)
    ctx = _ctx(prob)
    psi, phi, st, rc = ctx.amgt_solve(tol=1e-8, restart=20, maxit=2000,
                                      precond=AMGT_PREC_SWEEP, mode=AMGT_MODE_F64)
    assert st.relres < 1e-8
    # ||x - xo|| <= kappa * 1e-8 in principle; the bound observed is far smaller
    assert _rel(psi, xo) < 1e-6
    # scalar flux is positive inside the source region
    assert phi.min() > 0
    ctx.close()


def test_pure_absorber_single_iteration():
    from paper_2010_04559_gb300 import AMGT_MODE_F64, AMGT_PREC_SWEEP
    prob = W.random_problem(2, (5, 5), 1, 4, 61)
    prob["sigma_s"] = np.zeros_like(prob["sigma_s"])
    ctx = _ctx(prob)
    psi, phi, st, rc = ctx.amgt_solve(tol=1e-12, precond=AMGT_PREC_SWEEP, mode=AMGT_MODE_F64)
    assert st.iterations == 1 and st.relres < 1e-12
    ctx.close()


def test_infinite_medium_on_gpu():
    from paper_2010_04559_gb300 import AMGT_MODE_F64, AMGT_PREC_SWEEP
    C = 6 * 5
    st_, ss_, q = 3.0, 2.4, 1.0
    psi_inf = q / (4 * np.pi) / (st_ - ss_)
    prob = W.problem(2, (6, 5), np.full(C, st_), np.full(C, ss_), 6, W.hg_moments(0.8, 6),
                     np.full(C, q), 2, boundary=[(1, psi_inf)] * 4)
    ctx = _ctx(prob)
    psi, phi, st, rc = ctx.amgt_solve(tol=1e-13, precond=AMGT_PREC_SWEEP, mode=AMGT_MODE_F64)
    assert np.abs(psi - psi_inf).max() / psi_inf < 1e-10
    assert np.abs(phi - q / (st_ - ss_)).max() < 1e-9
    ctx.close()


def test_empty_source_gives_zero():
    from paper_2010_04559_gb300 import AMGT_MODE_F64, AMGT_PREC_SWEEP
    prob = W.random_problem(2, (3, 3), 1, 4, 62)
    prob["q"] = np.zeros_like(prob["q"])
    ctx = _ctx(prob)
    psi, phi, st, rc = ctx.amgt_solve(tol=1e-10, precond=AMGT_PREC_SWEEP, mode=AMGT_MODE_F64)
    assert np.abs(psi).max() == 0.0 and st.iterations == 0
    ctx.close()


def test_single_cell_mesh():
    prob = W.random_problem(2, (1, 1), 1, 4, 63, inflow=0.5)
    T = _oracle(prob)
    ctx = _ctx(prob)
    x = W.random_vector((T.nsdof, T.nadof), 64)
    y = torch.empty((T.nsdof, T.nadof), device="cuda", dtype=torch.float64)
    ctx.amgt_op_sweep(0, _dev(x), y)
    assert _rel(_host(y), T.sweep(x)) < 1e-12
    ctx.close()


def test_bad_arguments_raise():
    from paper_2010_04559_gb300 import AmgtError
    prob = W.random_problem(2, (3, 3), 1, 4, 65)
    ctx = _ctx(prob)
    x = torch.zeros((36 * 1, 96), device="cuda", dtype=torch.float64)
    with pytest.raises(AmgtError):
        ctx.amgt_op_sweep(0, x, x)          # aliasing in/out
    with pytest.raises(AmgtError):
        ctx.amgt_op_restrict(0, x, x)       # single-level hierarchy
    with pytest.raises(AmgtError):
        ctx.amgt_set_angular_uniform(1, 12)
    ctx.close()


@pytest.mark.parametrize("group", [1, 2, 4], ids=["G1", "G2", "G4"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_row_sweep_every_group_size(group, dtype):
    """The 2D row-pipelined sweep with 1, 2 and 4 patches per block on a
    32 x 32 mesh (block sizes that are multiples of 32 threads and several
    copy chunks per thread), sampled on two patches of every direction."""
    prob = W.random_problem(2, (32, 32), 1, 4, 33, inflow=0.2)
    T = _oracle(prob)
    ctx = _ctx(prob)
    ctx.amgt_set_tuning(2, group)
    td = torch.float64 if dtype == "f64" else torch.float32
    tol = 1e-12 if dtype == "f64" else 2e-5
    x = W.random_vector((T.nsdof, T.nadof), 34)
    y = torch.empty((T.nsdof, T.nadof), device="cuda", dtype=td)
    ctx.amgt_op_sweep(0, _dev(x, td), y)
    pats = [q for d in range(T.ndir) for q in T.patches_of(d)[:2]]
    ref = T.sweep(x, patches=pats)
    cols = np.concatenate([np.arange(q * T.a, (q + 1) * T.a) for q in pats])
    assert _rel(_host(y)[:, cols], ref[:, cols]) < tol
    ctx.close()


TC_CASES = [
    (2, (7, 5), 1, "lin"),      # N = K = 96: one partial 256-column tile, two K steps
    (2, (9, 4), 2, "const"),    # N = K = 128
    (2, (6, 6), 2, "lin"),      # N = K = 384: two column tiles, six K steps
    (3, (3, 4, 2), 1, "lin"),   # 3D, s = 8
]


@pytest.mark.parametrize("dim,nc,level,basis", TC_CASES,
                         ids=[f"{d}d-{'x'.join(map(str, n))}-l{l}-{b}" for d, n, l, b in TC_CASES])
def test_bf16_tensor_core_scatter(dim, nc, level, basis):
    """Scatter contraction on tcgen05 (BF16 inputs, FP32 accumulation) against
    the FP64 oracle; also its use inside (L - S) x."""
    prob = W.random_problem(dim, nc, level, 6, 35, basis=basis)
    T = _oracle(prob)
    ctx = _ctx(prob)
    x = W.random_vector((T.nsdof, T.nadof), 36)
    xd = _dev(x, torch.float32)
    y = torch.empty_like(xd)
    ctx.amgt_op_scatter(0, xd, y, tc=True)
    assert _rel(_host(y), T.scatter(x)) < 1e-2
    ctx.amgt_op_apply_A(0, xd, y, tc=True)
    assert _rel(_host(y), T.apply_A(x)) < 1e-2
    ctx.amgt_sync()        # no bounded device wait gave up
    ctx.close()


@pytest.mark.parametrize("dim,nc,level,basis", TC_CASES,
                         ids=[f"{d}d-{'x'.join(map(str, n))}-l{l}-{b}" for d, n, l, b in TC_CASES])
def test_fp16_three_product_scatter(dim, nc, level, basis):
    """FP32-accurate scatter on FP16 tensor cores (AMGT_F32_TC3: per-row power-
    of-two scales, hi/lo FP16 parts, three products in one GEMM) against the
    FP64 oracle at the FP32 operator tolerance, with rows whose magnitudes
    span 20 decades; also inside (L - S) x."""
    prob = W.random_problem(dim, nc, level, 6, 37, basis=basis)
    T = _oracle(prob)
    ctx = _ctx(prob)
    x = W.random_vector((T.nsdof, T.nadof), 38)
    x *= 10.0 ** np.linspace(-10, 10, T.nsdof)[:, None]
    xd = _dev(x, torch.float32)
    x32 = _host(xd)                # the FP32 input both sides see
    y = torch.empty_like(xd)
    ctx.amgt_op_scatter(0, xd, y, tc="tc3")
    ref = T.scatter(x32)
    # relative per spatial row: the rows' scales differ by 1e20
    rows = np.linalg.norm(_host(y) - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1e-300)
    assert rows.max() < 2e-5
    x2 = W.random_vector((T.nsdof, T.nadof), 39)
    xd2 = _dev(x2, torch.float32)
    ctx.amgt_op_apply_A(0, xd2, y, tc="tc3")
    assert _rel(_host(y), T.apply_A(_host(xd2))) < 2e-5
    ctx.amgt_sync()
    ctx.close()


@pytest.mark.parametrize("gs_kernel", [1, 2, 3, 4, 5, 6],
                         ids=["gs-per-patch", "gs-warp", "gs-group", "gs-grid", "gs-tc", "gs-rows"])
def test_coarse_gs_more_cells_per_level_than_groups(gs_kernel):
    """Up to 20 cells per wavefront level on a 20 x 40 mesh, with one-block
    clusters (8-16 groups) or 4 whole-GPU blocks, so every group handles
    several cells per level (the row-pipelined kernel: 4 blocks own 10 rows
    each); all must equal the oracle."""
    n = 20 * 40
    prob = W.random_problem(2, (20, 40), 1, 4, 37, g=0.8)
    prob["sigma_t"] = np.where(np.arange(n) % 7 < 3, 1.0, 4.0)
    prob["sigma_s"] = np.where(np.arange(n) % 7 < 3, 0.6, 3.7)
    prob["mg"] = dict(nlevels=1, Nr=[3], nu_pre=1, nu_post=1, coarse_sweeps=1)
    T = _oracle(prob, Nscat=3)
    ctx = _ctx(prob)
    ctx.amgt_set_tuning(1, gs_kernel)
    ctx.amgt_set_tuning(5, 1)     # one-block clusters
    ctx.amgt_set_tuning(4, 4)     # four whole-GPU blocks
    f = W.random_vector((T.nsdof, T.nadof), 38)
    x0 = W.random_vector((T.nsdof, T.nadof), 39)
    xd = _dev(x0, torch.float32)
    ctx.amgt_op_coarse_gs(1, _dev(f, torch.float32), xd)
    ctx.amgt_sync()
    ref = multigrid.coarse_gs(T, f, x0, 1)
    assert _rel(_host(xd), ref) < 2e-4
    ctx.close()


def test_row_pipelined_gs_3d_several_rows_per_block():
    """3D mesh of 4 x 3 x 5 cells: 15 rows shared by 2 blocks, each visiting
    its 7-8 rows in every direction's (y + z) wavefront order and waiting on
    face words from rows of the other block in both y and z."""
    prob = W.random_problem(3, (4, 3, 5), 1, 4, 53, g=0.8)
    prob["mg"] = dict(nlevels=1, Nr=[3], nu_pre=1, nu_post=1, coarse_sweeps=2)
    T = _oracle(prob, Nscat=3)
    ctx = _ctx(prob)
    ctx.amgt_set_tuning(1, 6)
    ctx.amgt_set_tuning(4, 2)
    f = W.random_vector((T.nsdof, T.nadof), 54)
    x0 = W.random_vector((T.nsdof, T.nadof), 55)
    for td, tol in ((torch.float64, 1e-12), (torch.float32, 2e-4)):
        xd = _dev(x0, td)
        ctx.amgt_op_coarse_gs(2, _dev(f, td), xd)
        ctx.amgt_sync()
        assert _rel(_host(xd), multigrid.coarse_gs(T, f, x0, 2)) < tol
    ctx.close()


GS_FORM_CASES = [
    ("2d-12x10-two-materials", 2, (12, 10), 2, 3, [8, 5, 4], 0),
    ("2d-6x5-per-cell", 2, (6, 5), 2, 3, [8, 4, 3], 0),
    ("2d-20x40-4-blocks", 2, (20, 40), 1, 1, [3], 4),
    ("3d-4x3x5-2-blocks", 3, (4, 3, 5), 1, 1, [3], 2),
]


@pytest.mark.parametrize("name,dim,nc,level,nlev,Nr,blocks", GS_FORM_CASES,
                         ids=[c[0] for c in GS_FORM_CASES])
@pytest.mark.parametrize("form", [1, 2], ids=["moment-form", "dense-form"])
def test_row_pipelined_gs_forms(name, dim, nc, level, nlev, Nr, blocks, form):
    """The row-pipelined coarse Gauss-Seidel with its scattering source in
    the moment form (flux moments kept per cell) and in the dense form
    (S_f rows of the direction minus S_dd^{L+D} times the cell's current
    unknowns, no moments), both against the oracle's block Gauss-Seidel:
    staged, tiled and per-cell materials, several rows per block, 3D, and
    in 2D the cell that ends one direction and starts the next."""
    from paper_2010_04559_gb300 import AMGT_TUNE_GS_FORM, AMGT_TUNE_GS_GRID_BLOCKS
    prob = _mg_problem(dim, nc, level, "lin", nlev, Nr, sweeps=2, seed=57)
    if nc == (20, 40):
        n = 20 * 40
        prob["sigma_t"] = np.where(np.arange(n) % 7 < 3, 1.0, 4.0)
        prob["sigma_s"] = np.where(np.arange(n) % 7 < 3, 0.6, 3.7)
    H = multigrid.Hierarchy(prob)
    Tc = H.levels[-1]
    ctx = _ctx(prob)
    ctx.amgt_set_tuning(1, 6)
    ctx.amgt_set_tuning(AMGT_TUNE_GS_FORM, form)
    if blocks:
        ctx.amgt_set_tuning(AMGT_TUNE_GS_GRID_BLOCKS, blocks)
    fc = W.random_vector((Tc.nsdof, Tc.nadof), 58)
    x0 = W.random_vector((Tc.nsdof, Tc.nadof), 59)
    ref = multigrid.coarse_gs(Tc, fc, x0, 2)
    for td, tol in ((torch.float64, 1e-12), (torch.float32, 2e-4)):
        xd = _dev(x0, td)
        ctx.amgt_op_coarse_gs(2, _dev(fc, td), xd)
        ctx.amgt_sync()
        assert _rel(_host(xd), ref) < tol
    ctx.close()


@pytest.mark.parametrize("group", [2, 4, 8], ids=["G2", "G4", "G8"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("nc", [(37, 29), (5, 21), (70, 24)], ids=["37x29", "5x21", "70x24"])
def test_warp_pipelined_sweep(group, dtype, nc):
    """The 2D warp-pipelined sweep (AMGT_TUNE_SWEEP_KERNEL = 2) against the
    oracle on two patches of every direction, and against the level-
    synchronous row sweep on all of them: ragged last warps, rows shorter than
    the hand-over ring and rows that wrap it several times, inflow faces."""
    from paper_2010_04559_gb300 import AMGT_TUNE_SWEEP_KERNEL
    prob = W.random_problem(2, nc, 2, 4, 35, inflow=0.3)
    T = _oracle(prob)
    ctx = _ctx(prob)
    ctx.amgt_set_tuning(2, group)
    td = torch.float64 if dtype == "f64" else torch.float32
    tol = 1e-12 if dtype == "f64" else 2e-5
    x = _dev(W.random_vector((T.nsdof, T.nadof), 36), td)
    yw = torch.empty_like(x)
    yr = torch.empty_like(x)
    ctx.amgt_set_tuning(AMGT_TUNE_SWEEP_KERNEL, 2)
    ctx.amgt_op_sweep(0, x, yw)
    ctx.amgt_sync()
    ctx.amgt_set_tuning(AMGT_TUNE_SWEEP_KERNEL, 1)
    ctx.amgt_op_sweep(0, x, yr)
    assert _rel(_host(yw), _host(yr)) < (1e-14 if dtype == "f64" else 1e-6)
    pats = [q for d in range(T.ndir) for q in T.patches_of(d)[:2]]
    ref = T.sweep(_host(x), patches=pats)
    cols = np.concatenate([np.arange(q * T.a, (q + 1) * T.a) for q in pats])
    assert _rel(_host(yw)[:, cols], ref[:, cols]) < tol
    ctx.close()


def test_kernel_timers_count_launches():
    """The library's per-kernel event timers: off by default (nothing
    recorded), on: one timed launch per operator call with positive time."""
    import paper_2010_04559_gb300 as pkg
    prob = W.random_problem(2, (12, 10), 2, 8, 91)
    ctx = _ctx(prob)
    ns, na = ctx.amgt_query_sizes(0)
    x = torch.randn((ns, na), device="cuda", dtype=torch.float32)
    y = torch.empty_like(x)
    ctx.amgt_op_sweep(0, x, y)
    assert ctx.amgt_query_kernel_time(pkg.AMGT_KT_SWEEP) == (0.0, 0)
    ctx.amgt_set_tuning(pkg.AMGT_TUNE_KERNEL_TIMERS, 1)
    for _ in range(3):
        ctx.amgt_op_sweep(0, x, y)
    ctx.amgt_op_apply_L(0, x, y)
    ms, n = ctx.amgt_query_kernel_time(pkg.AMGT_KT_SWEEP, reset=True)
    assert n == 3 and ms > 0
    assert ctx.amgt_query_kernel_time(pkg.AMGT_KT_APPLY_L)[1] == 1
    assert ctx.amgt_query_kernel_time(pkg.AMGT_KT_SWEEP) == (0.0, 0)
    ctx.amgt_set_tuning(pkg.AMGT_TUNE_KERNEL_TIMERS, 0)
    ctx.amgt_op_sweep(0, x, y)
    assert ctx.amgt_query_kernel_time(pkg.AMGT_KT_SWEEP)[1] == 0
    ctx.close()


def test_two_contexts_with_different_geometry_interleaved():
    """Each context carries its own spatial matrices: operators of two live
    contexts with different cell shapes, called alternately, each match
    their own oracle."""
    pa = W.random_problem(2, (6, 5), 1, 4, 141)
    pb = W.random_problem(2, (9, 7), 1, 4, 142)
    pb["hi"] = [2.0, 0.5, 1.0]
    Ta, Tb = _oracle(pa), _oracle(pb)
    ca, cb = _ctx(pa), _ctx(pb)
    ca.amgt_query_sizes(0)
    cb.amgt_query_sizes(0)
    xa = W.random_vector((Ta.nsdof, Ta.nadof), 143)
    xb = W.random_vector((Tb.nsdof, Tb.nadof), 144)
    ya = torch.empty((Ta.nsdof, Ta.nadof), device="cuda", dtype=torch.float64)
    yb = torch.empty((Tb.nsdof, Tb.nadof), device="cuda", dtype=torch.float64)
    for _ in range(2):
        ca.amgt_op_apply_A(0, _dev(xa), ya)
        cb.amgt_op_apply_A(0, _dev(xb), yb)
        assert _rel(_host(ya), Ta.apply_A(xa)) < 1e-12
        assert _rel(_host(yb), Tb.apply_A(xb)) < 1e-12
    ca.close()
    cb.close()


def test_fokker_planck_equivalent_moments_solve():
    """The paper's Fokker-Planck-equivalent Legendre moments (alpha = 1,
    N = 6: sigma_{s,0} = 21, strongly forward-peaked) with absorption 1:
    multigrid-preconditioned FP64 solve against the oracle."""
    from paper_2010_04559_gb300 import AMGT_MODE_F64, AMGT_PREC_MG
    s0, f = W.fp_moments(1.0, 6)
    prob = _mg_problem(2, (8, 7), 2, "lin", 3, [6, 4, 3], sweeps=10, seed=57)
    C = 8 * 7
    prob["sigma_s"] = np.full(C, s0)
    prob["sigma_t"] = np.full(C, s0 + 1.0)
    prob["fmom"] = f
    H = multigrid.Hierarchy(prob)
    T = H.levels[0]
    xo, _, _, _ = gmres.gmres(T.apply_A, T.source(), T.sweep, 1e-13, 20, 2000)
    ctx = _ctx(prob)
    psi, phi, st, _ = ctx.amgt_solve(tol=1e-13, restart=20, maxit=2000, precond=AMGT_PREC_MG,
                                     mode=AMGT_MODE_F64)
    assert st.relres < 1e-13
    assert _rel(psi, xo) < 1e-9
    ctx.close()


@pytest.mark.parametrize("precond", ["sweep", "mg"])
@pytest.mark.parametrize("mode", ["f64", "mixed"])
def test_bicgstab_solve_matches_oracle(precond, mode):
    """The paper's Krylov method (Sec. 3): right-preconditioned BiCGStab with
    the sweep or the multigrid cycle, FP64 or as the inner FP32 solver of the
    mixed refinement, against the oracle's BiCGStab solution."""
    from oracle import bicgstab
    from paper_2010_04559_gb300 import (AMGT_KRYLOV_BICGSTAB, AMGT_MODE_F64, AMGT_MODE_MIXED,
                                        AMGT_PREC_MG, AMGT_PREC_SWEEP)
    prob = _mg_problem(2, (8, 7), 2, "lin", 3, [8, 4, 4], sweeps=10, seed=61)
    H = multigrid.Hierarchy(prob)
    T = H.levels[0]
    xo, _, _, rel = bicgstab.bicgstab(T.apply_A, T.source(), T.sweep, 1e-13, 1000)
    assert rel < 1e-12
    ctx = _ctx(prob)
    pc = AMGT_PREC_SWEEP if precond == "sweep" else AMGT_PREC_MG
    md = AMGT_MODE_F64 if mode == "f64" else AMGT_MODE_MIXED
    tol = 1e-13 if mode == "f64" else 1e-10
    psi, phi, st, _ = ctx.amgt_solve(tol=tol, maxit=1000, precond=pc, mode=md,
                                     krylov=AMGT_KRYLOV_BICGSTAB)
    assert st.relres < tol
    assert _rel(psi, xo) < (1e-10 if mode == "f64" else 1e-6)
    ctx.close()


@pytest.mark.parametrize("dim,nc,level", [(2, (7, 6), 2), (3, (3, 4, 3), 1)])
def test_per_material_moment_shapes(dim, nc, level):
    """Two materials with different HG shapes (amgt_set_materials with mat_id,
    f[2][N+1]): the scatter (moment form with each cell's shape), the coarse
    Gauss-Seidel (per-patch form, shape-indexed tables), a V-cycle and the
    FP64 and mixed solves against the oracle."""
    from paper_2010_04559_gb300 import AMGT_MODE_F64, AMGT_MODE_MIXED, AMGT_PREC_MG
    prob = W.two_shape_problem(dim, nc, level, 6, 91)
    prob["mg"] = dict(nlevels=2, Nr=[6, 3], nu_pre=1, nu_post=1, coarse_sweeps=10)
    H = multigrid.Hierarchy(prob)
    T = H.levels[0]
    ctx = _ctx(prob)
    for td, tol in ((torch.float64, 1e-12), (torch.float32, 2e-5)):
        x = W.random_vector((T.nsdof, T.nadof), 92)
        y = torch.empty((T.nsdof, T.nadof), device="cuda", dtype=td)
        for tc in (False, True):           # the tensor-core flags fall back
            ctx.amgt_op_scatter(0, _dev(x, td), y, tc=tc)
            assert _rel(_host(y), T.scatter(x)) < tol
        ctx.amgt_op_apply_A(0, _dev(x, td), y)
        assert _rel(_host(y), T.apply_A(x)) < tol
        Tc = H.levels[-1]
        fc = W.random_vector((Tc.nsdof, Tc.nadof), 93)
        pc0 = W.random_vector((Tc.nsdof, Tc.nadof), 94)
        pc = _dev(pc0, td)
        ctx.amgt_op_coarse_gs(3, _dev(fc, td), pc)
        assert _rel(_host(pc), multigrid.coarse_gs(Tc, fc, pc0, 3)) < tol * 10
        out = torch.empty_like(y)
        ctx.amgt_op_vcycle(_dev(x, td), out)
        assert _rel(_host(out), H.vcycle(x)) < tol * 10
    xo, *_ = gmres.gmres(T.apply_A, T.source(), lambda v: H.vcycle(v), 1e-13, 20, 1000)
    psi, phi, st, _ = ctx.amgt_solve(tol=1e-13, precond=AMGT_PREC_MG, mode=AMGT_MODE_F64)
    assert st.relres < 1e-13 and _rel(psi, xo) < 1e-10
    psi, phi, st, _ = ctx.amgt_solve(tol=1e-11, precond=AMGT_PREC_MG, mode=AMGT_MODE_MIXED)
    assert st.relres < 1e-11 and _rel(psi, xo) < 1e-6
    ctx.close()


@pytest.mark.parametrize("dim,nc,level,basis", CASES, ids=IDS)
def test_double_float_L_apply(dim, nc, level, basis):
    """L x in double-float arithmetic (AMGT_F64_SPLIT; the refinement
    residual's L) against the oracle at 1e-12 per row, rows of very
    different magnitudes included (the mixed-solve tests above exercise it
    inside the refinement, where the split-form scatter applies)."""
    prob = W.random_problem(dim, nc, level, 4, 96, basis=basis, inflow=0.2)
    T = _oracle(prob)
    ctx = _ctx(prob)
    x = W.random_vector((T.nsdof, T.nadof), 97)
    x *= 10.0 ** np.linspace(-6, 6, T.nsdof)[:, None]
    y = torch.empty((T.nsdof, T.nadof), device="cuda", dtype=torch.float64)
    ctx.amgt_op_apply_L(0, _dev(x), y, tc=True)
    ref = T.apply_L(x)
    rows = np.linalg.norm(_host(y) - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert rows.max() < 1e-12
    ctx.close()


@pytest.mark.parametrize("nc,level,basis,dtype", [((5, 4, 6), 1, "lin", "f64"),
                                                  ((5, 4, 6), 1, "lin", "f32"),
                                                  ((3, 7, 2), 2, "const", "f64")])
def test_3d_grid_sweep(nc, level, basis, dtype):
    """The 3D sweep over every direction and patch at once (default) against
    the oracle's sweep and against the per-task level kernel
    (AMGT_TUNE_SWEEP_KERNEL = 1), with per-cell materials and inflow."""
    from paper_2010_04559_gb300 import AMGT_TUNE_SWEEP_KERNEL
    prob = W.random_problem(3, nc, level, 4, 98, basis=basis, inflow=0.3)
    T = _oracle(prob)
    ctx = _ctx(prob)
    td = torch.float64 if dtype == "f64" else torch.float32
    x = _dev(W.random_vector((T.nsdof, T.nadof), 99), td)
    yg = torch.empty_like(x)
    yl = torch.empty_like(x)
    ctx.amgt_op_sweep(0, x, yg)
    ctx.amgt_sync()
    ctx.amgt_set_tuning(AMGT_TUNE_SWEEP_KERNEL, 1)
    ctx.amgt_op_sweep(0, x, yl)
    ctx.amgt_sync()
    assert _rel(_host(yg), _host(yl)) < (1e-14 if dtype == "f64" else 1e-6)
    assert _rel(_host(yg), T.sweep(_host(x))) < (1e-12 if dtype == "f64" else 2e-5)
    ctx.close()
