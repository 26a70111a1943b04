"""The scatter contraction to FP64 accuracy from BF16 tensor-core products
(dtype AMGT_F64_SPLIT, error-free digit splitting): against the oracle's FP64
scatter and the library's FP64 SIMT contraction, in 2D and 3D, dense and
moment-form levels, one pass and several row passes; then the mixed solve
with split-form refinement residuals and the FP64 solve with every scatter
in split form, against the oracle and the FP64 SIMT solve."""
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


def _host(t):
    torch.cuda.synchronize()
    return t.detach().double().cpu().numpy()


# (dim, ncell, level, N): angular sizes 96 (level 1), 384 (level 2), 1536
# (level 3, moment form on the SIMT path), 3D with 8 spatial nodes per cell
CASES = [(2, (7, 5), 1, 4), (2, (6, 4), 2, 8), (2, (3, 5), 3, 12), (3, (3, 2, 3), 1, 6)]


@pytest.mark.parametrize("dim,nc,level,N", CASES)
def test_split_scatter_matches_oracle_and_fp64(dim, nc, level, N):
    from paper_2010_04559_gb300 import context_from_problem
    prob = W.random_problem(dim, nc, level, N, 131, g=0.9)
    T = transport.Transport(prob, angular.AngularMesh(angular.uniform_paths(level), "lin"))
    ctx = context_from_problem(prob, device=0)
    x = W.random_vector((T.nsdof, T.nadof), 132)
    # cells many orders of magnitude apart: each row has its own scale
    small = np.concatenate([np.arange(c * T.s, (c + 1) * T.s) for c in range(0, T.C, 3)])
    x[small] *= 1e-9
    x[T.s:2 * T.s] *= 1e6
    xd = torch.from_numpy(x).cuda()
    ys = torch.empty_like(xd)
    y64 = torch.empty_like(xd)
    ctx.amgt_op_scatter(0, xd, ys, tc=True)
    ctx.amgt_op_scatter(0, xd, y64)
    ref = T.scatter(x)
    es, e64 = _rel(_host(ys), ref), _rel(_host(y64), ref)
    assert es < 1e-13, (es, e64)
    assert e64 < 1e-13
    assert _rel(_host(ys)[small], ref[small]) < 1e-13
    # several passes over the rows (ragged last pass) give the same values
    from paper_2010_04559_gb300 import AMGT_TUNE_SPLIT_ROWS
    ctx.amgt_set_tuning(AMGT_TUNE_SPLIT_ROWS, 128)
    yc = torch.empty_like(xd)
    ctx.amgt_op_scatter(0, xd, yc, tc=True)
    assert torch.equal(yc, ys)
    ctx.close()


def test_split_apply_A_equals_fp64_apply_A():
    from paper_2010_04559_gb300 import context_from_problem
    prob = W.random_problem(2, (9, 8), 2, 8, 133, g=0.95)
    ctx = context_from_problem(prob, device=0)
    ns, na = ctx.amgt_query_sizes(0)
    x = torch.from_numpy(W.random_vector((ns, na), 134)).cuda()
    ys = torch.empty_like(x)
    y64 = torch.empty_like(x)
    ctx.amgt_op_apply_A(0, x, ys, tc=True)
    ctx.amgt_op_apply_A(0, x, y64)
    assert _rel(_host(ys), _host(y64)) < 1e-13
    ctx.close()


def _mg_problem(seed):
    prob = W.random_problem(2, (8, 7), 2, 8, seed, g=0.9)
    prob["mg"] = dict(nlevels=3, Nr=[8, 4, 4], nu_pre=1, nu_post=1, coarse_sweeps=10)
    return prob


def test_mixed_solve_with_split_residuals():
    """Default (split-form refinement residuals) against the FP64 SIMT
    residuals: same refinement, same answer; both against the oracle."""
    from paper_2010_04559_gb300 import (AMGT_MODE_MIXED, AMGT_PREC_MG, AMGT_TUNE_FP64_SCATTER,
                                        context_from_problem)
    prob = _mg_problem(135)
    H = multigrid.Hierarchy(prob)
    T = H.levels[0]
    xo, *_ = gmres.gmres(T.apply_A, T.source(), T.sweep, 1e-13, 20, 1000)
    out = {}
    for key in (0, 1):
        ctx = context_from_problem(prob, device=0)
        ctx.amgt_set_tuning(AMGT_TUNE_FP64_SCATTER, key)
        psi, _, st, _ = ctx.amgt_solve(tol=1e-11, precond=AMGT_PREC_MG, mode=AMGT_MODE_MIXED)
        assert st.relres < 1e-11
        assert _rel(psi, xo) < 1e-6
        out[key] = (psi, st.iterations, st.outer_iterations)
        ctx.close()
    assert out[0][1:] == out[1][1:]
    assert _rel(out[0][0], out[1][0]) < 1e-9


def test_fp64_solve_with_every_scatter_split():
    from paper_2010_04559_gb300 import (AMGT_MODE_F64, AMGT_PREC_MG, AMGT_TUNE_FP64_SCATTER,
                                        context_from_problem)
    prob = _mg_problem(136)
    H = multigrid.Hierarchy(prob)
    T = H.levels[0]
    xo, *_ = gmres.gmres(T.apply_A, T.source(), T.sweep, 1e-13, 20, 1000)
    ctx = context_from_problem(prob, device=0)
    ctx.amgt_set_tuning(AMGT_TUNE_FP64_SCATTER, 2)
    psi, phi, st, _ = ctx.amgt_solve(tol=1e-12, precond=AMGT_PREC_MG, mode=AMGT_MODE_F64)
    assert st.relres < 1e-12
    assert _rel(psi, xo) < 1e-10
    ctx.close()
