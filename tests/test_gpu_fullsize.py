"""Parity at the benchmark's full size: 128 x 128 cells, two-material
checkerboard, level-3 Lin mesh (512 patches, 1536 angular DOF), HG g = 0.9 at
order 16, 3-level multigrid -- the configuration bench.py times -- on outputs
the oracle computes independently: sampled patches (sweep), sampled cells
(L x, S x), full transfers, and for the coarse Gauss-Seidel sweep the block
equation every visited block must satisfy.  FP32, as in the timed solve.
"""
import numpy as np
import pytest

import workloads as W
from oracle import angular, transport

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL32 = 2e-5


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_04559_gb300 import build, context_from_problem
    build.build()
    prob = W.config2_checkerboard()
    ctx = context_from_problem(prob, device=0)
    # only the meshes and transfer the checks below need
    paths = angular.uniform_paths(3)
    m3 = angular.AngularMesh(paths, "lin")
    m2 = angular.AngularMesh(angular.coarsen_paths(paths, 2), "lin")
    m1 = angular.AngularMesh(angular.coarsen_paths(paths, 1), "lin")
    T3 = transport.Transport(prob, m3, prob["mg"]["Nr"][0])
    T1 = transport.Transport(prob, m1, prob["mg"]["Nr"][2])
    P32 = angular.prolongation(m3, m2)
    yield prob, ctx, T3, T1, P32
    ctx.close()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def test_fullsize_sweep_sampled_patches(setup):
    prob, ctx, T, _, _ = setup
    x = W.random_vector((T.nsdof, T.nadof), 81)
    xd = torch.from_numpy(x).to("cuda", torch.float32)
    y = torch.empty_like(xd)
    ctx.amgt_op_sweep(0, xd, y)
    # one patch per direction, at the start, middle and end of the groups
    pats = [int(T.patches_of(d)[k]) for d, k in zip(range(4), (0, 37, 64, 127))]
    ref = T.sweep(x, patches=pats)
    cols = np.concatenate([np.arange(q * 3, q * 3 + 3) for q in pats])
    assert _rel(_host(y)[:, cols], ref[:, cols]) < TOL32


def test_fullsize_warp_pipelined_sweep_sampled_patches(setup):
    from paper_2010_04559_gb300 import AMGT_TUNE_SWEEP_KERNEL
    prob, ctx, T, _, _ = setup
    x = W.random_vector((T.nsdof, T.nadof), 83)
    xd = torch.from_numpy(x).to("cuda", torch.float32)
    y = torch.empty_like(xd)
    ctx.amgt_set_tuning(AMGT_TUNE_SWEEP_KERNEL, 2)
    ctx.amgt_op_sweep(0, xd, y)
    ctx.amgt_sync()
    ctx.amgt_set_tuning(AMGT_TUNE_SWEEP_KERNEL, 0)
    pats = [int(T.patches_of(d)[k]) for d, k in zip(range(4), (3, 64, 100, 127))]
    ref = T.sweep(x, patches=pats)
    cols = np.concatenate([np.arange(q * 3, q * 3 + 3) for q in pats])
    assert _rel(_host(y)[:, cols], ref[:, cols]) < TOL32


def test_fullsize_apply_L_and_scatter_sampled_cells(setup):
    prob, ctx, T, _, _ = setup
    x = W.random_vector((T.nsdof, T.nadof), 82)
    xd = torch.from_numpy(x).to("cuda", torch.float32)
    y = torch.empty_like(xd)
    cells = [0, 127, 128 * 64 + 63, 128 * 127, 128 * 128 - 1, 5 * 128 + 77]
    rows = np.concatenate([np.arange(c * 4, c * 4 + 4) for c in cells])
    ctx.amgt_op_apply_L(0, xd, y)
    ref = T.apply_L(x, cells=cells)
    assert _rel(_host(y)[rows], ref[rows]) < TOL32
    ctx.amgt_op_scatter(0, xd, y)
    Sf = T.angular_scatter_matrix()
    got = _host(y)[rows]
    for i, c in enumerate(cells):
        blk = x[c * 4:c * 4 + 4]
        refc = T.sigma_s[c] * (T.cell.N @ (blk @ Sf.T))
        assert _rel(got[i * 4:i * 4 + 4], refc) < TOL32


def test_fullsize_bf16_tensor_core_scatter_sampled_cells(setup):
    prob, ctx, T, _, _ = setup
    x = W.random_vector((T.nsdof, T.nadof), 90)
    xd = torch.from_numpy(x).to("cuda", torch.float32)
    y = torch.empty_like(xd)
    ctx.amgt_op_scatter(0, xd, y, tc=True)
    ctx.amgt_sync()
    Sf = T.angular_scatter_matrix()
    got = _host(y)
    for c in [0, 127, 128 * 64 + 63, 128 * 128 - 1, 4095]:
        refc = T.sigma_s[c] * (T.cell.N @ (x[c * 4:c * 4 + 4] @ Sf.T))
        assert _rel(got[c * 4:c * 4 + 4], refc) < 1e-2


def test_fullsize_transfers(setup):
    prob, ctx, T, _, P = setup
    r = W.random_vector((T.nsdof, T.nadof), 83)
    rc = torch.empty((T.nsdof, P.shape[1]), device="cuda", dtype=torch.float32)
    ctx.amgt_op_restrict(0, torch.from_numpy(r).to("cuda", torch.float32), rc)
    sel = slice(0, T.nsdof, 97)
    assert _rel(_host(rc)[sel], r[sel] @ P) < TOL32
    xc = W.random_vector((T.nsdof, P.shape[1]), 84)
    xf = torch.zeros((T.nsdof, T.nadof), device="cuda", dtype=torch.float32)
    ctx.amgt_op_prolong(0, torch.from_numpy(xc).to("cuda", torch.float32), xf)
    assert _rel(_host(xf)[sel], xc[sel] @ P.T) < TOL32


def test_fullsize_coarse_gs_block_equations(setup):
    """After one Gauss-Seidel sweep from x0 on the coarsest level, each sampled
    block (c, q) satisfies its own equation with the newest values of the
    blocks visited before it and the old values of those visited after it."""
    prob, ctx, _, T1, _ = setup
    ns, na = ctx.amgt_query_sizes(2)
    assert (ns, na) == (T1.nsdof, T1.nadof)
    f = W.random_vector((ns, na), 85)
    x0 = W.random_vector((ns, na), 86)
    xd = torch.from_numpy(x0).to("cuda", torch.float32)
    ctx.amgt_op_coarse_gs(1, torch.from_numpy(f).to("cuda", torch.float32), xd)
    x1 = _host(xd)
    s, a = T1.s, T1.a
    Sf = T1.angular_scatter_matrix()
    N = T1.cell.N
    pos = [{cc: i for i, cc in enumerate(T1.sweep_order(dd))} for dd in range(T1.ndir)]
    rng = np.random.default_rng(87)
    for _ in range(24):
        c = int(rng.integers(T1.C))
        q = int(rng.integers(T1.P))
        d = int(T1.pdir[q])
        # which blocks are "new" when (c, q) is solved
        def newer(c2, p2):
            d2 = int(T1.pdir[p2])
            if d2 != d:
                return d2 < d
            if c2 == c:
                return p2 <= q
            # same direction, other cell: visited earlier iff ordered before
            return pos[d][c2] < pos[d][c]
        xb = lambda c2, p2: (x1 if newer(c2, p2) else x0)[c2 * s:(c2 + 1) * s, p2 * a:(p2 + 1) * a]
        lhs = T1.block(c, q) @ xb(c, q).reshape(-1)
        for fc in range(4):
            nb = T1.neighbour(c, fc)
            if nb >= 0 and not T1.outflow[fc, q]:
                lhs += T1.U[fc, q] @ xb(nb, q).reshape(-1)
        src = np.zeros((s, a))
        for p in range(T1.P):
            src += N @ xb(c, p) @ Sf[q * a:(q + 1) * a, p * a:(p + 1) * a].T
        res = lhs - T1.sigma_s[c] * src.reshape(-1) - f[c * s:(c + 1) * s, q * a:(q + 1) * a].reshape(-1)
        scale = np.abs(f[c * s:(c + 1) * s]).max() + np.abs(lhs).max()
        assert np.abs(res).max() < 1e-4 * scale


def test_fullsize_vcycle_is_linear(setup):
    prob, ctx, T, _, _ = setup
    f1 = torch.from_numpy(W.random_vector((T.nsdof, T.nadof), 88)).to("cuda", torch.float32)
    f2 = torch.from_numpy(W.random_vector((T.nsdof, T.nadof), 89)).to("cuda", torch.float32)
    out = [torch.empty_like(f1) for _ in range(3)]
    ctx.amgt_op_vcycle(f1, out[0])
    ctx.amgt_op_vcycle(f2, out[1])
    ctx.amgt_op_vcycle(2.0 * f1 - 0.5 * f2, out[2])
    lin = 2.0 * out[0] - 0.5 * out[1]
    torch.cuda.synchronize()
    assert float(torch.linalg.norm(out[2] - lin) / torch.linalg.norm(lin)) < 1e-4
