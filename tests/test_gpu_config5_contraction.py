"""Oracle parity of the scatter contraction at the shapes of the 256x256 beam
workload (uniform level 4: 2048 patches, K = N = Nadof = 6144, order 64;
coarse levels at order 12), on sampled cells.

S couples only the rows of one cell (Sec. 4.2), so each sampled cell's
output rows depend on that cell's input rows alone: the full-size input is
filled on the device, the sampled cells' rows are overwritten with seeded
values, and the oracle computes those cells' rows.  The cells are spread
over the row passes of the split FP64 form and of the FP16 three-product
form, the last, partial pass included.  The oracle's angular table X to
degree 64 (2048 patches) is built by chunks of patches in spawned processes:
a patch's row of X depends on that patch alone."""
import multiprocessing
import os

import numpy as np
import pytest

import workloads as W
from oracle import angular, transport

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N_CELLS = 256
CELLS = [0, 1, 7000, 14559, 14560, 14561, 29120, 40000, 58239, 58240, 65535]


def _x_chunk(args):
    paths, basis, N = args
    return angular.AngularMesh(paths, basis).X(N)


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_04559_gb300 import build, context_from_problem
    build.build()
    prob = W.config5_beam()
    paths = angular.uniform_paths(4)
    chunks = [paths[i:i + 64] for i in range(0, len(paths), 64)]
    nproc = min(len(chunks), max(1, (os.cpu_count() or 2) - 1))
    with multiprocessing.get_context("spawn").Pool(nproc) as pool:
        parts = pool.map(_x_chunk, [(c, "lin", prob["N"]) for c in chunks])
    X = np.concatenate(parts, axis=0)
    am = angular.AngularMesh(paths, "lin")
    am.X = lambda N, _X=X: _X          # the table built above, same rows
    T = transport.Transport(prob, am)
    stream = torch.cuda.Stream()
    ctx = context_from_problem(prob, device=0, stream=stream.cuda_stream)
    yield prob, T, ctx, stream
    ctx.close()


def _rows(cells, s):
    return np.concatenate([np.arange(c * s, (c + 1) * s) for c in cells])


def _row_rel(y, ref):
    return (np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)).max()


def _fill(ns, na, dtype, xs, rows):
    x = torch.randn((ns, na), device="cuda", dtype=torch.float32,
                    generator=torch.Generator(device="cuda").manual_seed(5)).to(dtype)
    x[torch.from_numpy(rows).cuda()] = torch.from_numpy(xs).to(device="cuda", dtype=dtype)
    return x


def test_shapes(setup):
    prob, T, ctx, _ = setup
    assert ctx.amgt_query_sizes(0) == (4 * N_CELLS * N_CELLS, 6144)
    assert T.X.shape == (6144, 65 * 65)


@pytest.mark.parametrize("path,tol", [("split", 1e-12), ("tc3", 1e-4), ("simt32", 1e-4),
                                      ("bf16", 1e-2)])
def test_fine_level_scatter_matches_oracle(setup, path, tol):
    """amgt_op_scatter on level 0 (K = 6144): the FP64-accurate split form
    (5-bit digits, 10 slices, row passes of ~8 GB), the FP32-accurate FP16
    three-product form (row passes of ~4 GB), the FP32 SIMT contraction and
    the BF16 form, each against the oracle's moment-form scatter of the
    sampled cells.  Tolerances per row: FP64 1e-12 (with random-sign rows the
    oracle's own FP64 sums over 6144 angular DOF and 4225 moments carry
    ~1e-16 sqrt(K) |x||S| / |x S| ~ 1e-13 of rounding); FP32 1e-4, the unit
    roundoff 6e-8 times the sum length 6144 (the 2e-5 of the smaller parity
    cases is 6e-8 times their sums of a few hundred)."""
    prob, T, ctx, stream = setup
    ns, na = ctx.amgt_query_sizes(0)
    rows = _rows(CELLS, T.s)
    xs = W.random_vector((len(rows), na), 71)
    xs *= 10.0 ** np.linspace(-3, 3, len(rows))[:, None]
    dtype = torch.float64 if path == "split" else torch.float32
    if dtype == torch.float32:
        xs = xs.astype(np.float32).astype(np.float64)   # the input both sides see
    with torch.cuda.stream(stream):
        x = _fill(ns, na, dtype, xs, rows)
        y = torch.empty_like(x)
        ctx.amgt_op_scatter(0, x, y, tc={"split": True, "tc3": "tc3", "simt32": False,
                                         "bf16": True}[path])
        ctx.amgt_sync()
        ys = y[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    del x, y
    torch.cuda.empty_cache()
    ref = T.scatter(xs, cells=CELLS)
    assert _row_rel(ys, ref) < tol


@pytest.mark.parametrize("level", [1, 2, 3])
def test_coarse_level_scatter_matches_oracle(setup, level):
    """Levels 1-3 of the 4-level hierarchy (1536, 384 and 96 angular DOF)
    with the reduced order N_r = 12, FP64 and the BF16 form."""
    prob, _, ctx, stream = setup
    am = angular.AngularMesh(angular.uniform_paths(4 - level), "lin")
    Tc = transport.Transport(prob, am, prob["mg"]["Nr"][level])
    ns, na = ctx.amgt_query_sizes(level)
    assert na == Tc.nadof
    rows = _rows(CELLS, Tc.s)
    xs = W.random_vector((len(rows), na), 72 + level)
    ref = Tc.scatter(xs, cells=CELLS)
    for dtype, tc, tol in ((torch.float64, False, 1e-12), (torch.float32, True, 1e-2)):
        with torch.cuda.stream(stream):
            x = _fill(ns, na, dtype, xs, rows)
            y = torch.empty_like(x)
            ctx.amgt_op_scatter(level, x, y, tc=tc)
            ctx.amgt_sync()
            ys = y[torch.from_numpy(rows).cuda()].double().cpu().numpy()
        if dtype == torch.float32:
            ref32 = Tc.scatter(xs.astype(np.float32).astype(np.float64), cells=CELLS)
            assert _row_rel(ys, ref32) < tol
        else:
            assert _row_rel(ys, ref) < tol
