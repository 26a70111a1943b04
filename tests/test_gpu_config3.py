"""The 3D workload with a different sigma_t in every cell: 32^3 hex cells,
lognormal sigma_t, sigma_s = 0.9 sigma_t, HG g = 0.95 at order 32, level-2
Lin angular mesh (128 patches), 3-level multigrid -- 32768 materials, so one
block inverse per (cell, patch).  Sampled parity of the sweep and of L
against the oracle, the mixed-precision solve to 1e-8, and the detector
response of the corner 8^3 block: adjoint gradients against central finite
differences of the GPU response."""
import numpy as np
import pytest

import workloads as W
from oracle import angular, transport

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N3 = 32


def _corner_weight():
    w = np.zeros(N3 ** 3)
    for iz in range(8):
        for iy in range(8):
            w[(iz * N3 + iy) * N3:(iz * N3 + iy) * N3 + 8] = 1.0
    return w


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_04559_gb300 import build, context_from_problem
    build.build()
    prob = W.config3_cube()
    ctx = context_from_problem(prob, device=0)
    yield prob, ctx
    ctx.close()


def test_config3_sampled_operators(setup):
    prob, ctx = setup
    T = transport.Transport(prob, angular.AngularMesh(angular.uniform_paths(2), "lin"), Nscat=2)
    assert ctx.amgt_query_sizes(0) == (T.nsdof, T.nadof)
    x = W.random_vector((T.nsdof, T.nadof), 121)
    xd = torch.from_numpy(x).to("cuda", torch.float32)
    y = torch.empty_like(xd)
    ctx.amgt_op_sweep(0, xd, y)
    torch.cuda.synchronize()
    pats = [int(T.patches_of(d)[0]) for d in (0, 7)]
    ref = T.sweep(x, patches=pats)
    cols = np.concatenate([np.arange(q * 3, q * 3 + 3) for q in pats])
    assert _rel(y.double().cpu().numpy()[:, cols], ref[:, cols]) < 2e-5
    cells = [0, 31, 32 * 32 * 16 + 32 * 7 + 5, N3 ** 3 - 1]
    rows = np.concatenate([np.arange(c * 8, c * 8 + 8) for c in cells])
    ctx.amgt_op_apply_L(0, xd, y)
    torch.cuda.synchronize()
    assert _rel(y.double().cpu().numpy()[rows], T.apply_L(x, cells=cells)[rows]) < 2e-5


def test_config3_mixed_solve_adjoint_and_finite_differences(setup):
    from paper_2010_04559_gb300 import AMGT_MODE_MIXED, AMGT_PREC_MG, context_from_problem
    from paper_2010_04559_gb300.adjoint import response_problem
    prob, ctx = setup
    weight = _corner_weight()
    ns, na = ctx.amgt_query_sizes(0)
    psi = torch.empty((ns, na), device="cuda", dtype=torch.float64)
    phi = torch.empty(ns, device="cuda", dtype=torch.float64)
    kw = dict(precond=AMGT_PREC_MG, mode=AMGT_MODE_MIXED, phi=phi, device_ptrs=True)
    _, _, st, _ = ctx.amgt_solve(tol=1e-12, psi=psi, **kw)
    assert st.relres < 1e-12
    actx = context_from_problem(response_problem(prob, weight), device=0)
    actx.amgt_set_adjoint(1)
    lam = torch.empty_like(psi)
    _, _, sta, _ = actx.amgt_solve(tol=1e-12, psi=lam, **kw)
    assert sta.relres < 1e-12
    R = actx.amgt_response(psi)
    C = N3 ** 3
    dt = torch.empty(C, device="cuda", dtype=torch.float64)
    ds = torch.empty_like(dt)
    df = torch.empty(prob["N"] + 1, device="cuda", dtype=torch.float64)
    ctx.amgt_response_gradients(psi, lam, dt, ds, df)
    dt, df = dt.cpu().numpy(), df.cpu().numpy()
    assert R > 0 and dt.sum() < 0

    def resp(key, idx, h):
        p = {k: (np.array(v, dtype=float) if k in ("sigma_t", "fmom") else v)
             for k, v in prob.items()}
        p[key][idx] += h
        c = context_from_problem(p, device=0)
        x = torch.empty_like(psi)
        c.amgt_solve(tol=1e-12, psi=x, **kw)
        c.close()
        return actx.amgt_response(x)

    # one cell of width 1/32 is optically thin: R is nearly linear in its
    # sigma_t, so a wide step keeps the solver noise small against the change
    c = int(np.argmax(np.abs(dt)))
    h = 3e-2 * prob["sigma_t"][c]
    fd = (resp("sigma_t", c, h) - resp("sigma_t", c, -h)) / (2 * h)
    assert abs(fd - dt[c]) < 1e-5 * abs(dt[c]), (c, fd, dt[c])
    h = 1e-3
    fd = (resp("fmom", 1, h) - resp("fmom", 1, -h)) / (2 * h)
    assert abs(fd - df[1]) < 1e-5 * abs(df[1]), (fd, df[1])
    actx.close()
