"""GPU parity of the adjoint path: the transposed operators of a context with
amgt_set_adjoint(1) against the oracle's reversed-direction operators, the
forward/adjoint solves and the response gradients against the oracle's dense
solves and gradients, and the autograd gradients against central finite
differences of the GPU response."""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint as oadj
from oracle import angular, transport

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


def _dev(x, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def _host(t):
    torch.cuda.synchronize()
    return t.detach().double().cpu().numpy()


OPS = [(2, (6, 5), 1, "lin"), (2, (5, 4), 1, "const"), (3, (3, 2, 3), 1, "lin")]


@pytest.mark.parametrize("dim,nc,level,basis", OPS)
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_adjoint_operators_match_reversed_oracle(dim, nc, level, basis, dtype):
    from paper_2010_04559_gb300 import context_from_problem
    prob = W.random_problem(dim, nc, level, 4, 101, basis=basis, g=0.8)
    am = angular.AngularMesh(angular.uniform_paths(level), basis)
    Ta = transport.Transport(prob, oadj.ReversedMesh(am))
    ctx = context_from_problem(prob, device=0)
    ctx.amgt_set_adjoint(1)
    td = torch.float64 if dtype == "f64" else torch.float32
    tol = 1e-12 if dtype == "f64" else 2e-5
    x = W.random_vector((Ta.nsdof, Ta.nadof), 102)
    y = torch.empty((Ta.nsdof, Ta.nadof), device="cuda", dtype=td)
    ctx.amgt_op_apply_L(0, _dev(x, td), y)
    assert _rel(_host(y), Ta.apply_L(x)) < tol
    ctx.amgt_op_sweep(0, _dev(x, td), y)
    assert _rel(_host(y), Ta.sweep(x)) < tol
    ctx.amgt_op_apply_A(0, _dev(x, td), y)
    assert _rel(_host(y), Ta.apply_A(x)) < tol
    ctx.close()


def _problem(dim, nc, level, N, seed, nlev=2):
    prob = W.random_problem(dim, nc, level, N, seed, g=0.8)
    prob["mg"] = dict(nlevels=nlev, Nr=[N, 2][:nlev], nu_pre=1, nu_post=1, coarse_sweeps=4)
    C = int(np.prod(nc))
    weight = np.zeros(C)
    weight[C - 1] = 1.0
    weight[C // 3] = 1.0
    return prob, weight


@pytest.mark.parametrize("dim,nc,level,nlev", [(2, (4, 3), 1, 2), (3, (2, 3, 2), 0, 1)],
                         ids=["2d", "3d"])
def test_solves_and_gradients_match_oracle(dim, nc, level, nlev):
    from paper_2010_04559_gb300.adjoint import solve_response
    prob, weight = _problem(dim, nc, level, 4, 103, nlev)
    am = angular.AngularMesh(angular.uniform_paths(level), "lin")
    T = transport.Transport(prob, am)
    Ta = oadj.adjoint_transport(prob, am, weight)
    psi_ref = oadj.dense_solve(T, T.source())
    lam_ref = oadj.dense_solve(Ta, Ta.source())
    R_ref = oadj.response(T, psi_ref, weight)
    dt_ref, ds_ref, df_ref = oadj.gradients(T, psi_ref, lam_ref)
    R, psi, lam, dt, ds, df = solve_response(prob, weight, tol=1e-13)
    assert _rel(_host(psi), psi_ref) < 1e-10
    assert _rel(_host(lam), lam_ref) < 1e-10
    assert abs(R - R_ref) < 1e-10 * abs(R_ref)
    assert _rel(_host(dt), dt_ref) < 1e-9
    assert _rel(_host(ds), ds_ref) < 1e-9
    assert _rel(_host(df), df_ref) < 1e-9


def test_mixed_precision_adjoint_solve():
    from paper_2010_04559_gb300 import AMGT_MODE_MIXED
    from paper_2010_04559_gb300.adjoint import solve_response
    prob, weight = _problem(2, (12, 10), 2, 6, 104)
    R64, _, lam64, dt64, _, _ = solve_response(prob, weight, tol=1e-12)
    R32, _, lam32, dt32, _, _ = solve_response(prob, weight, tol=1e-10, mode=AMGT_MODE_MIXED)
    assert abs(R32 - R64) < 1e-8 * abs(R64)
    assert float(torch.linalg.norm(lam32 - lam64) / torch.linalg.norm(lam64)) < 1e-6
    assert float(torch.linalg.norm(dt32 - dt64) / torch.linalg.norm(dt64)) < 1e-6


def test_autograd_gradients_match_central_differences():
    """dR/dsigma_t, dR/dsigma_s, dR/df_n through torch.autograd against
    central differences of the GPU response, 1e-5 relative."""
    from paper_2010_04559_gb300.adjoint import DetectorResponse, solve_response
    prob, weight = _problem(2, (6, 5), 1, 4, 105)
    st = torch.tensor(prob["sigma_t"], dtype=torch.float64, requires_grad=True)
    ss = torch.tensor(prob["sigma_s"], dtype=torch.float64, requires_grad=True)
    fm = torch.tensor(prob["fmom"], dtype=torch.float64, requires_grad=True)
    R = DetectorResponse.apply(st, ss, fm, prob, weight, tol=1e-13)
    R.backward()
    gt, gs, gf = st.grad.numpy(), ss.grad.numpy(), fm.grad.numpy()

    def resp(key, idx, h):
        p = {k: (np.array(v, dtype=float) if k in ("sigma_t", "sigma_s", "fmom") else v)
             for k, v in prob.items()}
        p[key][idx] += h
        return solve_response(p, weight, tol=1e-13)[0]

    C = st.numel()
    for key, grad, idxs in (("sigma_t", gt, (0, C // 2, C - 1)), ("sigma_s", gs, (1, C - 1)),
                            ("fmom", gf, (1, 2, 4))):
        for i in idxs:
            h = 1e-4 * max(1.0, abs(prob[key][i]))
            fd = (resp(key, i, h) - resp(key, i, -h)) / (2 * h)
            assert abs(fd - grad[i]) < 1e-5 * np.abs(grad).max(), (key, i, fd, grad[i])


def test_per_material_shape_gradients_match_the_oracle():
    """dR/df for two materials with different moment shapes: the library's
    [nmat][N+1] gradient against the oracle's adjoint gradients."""
    from oracle import adjoint as oadj
    from paper_2010_04559_gb300.adjoint import solve_response
    prob = W.two_shape_problem(2, (4, 3), 1, 4, 95)
    weight = np.zeros(12)
    weight[[0, 5, 7]] = 1.0
    am = angular.AngularMesh(angular.uniform_paths(1), "lin")
    T = transport.Transport(prob, am)
    psi = oadj.dense_solve(T, T.source())
    Ta = oadj.adjoint_transport(prob, am, weight)
    lam = oadj.dense_solve(Ta, Ta.source())
    dt_o, ds_o, df_o = oadj.gradients(T, psi, lam)
    R, _, _, dt, ds, df = solve_response(prob, weight, tol=1e-13)
    assert abs(R - oadj.response(T, psi, weight)) < 1e-10 * abs(R)
    assert df.shape == (2, 5)
    for a, b in ((dt, dt_o), (ds, ds_o), (df, df_o)):
        a = a.cpu().numpy()
        assert np.abs(a - b).max() < 1e-9 * np.abs(b).max()
