"""Failure paths of the library on the GPU, in forms that fault nothing: bad
inputs are refused before any device work, a non-finite iterate and a too
small iteration cap come back as status codes, and a device-side wait that
runs out (a progress counter that nothing publishes, under a test-only
tuning key that also shortens the wait to 10 ms) is reported by amgt_sync
while the context stays usable."""
import numpy as np
import pytest

import workloads as W
from oracle import angular, transport

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_04559_gb300 import build
    build.build()


def _ctx(prob):
    from paper_2010_04559_gb300 import context_from_problem
    return context_from_problem(prob, device=0)


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b)


def test_non_finite_inputs_are_refused():
    from paper_2010_04559_gb300 import AMGT_ERR_ARG, AmgtError
    prob = W.random_problem(2, (6, 5), 1, 4, 61)
    ctx = _ctx(prob)
    for bad in (np.nan, np.inf):
        q = prob["q"].copy()
        q[3] = bad
        with pytest.raises(AmgtError) as e:
            ctx.amgt_set_source_iso(q)
        assert e.value.code == AMGT_ERR_ARG
        with pytest.raises(AmgtError) as e:
            ctx.amgt_set_boundary(0, 1, bad)
        assert e.value.code == AMGT_ERR_ARG
        f = prob["fmom"].copy()
        f[2] = bad
        with pytest.raises(AmgtError) as e:
            ctx.amgt_set_materials(prob["sigma_t"], prob["sigma_s"], prob["N"], f)
        assert e.value.code == AMGT_ERR_ARG
    # the refused calls changed nothing: the context still solves its problem
    from paper_2010_04559_gb300 import AMGT_MODE_F64, AMGT_PREC_SWEEP
    psi, _, st, _ = ctx.amgt_solve(tol=1e-12, precond=AMGT_PREC_SWEEP, mode=AMGT_MODE_F64)
    am = angular.AngularMesh(angular.uniform_paths(1), "lin")
    T = transport.Transport(prob, am)
    assert st.relres < 1e-12
    assert _rel(T.apply_A(psi), T.source()) < 1e-10
    ctx.close()


@pytest.mark.parametrize("mode", ["f64", "mixed"])
def test_non_finite_initial_guess_gives_nan_status(mode):
    from paper_2010_04559_gb300 import (AMGT_ERR_NAN, AMGT_MODE_F64, AMGT_MODE_MIXED,
                                        AMGT_PREC_MG, AmgtError)
    prob = W.random_problem(2, (6, 5), 2, 4, 62)
    prob["mg"] = dict(nlevels=2, Nr=[4, 2], nu_pre=1, nu_post=1, coarse_sweeps=10)
    ctx = _ctx(prob)
    ns, na = ctx.amgt_query_sizes(0)
    x0 = np.zeros((ns, na))
    x0[5, 7] = np.nan
    md = AMGT_MODE_F64 if mode == "f64" else AMGT_MODE_MIXED
    with pytest.raises(AmgtError) as e:
        ctx.amgt_solve(tol=1e-8, precond=AMGT_PREC_MG, mode=md, x0=x0)
    assert e.value.code == AMGT_ERR_NAN
    # the next solve from a finite guess converges
    _, _, st, _ = ctx.amgt_solve(tol=1e-8, precond=AMGT_PREC_MG, mode=md)
    assert st.relres < 1e-8
    ctx.close()


@pytest.mark.parametrize("mode", ["f64", "mixed"])
def test_iteration_cap_gives_not_converged(mode):
    from paper_2010_04559_gb300 import (AMGT_ERR_NOT_CONVERGED, AMGT_MODE_F64, AMGT_MODE_MIXED,
                                        AMGT_PREC_SWEEP)
    prob = W.random_problem(2, (8, 7), 1, 6, 63, g=0.9)
    prob["sigma_s"] = 0.98 * prob["sigma_t"]     # many sweep-preconditioned iterations
    ctx = _ctx(prob)
    md = AMGT_MODE_F64 if mode == "f64" else AMGT_MODE_MIXED
    _, _, st, rc = ctx.amgt_solve(tol=1e-12, maxit=2, precond=AMGT_PREC_SWEEP, mode=md,
                                  allow_not_converged=True)
    assert rc == AMGT_ERR_NOT_CONVERGED
    assert st.iterations <= 2 and st.relres > 1e-12
    ctx.close()


def test_device_wait_that_runs_out_is_reported_and_the_context_recovers():
    """Under AMGT_TUNE_TEST_SWEEP_HOLD the warp-pipelined sweep's first warp
    of each block never publishes its progress, so its neighbour's bounded
    wait gives up after 10 ms, every other wait returns at once, and the
    launch ends: amgt_sync reports AMGT_ERR_DEVICE_TIMEOUT.  With the key
    cleared the same context sweeps correctly again, and so does a new one."""
    from paper_2010_04559_gb300 import (AMGT_ERR_DEVICE_TIMEOUT, AMGT_TUNE_SWEEP_GROUP,
                                        AMGT_TUNE_SWEEP_KERNEL, AMGT_TUNE_TEST_SWEEP_HOLD,
                                        AmgtError)
    prob = W.random_problem(2, (20, 24), 2, 4, 64)
    am = angular.AngularMesh(angular.uniform_paths(2), "lin")
    T = transport.Transport(prob, am)
    x = W.random_vector((T.nsdof, T.nadof), 65)
    ref = T.sweep(x)
    ctx = _ctx(prob)
    # the warp-pipelined form: 4 patches per block, 8 rows per warp, 3 warps
    ctx.amgt_set_tuning(AMGT_TUNE_SWEEP_GROUP, 4)
    ctx.amgt_set_tuning(AMGT_TUNE_SWEEP_KERNEL, 2)
    xd = torch.from_numpy(x).to(device="cuda", dtype=torch.float32)
    yd = torch.empty_like(xd)
    ctx.amgt_set_tuning(AMGT_TUNE_TEST_SWEEP_HOLD, 1)
    ctx.amgt_op_sweep(0, xd, yd)
    with pytest.raises(AmgtError) as e:
        ctx.amgt_sync()
    assert e.value.code == AMGT_ERR_DEVICE_TIMEOUT
    ctx.amgt_set_tuning(AMGT_TUNE_TEST_SWEEP_HOLD, 0)
    ctx.amgt_op_sweep(0, xd, yd)
    ctx.amgt_sync()
    assert _rel(yd.double().cpu().numpy(), ref) < 2e-5
    ctx.close()
    ctx2 = _ctx(prob)
    ctx2.amgt_set_tuning(AMGT_TUNE_SWEEP_GROUP, 4)
    ctx2.amgt_set_tuning(AMGT_TUNE_SWEEP_KERNEL, 2)
    yd.zero_()
    ctx2.amgt_op_sweep(0, xd, yd)
    ctx2.amgt_sync()
    assert _rel(yd.double().cpu().numpy(), ref) < 2e-5
    ctx2.close()
