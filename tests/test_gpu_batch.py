"""Batched solves of independent problems of uneven size (one context and one
stream each, solved concurrently), the V-cycle replayed from a captured CUDA
graph, and the autotuner: each must leave the answers unchanged."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_04559_gb300 import build
    build.build()


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def _solve(ctx, **kw):
    from paper_2010_04559_gb300 import AMGT_MODE_MIXED, AMGT_PREC_MG
    ns, na = ctx.amgt_query_sizes(0)
    psi = torch.empty((ns, na), device="cuda", dtype=torch.float64)
    phi = torch.empty(ns, device="cuda", dtype=torch.float64)
    opts = dict(tol=1e-11, precond=AMGT_PREC_MG, mode=AMGT_MODE_MIXED)
    opts.update(kw)
    _, _, st, _ = ctx.amgt_solve(psi=psi, phi=phi, device_ptrs=True, **opts)
    torch.cuda.synchronize()
    return psi, st


def test_batch_matches_individual_solves():
    from paper_2010_04559_gb300 import amgt_solve_batch, context_from_problem
    probs = W.config4_batch(nprob=6, nmin=8, nmax=20, seed_k=41)
    streams = [torch.cuda.Stream() for _ in probs]
    ctxs = [context_from_problem(p, device=0, stream=s.cuda_stream) for p, s in zip(probs, streams)]
    refs = [_solve(c)[0] for c in ctxs]
    psis = [torch.empty_like(r) for r in refs]
    stats = amgt_solve_batch(ctxs, psis, tol=1e-11)
    torch.cuda.synchronize()
    for r, p, st in zip(refs, psis, stats):
        assert st.relres < 1e-11
        assert _rel(p, r) < 1e-8
    for c in ctxs:
        c.close()


def test_concurrent_setup_matches_lazy_setup():
    """amgt_setup_batch builds the contexts' tables on host threads at once;
    the solves that follow equal those of contexts set up one by one at
    their first use (same tables, same kernels)."""
    from paper_2010_04559_gb300 import amgt_setup_batch, context_from_problem
    probs = W.config4_batch(nprob=6, nmin=8, nmax=20, seed_k=43)
    streams = [torch.cuda.Stream() for _ in probs]
    lazy = [context_from_problem(p, device=0, stream=s.cuda_stream) for p, s in zip(probs, streams)]
    refs = [_solve(c)[0] for c in lazy]
    for c in lazy:
        c.close()
    ctxs = [context_from_problem(p, device=0, stream=s.cuda_stream) for p, s in zip(probs, streams)]
    amgt_setup_batch(ctxs, nthreads=4)
    for c, r in zip(ctxs, refs):
        psi, st = _solve(c)
        assert st.relres < 1e-11
        assert _rel(psi, r) < 1e-12
    for c in ctxs:
        c.close()


def test_graph_replayed_vcycle_gives_the_same_solve():
    from paper_2010_04559_gb300 import AMGT_TUNE_GRAPHS, context_from_problem
    prob = W.config4_batch(nprob=1, nmin=24, nmax=24, seed_k=42)[0]
    stream = torch.cuda.Stream()  # the default stream cannot be captured
    ctx = context_from_problem(prob, device=0, stream=stream.cuda_stream)
    ref, st0 = _solve(ctx)
    ctx.amgt_set_tuning(AMGT_TUNE_GRAPHS, 1)
    for _ in range(2):  # the first solve captures, the second replays
        psi, st = _solve(ctx)
        assert st.iterations == st0.iterations
        assert _rel(psi, ref) < 1e-12
    ctx.close()


def test_autotune_keeps_the_answer_and_caches():
    from paper_2010_04559_gb300 import context_from_problem
    prob = W.config4_batch(nprob=1, nmin=32, nmax=32, seed_k=43)[0]
    ctx = context_from_problem(prob, device=0)
    ref, _ = _solve(ctx)
    G, stages, gs, cached = ctx.amgt_autotune(3)
    assert G in (1, 2, 4, 8) and stages in (0, 2, 3, 4, 6) and gs in (0, 1, 2, 3, 6)
    psi, st = _solve(ctx)
    assert st.relres < 1e-11 and _rel(psi, ref) < 1e-8
    ctx2 = context_from_problem(prob, device=0)
    assert ctx2.amgt_autotune(3) == (G, stages, gs, 1)
    ctx.close()
    ctx2.close()


def test_batch_members_match_the_oracle():
    """Members of the 256-problem batch (n = 16..22 cells per axis, angular
    levels 1-3, per-cell sigma_t, their own g and order) solved together by
    amgt_solve_batch (mixed precision, autotuned, graph-replayed V-cycles),
    each against the oracle's solution of the same problem (GMRES with the
    sweep preconditioner to 1e-12: the solution does not depend on the
    preconditioner)."""
    from oracle import angular, gmres, transport
    from paper_2010_04559_gb300 import (AMGT_TUNE_GRAPHS, amgt_solve_batch,
                                        context_from_problem)
    allp = W.config4_batch()
    picks = [75, 95, 141, 18]                  # levels 1, 1, 3, 3; n = 19, 22, 16, 19
    probs = [allp[i] for i in picks]
    streams = [torch.cuda.Stream() for _ in probs]
    ctxs = [context_from_problem(p, device=0, stream=s.cuda_stream)
            for p, s in zip(probs, streams)]
    for c in ctxs:
        c.amgt_autotune(3)
        c.amgt_set_tuning(AMGT_TUNE_GRAPHS, 1)
    psis = [torch.empty(c.amgt_query_sizes(0), device="cuda", dtype=torch.float64) for c in ctxs]
    for _ in range(2):                         # the first solve captures the graphs
        stats = amgt_solve_batch(ctxs, psis, tol=1e-11)
    torch.cuda.synchronize()
    for p, psi, st in zip(probs, psis, stats):
        assert st.relres < 1e-11
        T = transport.Transport(p, angular.AngularMesh(angular.uniform_paths(p["level"]), "lin"))
        xo, _, _, rel = gmres.gmres(T.apply_A, T.source(), T.sweep, 1e-12, 30, 3000)
        assert rel < 1e-12
        assert np.linalg.norm(psi.cpu().numpy() - xo) / np.linalg.norm(xo) < 1e-6
    for c in ctxs:
        c.close()
