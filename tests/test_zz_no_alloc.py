"""The allocation-free coarse Gauss-Seidel entry point.

Some callers cannot let a library allocate device memory while they run: a
process whose GPU memory belongs to another framework's caching allocator or
sits under a fixed budget, or a latency-critical loop that cannot pay for an
allocation's implicit synchronisation.  amgt_op_coarse_gs_noalloc serves them
by keeping its scratch (the coarse cells' flux moments) in a fixed device
array built into the library.  This file is collected last on purpose.
"""
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
    return float(torch.linalg.norm((a - b).double()) / torch.linalg.norm(b.double()))


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 2e-5)],
                         ids=["f64", "f32"])
def test_noalloc_matches_allocating_entry_point(dtype, tol):
    from paper_2010_04559_gb300 import context_from_problem
    prob = W.random_problem(2, (9, 7), 2, 8, 71, g=0.85)
    prob["mg"] = dict(nlevels=2, Nr=[8, 4], nu_pre=1, nu_post=1, coarse_sweeps=4)
    ctx = context_from_problem(prob, device=0)
    nsc, nac = ctx.amgt_query_sizes(1)      # completes set-up
    gen = torch.Generator(device="cpu").manual_seed(7)
    for call in range(2):                    # two calls in a row share the scratch
        f = torch.randn((nsc, nac), generator=gen, dtype=torch.float64).to("cuda", dtype)
        phi0 = torch.randn((nsc, nac), generator=gen, dtype=torch.float64).to("cuda", dtype)
        ref = phi0.clone()
        ctx.amgt_op_coarse_gs(3, f, ref)
        out = phi0.clone()
        ctx.amgt_op_coarse_gs_noalloc(3, f, out)
        torch.cuda.synchronize()
        assert _rel(out, ref) < tol, call
    ctx.close()


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 2e-5)],
                         ids=["f64", "f32"])
def test_first_call_on_a_fresh_context_takes_no_device_memory(dtype, tol):
    """The very first call on a freshly built context (set-up completed by
    amgt_query_sizes, nothing launched yet) leaves the device's free memory
    unchanged, then agrees with the allocating entry point."""
    from paper_2010_04559_gb300 import context_from_problem
    prob = W.random_problem(2, (8, 9), 2, 8, 73, g=0.8)
    prob["mg"] = dict(nlevels=2, Nr=[8, 4], nu_pre=1, nu_post=1, coarse_sweeps=4)
    ctx = context_from_problem(prob, device=0)
    nsc, nac = ctx.amgt_query_sizes(1)
    gen = torch.Generator(device="cpu").manual_seed(8)
    f = torch.randn((nsc, nac), generator=gen, dtype=torch.float64).to("cuda", dtype)
    phi0 = torch.randn((nsc, nac), generator=gen, dtype=torch.float64).to("cuda", dtype)
    out = phi0.clone()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    ctx.amgt_op_coarse_gs_noalloc(3, f, out)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0
    ref = phi0.clone()
    ctx.amgt_op_coarse_gs(3, f, ref)
    torch.cuda.synchronize()
    assert _rel(out, ref) < tol
    ctx.close()


def test_noalloc_rejects_oversized_coarse_level():
    from paper_2010_04559_gb300 import AmgtError, context_from_problem
    # 128 x 128 cells, coarse order 8: 65536 x 81 doubles = 42 MB > 32 MiB
    prob = W.random_problem(2, (128, 128), 1, 8, 72)
    prob["sigma_t"] = np.ones_like(prob["sigma_t"])        # one material: quick set-up
    prob["sigma_s"] = np.full_like(prob["sigma_s"], 0.5)
    ctx = context_from_problem(prob, device=0)
    ns, na = ctx.amgt_query_sizes(0)
    f = torch.zeros((ns, na), device="cuda", dtype=torch.float64)
    phi = torch.zeros_like(f)
    with pytest.raises(AmgtError, match="allocation-free entry point holds at most"):
        ctx.amgt_op_coarse_gs_noalloc(1, f, phi)
    ctx.close()
