"""Benchmark of the transport hot path on GB300.

Workload: 2D 128x128 DG-Q1 quads, two-material checkerboard (sigma_t 1/10,
scatter ratio 0.5/0.99, seeded 16x16-cell tiles), angular level 3 (512 Lin
patches, 1536 angular DOF), HG g = 0.9 at Legendre order 16, centred unit
source, vacuum; 3-level angular multigrid V(1,1), coarse order 4, 10 coarse
Gauss-Seidel sweeps; 1.01e8 unknowns.

One step = one complete solve to ||b - A x|| / ||b|| < 1e-8 (mixed mode:
FP64 GMRES refinement around an FP32 flexible GMRES(20) whose V-cycle and
operator run the FP32 sweeps/transfers and the scatter contraction on BF16
tensor cores), i.e. every hot-path operator: sweep, scatter, operator apply,
restriction/prolongation, smoother, coarse Gauss-Seidel, GMRES and the scalar
flux.  value = unknowns x Krylov iterations / step time (GDOF/s of
preconditioned transport-operator applications); ms_per_step is the time to
residual 1e-8.

--impl reference times the CPU FP64 oracle instead (bounded sample, see
cpu_baseline.sample).  Multi-GPU: replicas only (the method has no data-path
exchange on one problem); each rank solves its own copy.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

WORKLOAD = "2D 128x128 Q1, checkerboard sigma_t 1/10 c 0.5/0.99, level-3 Lin (512 patches), HG g=0.9 N=16, 3-level MG Nr=4"
METRIC = "transport-operator GDOF/s; time-to-residual 1e-8, mixed/batched vs FP64 GPU"

KERNEL_NAMES = {
    "sweep": "sweep2d_warp_kernel<float,3,4,4,3>",
    "apply_L": "apply_L_kernel<float,2,3>",
    "scatter_prep": "tc_prep_kernel<4>",
    "scatter_tc": "tc_gemm_kernel (tcgen05, persistent)",
    "scatter_f32": "gemm_kernel<float>",
    "scatter_f64": "gemm_kernel<double>",
    "coarse_gs": "coarse_gs_rows_kernel<float,2,3>",
    "split_tc": "tc_gemm_kernel (tcgen05, slice products of the split FP64 scatter)",
    "split_aux": "split_rows_kernel + split_flush_kernel (digit slicing, FP64 accumulation)",
}
# DRAM bytes (read + write) per launch on this workload from the ncu captures
# summarised under profiles/; a kernel changed since its capture has no entry
TRAFFIC = {
    "sweep": 773.4e6,       # profiles/ncu_sweep_warp_config2.md
    "scatter_tc": 554.7e6,  # profiles/ncu_top_kernels_config2.md
    "coarse_gs": 243.8e6,   # profiles/ncu_coarse_gs_rows_config2.md (10-sweep launch)
}
NMOM_FINE = 289           # (N + 1)^2 Legendre moments at order 16
FP64_PEAK = 1.25          # TFLOP/s, nominal GB300 FP64 rate
PEAK_KINDS = {
    "alu": "FP32 FMA units x clock (152 x 128 x 2 x 2.07 GHz)",
    "alu64": "nominal GB300 FP64 rate, 1.25 TFLOP/s",
    "hbm": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
    "tensor": "measured BF16 GEMM burst (MEASURED_PEAKS.json bf16_tflops)",
}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p["hbm_gbs"], p["bf16_tflops"], "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, gpu):
        self.gpu = gpu
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx = float(r[1])
                for n, v in zip(names, r[3:7]):
                    if v.lower() == "active":
                        reasons.add(n)
            except Exception:
                continue
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sampler():
    """The oracle on a bounded sample of the workload: a 16x16-cell window
    (same angular mesh, order, materials and multigrid).  Returns a function
    timing one preconditioned GMRES iteration (one V-cycle plus one operator
    apply, FP64) and returning the cpu_baseline record; the set-up (tables,
    hierarchy) is done once, outside the timing."""
    from oracle import multigrid
    import multiprocessing
    prob = W.config2_checkerboard(n=16, block=16)
    H = multigrid.Hierarchy(prob)
    T = H.levels[0]
    f = T.source()
    dof = T.nsdof * T.nadof
    try:
        cores = len(os.sched_getaffinity(0))
    except Exception:
        cores = multiprocessing.cpu_count()

    def step():
        t0 = time.perf_counter()
        z = H.vcycle(f)
        _ = T.apply_A(z)
        dt = time.perf_counter() - t0
        return {"value": dof / dt / 1e9, "unit": "GDOF/s", "cores": cores, "kind": "oracle",
                "sample": (f"16x16-cell window of the 128x128 workload ({dof} unknowns, all 512 "
                           f"patches, N=16, 3-level MG): one V-cycle + one operator apply "
                           f"(= one preconditioned GMRES iteration) in {dt:.1f} s, NumPy FP64")}
    return step


def cpu_baseline():
    """One oracle sample (see oracle_sampler)."""
    return oracle_sampler()()


def max_over_ranks(x, dist, device="cpu"):
    """x on this rank -> max over the ranks of the process group (x itself
    without one); the job's time is its slowest rank's."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gdofs(world, unknowns, iterations, seconds):
    """Whole-job throughput: every rank solves its own replica of the
    workload, so the job's unknown-iterations are world times one rank's."""
    return world * unknowns * float(iterations) / seconds / 1e9


def run_reference(args, baseline=None):
    """The oracle (the method restated from the paper, NumPy FP64) on the
    host cores: W untimed warm-up samples, then K timed ones.  Under torchrun
    only rank 0 runs; the other ranks exit without work."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    baseline = baseline or oracle_sampler()
    for _ in range(max(0, args.warmup)):
        baseline()
    vals = []
    t0 = time.perf_counter()
    for _ in range(max(1, args.steps)):
        vals.append(baseline())
    t_step = (time.perf_counter() - t0) / max(1, args.steps)
    v = float(np.median([c["value"] for c in vals]))
    cb = dict(vals[0])
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GDOF/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + " (oracle sample: 16x16-cell window)"},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "GDOF/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_profile(args):
    """One mixed-precision solve, or one launch each of the sweep, the tensor-
    core scatter and one coarse Gauss-Seidel sweep, on the benchmark workload."""
    import torch
    from paper_2010_04559_gb300 import AMGT_MODE_MIXED, AMGT_PREC_MG, context_from_problem
    from paper_2010_04559_gb300 import build as _b
    _b.build()
    prob = W.config2_checkerboard(n=args.n)
    ctx = context_from_problem(prob, device=0)
    ns, na = ctx.amgt_query_sizes(0)
    if args.profile == "gs":
        # the coarse Gauss-Seidel launch of one V-cycle (10 sweeps), once to
        # warm up and once more
        nsc, nac = ctx.amgt_query_sizes(2)
        fc = torch.randn((nsc, nac), device="cuda", dtype=torch.float32)
        pc = torch.zeros_like(fc)
        for _ in range(2):
            ctx.amgt_op_coarse_gs(10, fc, pc)
        ctx.amgt_sync()
        print("kernels: coarse Gauss-Seidel, 10 sweeps (x2)")
    elif args.profile == "sweeps":
        from paper_2010_04559_gb300 import AMGT_TUNE_SWEEP_KERNEL
        x = torch.randn((ns, na), device="cuda", dtype=torch.float32)
        y = torch.empty_like(x)
        for _ in range(2):  # one warm-up launch of each variant, then one each
            for k in (1, 2):
                ctx.amgt_set_tuning(AMGT_TUNE_SWEEP_KERNEL, k)
                ctx.amgt_op_sweep(0, x, y)
        ctx.amgt_sync()
        print("kernels: level-synchronous row sweep, warp-pipelined sweep (x2)")
    elif args.profile == "solve":
        psi = torch.empty((ns, na), device="cuda", dtype=torch.float64)
        phi = torch.empty(ns, device="cuda", dtype=torch.float64)
        _, _, st, _ = ctx.amgt_solve(tol=1e-8, precond=AMGT_PREC_MG, mode=AMGT_MODE_MIXED,
                                     psi=psi, phi=phi, device_ptrs=True)
        print(f"solve: {st.iterations} iterations, relres {st.relres:.3e}")
    else:
        x = torch.randn((ns, na), device="cuda", dtype=torch.float32)
        y = torch.empty_like(x)
        nsc, nac = ctx.amgt_query_sizes(2)
        fc = torch.randn((nsc, nac), device="cuda", dtype=torch.float32)
        pc = torch.zeros_like(fc)
        ctx.amgt_op_sweep(0, x, y)
        ctx.amgt_op_scatter(0, x, y, tc=True)
        ctx.amgt_op_coarse_gs(1, fc, pc)
        x64 = x.double()
        ctx.amgt_op_scatter(0, x64, torch.empty_like(x64))
        ctx.amgt_op_scatter(0, x64, torch.empty_like(x64), tc=True)
        ctx.amgt_sync()
        print("kernels: sweep, tensor-core scatter, coarse Gauss-Seidel (1 sweep), FP64 scatter "
              "(SIMT, then split form)")
    torch.cuda.synchronize()
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=128, help="cells per axis")
    ap.add_argument("--fp64-ref", action="store_true", help="also time one FP64 GPU solve")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint timing")
    ap.add_argument("--batch", type=int, default=32,
                    help="problems of the uneven 2D batch solved concurrently (0: skip)")
    ap.add_argument("--inner-tol", type=float, default=0.0,
                    help="tolerance of each inner FP32 solve (0: adaptive)")
    ap.add_argument("--profile", choices=["solve", "kernels", "sweeps", "gs"], default=None,
                    help="run one solve, or one launch of each hot kernel, and exit (for ncu)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile:
        return run_profile(args)

    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if args.warmup < 3:
        print("warmup must be >= 3", file=sys.stderr)
        return 2

    import paper_2010_04559_gb300 as pkg
    from paper_2010_04559_gb300 import (AMGT_F32, AMGT_F32_BF16TC, AMGT_MODE_F64,
                                        AMGT_MODE_MIXED, AMGT_PREC_MG, AMGT_TUNE_KERNEL_TIMERS,
                                        amgt_query_launches, context_from_problem)
    kt_ids = {"sweep": pkg.AMGT_KT_SWEEP, "apply_L": pkg.AMGT_KT_APPLY_L,
              "scatter_prep": pkg.AMGT_KT_SCATTER_PREP, "scatter_tc": pkg.AMGT_KT_SCATTER_TC,
              "scatter_f32": pkg.AMGT_KT_SCATTER_F32, "scatter_f64": pkg.AMGT_KT_SCATTER_F64,
              "coarse_gs": pkg.AMGT_KT_COARSE_GS, "split_tc": pkg.AMGT_KT_SPLIT_TC,
              "split_aux": pkg.AMGT_KT_SPLIT_AUX}

    def kt_read(reset=True):
        return {k: ctx.amgt_query_kernel_time(i, reset=reset) for k, i in kt_ids.items()}
    from paper_2010_04559_gb300 import build as _b
    _b.build()
    stream = torch.cuda.Stream()
    prob = W.config2_checkerboard(n=args.n)
    ctx = context_from_problem(prob, device=local, stream=stream.cuda_stream)
    nsdof, nadof = ctx.amgt_query_sizes(0)
    dof = nsdof * nadof
    psi = torch.empty((nsdof, nadof), device="cuda", dtype=torch.float64)
    phi = torch.empty(nsdof, device="cuda", dtype=torch.float64)

    def solve():
        _, _, st, _ = ctx.amgt_solve(tol=1e-8, restart=20, maxit=400, precond=AMGT_PREC_MG,
                                     mode=AMGT_MODE_MIXED, psi=psi, phi=phi, device_ptrs=True,
                                     inner_tol=args.inner_tol, inner_maxit=200)
        return st

    for _ in range(args.warmup):
        st = solve()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    its = []
    outer = []
    relres = []
    l0 = amgt_query_launches()
    # the library records CUDA events on its stream around each launch of its
    # main kernels while the timers are on: per-kernel device time in the solve
    ctx.amgt_set_tuning(AMGT_TUNE_KERNEL_TIMERS, 1)
    kt_read()
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            st = solve()
            its.append(st.iterations)
            outer.append(st.outer_iterations)
            relres.append(st.relres)
        e1.record(stream)
        torch.cuda.synchronize()
    launches = amgt_query_launches() - l0
    elapsed = e0.elapsed_time(e1) / 1e3
    kt_solve = kt_read()
    ctx.amgt_set_tuning(AMGT_TUNE_KERNEL_TIMERS, 0)
    elapsed = max_over_ranks(elapsed, dist, "cuda")
    ms = elapsed / args.steps * 1e3
    value = job_gdofs(world, dof, np.sum(its), elapsed)

    # ---- end to end through the public API with host buffers
    qsrc = np.ascontiguousarray(prob["q"])
    psi_h = torch.empty((nsdof, nadof), dtype=torch.float64, pin_memory=True).numpy()
    phi_h = torch.empty(nsdof, dtype=torch.float64, pin_memory=True).numpy()
    e2e_its = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.amgt_set_source_iso(qsrc)
        _, _, st2, _ = ctx.amgt_solve(tol=1e-8, restart=20, maxit=400, precond=AMGT_PREC_MG,
                                      mode=AMGT_MODE_MIXED, psi=psi_h, phi=phi_h,
                                      inner_tol=args.inner_tol, inner_maxit=200)
        e2e_its += st2.iterations
    e2e_t = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e = {"value": job_gdofs(world, dof, e2e_its, e2e_t), "unit": "GDOF/s",
           "h2d_bytes_per_step": int(qsrc.nbytes),
           "d2h_bytes_per_step": int(psi_h.nbytes + phi_h.nbytes)}

    # ---- per-kernel roofline, timed with events on the library's stream
    hbm, bf16, peak_kind = _peaks()
    kern = {}
    x32 = torch.randn((nsdof, nadof), device="cuda", dtype=torch.float32)
    y32 = torch.empty_like(x32)
    nsc, nac = ctx.amgt_query_sizes(2)
    fc = torch.randn((nsc, nac), device="cuda", dtype=torch.float32)
    pc = torch.zeros_like(fc)
    with torch.cuda.stream(stream):
        def timeit(fn, reps=10):
            for _ in range(2):
                fn()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            ctx.amgt_set_tuning(AMGT_TUNE_KERNEL_TIMERS, 1)
            kt_read()
            a.record(stream)
            for _ in range(reps):
                fn()
            b.record(stream)
            torch.cuda.synchronize()
            k = kt_read()
            ctx.amgt_set_tuning(AMGT_TUNE_KERNEL_TIMERS, 0)
            # seconds per call, and per kernel class: seconds per launch
            per = {n: (v[0] / 1e3 / v[1]) for n, v in k.items() if v[1] > 0}
            return a.elapsed_time(b) / reps / 1e3, per
        t_sweep, k_sw = timeit(lambda: ctx.amgt_op_sweep(0, x32, y32))
        kern["sweep_f32"] = {"s": t_sweep, "GB/s": 8.0 * dof / k_sw["sweep"] / 1e9}
        use_tc = True
        try:
            t_sc, k_sc = timeit(lambda: ctx.amgt_op_scatter(0, x32, y32, tc=True))
            kern["scatter_bf16tc"] = {"s": t_sc, "gemm_s": k_sc["scatter_tc"],
                                      "prep_s": k_sc["scatter_prep"],
                                      "gemm_TFLOP/s": 2.0 * nsdof * nadof * nadof / k_sc["scatter_tc"] / 1e12}
        except Exception as ex:
            use_tc = False
            t_sc, k_sc = timeit(lambda: ctx.amgt_op_scatter(0, x32, y32))
            kern["scatter_f32"] = {"s": t_sc, "note": str(ex)[:80]}
        x64 = x32.double()
        y64 = torch.empty_like(x64)
        t_sp, k_sp = timeit(lambda: ctx.amgt_op_scatter(0, x64, y64, tc=True), reps=3)
        if k_sp.get("split_tc"):
            kern["scatter_f64_split"] = {"s": t_sp, "gemm_s_per_launch": k_sp["split_tc"],
                                         "gemm_TFLOP/s": 2.0 * nsdof * nadof * nadof / k_sp["split_tc"] / 1e12}
        t_64, k_64 = timeit(lambda: ctx.amgt_op_scatter(0, x64, y64), reps=2)
        kern["scatter_f64_simt"] = {"s": t_64}
        del x64, y64
        t_L, k_L = timeit(lambda: ctx.amgt_op_apply_L(0, x32, y32))
        kern["apply_L_f32"] = {"s": t_L, "GB/s": 8.0 * dof / k_L["apply_L"] / 1e9}
        t_gs, k_gs = timeit(lambda: ctx.amgt_op_coarse_gs(10, fc, pc), reps=3)
        kern["coarse_gs_f32_10sweeps"] = {"s": t_gs, "kernel_s": k_gs["coarse_gs"]}
        t_v, _ = timeit(lambda: ctx.amgt_op_vcycle(x32, y32, tc=use_tc), reps=3)
        kern["vcycle_bf16tc" if use_tc else "vcycle_f32"] = {"s": t_v}
    # FP32 ALU peak from unit counts and clock: 152 SMs x 128 FMA/clk x 2 x 2.07 GHz
    alu_peak = 152 * 128 * 2 * 2.07e9 / 1e12
    # coarse Gauss-Seidel algorithmic work: per cell, per sweep direction and
    # per sweep, the sequential per-patch form of the block solves
    # (moments source s*a*nm, self-scatter s*a*a, mass mix s*a*s, block solve
    # (s*a)^2, moment update s*nm*a per patch) -> 2 flop per FMA
    nsc_cells = nsc // 4
    npd = nac // 3 // 4
    nm = 25
    per_patch = 4 * 3 * nm + 4 * 3 * 3 + 4 * 3 * 4 + (4 * 3) ** 2 + 4 * nm * 3
    gs_flop = 2.0 * per_patch * npd * 4 * nsc_cells * 10
    gs_alg = f"{gs_flop/1e9:.2f} GFLOP per launch of 10 sweeps (sequential per-patch form)"
    tc_flop = 2.0 * nsdof * nadof * nadof
    # work per launch of each kernel class on the benchmark workload
    work = {
        "sweep": ("hbm", 8.0 * dof / 1e9, hbm, "GB/s", "8 B per unknown (read b, write psi, FP32)"),
        "apply_L": ("hbm", 8.0 * dof / 1e9, hbm, "GB/s", "8 B per unknown (read x, write y, FP32)"),
        "scatter_prep": ("hbm", 6.0 * dof / 1e9, hbm, "GB/s",
                         "6 B per unknown (read FP32 x, write BF16 operand)"),
        "scatter_tc": ("tensor", tc_flop / 1e12, bf16, "TFLOP/s", "2 Nsdof Nadof^2 flop (dense S_f, BF16)"),
        "coarse_gs": ("alu", gs_flop / 1e12, alu_peak, "TFLOP/s", gs_alg),
        # FP64 moment form of the scatter in each refinement residual:
        # Phi = psi X and Y = Phi (F X^T), 2 Nsdof Nadof nmom flop each
        "scatter_f64": ("alu", 4.0 * nsdof * nadof * NMOM_FINE / 1e12, FP64_PEAK, "TFLOP/s",
                        "4 Nsdof Nadof nmom flop per residual (two FP64 GEMMs, nmom = 289)"),
        "scatter_f32": ("alu", 4.0 * nsdof * nadof * NMOM_FINE / 1e12, alu_peak, "TFLOP/s",
                        "4 Nsdof Nadof nmom flop per apply (two FP32 GEMMs, nmom = 289)"),
        # one slice-pair product of the split FP64 scatter per launch
        "split_tc": ("tensor", tc_flop / 1e12, bf16, "TFLOP/s",
                     "2 Nsdof Nadof^2 flop per slice-pair GEMM (BF16 digits, dense S_f)"),
    }
    rl = {}
    for name, per_launch in (("sweep", k_sw.get("sweep")), ("apply_L", k_L.get("apply_L")),
                             ("scatter_prep", k_sc.get("scatter_prep")),
                             ("scatter_tc", k_sc.get("scatter_tc")),
                             ("split_tc", k_sp.get("split_tc")),
                             ("coarse_gs", k_gs.get("coarse_gs"))):
        if not per_launch:
            continue
        bound, w, peak, unit, alg = work[name]
        rl[name] = {"kernel": KERNEL_NAMES[name], "bound": bound, "achieved": w / per_launch,
                    "peak": peak, "unit": unit, "frac": w / per_launch / peak,
                    "launch_s": per_launch, "traffic": TRAFFIC.get(name), "algorithmic": alg}
    # in-solve device time per kernel class (timed region, library events)
    solve_k = {}
    for name, (msum, n) in kt_solve.items():
        if n > 0:
            solve_k[name] = {"ms_per_step": msum / args.steps, "launches_per_step": n / args.steps,
                             "share": msum / 1e3 / elapsed}
    dom_name = max(solve_k, key=lambda k: solve_k[k]["share"]) if solve_k else "coarse_gs"
    if dom_name in work:
        bound, w, peak, unit, alg = work[dom_name]
        msum, n = kt_solve[dom_name]
        per_launch = msum / 1e3 / n
        roof = {"kernel": KERNEL_NAMES[dom_name], "bound": bound, "achieved": w / per_launch,
                "peak": peak, "unit": unit, "frac": w / per_launch / peak,
                "traffic": TRAFFIC.get(dom_name), "share_of_solve": solve_k[dom_name]["share"],
                "peak_kind": PEAK_KINDS["alu64"] if dom_name == "scatter_f64"
                else PEAK_KINDS.get(bound, peak_kind), "algorithmic": alg}
    else:
        roof = {"kernel": dom_name, "bound": None, "achieved": None, "peak": None,
                "unit": None, "frac": None, "traffic": None,
                "share_of_solve": solve_k[dom_name]["share"]}

    # ---- adjoint: lambda = A^-T g for the flux integral over a 16x16-cell
    # corner block, then the response and its gradients (mixed solve to 1e-8)
    adj = None
    if not args.no_adjoint:
        from paper_2010_04559_gb300.adjoint import response_problem
        nx = args.n
        weight = np.zeros(nx * nx)
        for iy in range(16):
            weight[iy * nx:iy * nx + 16] = 1.0
        actx = context_from_problem(response_problem(prob, weight), device=local,
                                    stream=stream.cuda_stream)
        actx.amgt_set_adjoint(1)
        lam = torch.empty_like(psi)
        C = nx * nx
        dt = torch.empty(C, device="cuda", dtype=torch.float64)
        ds = torch.empty_like(dt)
        df = torch.empty(prob["N"] + 1, device="cuda", dtype=torch.float64)

        def adjoint_step():
            _, _, sta, _ = actx.amgt_solve(tol=1e-8, restart=20, maxit=400, precond=AMGT_PREC_MG,
                                           mode=AMGT_MODE_MIXED, psi=lam, phi=phi,
                                           device_ptrs=True, inner_tol=args.inner_tol)
            R = actx.amgt_response(psi)
            ctx.amgt_response_gradients(psi, lam, dt, ds, df)
            return sta, R
        solve()                     # psi of the forward problem
        adjoint_step()              # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sta, R = adjoint_step()
        torch.cuda.synchronize()
        t_adj = time.perf_counter() - t0
        t0 = time.perf_counter()
        ctx.amgt_response_gradients(psi, lam, dt, ds, df)
        t_grad = time.perf_counter() - t0
        adj = {"workload": "flux integral over the 16x16-cell corner block; dR/dsigma_t, "
                           "dR/dsigma_s per cell and dR/df_n (N=16)",
               "adjoint_solve_and_gradients_s": t_adj, "gradients_s": t_grad,
               "iterations": sta.iterations, "relres": sta.relres, "response": R}
        actx.close()

    # ---- batched: the first problems of the 256-problem batch of uneven 2D
    # problems, each on its own context and stream, autotuned, V-cycles
    # replayed from captured graphs, solved concurrently (mixed, 1e-8)
    batch = None
    if args.batch > 0:
        from paper_2010_04559_gb300 import AMGT_TUNE_GRAPHS, amgt_solve_batch
        probs = W.config4_batch()[:args.batch]
        bstreams = [torch.cuda.Stream() for _ in probs]
        bctx = [context_from_problem(p, device=local, stream=s.cuda_stream)
                for p, s in zip(probs, bstreams)]
        t0 = time.perf_counter()
        tunes = [c.amgt_autotune(3) for c in bctx]
        t_tune = time.perf_counter() - t0
        for c in bctx:
            c.amgt_set_tuning(AMGT_TUNE_GRAPHS, 1)
        bpsi = [torch.empty(c.amgt_query_sizes(0), device="cuda", dtype=torch.float64)
                for c in bctx]
        bdof = [int(np.prod(c.amgt_query_sizes(0))) for c in bctx]
        amgt_solve_batch(bctx, bpsi, tol=1e-8)  # warm-up: captures the graphs
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bst = amgt_solve_batch(bctx, bpsi, tol=1e-8)
        torch.cuda.synchronize()
        t_batch = time.perf_counter() - t0
        t0 = time.perf_counter()
        for c, p in zip(bctx, bpsi):
            c.amgt_solve(tol=1e-8, precond=AMGT_PREC_MG, mode=AMGT_MODE_MIXED, psi=p,
                         phi=None, device_ptrs=True)
        torch.cuda.synchronize()
        t_seq = time.perf_counter() - t0
        dof_its = sum(d * st.iterations for d, st in zip(bdof, bst))
        batch = {"workload": f"first {len(probs)} problems of the 256-problem batch (2D, n in "
                             f"16..96, level 1..3, per-cell lognormal sigma_t, N = 2 level + 4)",
                 "problems": len(probs), "unknowns": sum(bdof),
                 "value": dof_its / t_batch / 1e9, "unit": "GDOF/s",
                 "time_to_tol_s": t_batch, "sequential_time_to_tol_s": t_seq,
                 "max_relres": max(st.relres for st in bst),
                 "iterations": [st.iterations for st in bst], "autotune_s": t_tune,
                 "tuned": [list(t[:3]) for t in tunes]}
        for c in bctx:
            c.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            cpu = cpu_baseline()
        except Exception as ex:
            cpu = {"error": str(ex)[:200]}
    fp64 = None
    if args.fp64_ref:
        t0 = time.perf_counter()
        _, _, st3, _ = ctx.amgt_solve(tol=1e-8, restart=20, maxit=400, precond=AMGT_PREC_MG,
                                      mode=AMGT_MODE_F64, psi=psi, phi=phi, device_ptrs=True,
                                      allow_not_converged=True)
        fp64 = {"time_to_tol_s": time.perf_counter() - t0, "iterations": st3.iterations,
                "relres": st3.relres}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32/bf16 (f64 refinement)", "data": "synthetic",
                "config": {"workload": WORKLOAD if args.n == 128 else WORKLOAD.replace("128x128", f"{args.n}x{args.n}"),
                           "unknowns": dof, "mode": "mixed", "precond": "MG V(1,1)",
                           "tol": 1e-8, "inner_tol": args.inner_tol if args.inner_tol > 0 else "adaptive",
                           "l2": "inputs larger than L2 (0.4-0.8 GB per vector)",
                           "parallelism": f"replicas x{world}"},
                "time_to_tol_s": ms / 1e3, "krylov_iterations": its, "refinement_steps": outer, "relres": relres,
                "gpu_launches": int(launches), "roofline": roof, "rooflines": rl,
                "solve_kernels": solve_k, "kernels": kern,
                "clocks": clk.summary(), "e2e": e2e, "cpu_baseline": cpu}
        if fp64:
            line["fp64_gpu"] = fp64
        if adj:
            line["adjoint"] = adj
        if batch:
            line["batched"] = batch
        print(json.dumps(line))
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
