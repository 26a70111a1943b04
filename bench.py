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


def cpu_baseline(seconds_cap=60.0):
    """Oracle timed on a bounded sample: a 16x16-cell window of the workload
    (same angular mesh, order, materials and multigrid), one preconditioned
    GMRES iteration = one V-cycle plus one operator apply, FP64."""
    from oracle import multigrid
    import multiprocessing
    prob = W.config2_checkerboard(n=16, block=16)
    H = multigrid.Hierarchy(prob)
    T = H.levels[0]
    f = T.source()
    t0 = time.perf_counter()
    z = H.vcycle(f)
    _ = T.apply_A(z)
    dt = time.perf_counter() - t0
    dof = T.nsdof * T.nadof
    try:
        cores = len(os.sched_getaffinity(0))
    except Exception:
        cores = multiprocessing.cpu_count()
    return {"value": dof / dt / 1e9, "unit": "GDOF/s", "cores": cores, "kind": "oracle",
            "sample": (f"16x16-cell window of the 128x128 workload ({dof} unknowns, all 512 "
                       f"patches, N=16, 3-level MG): one V-cycle + one operator apply "
                       f"(= one preconditioned GMRES iteration) in {dt:.1f} s, NumPy FP64")}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    for _ in range(args.warmup if args.warmup < 1 else 0):
        pass
    vals = []
    for _ in range(max(1, args.steps)):
        vals.append(cpu_baseline())
    v = float(np.median([c["value"] for c in vals]))
    cb = dict(vals[0])
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GDOF/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
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
    if args.profile == "solve":
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
        ctx.amgt_sync()
        print("kernels: sweep, tensor-core scatter, coarse Gauss-Seidel (1 sweep)")
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
    ap.add_argument("--profile", choices=["solve", "kernels"], default=None,
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

    from paper_2010_04559_gb300 import (AMGT_F32, AMGT_F32_BF16TC, AMGT_MODE_F64,
                                        AMGT_MODE_MIXED, AMGT_PREC_MG, amgt_query_launches,
                                        context_from_problem)
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
                                     inner_tol=1e-4, inner_maxit=200)
        return st

    for _ in range(args.warmup):
        st = solve()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    its = []
    relres = []
    l0 = amgt_query_launches()
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            st = solve()
            its.append(st.iterations)
            relres.append(st.relres)
        e1.record(stream)
        torch.cuda.synchronize()
    launches = amgt_query_launches() - l0
    elapsed = e0.elapsed_time(e1) / 1e3
    if dist:
        t = torch.tensor([elapsed], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed = float(t.item())
    ms = elapsed / args.steps * 1e3
    value = world * dof * float(np.sum(its)) / elapsed / 1e9

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
                                      inner_tol=1e-4, inner_maxit=200)
        e2e_its += st2.iterations
    e2e_t = time.perf_counter() - t0
    e2e = {"value": world * dof * e2e_its / e2e_t / 1e9, "unit": "GDOF/s",
           "h2d_bytes_per_step": int(qsrc.nbytes),
           "d2h_bytes_per_step": int(psi_h.nbytes + phi_h.nbytes)}

    # ---- per-kernel roofline, timed with events on the library's stream
    hbm, bf16, peak_kind = _peaks()
    kern = {}
    x32 = torch.randn((nsdof, nadof), device="cuda", dtype=torch.float32)
    y32 = torch.empty_like(x32)
    with torch.cuda.stream(stream):
        def timeit(fn, reps=10):
            for _ in range(2):
                fn()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                fn()
            b.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(b) / reps / 1e3
        t_sweep = timeit(lambda: ctx.amgt_op_sweep(0, x32, y32))
        kern["sweep_f32"] = {"s": t_sweep, "GB/s": 8.0 * dof / t_sweep / 1e9}
        use_tc = True
        try:
            t_sc = timeit(lambda: ctx.amgt_op_scatter(0, x32, y32, tc=True))
            kern["scatter_bf16tc"] = {"s": t_sc, "TFLOP/s": 2.0 * nsdof * nadof * nadof / t_sc / 1e12}
        except Exception as ex:
            use_tc = False
            t_sc = timeit(lambda: ctx.amgt_op_scatter(0, x32, y32))
            kern["scatter_f32"] = {"s": t_sc, "note": str(ex)[:80]}
        t_L = timeit(lambda: ctx.amgt_op_apply_L(0, x32, y32))
        kern["apply_L_f32"] = {"s": t_L, "GB/s": 8.0 * dof / t_L / 1e9}
        nsc, nac = ctx.amgt_query_sizes(2)
        fc = torch.randn((nsc, nac), device="cuda", dtype=torch.float32)
        pc = torch.zeros_like(fc)
        t_gs = timeit(lambda: ctx.amgt_op_coarse_gs(10, fc, pc), reps=2)
        kern["coarse_gs_f32_10sweeps"] = {"s": t_gs}
        t_v = timeit(lambda: ctx.amgt_op_vcycle(x32, y32, tc=use_tc), reps=3)
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
    rl = {
        "sweep": {"kernel": "sweep2d_rows_kernel<float,3,4>", "bound": "hbm",
                  "achieved": 8.0 * dof / t_sweep / 1e9, "peak": hbm, "unit": "GB/s",
                  "algorithmic": "8 B per unknown (read b, write psi, FP32)"},
        "apply_L": {"kernel": "apply_L_kernel<float,2,3>", "bound": "hbm",
                    "achieved": 8.0 * dof / t_L / 1e9, "peak": hbm, "unit": "GB/s",
                    "algorithmic": "8 B per unknown (read x, write y, FP32)"},
        "coarse_gs": {"kernel": "coarse_gs_group_kernel<float,2,3>", "bound": "alu",
                      "achieved": gs_flop / t_gs / 1e12, "peak": alu_peak, "unit": "TFLOP/s",
                      "algorithmic": f"{gs_flop/1e9:.2f} GFLOP per 10 sweeps (sequential per-patch form)"},
    }
    if use_tc:
        rl["scatter"] = {"kernel": "tc_prep_kernel + tc_gemm_kernel (tcgen05)", "bound": "tensor",
                         "achieved": 2.0 * nsdof * nadof * nadof / t_sc / 1e12, "peak": bf16,
                         "unit": "TFLOP/s", "algorithmic": "2 Nsdof Nadof^2 flop (dense S_f)"}
    for v in rl.values():
        v["frac"] = v["achieved"] / v["peak"]
    # dominant kernel by its share of one solve (launch list: coarse Gauss-Seidel)
    dom = dict(rl["coarse_gs"])
    roof = {"kernel": dom["kernel"], "bound": dom["bound"], "achieved": dom["achieved"],
            "peak": dom["peak"], "unit": dom["unit"], "frac": dom["frac"], "traffic": None,
            "peak_kind": "FP32 FMA units x clock (152 x 128 x 2 x 2.07 GHz)",
            "algorithmic": dom["algorithmic"]}

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
                           "tol": 1e-8, "l2": "inputs larger than L2 (0.4-0.8 GB per vector)",
                           "parallelism": f"replicas x{world}"},
                "time_to_tol_s": ms / 1e3, "krylov_iterations": its, "relres": relres,
                "gpu_launches": int(launches), "roofline": roof, "rooflines": rl, "kernels": kern,
                "clocks": clk.summary(), "e2e": e2e, "cpu_baseline": cpu}
        if fp64:
            line["fp64_gpu"] = fp64
        print(json.dumps(line))
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
