"""Benchmark of the transport hot path on GB300.

Headline workload (the largest configuration that fits one GPU): 2D 256x256
DG-Q1 quads, sigma_t = 5, sigma_s = 4.95, Henyey-Greenstein g = 0.98 at
Legendre order 64, a normally incident pencil beam of unit strength on the
low-x edge, vacuum elsewhere, uniform angular level 4 (2048 Lin patches, 6144
angular DOF), 4-level angular multigrid V(1,1) with coarse scatter order 12
and 10 coarse Gauss-Seidel sweeps: 1.61e9 unknowns.

One step = one complete mixed-precision solve to ||b - A x|| / ||b|| < 1e-8:
FP64 GMRES refinement around an FP32 flexible GMRES(8) whose operator takes
the FP32-accurate FP16 three-product scatter and whose V-cycle runs FP32
sweeps/transfers, the BF16 tensor-core scatter and the coarse Gauss-Seidel;
the refinement residuals take the FP64-accurate split scatter.  Every
hot-path operator runs in it: sweep, scatter, operator apply, restriction /
prolongation, smoother, coarse Gauss-Seidel, GMRES and the scalar flux.
value = unknowns x Krylov iterations / step time (GDOF/s of preconditioned
transport-operator applications); ms_per_step is the time to residual 1e-8.
The timed steps run with the library's kernel timers off and the V-cycle
replayed from a captured CUDA graph; a separate instrumented solve gives the
per-kernel shares and the rooflines.  fp64_gpu times the plain FP64 GPU solve
of the same inputs (BiCGStab, the paper's Krylov method, whose FP64 basis
fits in memory at this size; every FP64 scatter in the split form).  The
128x128 two-material checkerboard workload (1.01e8 unknowns) is timed the
same way under extra.config2.

--impl reference times the CPU FP64 oracle instead (bounded sample, see
cpu_baseline.sample).  Multi-GPU: replicas only (the method has no data-path
exchange on one problem); each rank solves its own copy.
"""
import argparse
import json
import multiprocessing
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

WORKLOAD = ("2D 256x256 Q1, sigma_t 5 sigma_s 4.95, HG g=0.98 N=64, normally incident pencil "
            "beam on the low-x edge, uniform level-4 Lin (2048 patches), 4-level MG Nr=12")
WORKLOAD2 = ("2D 128x128 Q1, checkerboard sigma_t 1/10 c 0.5/0.99, level-3 Lin (512 patches), "
             "HG g=0.9 N=16, 3-level MG Nr=4")
METRIC = "transport-operator GDOF/s; time-to-residual 1e-8, mixed/batched vs FP64 GPU"
HEAD_RESTART = 8   # FGMRES(8): 17 FP32 basis vectors of 6.4 GB each at 1.61e9 unknowns

# kernel class -> (kernel, bound, work unit); the work per launch is counted by
# the library (amgt_query_kernel_stats) from each launch's shapes
CLASSES = {
    "sweep": ("sweep2d_warp_kernel", "hbm", "B"),
    "apply_L": ("apply_L_kernel", "hbm", "B"),
    "scatter_prep": ("tc_prep_kernel", "hbm", "B"),
    "scatter_tc": ("tc_gemm_kernel<bf16> (tcgen05, V-cycle scatter)", "tensor", "flop"),
    "scatter_f32": ("gemm_kernel<float> (SIMT)", "alu", "flop"),
    "scatter_f64": ("gemm_kernel<double> (SIMT)", "alu64", "flop"),
    "coarse_gs": ("coarse_gs_rows_fast_kernel (register form, dense S_f source)", "alu", "flop"),
    "split_tc": ("tc_gemm_kernel<bf16> (tcgen05, slice products of the split FP64 scatter)",
                 "tensor", "flop"),
    "split_aux": ("split_rows_kernel + split_flush_kernel", "hbm", "B"),
    "tc3": ("tc_gemm_kernel<f16> (tcgen05, FP32-accurate three-product scatter)", "tensor", "flop"),
    "tc3_prep": ("tc3_prep_kernel", "hbm", "B"),
}
# DRAM bytes (read + write) per launch from the ncu captures summarised under
# profiles/, per workload; a kernel changed since its capture has no entry
TRAFFIC = {
    # split_tc, tc3: captured at 16384 rows (profiles/ncu_split_gemm_config5shape.md,
    # ncu_tc3_gemm_config5shape.md), scaled to the mean launch's rows (52428 and
    # 87381); coarse_gs: one 10-sweep launch (profiles/ncu_coarse_gs_rows_config5.md,
    # ncu_coarse_gs_rows_config2.md)
    "config5": {"split_tc": 3.72e9, "tc3": 21.1e9, "coarse_gs": 6.60e9},
    "config2": {"coarse_gs": 0.118e9},
}
FP64_PEAK = 1.25          # TFLOP/s, nominal GB300 FP64 rate
ALU_PEAK = 152 * 128 * 2 * 2.07e9 / 1e12   # FP32: 152 SMs x 128 FMA/clk x 2 x 2.07 GHz
PEAK_KINDS = {
    "alu": "FP32 FMA units x clock (152 x 128 x 2 x 2.07 GHz)",
    "alu64": "nominal GB300 FP64 rate, 1.25 TFLOP/s",
    "hbm": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
    "tensor": "measured BF16 GEMM burst (MEASURED_PEAKS.json bf16_tflops; FP16 runs at the "
              "same dense rate)",
}


_T0 = time.perf_counter()


def log(msg):
    """Progress on stderr (the JSON line alone goes to stdout)."""
    print(f"[bench {time.perf_counter() - _T0:7.1f} s] {msg}", file=sys.stderr, flush=True)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p["hbm_gbs"], p["bf16_tflops"], "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


def gpu_identity(local):
    """The CUDA device's UUID in nvidia-smi's form (GPU-xxxxxxxx-...), which
    names the same GPU whatever CUDA_VISIBLE_DEVICES renumbers; None if
    unavailable."""
    try:
        import torch
        u = str(torch.cuda.get_device_properties(local).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons of one GPU, named by its UUID,
    sampled during the timed region."""

    def __init__(self, gpu_id):
        self.gpu = gpu_id
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        if self.gpu is None:
            return self
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
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
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"],
                    "gpu": self.gpu}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm), "gpu": self.gpu}


# ------------------------------------------------------------------ CPU oracle
def oracle_sampler():
    """The oracle on a bounded sample of the headline workload: a 4x4-cell
    window of it (same angular mesh, order, materials, beam and multigrid).
    Returns a function timing one preconditioned Krylov iteration (one
    V-cycle plus one operator apply, FP64) and returning the cpu_baseline
    record; the set-up (tables, hierarchy) is done once, outside the timing."""
    from oracle import multigrid
    prob = W.config5_beam(n=4)
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
                "sample": (f"4x4-cell window of the 256x256 beam workload ({dof} unknowns, all "
                           f"2048 patches, N=64, 4-level MG): one V-cycle + one operator apply "
                           f"(= one preconditioned Krylov iteration) in {dt:.2f} s, NumPy FP64")}
    return step


def _oracle_child(conn):
    """Spawned process: builds the oracle sample, then times one sample per
    request (so the set-up overlaps the GPU work of the parent)."""
    try:
        step = oracle_sampler()
        conn.send(("ready", None))
        while True:
            msg = conn.recv()
            if msg != "go":
                break
            conn.send(("sample", step()))
    except Exception as ex:  # reported in the bench line
        conn.send(("error", str(ex)[:200]))


class OracleBaseline:
    """The CPU baseline in a spawned process started before any CUDA call."""

    def __init__(self):
        ctx = multiprocessing.get_context("spawn")
        self.conn, child = ctx.Pipe()
        self.proc = ctx.Process(target=_oracle_child, args=(child,), daemon=True)
        self.proc.start()

    def sample(self):
        try:
            kind, val = self.conn.recv()
            if kind != "ready":
                return {"error": val}
            self.conn.send("go")
            kind, val = self.conn.recv()
            return val if kind == "sample" else {"error": val}
        finally:
            try:
                self.conn.send("stop")
            except Exception:
                pass
            self.proc.join(timeout=10)


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


def head_config(world):
    return {"workload": WORKLOAD, "unknowns": 4 * 256 * 256 * 6144, "mode": "mixed",
            "krylov": f"FP64 refinement around FP32 FGMRES({HEAD_RESTART})",
            "precond": "MG V(1,1)", "tol": 1e-8, "inner_tol": "adaptive",
            "l2": "inputs larger than L2 (6.4-12.9 GB per vector)",
            "parallelism": f"replicas x{world}"}


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
            "config": head_config(args.gpus),
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "GDOF/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ GPU parts
def _kt_ids(pkg):
    return {"sweep": pkg.AMGT_KT_SWEEP, "apply_L": pkg.AMGT_KT_APPLY_L,
            "scatter_prep": pkg.AMGT_KT_SCATTER_PREP, "scatter_tc": pkg.AMGT_KT_SCATTER_TC,
            "scatter_f32": pkg.AMGT_KT_SCATTER_F32, "scatter_f64": pkg.AMGT_KT_SCATTER_F64,
            "coarse_gs": pkg.AMGT_KT_COARSE_GS, "split_tc": pkg.AMGT_KT_SPLIT_TC,
            "split_aux": pkg.AMGT_KT_SPLIT_AUX, "tc3": pkg.AMGT_KT_TC3,
            "tc3_prep": pkg.AMGT_KT_TC3_PREP}


def kt_read(ctx, pkg):
    return {k: ctx.amgt_query_kernel_stats(i, reset=True) for k, i in _kt_ids(pkg).items()}


def class_roofline(name, ms, n, work, peaks, traffic):
    """Achieved rate of one kernel class over its timed launches: summed
    algorithmic work / summed launch time, against the class's peak."""
    hbm, bf16, peak_src = peaks
    kernel, bound, unit = CLASSES[name]
    sec = ms / 1e3
    if unit == "B":
        achieved, peak, u = work / sec / 1e9, hbm, "GB/s"
    else:
        achieved, u = work / sec / 1e12, "TFLOP/s"
        peak = {"tensor": bf16, "alu": ALU_PEAK, "alu64": FP64_PEAK}[bound]
    return {"kernel": kernel, "bound": "alu" if bound == "alu64" else bound,
            "achieved": achieved, "peak": peak, "unit": u, "frac": achieved / peak,
            "launches": n, "mean_launch_s": sec / max(n, 1),
            "work_per_launch": work / max(n, 1), "work_unit": unit,
            "traffic": traffic.get(name),
            "peak_kind": PEAK_KINDS[bound] + ("" if bound in ("alu", "alu64") else
                                              f" ({peak_src})")}


def solve_timed(ctx, solve, steps, stream, torch):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    its, outer, relres = [], [], []
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        st = solve()
        its.append(st.iterations)
        outer.append(st.outer_iterations)
        relres.append(st.relres)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3, its, outer, relres


def coarse_f64_variant(ctx, solve, stream, torch, steps):
    """The same mixed solve with the coarsest Gauss-Seidel solve of the FP32
    V-cycle in FP64 (AMGT_TUNE_COARSE_F64): one warm-up solve, `steps` timed."""
    from paper_2010_04559_gb300 import AMGT_TUNE_COARSE_F64
    ctx.amgt_set_tuning(AMGT_TUNE_COARSE_F64, 1)
    with torch.cuda.stream(stream):
        solve()
        el, its, outer, rel = solve_timed(ctx, solve, steps, stream, torch)
    ctx.amgt_set_tuning(AMGT_TUNE_COARSE_F64, 0)
    return {"time_to_tol_s": el / steps, "krylov_iterations": its, "refinement_steps": outer,
            "relres": rel}


def instrumented(ctx, solve, pkg, peaks, traffic, torch):
    """One solve with the library's per-launch event timers on: per kernel
    class its device time, launches, share of the solve and roofline."""
    from paper_2010_04559_gb300 import AMGT_TUNE_KERNEL_TIMERS
    ctx.amgt_set_tuning(AMGT_TUNE_KERNEL_TIMERS, 1)
    kt_read(ctx, pkg)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = solve()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    k = kt_read(ctx, pkg)
    ctx.amgt_set_tuning(AMGT_TUNE_KERNEL_TIMERS, 0)
    out = {}
    for name, (ms, n, work) in k.items():
        if n > 0:
            r = class_roofline(name, ms, n, work, peaks, traffic)
            r["ms"] = ms
            r["share"] = ms / 1e3 / wall
            out[name] = r
    return out, wall, st


def operators_alone(ctx, nsdof, nadof, nmom, peaks, torch, stream, pkg):
    """One call of each operator on the finest level (FP32 unless stated),
    timed with events on the library's stream: GDOF/s per operator, and for
    the scatter the method's own work, 2 min(Nadof, 2 nmom) flop per unknown
    (dense S_f or the moment form, whichever is cheaper)."""
    from paper_2010_04559_gb300 import AMGT_TUNE_KERNEL_TIMERS
    dof = nsdof * nadof
    x32 = torch.randn((nsdof, nadof), device="cuda", dtype=torch.float32)
    y32 = torch.empty_like(x32)
    method_flop = 2.0 * dof * min(nadof, 2 * nmom)
    out = {}

    def timeit(fn, reps):
        fn()
        ctx.amgt_set_tuning(AMGT_TUNE_KERNEL_TIMERS, 1)
        kt_read(ctx, pkg)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        k = kt_read(ctx, pkg)
        ctx.amgt_set_tuning(AMGT_TUNE_KERNEL_TIMERS, 0)
        return a.elapsed_time(b) / reps / 1e3, {n: v for n, v in k.items() if v[1] > 0}

    with torch.cuda.stream(stream):
        t, _ = timeit(lambda: ctx.amgt_op_sweep(0, x32, y32), 5)
        out["sweep_f32"] = {"s": t, "GDOF/s": dof / t / 1e9, "GB/s": 8.0 * dof / t / 1e9}
        t, _ = timeit(lambda: ctx.amgt_op_apply_L(0, x32, y32), 5)
        out["apply_L_f32"] = {"s": t, "GDOF/s": dof / t / 1e9, "GB/s": 8.0 * dof / t / 1e9}
        t, k = timeit(lambda: ctx.amgt_op_scatter(0, x32, y32, tc=True), 5)
        out["scatter_bf16tc"] = {"s": t, "GDOF/s": dof / t / 1e9,
                                 "method_TFLOP/s": method_flop / t / 1e12,
                                 "gemm_TFLOP/s": k["scatter_tc"][2] / k["scatter_tc"][0] / 1e9}
        t, k = timeit(lambda: ctx.amgt_op_scatter(0, x32, y32, tc="tc3"), 3)
        if "tc3" in k:
            out["scatter_f32_tc3"] = {"s": t, "GDOF/s": dof / t / 1e9,
                                      "method_TFLOP/s": method_flop / t / 1e12,
                                      "gemm_TFLOP/s": k["tc3"][2] / k["tc3"][0] / 1e9}
        t, _ = timeit(lambda: ctx.amgt_op_vcycle(x32, y32, tc=True), 2)
        out["vcycle_bf16tc"] = {"s": t, "GDOF/s": dof / t / 1e9}
        del x32, y32
        x64 = torch.randn((nsdof, nadof), device="cuda", dtype=torch.float64)
        y64 = torch.empty_like(x64)
        t, k = timeit(lambda: ctx.amgt_op_scatter(0, x64, y64, tc=True), 1)
        if "split_tc" in k:
            out["scatter_f64_split"] = {"s": t, "GDOF/s": dof / t / 1e9,
                                        "method_TFLOP/s": method_flop / t / 1e12,
                                        "gemm_TFLOP/s": k["split_tc"][2] / k["split_tc"][0] / 1e9,
                                        "gemm_launches": k["split_tc"][1]}
        del x64, y64
    return out


def fp64_solve(prob, local, krylov, restart, torch, maxit=400):
    """Time to relres 1e-8 of the plain FP64 GPU solve on its own context
    (every FP64 scatter in the split form on the tensor cores), after one
    warm-up operator apply and V-cycle that build the lazily made tables."""
    from paper_2010_04559_gb300 import (AMGT_MODE_F64, AMGT_PREC_MG, AMGT_TUNE_FP64_SCATTER,
                                        context_from_problem)
    stream = torch.cuda.Stream()
    ctx = context_from_problem(prob, device=local, stream=stream.cuda_stream)
    ctx.amgt_set_tuning(AMGT_TUNE_FP64_SCATTER, 2)
    ns, na = ctx.amgt_query_sizes(0)
    psi = torch.empty((ns, na), device="cuda", dtype=torch.float64)
    phi = torch.empty(ns, device="cuda", dtype=torch.float64)
    with torch.cuda.stream(stream):
        tmp = torch.empty_like(psi)
        ctx.amgt_op_apply_A(0, psi.zero_(), tmp, tc=True)
        ctx.amgt_op_vcycle(psi, tmp, tc=True)
        del tmp
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, st, _ = ctx.amgt_solve(tol=1e-8, restart=restart, maxit=maxit,
                                     precond=AMGT_PREC_MG, mode=AMGT_MODE_F64, psi=psi, phi=phi,
                                     device_ptrs=True, allow_not_converged=True, krylov=krylov)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
    ctx.close()
    del psi, phi
    torch.cuda.empty_cache()
    return {"time_to_tol_s": t, "iterations": st.iterations, "restarts": st.outer_iterations,
            "relres": st.relres,
            "krylov": "BiCGStab" if krylov == 1 else f"GMRES({restart})",
            "scatter": "FP64-accurate split form on BF16 tensor cores (AMGT_F64_SPLIT)",
            "warmup": "one operator apply and one V-cycle (lazy tables and workspaces)"}


def config2_extra(local, torch, pkg, peaks, steps=3, warmup=3):
    """The 128x128 checkerboard workload: mixed solve time (events, timers
    off), its kernel shares, and the FP64 GPU solve of the same inputs."""
    from paper_2010_04559_gb300 import (AMGT_MODE_MIXED, AMGT_PREC_MG, AMGT_TUNE_GRAPHS,
                                        context_from_problem)
    prob = W.config2_checkerboard()
    stream = torch.cuda.Stream()
    ctx = context_from_problem(prob, device=local, stream=stream.cuda_stream)
    ctx.amgt_set_tuning(AMGT_TUNE_GRAPHS, 1)
    ns, na = ctx.amgt_query_sizes(0)
    psi = torch.empty((ns, na), device="cuda", dtype=torch.float64)
    phi = torch.empty(ns, device="cuda", dtype=torch.float64)

    def solve():
        _, _, st, _ = ctx.amgt_solve(tol=1e-8, restart=20, maxit=400, precond=AMGT_PREC_MG,
                                     mode=AMGT_MODE_MIXED, psi=psi, phi=phi, device_ptrs=True)
        return st
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            solve()
        el, its, outer, rel = solve_timed(ctx, solve, steps, stream, torch)
        kin, wall, _ = instrumented(ctx, solve, pkg, peaks, TRAFFIC["config2"], torch)
    cf64 = coarse_f64_variant(ctx, solve, stream, torch, steps)
    ctx.close()
    del psi, phi
    torch.cuda.empty_cache()
    t_mixed = el / steps
    f64 = fp64_solve(prob, local, 0, 20, torch)
    dof = ns * na
    dom = max(kin, key=lambda n: kin[n]["share"])
    return {"workload": WORKLOAD2, "unknowns": dof,
            "mixed": {"time_to_tol_s": t_mixed, "GDOF/s": dof * np.mean(its) / t_mixed / 1e9,
                      "krylov_iterations": its, "refinement_steps": outer, "relres": rel,
                      "krylov": "FP64 refinement around FP32 FGMRES(20)"},
            "fp64_gpu": f64, "mixed_speedup_vs_fp64": f64["time_to_tol_s"] / t_mixed,
            "mixed_coarse_f64": cf64,
            "solve_kernels": {n: {"ms": v["ms"], "share": v["share"], "launches": v["launches"]}
                              for n, v in kin.items()},
            "dominant": dict(kin[dom], name=dom)}


def adjoint_extra(local, torch):
    """Adjoint solve (mixed, 1e-8) for the flux integral over a 16x16-cell
    corner block of the 128x128 workload, then the response and all its
    gradients."""
    from paper_2010_04559_gb300 import AMGT_MODE_MIXED, AMGT_PREC_MG, context_from_problem
    from paper_2010_04559_gb300.adjoint import response_problem
    prob = W.config2_checkerboard()
    nx = 128
    weight = np.zeros(nx * nx)
    for iy in range(16):
        weight[iy * nx:iy * nx + 16] = 1.0
    stream = torch.cuda.Stream()
    ctx = context_from_problem(prob, device=local, stream=stream.cuda_stream)
    actx = context_from_problem(response_problem(prob, weight), device=local,
                                stream=stream.cuda_stream)
    actx.amgt_set_adjoint(1)
    ns, na = ctx.amgt_query_sizes(0)
    psi = torch.empty((ns, na), device="cuda", dtype=torch.float64)
    lam = torch.empty_like(psi)
    phi = torch.empty(ns, device="cuda", dtype=torch.float64)
    C = nx * nx
    dt = torch.empty(C, device="cuda", dtype=torch.float64)
    ds = torch.empty_like(dt)
    df = torch.empty(prob["N"] + 1, device="cuda", dtype=torch.float64)
    with torch.cuda.stream(stream):
        ctx.amgt_solve(tol=1e-8, precond=AMGT_PREC_MG, mode=AMGT_MODE_MIXED, psi=psi, phi=phi,
                       device_ptrs=True)

        def step():
            _, _, sta, _ = actx.amgt_solve(tol=1e-8, restart=20, maxit=400,
                                           precond=AMGT_PREC_MG, mode=AMGT_MODE_MIXED, psi=lam,
                                           phi=phi, device_ptrs=True)
            R = actx.amgt_response(psi)
            ctx.amgt_response_gradients(psi, lam, dt, ds, df)
            return sta, R
        step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sta, R = step()
        torch.cuda.synchronize()
        t_adj = time.perf_counter() - t0
        t0 = time.perf_counter()
        ctx.amgt_response_gradients(psi, lam, dt, ds, df)
        t_grad = time.perf_counter() - t0
    actx.close()
    ctx.close()
    return {"workload": "128x128 checkerboard workload: flux integral over the 16x16-cell corner "
                        "block; dR/dsigma_t, dR/dsigma_s per cell and dR/df_n (N=16)",
            "adjoint_solve_and_gradients_s": t_adj, "gradients_s": t_grad,
            "iterations": sta.iterations, "relres": sta.relres, "response": R}


def batch_extra(local, torch, nprob, wave=16):
    """The 256-problem batch of uneven 2D problems (n = 16..96 cells per axis,
    levels 1..3, per-cell lognormal sigma_t, own g and order), in waves of
    `wave` problems: each wave's contexts are set up concurrently by
    amgt_setup_batch (block inverses on the GPU), solved concurrently by
    amgt_solve_batch (each problem on its own
    stream, V-cycles replayed from captured graphs; a first solve captures
    them), then solved one after another for comparison.  Times are sums over
    the waves of the timed solves only."""
    from paper_2010_04559_gb300 import (AMGT_MODE_MIXED, AMGT_PREC_MG, AMGT_TUNE_GRAPHS,
                                        amgt_setup_batch, amgt_solve_batch,
                                        context_from_problem)
    probs = W.config4_batch()[:nprob]
    t_conc = t_seq = t_setup = 0.0
    dof_its = 0
    unknowns = 0
    iters, maxrel = [], 0.0
    for w0 in range(0, len(probs), wave):
        part = probs[w0:w0 + wave]
        bstreams = [torch.cuda.Stream() for _ in part]
        t0 = time.perf_counter()
        bctx = [context_from_problem(p, device=local, stream=s.cuda_stream)
                for p, s in zip(part, bstreams)]
        amgt_setup_batch(bctx)                          # the wave's set-up, concurrently
        bdof = [int(np.prod(c.amgt_query_sizes(0))) for c in bctx]
        torch.cuda.synchronize()
        t_setup += time.perf_counter() - t0
        for c in bctx:
            c.amgt_set_tuning(AMGT_TUNE_GRAPHS, 1)
        bpsi = [torch.empty(c.amgt_query_sizes(0), device="cuda", dtype=torch.float64)
                for c in bctx]
        amgt_solve_batch(bctx, bpsi, tol=1e-8)          # warm-up: captures the graphs
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bst = amgt_solve_batch(bctx, bpsi, tol=1e-8)
        torch.cuda.synchronize()
        t_conc += time.perf_counter() - t0
        t0 = time.perf_counter()
        for c, p in zip(bctx, bpsi):
            c.amgt_solve(tol=1e-8, precond=AMGT_PREC_MG, mode=AMGT_MODE_MIXED, psi=p, phi=None,
                         device_ptrs=True)
        torch.cuda.synchronize()
        t_seq += time.perf_counter() - t0
        dof_its += sum(d * st.iterations for d, st in zip(bdof, bst))
        unknowns += sum(bdof)
        iters += [st.iterations for st in bst]
        maxrel = max(maxrel, max(st.relres for st in bst))
        for c in bctx:
            c.close()
        del bpsi
        torch.cuda.empty_cache()
    return {"workload": f"{len(probs)} problems of the uneven 2D batch (n in 16..96, level "
                        f"1..3, per-cell lognormal sigma_t, N = 2 level + 4), waves of {wave}",
            "problems": len(probs), "unknowns": unknowns, "value": dof_its / t_conc / 1e9,
            "unit": "GDOF/s", "time_to_tol_s": t_conc, "sequential_time_to_tol_s": t_seq,
            "concurrency_speedup": t_seq / t_conc, "setup_s": t_setup, "max_relres": maxrel,
            "iterations": iters}


# the paper's Table 1, Lin basis, level 3 (Sec. 5.1): Krylov (BiCGStab)
# iterations to 1e-8, single grid (SG) and V(1,1) with N_r = 1, 2, 3
TABLE1 = {4: {"SG": 44, 1: 4, 2: 4}, 8: {"SG": 124, 1: 11, 2: 8, 3: 4},
          16: {"SG": 284, 1: 31, 2: 22, 3: 22}}


def run_table1(args):
    """Context run of the paper's Table 1 set-up (workloads.table1_cube): FP64
    BiCGStab to relres 1e-8 on the GPU, single grid (sweep preconditioner)
    and V(1,1) multigrid with the reduced coarse orders, iteration counts
    beside the paper's.  Context only: the coarse solve and the absorption
    are readings (see workloads.table1_cube)."""
    import torch
    from paper_2010_04559_gb300 import (AMGT_MODE_F64, AMGT_PREC_MG, AMGT_PREC_SWEEP,
                                        AMGT_TUNE_FP64_SCATTER, context_from_problem)
    from paper_2010_04559_gb300 import build as _b
    _b.build()
    out = []
    for N in args.table1_orders:
        runs = [("SG", 2)] + [(nr, nr) for nr in (1, 2, 3) if nr in TABLE1.get(N, {})]
        for label, nr in runs:
            prob = W.table1_cube(N, Nr=nr)
            if label == "SG":
                prob["mg"] = None
            stream = torch.cuda.Stream()
            t0 = time.perf_counter()
            ctx = context_from_problem(prob, device=0, stream=stream.cuda_stream)
            ctx.amgt_set_tuning(AMGT_TUNE_FP64_SCATTER, 2)
            ns, na = ctx.amgt_query_sizes(0)
            t_set = time.perf_counter() - t0
            psi = torch.empty((ns, na), device="cuda", dtype=torch.float64)
            phi = torch.empty(ns, device="cuda", dtype=torch.float64)
            with torch.cuda.stream(stream):
                t0 = time.perf_counter()
                _, _, st, _ = ctx.amgt_solve(
                    tol=1e-8, maxit=2000, precond=AMGT_PREC_SWEEP if label == "SG" else AMGT_PREC_MG,
                    mode=AMGT_MODE_F64, psi=psi, phi=phi, device_ptrs=True,
                    allow_not_converged=True, krylov=1)
                torch.cuda.synchronize()
                t = time.perf_counter() - t0
            ctx.close()
            del psi, phi
            torch.cuda.empty_cache()
            rec = {"N": N, "run": "SG" if label == "SG" else f"V(1,1) N_r={nr}",
                   "iterations": st.iterations, "paper_iterations": TABLE1[N][label],
                   "relres": st.relres, "solve_s": t, "setup_s": t_set}
            log(json.dumps(rec))
            out.append(rec)
    line = {"table1": out, "workload": "5 cm cube, 30^3 Q1 hexes, uniform isotropic unit "
            "source, vacuum, FP-equivalent moments alpha = 1 (sigma_t = sigma_s0 = N(N+1)/2, "
            "no absorption), Lin level 3 (512 patches), BiCGStab FP64 to 1e-8, multigrid down "
            "to level 0 with 30 coarse Gauss-Seidel sweeps", "context_only": True}
    print(json.dumps(line))
    return 0


def run_profile(args):
    """Small launches for ncu: one launch of a chosen kernel on a chosen
    workload, warm-up launch first."""
    import torch
    from paper_2010_04559_gb300 import (AMGT_MODE_MIXED, AMGT_PREC_MG, AMGT_TUNE_SWEEP_KERNEL,
                                        context_from_problem)
    from paper_2010_04559_gb300 import build as _b
    _b.build()
    if args.profile in ("gemm5", "tc3_5", "split5", "ops5"):
        # the headline's contraction shape on a 64x64-cell slab of its rows:
        # K = N = 6144, 65536 rows (a few GB on the device, larger than L2)
        prob = W.config5_beam(n=64)
    elif args.profile in ("solve5", "gs5"):
        prob = W.config5_beam()
    elif args.profile == "sweep3d":
        prob = W.config3_cube(n=args.n if args.n != 128 else 32)
    else:
        prob = W.config2_checkerboard(n=args.n)
    t0 = time.perf_counter()
    ctx = context_from_problem(prob, device=0)
    ns, na = ctx.amgt_query_sizes(0)
    print(f"set-up {time.perf_counter() - t0:.2f} s")
    if args.profile == "sweep3d":
        # the 32^3 cube (32768 materials, level 2): FP32 then FP64 sweeps, twice
        for td in (torch.float32, torch.float64):
            x = torch.randn((ns, na), device="cuda", dtype=td)
            y = torch.empty_like(x)
            for _ in range(2):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                ctx.amgt_op_sweep(0, x, y)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
            print(f"3D sweep {td}: {dt * 1e3:.2f} ms, {2 * x.element_size() * ns * na / dt / 1e9:.0f} "
                  f"GB/s algorithmic")
            del x, y
    elif args.profile == "gs5":
        # the headline's coarse Gauss-Seidel launch (level 1: 32 patches, 10 sweeps)
        nsc, nac = ctx.amgt_query_sizes(3)
        fc = torch.randn((nsc, nac), device="cuda", dtype=torch.float32)
        pc = torch.zeros_like(fc)
        for _ in range(2):
            ctx.amgt_op_coarse_gs(10, fc, pc)
        print("kernels: coarse Gauss-Seidel of the beam workload, 10 sweeps (x2)")
    elif args.profile == "gs":
        nsc, nac = ctx.amgt_query_sizes(2)
        fc = torch.randn((nsc, nac), device="cuda", dtype=torch.float32)
        pc = torch.zeros_like(fc)
        for _ in range(2):
            ctx.amgt_op_coarse_gs(10, fc, pc)
        print("kernels: coarse Gauss-Seidel, 10 sweeps (x2)")
    elif args.profile == "sweeps":
        x = torch.randn((ns, na), device="cuda", dtype=torch.float32)
        y = torch.empty_like(x)
        for _ in range(2):
            for k in (1, 2):
                ctx.amgt_set_tuning(AMGT_TUNE_SWEEP_KERNEL, k)
                ctx.amgt_op_sweep(0, x, y)
        print("kernels: level-synchronous row sweep, warp-pipelined sweep (x2)")
    elif args.profile in ("gemm5", "tc3_5"):
        x = torch.randn((ns, na), device="cuda", dtype=torch.float32)
        y = torch.empty_like(x)
        for _ in range(2):
            ctx.amgt_op_scatter(0, x, y, tc=True if args.profile == "gemm5" else "tc3")
        print("kernels: scatter contraction at K = N = 6144 (x2)")
    elif args.profile == "ops5":
        # the finest level's FP32 L apply and sweep and the double-float L
        # apply on the 64x64-cell slab (6144 angular DOF, 403 MB per FP32 vector)
        x = torch.randn((ns, na), device="cuda", dtype=torch.float32)
        y = torch.empty_like(x)
        for _ in range(2):
            ctx.amgt_op_apply_L(0, x, y)
            ctx.amgt_op_sweep(0, x, y)
        del x, y
        x = torch.randn((ns, na), device="cuda", dtype=torch.float64)
        y = torch.empty_like(x)
        for _ in range(2):
            ctx.amgt_op_apply_L(0, x, y, tc=True)
        print("kernels: FP32 L apply and sweep, double-float L apply, on level 0 (x2)")
    elif args.profile == "split5":
        x = torch.randn((ns, na), device="cuda", dtype=torch.float64)
        y = torch.empty_like(x)
        ctx.amgt_op_scatter(0, x, y, tc=True)
        print("kernels: split FP64 scatter at K = N = 6144")
    elif args.profile in ("solve", "solve5"):
        psi = torch.empty((ns, na), device="cuda", dtype=torch.float64)
        phi = torch.empty(ns, device="cuda", dtype=torch.float64)
        _, _, st, _ = ctx.amgt_solve(tol=1e-8, restart=HEAD_RESTART if args.profile == "solve5"
                                     else 20, precond=AMGT_PREC_MG, mode=AMGT_MODE_MIXED,
                                     psi=psi, phi=phi, device_ptrs=True)
        print(f"solve: {st.iterations} iterations, relres {st.relres:.3e}")
    ctx.amgt_sync()
    torch.cuda.synchronize()
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the FP64 arm, the 128x128 workload, the adjoint and the batch")
    ap.add_argument("--graphs", type=int, default=1, help="V-cycle graph replay (1) or not (0)")
    ap.add_argument("--batch", type=int, default=256,
                    help="problems of the uneven 2D batch, solved in concurrent waves (0: skip)")
    ap.add_argument("--n", type=int, default=128, help="cells per axis of --profile's workload")
    ap.add_argument("--profile", choices=["solve", "solve5", "sweeps", "gs", "gs5", "gemm5",
                                          "tc3_5", "split5", "sweep3d", "ops5"],
                    default=None, help="one launch of a hot kernel, and exit (for ncu)")
    ap.add_argument("--table1", action="store_true",
                    help="context run of the paper's Table 1 set-up (iteration counts), and exit")
    ap.add_argument("--table1-orders", type=int, nargs="*", default=[4, 8, 16])
    args = ap.parse_args()
    if args.table1:
        return run_table1(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.profile:
        return run_profile(args)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    # the oracle's set-up starts before any CUDA call, in a spawned process
    oracle = OracleBaseline() if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if args.warmup < 3:
        print("warmup must be >= 3", file=sys.stderr)
        return 2

    import paper_2010_04559_gb300 as pkg
    from paper_2010_04559_gb300 import (AMGT_MODE_MIXED, AMGT_PREC_MG, AMGT_TUNE_GRAPHS,
                                        amgt_query_launches, context_from_problem)
    from paper_2010_04559_gb300 import build as _b
    _b.build()
    peaks = _peaks()
    stream = torch.cuda.Stream()
    prob = W.config5_beam()
    t0 = time.perf_counter()
    ctx = context_from_problem(prob, device=local, stream=stream.cuda_stream)
    nsdof, nadof = ctx.amgt_query_sizes(0)
    t_setup = time.perf_counter() - t0
    ctx.amgt_set_tuning(AMGT_TUNE_GRAPHS, args.graphs)
    dof = nsdof * nadof
    psi = torch.empty((nsdof, nadof), device="cuda", dtype=torch.float64)
    phi = torch.empty(nsdof, device="cuda", dtype=torch.float64)

    def solve():
        _, _, st, _ = ctx.amgt_solve(tol=1e-8, restart=HEAD_RESTART, maxit=400,
                                     precond=AMGT_PREC_MG, mode=AMGT_MODE_MIXED, psi=psi,
                                     phi=phi, device_ptrs=True, inner_maxit=200)
        return st

    log(f"headline context ready ({t_setup:.1f} s)")
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            st = solve()
            log(f"warm-up solve: {st.iterations} iterations, relres {st.relres:.2e}")
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        l0 = amgt_query_launches()
        with ClockSampler(gpu_identity(local)) as clk:
            elapsed, its, outer, relres = solve_timed(ctx, solve, args.steps, stream, torch)
        launches = amgt_query_launches() - l0
    elapsed = max_over_ranks(elapsed, dist, "cuda")
    ms = elapsed / args.steps * 1e3
    value = job_gdofs(world, dof, np.sum(its), elapsed)

    log(f"timed: {ms:.1f} ms per solve")
    # ---- end to end through the public API with host buffers: the source
    # upload and the psi/phi download inside the timed region
    e2e_steps = min(args.steps, 2)
    qsrc = np.ascontiguousarray(prob["q"])
    psi_h = torch.empty((nsdof, nadof), dtype=torch.float64, pin_memory=True).numpy()
    phi_h = torch.empty(nsdof, dtype=torch.float64, pin_memory=True).numpy()
    e2e_its = 0
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.amgt_set_source_iso(qsrc)
        _, _, st2, _ = ctx.amgt_solve(tol=1e-8, restart=HEAD_RESTART, maxit=400,
                                      precond=AMGT_PREC_MG, mode=AMGT_MODE_MIXED, psi=psi_h,
                                      phi=phi_h, inner_maxit=200)
        e2e_its += st2.iterations
    e2e_t = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e = {"value": job_gdofs(world, dof, e2e_its, e2e_t), "unit": "GDOF/s",
           "h2d_bytes_per_step": int(qsrc.nbytes),
           "d2h_bytes_per_step": int(psi_h.nbytes + phi_h.nbytes), "steps": e2e_steps,
           "time_to_tol_s": e2e_t / e2e_steps}
    del psi_h, phi_h

    log(f"e2e: {e2e['time_to_tol_s']:.2f} s per solve")
    # ---- one instrumented solve: kernel shares and rooflines
    with torch.cuda.stream(stream):
        kin, wall, _ = instrumented(ctx, solve, pkg, peaks, TRAFFIC["config5"], torch)
    dom = max(kin, key=lambda n: kin[n]["share"])
    roof = dict(kin[dom])
    roof["class"] = dom
    tc_classes = [n for n in kin if CLASSES[n][0].startswith("tc_gemm_kernel")]
    tc_gemm = {"classes": tc_classes,
               "share": sum(kin[n]["share"] for n in tc_classes),
               "TFLOP/s": (sum(kin[n]["work_per_launch"] * kin[n]["launches"] for n in tc_classes)
                           / max(1e-9, sum(kin[n]["ms"] for n in tc_classes) / 1e3) / 1e12)}
    tc_gemm["frac"] = tc_gemm["TFLOP/s"] / peaks[1]
    log(f"instrumented solve {wall:.2f} s, dominant {dom}")
    ops = operators_alone(ctx, nsdof, nadof, (prob["N"] + 1) ** 2, peaks, torch, stream, pkg)
    cf64 = coarse_f64_variant(ctx, solve, stream, torch, 1)
    log(f"coarse FP64 variant: {cf64['time_to_tol_s']:.2f} s")
    ctx.close()
    del psi, phi
    torch.cuda.empty_cache()

    extra = {}
    fp64 = None
    if not args.no_extra:
        log("operators timed; FP64 arm")
        fp64 = fp64_solve(prob, local, 1, 20, torch, maxit=200)
        log(f"FP64 arm: {fp64['time_to_tol_s']:.1f} s, {fp64['iterations']} iterations")
        extra["config2"] = config2_extra(local, torch, pkg, peaks)
        log("128x128 workload done")
        extra["adjoint"] = adjoint_extra(local, torch)
        if args.batch > 0:
            extra["batched"] = batch_extra(local, torch, args.batch)

    log("GPU parts done; CPU oracle sample")
    cpu = oracle.sample() if oracle else None
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32/bf16/f16 (f64 refinement)", "data": "synthetic",
                "config": head_config(world),
                "time_to_tol_s": ms / 1e3, "krylov_iterations": its,
                "refinement_steps": outer, "relres": relres,
                "gpu_launches": int(launches), "graphs": bool(args.graphs),
                "setup_s": t_setup, "roofline": roof, "tensor_core_gemm": tc_gemm,
                "solve_kernels": kin, "instrumented_solve_s": wall, "operators": ops,
                "clocks": clk.summary(), "e2e": e2e, "cpu_baseline": cpu}
        line["mixed_coarse_f64"] = cf64
        if fp64:
            line["fp64_gpu"] = fp64
            line["mixed_speedup_vs_fp64"] = fp64["time_to_tol_s"] / (ms / 1e3)
        line["extra"] = extra
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
