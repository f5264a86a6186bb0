"""Benchmark: auxiliary-space PCG to relative residual 1e-8 on the P4 Poisson problem of a
48^3-cube jittered Kuhn mesh (663,552 tetrahedra, 6,967,871 unknowns, 512.8M nonzeros),
kappa_e = exp(N(0,1)) per element (seed 1), sine source, additive preconditioner (one
symmetric multicolour GS sweep + one P1 AMG V(1,1)-cycle, PMIS + extended+i, theta =
0.25, l1-Jacobi level smoothing). value: the all-FP64 solve; beside it, timed the same
way (CUDA events around the same number of solves), the mixed-precision solve (FP32
smoother / I_P / AMG hierarchy, FP64 flexible CG) and both with the l1-Jacobi smoother.

One step = one complete PCG solve from x0 = 0 (setup excluded, reported separately).
The metric is MDOF*iter/s = n_h * iterations / solve time; the time to solution and the
HBM roofline of the dominant kernel are reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload p4_n48_lognormal | p3_n32 | p2_n8 | p2_n64_batched48 |
                                p3_n24_adjoint | ...]

p3_n32 is the P3 problem on 32^3 cubes (857,375 unknowns, kappa = 1), p2_n8 the P2
problem on 8^3 cubes (3,375 unknowns; launch-latency bound). p2_n64_batched48 is the
multi-RHS solve: the P2 vector Laplacian (3 velocity components, identical scalar
blocks) on a 64^3 jittered Kuhn mesh with 16 right-hand sides of i.i.d. N(0,1) entries
(seed 2), i.e. 48 columns of the scalar system in one blocked PCG, FP32 preconditioner
and FP64 outer iteration. p3_n24_adjoint is the differentiable solve: P3 on 24^3 cubes
with lognormal kappa, one step = forward PCG + adjoint PCG + dL/dkappa for
L = 0.5 ||u - u_obs||^2.

Multi-GPU: the path runs as independent replicas (one solve per rank, no collective on
the data path); value sums the ranks' work over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(name="p3_n32", k=3, n=32, jitter=0.2, mesh_seed=0)
METRIC = "P_k PCG time to rel. residual 1e-8 (s), MDOF*iter/s, HBM GB/s vs peak"
UNIT = "MDOF*iter/s"
CONFIG = {
    "workload": "P3 Poisson, kappa=1, 32^3 jittered Kuhn cubes (196,608 tets, 857,375 unknowns), "
                "sine source, FP64, PCG to rel. residual 1e-8, additive aux-space preconditioner "
                "(1 SGS sweep + 1 P1 AMG V-cycle, PMIS + ext+i, theta=0.25, l1-Jacobi level smoothing)",
    "mesh": "unit cube, 32^3 cubes x 6 Kuhn tets, interior vertices jittered by <=0.2h (seed 0)",
    "k": 3,
    "n_h": 857375,
    "l2_flush": "inputs larger than L2: A_h alone is 480 MB (12 B/nnz x 39,951,635 nnz) vs 129 MB L2",
    "parallelism": "replicas (one independent solve per GPU)",
}
P4 = dict(name="p4_n48_lognormal", k=4, n=48, jitter=0.2, mesh_seed=0, kappa_seed=1)
CONFIG_P4 = {
    "workload": "P4 Poisson, kappa_e = exp(N(0,1)) per tet (seed 1), 48^3 jittered Kuhn cubes (663,552 tets, "
                "6,967,871 unknowns, 512,842,207 nonzeros), sine source, PCG to rel. residual 1e-8, "
                "additive aux-space preconditioner (1 SGS sweep + 1 P1 AMG V-cycle, theta=0.25, l1-Jacobi "
                "levels); value: FP64 throughout; the mixed-precision solve (FP32 preconditioner, FP64 "
                "flexible CG) is reported beside it",
    "mesh": "unit cube, 48^3 cubes x 6 Kuhn tets, interior vertices jittered by <=0.2h (seed 0)",
    "k": 4,
    "n_h": 6967871,
    "l2_flush": "inputs larger than L2: A_h alone is 6.2 GB vs 129 MB L2",
    "parallelism": "replicas (one independent solve per GPU)",
}
P2_8 = dict(name="p2_n8", k=2, n=8, jitter=0.2, mesh_seed=0)
CONFIG_P2_8 = {
    "workload": "P2 Poisson, kappa=1, 8^3 jittered Kuhn cubes (3,072 tets, 3,375 unknowns), sine source, "
                "FP64, PCG to rel. residual 1e-8, additive aux-space preconditioner (1 SGS sweep + 1 P1 AMG "
                "V-cycle, theta=0.25, l1-Jacobi level smoothing); launch-latency bound at this size",
    "mesh": "unit cube, 8^3 cubes x 6 Kuhn tets, interior vertices jittered by <=0.2h (seed 0)",
    "k": 2,
    "n_h": 3375,
    "l2_flush": "none: the whole problem (under 1 MB) stays in L2; a latency measurement",
    "parallelism": "replicas (one independent solve per GPU)",
}
SINGLE = {WORKLOAD["name"]: (WORKLOAD, CONFIG), P4["name"]: (P4, CONFIG_P4), P2_8["name"]: (P2_8, CONFIG_P2_8)}
ADJOINT = dict(name="p3_n24_adjoint", k=3, n=24, jitter=0.2, mesh_seed=0, kappa_seed=1, obs_kappa_seed=3)
CONFIG_ADJOINT = {
    "workload": "P3 Poisson on 24^3 jittered Kuhn cubes (82,944 tets, 357,911 unknowns), kappa_e = exp(N(0,1)) "
                "(seed 1), sine source; loss L = 0.5 ||u - u_obs||^2 with u_obs solved for a second kappa "
                "field (seed 3); one step = forward PCG + adjoint PCG (right-hand side u - u_obs) + dL/dkappa "
                "for every element (dL/db = the adjoint solution); FP32 preconditioner, FP64 outer "
                "flexible CG, rel. residual 1e-8; value counts forward and adjoint iterations",
    "mesh": "unit cube, 24^3 cubes x 6 Kuhn tets, interior vertices jittered by <=0.2h (seed 0)",
    "k": 3,
    "n_h": 357911,
    "l2_flush": "none: A_h (about 170 MB) is only a little larger than L2",
    "parallelism": "replicas (one independent solve per GPU)",
}
DEFAULT_WORKLOAD = P4["name"]
BATCHED = dict(name="p2_n64_batched48", k=2, n=64, jitter=0.2, mesh_seed=0, rhs_seed=2, ncols=48)
CONFIG_BATCHED = {
    "workload": "P2 vector Laplacian (3 components x 16 right-hand sides = 48 columns of the scalar "
                "system), kappa=1, 64^3 jittered Kuhn cubes (1,572,864 tets, 2,048,383 unknowns per column), "
                "RHS entries i.i.d. N(0,1) (seed 2), one blocked PCG to rel. residual 1e-8 per column, "
                "FP32 preconditioner (1 SGS sweep + 1 P1 AMG V-cycle, l1-Jacobi levels), FP64 outer "
                "flexible CG, CUDA-graph loop",
    "mesh": "unit cube, 64^3 cubes x 6 Kuhn tets, interior vertices jittered by <=0.2h (seed 0)",
    "k": 2,
    "n_h": 2048383,
    "ncols": 48,
    "l2_flush": "inputs larger than L2: every [n_h][48] FP64 block is 787 MB vs 129 MB L2",
    "parallelism": "replicas (one independent blocked solve per GPU)",
}
# peak of the FP64 pipe derived from unit counts and clocks: 152 SMs x 2,070 MHz x 4 flop
# per clock per SM (2 FP64 FMA per clock per SM) = 1.259 TFLOP/s (nominal 1.25)
FP64_PEAK_TFLOPS = 152 * 2.070e9 * 4 / 1e12
ORACLE_SAMPLE_ITERS = 12
# ncu dram__bytes_read.sum + dram__bytes_write.sum per launch (summed over the phases of
# one S_k application), keyed by (workload, cubes per side, smoother layout); a kernel
# changed since the capture has no entry (traffic null)
SMOOTHER_TRAFFIC = {}
SPMV_TRAFFIC = {("p4_n48_lognormal", 48): (6843905536 + 82143744 + 6831242496 + 91436544 + 6832146176 + 91604224) / 3}
NOMINAL_HBM_GBS = 8000.0  # GB300's nominal HBM3e bandwidth, for the second fraction
# AMG level smoother: l1-Jacobi (1), one kernel per smoothing step; multicolour GS on the
# dense coarse levels needs one launch per colour and costs ~25x more per V-cycle here
LEVEL_SMOOTHER = 1


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def replica_totals(ms, work, device="cuda"):
    """Whole-job figures of independent replicas (one per rank): the slowest rank's time
    and the work of all ranks summed. A single process returns its own figures."""
    import torch

    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return float(ms), float(work)
    t = torch.tensor([float(ms), float(work)], dtype=torch.float64, device=device)
    mx = t[:1].clone()
    torch.distributed.all_reduce(mx, op=torch.distributed.ReduceOp.MAX)
    sm = t[1:].clone()
    torch.distributed.all_reduce(sm, op=torch.distributed.ReduceOp.SUM)
    return float(mx.item()), float(sm.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_kappa(wl, nt):
    from paper_1204_2586_gb300.inputs import kappa_lognormal

    return kappa_lognormal(nt, wl["kappa_seed"]) if wl.get("kappa_seed") is not None else None


def make_problem():
    from paper_1204_2586_gb300 import Problem
    from paper_1204_2586_gb300.inputs import kuhn_mesh

    xyz, t = kuhn_mesh(WORKLOAD["n"], WORKLOAD["jitter"], WORKLOAD["mesh_seed"])
    return xyz, t, Problem(xyz, t, WORKLOAD["k"], workload_kappa(WORKLOAD, t.shape[0]))


def host_cpu():
    """CPU model and logical core count of the host (for the baseline record)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu model")):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"cpu_model": model or "unknown", "nproc": os.cpu_count()}


def run_cpu_oracle(steps, warmup, sample_iters=ORACLE_SAMPLE_ITERS, batched=False, mesh_n=0):
    """The oracle, as it stands, on one host core: assembly and setup timed separately
    (not part of the metric), then timed bounded samples of the solve (sample_iters PCG
    iterations each). The oracle solves one right-hand side at a time; on the multi-RHS
    workload a sample is one column."""
    import oracle
    from paper_1204_2586_gb300.inputs import kuhn_mesh, rhs_normal

    wl = dict(BATCHED if batched else WORKLOAD)
    if mesh_n:
        wl["n"] = mesh_n
    xyz, t = kuhn_mesh(wl["n"], wl["jitter"], wl["mesh_seed"])
    t0 = time.perf_counter()
    P = oracle.Problem(xyz, t, wl["k"], workload_kappa(wl, t.shape[0]))
    t1 = time.perf_counter()
    if batched:
        P.setup(theta=0.25, level_smoother=LEVEL_SMOOTHER, max_iter=sample_iters, flexible=1)
        b = rhs_normal(P.nh, 1, wl["rhs_seed"])[:, 0]
    else:
        P.setup(theta=0.25, level_smoother=LEVEL_SMOOTHER, max_iter=sample_iters)
        b = None
    t2 = time.perf_counter()
    times, iters = [], []
    for i in range(warmup + steps):
        t0s = time.perf_counter()
        out = P.solve(b)
        dt = time.perf_counter() - t0s
        if i >= warmup:
            times.append(dt)
            iters.append(out["iters"])
    tot = sum(times)
    value = P.nh * sum(iters) / tot / 1e6
    what = "one column (FP64 flexible CG)" if batched else "the solve"
    rec = dict(value=value, unit=UNIT, cores=1, kind="oracle",
               sample=f"{steps} timed runs of {sample_iters} PCG iterations each of {what} on the "
                      f"full workload (n_h={P.nh}); single-threaded C oracle; assembly and setup "
                      "timed separately, outside the metric",
               seconds=tot, oracle_assemble_s=t1 - t0, oracle_setup_s=t2 - t1,
               seconds_per_iteration=tot / max(1, sum(iters)))
    rec.update(host_cpu())
    return value, rec


def reference_arm(args):
    """The oracle as it stands, timed on the host's cores for the same workload: one
    step = a bounded sample of the solve (PCG from x0 = 0 stopped after a few iterations).
    Steps are independent, so they run concurrently on one thread per core (the oracle
    is plain single-threaded C; each call allocates its own work vectors and reads the
    assembled problem only), args.warmup untimed steps first, then exactly args.steps
    timed ones. value = n_h x iterations of the timed steps / their wall time."""
    ws, rank, _ = dist_env()
    if ws > 1 and rank != 0:
        return
    import concurrent.futures as cf

    import oracle
    from paper_1204_2586_gb300.inputs import kuhn_mesh, rhs_normal

    batched = args.workload == BATCHED["name"]
    wl = dict(BATCHED if batched else WORKLOAD)
    # iterations per step: P4 48^3 takes ~12 s per oracle iteration on one core
    sample = 2 if args.workload == P4["name"] else 4
    xyz, t = kuhn_mesh(wl["n"], wl["jitter"], wl["mesh_seed"])
    t0 = time.perf_counter()
    P = oracle.Problem(xyz, t, wl["k"], workload_kappa(wl, t.shape[0]))
    t1 = time.perf_counter()
    P.setup(theta=0.25, level_smoother=LEVEL_SMOOTHER, max_iter=sample, flexible=1 if batched else 0)
    t2 = time.perf_counter()
    b = rhs_normal(P.nh, 1, wl["rhs_seed"])[:, 0] if batched else P.rhs()
    threads = max(1, min(os.cpu_count() or 1, 16, args.steps))

    def one(_):
        return P.solve(b)["iters"]

    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(one, range(args.warmup)))
        ts = time.perf_counter()
        its = list(ex.map(one, range(args.steps)))
        wall = time.perf_counter() - ts
    value = P.nh * sum(its) / wall / 1e6
    cpu = dict(value=value, unit=UNIT, cores=threads, kind="oracle",
               sample=f"each step: PCG from x0 = 0 stopped after {sample} iterations "
                      f"({'one column, FP64 flexible CG' if batched else 'the solve'}) on the full workload "
                      f"(n_h={P.nh}); {args.steps} timed steps run concurrently on {threads} threads of the "
                      "single-threaded C oracle; assembly and setup timed separately, outside the metric",
               oracle_assemble_s=t1 - t0, oracle_setup_s=t2 - t1)
    cpu.update(host_cpu())
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": CONFIG_BATCHED if batched else CONFIG,
            "cpu_baseline": cpu, "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                                         "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def smoother_layout_name(code):
    if code == 0:
        return "SELL-32"
    if code == -1:
        return "CSR, lanes per colour"
    if code < -1:
        return f"one cooperative launch, CSR x{-code} lanes"
    if code > 400:
        return f"CSR x{code % 100} lanes, grid-stride over the resident blocks"
    if code > 100:
        return f"CSR x{code - 100} lanes, two rows per lane group"
    return f"CSR x{code} lanes"


def timed_solves(G, b, x, steps, warmup, clock=None):
    """warmup untimed solves, then `steps` solves bracketed by CUDA events on the
    launching stream (a device synchronize on both sides). Returns (ms total, iteration
    counts, kernel launches, last stats)."""
    import torch

    stream = torch.cuda.current_stream()

    def step():
        x.zero_()
        _, st = G.solve(b, x)
        assert st["status"][0] == 0, st
        return st

    for _ in range(warmup):
        step()
    ws, _, _ = dist_env()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    iters, launches, st = [], 0, None
    if clock is not None:
        clock.__enter__()
    try:
        torch.cuda.nvtx.range_push("timed_solves")  # lets ncu --nvtx-include select them
        e0.record(stream)
        for _ in range(steps):
            st = step()
            iters.append(st["iters"][0])
            launches += st["kernel_launches"]
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    finally:
        if clock is not None:
            clock.__exit__(None, None, None)
    if ws > 1:
        torch.distributed.barrier()
    return e0.elapsed_time(e1), iters, launches, st


def main():
    global WORKLOAD, CONFIG
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    choices=[WORKLOAD["name"], P4["name"], P2_8["name"], BATCHED["name"], ADJOINT["name"],
                             "theta_study", "cop_study", "stokes_study"])
    ap.add_argument("--smoother-layout", type=int, default=0,
                    help="pin the fine smoother layout (pkasp_options.smoother_layout) instead of "
                         "autotuning it; for profiler runs, under which the autotuner's timings "
                         "are distorted")
    ap.add_argument("--smoother-layout-fp32", type=int, default=0,
                    help="the same for the FP32-preconditioner solves")
    ap.add_argument("--mesh-n", type=int, default=0,
                    help="cubes per side of the mesh instead of the workload's own (a smaller case "
                         "of the same kernels for profiler captures; the JSON line states the size)")
    ap.add_argument("--eager", action="store_true",
                    help="launch the same kernels without the CUDA graph (profilers cannot see "
                         "kernels inside graphs that hold conditional nodes)")
    ap.add_argument("--only-fp64", action="store_true",
                    help="time the FP64 solve only (profiler runs): no e2e, FP32, l1-Jacobi or "
                         "FGMRES legs")
    ap.add_argument("--only-fp32", action="store_true",
                    help="time the FP32-preconditioner solve only (profiler runs), with "
                         "--smoother-layout-fp32")
    args = ap.parse_args()
    if args.mesh_n and args.workload not in SINGLE and args.workload != BATCHED["name"]:
        ap.error("--mesh-n applies to the p3, p4 and multi-RHS workloads")
    if args.warmup < 3:
        args.warmup = 3
    if args.workload == ADJOINT["name"]:
        WORKLOAD, CONFIG = ADJOINT, CONFIG_ADJOINT
    if args.workload in SINGLE:
        WORKLOAD, CONFIG = SINGLE[args.workload]
        if args.mesh_n:  # a smaller case of the same workload (profiler captures)
            WORKLOAD = dict(WORKLOAD, n=args.mesh_n)
            CONFIG = dict(CONFIG, workload=f"{CONFIG['workload']} -- REDUCED to {args.mesh_n}^3 cubes "
                                           "(--mesh-n), not the named workload")
    if args.impl == "reference":
        reference_arm(args)
        return

    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    from paper_1204_2586_gb300 import build

    build.build()
    if args.workload == "theta_study":
        run_theta_study(args)
        return
    if args.workload == "cop_study":
        run_cop_study(args)
        return
    if args.workload == "stokes_study":
        run_stokes_study(args)
        return
    if args.workload == ADJOINT["name"]:
        run_adjoint(args, ws, rank, local)
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    if args.workload == BATCHED["name"]:
        run_batched(args, ws, rank, local)
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    t_as = time.perf_counter()
    xyz, tets, G = make_problem()
    torch.cuda.synchronize()
    assemble_s = time.perf_counter() - t_as
    graph = 0 if args.eager else 1
    t_su = time.perf_counter()
    if args.only_fp32:
        G.setup(theta=0.25, level_smoother=LEVEL_SMOOTHER, use_graph=graph, precond_precision=1,
                smoother_layout=args.smoother_layout_fp32)
    else:
        G.setup(theta=0.25, level_smoother=LEVEL_SMOOTHER, use_graph=graph, smoother_layout=args.smoother_layout)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_su
    b = G.rhs()
    x = torch.zeros_like(b)
    nh = G.nh

    clk = ClockSampler(local)
    ms, iters, launches, st = timed_solves(G, b, x, args.steps, args.warmup, clock=clk)
    ms, work = replica_totals(ms, nh * sum(iters))
    value = work / (ms / 1e3) / 1e6
    sol_s = ms / 1e3 / args.steps
    true_rel64 = st["true_rel"][0]
    info64 = G.info
    if args.only_fp64 or args.only_fp32:
        if rank == 0:
            flag = "--only-fp32" if args.only_fp32 else "--only-fp64"
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                              "warmup": args.warmup, "ms_per_step": ms / args.steps, "config": CONFIG,
                              "note": f"{flag} profiler run: not a bench line"}))
        return

    # end to end through the C ABI with pinned host buffers: H2D of b, D2H of x (the solve
    # starts from x0 = 0 through pkasp_solve_from_zero, so no x0 is uploaded)
    bh = torch.empty(nh, dtype=torch.float64, pin_memory=True)
    bh.copy_(b.cpu())
    xh = torch.zeros(nh, dtype=torch.float64, pin_memory=True)
    bnp, xnp = bh.numpy(), xh.numpy()
    for _ in range(2):
        G.solve(bnp, xnp, from_zero=True)
    torch.cuda.synchronize()
    e_iters, e_dev = [], []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _, ste = G.solve(bnp, xnp, from_zero=True)
        e_dev.append(ste["solve_ms"])
        e_iters.append(ste["iters"][0])
    e2e_s = time.perf_counter() - t0
    e2e_ms, e2e_work = replica_totals(e2e_s * 1e3, nh * sum(e_iters))
    e2e_value = e2e_work / (e2e_ms / 1e3) / 1e6

    # Rooflines, measured with CUDA events on the launching stream (pkasp_time_kernel).
    # Dominant kernel by the launch list of a solve: the colour phases of the fine
    # smoother S_k. Algorithmic bytes of one S_k application (all its phases): each
    # off-diagonal entry once (FP64 value + int32 column = 12 B) and per row 52 B (inverse
    # diagonal, r, y written then read-modified, two part pointers, row index); a phase's
    # average rate is this total over the application's time. Its FP64 work: one FMA per
    # off-diagonal entry and 3 flops per row and half sweep. The fine SpMV: 12 B per
    # nonzero + 20 B per row.
    spmv_ms = G.time_kernel(0, 50)
    smoother_ms = G.time_kernel(1, 20)
    # the same loads without the colour dependencies (all rows at once): the memory work
    # of one S_k application with no barrier between its phases
    nodep_ms = G.time_kernel(7, 20)
    # the GPU's random 8-byte gather rate from a vector of n_h values (pkasp_time_kernel
    # mode 8 returns nanoseconds per gather): the colour phases gather one value per
    # off-diagonal entry, and their L2 sector traffic, not DRAM bytes, binds them
    gather_ns = G.time_kernel(8, 5)
    nnz = int(info64.nnz_h)
    spmv_bytes = 12 * nnz + 20 * nh
    smoother_bytes = 12 * (nnz - nh) + 52 * nh
    smoother_flops = 2.0 * (nnz - nh) + 6.0 * nh
    pk = peaks()
    hbm = pk.get("hbm_gbs")
    peak = hbm if hbm else 6800.0
    src = "measured (MEASURED_PEAKS.json hbm_gbs)" if hbm else "fallback"
    s_ach = smoother_bytes / (smoother_ms / 1e3) / 1e9
    s_tf = smoother_flops / (smoother_ms / 1e3) / 1e12
    roof = {"bound": "hbm", "kernel": "k_gs_phase (colour phases of the fine SGS S_k, FP64)",
            "achieved": s_ach, "peak": peak, "unit": "GB/s", "frac": s_ach / peak,
            "traffic": SMOOTHER_TRAFFIC.get((WORKLOAD["name"], WORKLOAD["n"], smoother_layout_name(
                info64.smoother_layout))),
            "traffic_note": "ncu dram__bytes_read+write summed over the 81 launches of one application, "
                            "profiles/k_gs_phase_p4_n48.md",
            "frac_of_nominal_8000": s_ach / NOMINAL_HBM_GBS,
            "peak_source": src, "bytes_per_application": smoother_bytes, "ms_per_application": smoother_ms,
            "phases_per_application": 2 * int(info64.fine_colours) - 1,
            "dependency_free_pass_ms": nodep_ms,
            "gather_roof": {"achieved_Ggathers_per_s": (nnz - nh) / (smoother_ms / 1e3) / 1e9,
                            "peak_Ggathers_per_s": 1.0 / gather_ns,
                            "frac": (nnz - nh) / (smoother_ms / 1e3) / 1e9 * gather_ns,
                            "peak_source": "measured live: random 8-byte gathers from an n_h vector "
                                           "(pkasp_time_kernel mode 8)"},
            "dependency_free_pass_frac": (smoother_bytes / (nodep_ms / 1e3) / 1e9) / peak,
            "fp64_pipe": {"achieved_tflops": s_tf, "peak_tflops": FP64_PEAK_TFLOPS,
                          "frac": s_tf / FP64_PEAK_TFLOPS, "flops_per_application": smoother_flops,
                          "peak_source": "derived: 152 SMs x 2.07 GHz x 4 FP64 flop/clk/SM"}}
    achieved = spmv_bytes / (spmv_ms / 1e3) / 1e9
    roof_spmv = {"bound": "hbm", "kernel": "k_spmv_q / k_sell_spmv (fine SpMV, SELL-32, FP64)",
                 "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                 "frac_of_nominal_8000": achieved / NOMINAL_HBM_GBS,
                 "traffic": SPMV_TRAFFIC.get((WORKLOAD["name"], WORKLOAD["n"])),
                 "traffic_note": "ncu dram__bytes_read+write per launch (mean of 3), profiles/k_spmv_q_p4_n48.md",
                 "peak_source": src, "bytes_per_launch": spmv_bytes, "ms_per_launch": spmv_ms}

    def leg(**kw):
        """Another configuration of the same solve, timed like the headline: CUDA events
        around args.steps solves after the warm-up ones; mean time per solve."""
        G.setup(theta=0.25, level_smoother=LEVEL_SMOOTHER, use_graph=graph, **kw)
        lms, lit, _, lst = timed_solves(G, b, x, args.steps, args.warmup)
        return {"iterations": lit[-1], "time_to_solution_s": lms / args.steps / 1e3,
                "true_rel_residual": lst["true_rel"][0],
                "mdof_iter_per_s": nh * sum(lit) / (lms / 1e3) / 1e6,
                "smoother_layout": smoother_layout_name(G.info.smoother_layout)}, x.clone()

    x64 = x.clone()
    # the mixed-precision variant: FP32 smoother / I_P / AMG, FP64 flexible CG
    fp32, x32 = leg(precond_precision=1, smoother_layout=args.smoother_layout_fp32)
    fp32["speedup_vs_fp64"] = sol_s / fp32["time_to_solution_s"]
    fp32["rel_diff_vs_fp64_solution"] = float(torch.linalg.norm(x32 - x64) / torch.linalg.norm(x64))
    # the l1-Jacobi smoother for S_k (the benchmark spec allows it): no pass over A_h from zero
    l1_64, _ = leg(smoother=1)
    l1_32, _ = leg(smoother=1, precond_precision=1)
    # the paper's own outer setting (Sec. 6.2): FGMRES(30) with the multiplicative form
    # (Algorithm 2.1 with pre-smoothing), FP64, same tolerance; and FGMRES with the additive form
    krylov_cmp = {}
    for mode, name in ((1, "fgmres_multiplicative"), (0, "fgmres_additive")):
        G.setup(theta=0.25, level_smoother=LEVEL_SMOOTHER, mode=mode, krylov=1, restart=30, use_graph=graph)
        msg = []
        for i in range(5):
            x.zero_()
            _, stg = G.solve(b, x)
            if i >= 2:
                msg.append(stg["solve_ms"])
        krylov_cmp[name] = {"iterations": stg["iters"][0], "time_to_solution_s": sum(msg) / len(msg) / 1e3,
                            "true_rel_residual": stg["true_rel"][0], "restarts": stg["restarts"]}
    extra = {"time_to_solution_s": sol_s, "iterations": iters[-1], "true_rel_residual": true_rel64,
             "setup_s": setup_s, "assemble_s": assemble_s, "levels": int(info64.levels),
             "l2_persist_bytes": int(info64.l2_persist_bytes),
             "level_rows": [int(v) for v in info64.level_rows[: info64.levels]],
             "fine_colours": int(info64.fine_colours), "op_complexity": info64.op_complexity,
             "spmv_layout": "SELL-32" if info64.spmv_layout == 0 else f"CSR x{info64.spmv_layout} lanes",
             "smoother_layout": smoother_layout_name(info64.smoother_layout),
             "smoother_ms": smoother_ms, "smoother_GBps": s_ach, "spmv_ms": spmv_ms,
             "fp32_preconditioner": fp32,
             "fp32_precond_time_to_solution_s": fp32["time_to_solution_s"],
             "fp32_precond_speedup_vs_fp64": fp32["speedup_vs_fp64"],
             "l1_jacobi_smoother": {"fp64": l1_64, "fp32_preconditioner": l1_32},
             "outer_iteration_comparison": krylov_cmp}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        try:
            p3 = WORKLOAD["name"] == "p3_n32"
            _, cpu = run_cpu_oracle(1, 0, sample_iters=ORACLE_SAMPLE_ITERS if p3 else 2)
            cpu.pop("seconds", None)
        except Exception as e:  # the baseline must not sink the GPU line
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {e}"}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": CONFIG, "clocks": clk.summary(),
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * nh,
                        "d2h_bytes_per_step": 8 * nh, "ms_per_step": e2e_ms / args.steps,
                        "solve_ms_per_step": sum(e_dev) / len(e_dev)},
                "gpu_launches": launches, "roofline": roof, "roofline_spmv": roof_spmv,
                "cpu_baseline": cpu}
        line.update(extra)
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


THETA_STUDY = [(2, 32), (3, 24), (4, 16)]  # (k, cubes per side)


def run_theta_study(args):
    """Iteration counts and times of the auxiliary-space preconditioner (additive PCG)
    against plain AMG on A_h (one V-cycle, PCG), for strength thresholds 0.25 / 0.5 / 0.8:
    the comparison of the paper's Table 1 (AMG on P_k matrices degrades as theta and k
    grow) and Tables 2-4 (the auxiliary space is robust in theta). Prints one JSON line."""
    import torch

    from paper_1204_2586_gb300 import Problem
    from paper_1204_2586_gb300.inputs import kuhn_mesh

    rows = []
    for k, n in THETA_STUDY:
        xyz, t = kuhn_mesh(n, 0.2, 0)
        G = Problem(xyz, t, k)
        b = G.rhs()
        for theta in (0.25, 0.5, 0.8):
            for mode, name in ((0, "aux_space_additive"), (2, "plain_amg")):
                t0 = time.perf_counter()
                G.setup(theta=theta, mode=mode, level_smoother=LEVEL_SMOOTHER, max_iter=2000)
                torch.cuda.synchronize()
                setup_s = time.perf_counter() - t0
                x = torch.zeros_like(b)
                G.solve(b, x, raise_on_fail=False)
                x.zero_()
                _, st = G.solve(b, x, raise_on_fail=False)
                info = G.info
                rows.append({"k": k, "n": n, "n_h": G.nh, "theta": theta, "method": name,
                             "iterations": st["iters"][0], "status": st["status"][0],
                             "solve_s": st["solve_ms"] / 1e3, "setup_s": setup_s,
                             "levels": int(info.levels), "op_complexity": info.op_complexity})
        G.close()
    print(json.dumps({"study": "theta", "tol": 1e-8, "krylov": "PCG", "rows": rows}))


def run_cop_study(args):
    """Operator complexities against the paper's Table 6 (PMIS, theta 0.25): plain AMG on
    A_h (sum nnz(A_l) / nnz(A_h)), the P1 AMG of the auxiliary space (relative to A_H) and
    the whole auxiliary-space hierarchy relative to A_h ("GAMG": (nnz(A_h) + sum nnz of
    the P1 levels) / nnz(A_h)); with extended+i and extended+i+cc interpolation (the
    paper's), each without truncation and with at most 4 interpolation weights per row.
    Iterations and times beside them. One JSON line."""
    import torch

    from paper_1204_2586_gb300 import Problem
    from paper_1204_2586_gb300.inputs import kuhn_mesh

    rows = []
    for k, n in THETA_STUDY:
        xyz, t = kuhn_mesh(n, 0.2, 0)
        G = Problem(xyz, t, k)
        b = G.rhs()
        nnz_h = int(G.info.nnz_h)
        for cc, pmax in ((0, 0), (0, 4), (1, 0), (1, 4)):
            for mode, name in ((0, "aux_space_additive"), (2, "plain_amg")):
                t0 = time.perf_counter()
                G.setup(theta=0.25, mode=mode, level_smoother=LEVEL_SMOOTHER, interp_pmax=pmax, interp_cc=cc,
                        max_iter=2000)
                torch.cuda.synchronize()
                setup_s = time.perf_counter() - t0
                x = torch.zeros_like(b)
                G.solve(b, x, raise_on_fail=False)
                x.zero_()
                _, st = G.solve(b, x, raise_on_fail=False)
                info = G.info
                lev_nnz = [int(info.level_nnz[l]) for l in range(info.levels)]
                row = {"k": k, "n": n, "n_h": G.nh, "interp": "ext+i+cc" if cc else "ext+i",
                       "interp_pmax": pmax, "method": name,
                       "iterations": st["iters"][0], "solve_s": st["solve_ms"] / 1e3, "setup_s": setup_s,
                       "levels": int(info.levels)}
                if mode == 2:
                    row["cop_amg_on_Ah"] = sum(lev_nnz) / lev_nnz[0]
                else:
                    row["cop_p1_amg"] = sum(lev_nnz) / lev_nnz[0]
                    row["cop_gamg_rel_Ah"] = (nnz_h + sum(lev_nnz)) / nnz_h
                rows.append(row)
        G.close()
    print(json.dumps({"study": "operator_complexity", "theta": 0.25, "rows": rows,
                      "paper_table6": {"P2": {"AMG": 1.67, "P1-AMG": 1.76, "GAMG": 1.12},
                                       "P3": {"AMG": 1.56, "P1-AMG": 1.96, "GAMG": 1.02},
                                       "P4": {"AMG": 1.36, "P1-AMG": 1.70, "GAMG": 1.01}}}))


STOKES_STUDY = [(2, 12), (2, 24), (3, 8), (3, 16), (4, 6), (4, 12)]  # (k, cubes per side)


def run_stokes_study(args):
    """Taylor-Hood P_k - P_{k-1} Stokes (Sec. 5, Sec. 6.3): FGMRES(30) with the block
    upper-triangular preconditioner Q_t (one auxiliary-space cycle per velocity component,
    10 diagonal-PCG steps on the pressure mass matrix), theta = 0.8 as in Sec. 6.3, to
    relative residual 1e-8; two mesh sizes per k show whether the step count grows with
    the number of unknowns. The right-hand side has i.i.d. N(0,1) velocity entries
    (seed 2) and a zero pressure part. One JSON line."""
    import numpy as np
    import torch

    from paper_1204_2586_gb300 import Problem
    from paper_1204_2586_gb300.inputs import kuhn_mesh, rhs_normal

    rows = []
    for k, n in STOKES_STUDY:
        xyz, t = kuhn_mesh(n, 0.2, 0)
        G = Problem(xyz, t, k)
        G.setup(theta=0.8, level_smoother=LEVEL_SMOOTHER, max_iter=1000)
        t0 = time.perf_counter()
        G.stokes_setup(10)
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        nu = 3 * G.stokes_nh
        b = torch.tensor(np.concatenate([rhs_normal(nu, 1, 2)[:, 0], np.zeros(G.stokes_np)]), device="cuda")
        x = torch.zeros_like(b)
        G.stokes_solve(b, x)
        x.zero_()
        _, st = G.stokes_solve(b, x)
        rows.append({"k": k, "n": n, "velocity_unknowns": nu, "pressure_unknowns": G.stokes_np,
                     "unknowns": G.stokes_n, "iterations": st["iters"], "restarts": st["restarts"],
                     "status": st["status"], "true_rel_residual": st["true_rel"],
                     "solve_s": st["solve_ms"] / 1e3, "stokes_setup_s": setup_s})
        G.close()
    print(json.dumps({"study": "stokes_taylor_hood", "krylov": "FGMRES(30)", "preconditioner": "Q_t",
                      "theta": 0.8, "tol": 1e-8, "rows": rows}))


def run_batched(args, ws, rank, local):
    """One step = one blocked PCG solve of all 48 columns from X0 = 0. value counts every
    column's iterations: n_h * sum_c iters_c / time."""
    import numpy as np
    import torch

    from paper_1204_2586_gb300 import Problem
    from paper_1204_2586_gb300.inputs import kuhn_mesh, rhs_normal

    wl = dict(BATCHED)
    config = dict(CONFIG_BATCHED)
    if args.mesh_n:
        wl["n"] = args.mesh_n
        config["workload"] = f"{wl['n']}^3-cube case of: " + config["workload"]
    t_as = time.perf_counter()
    xyz, tets = kuhn_mesh(wl["n"], wl["jitter"], wl["mesh_seed"])
    G = Problem(xyz, tets, wl["k"])
    torch.cuda.synchronize()
    assemble_s = time.perf_counter() - t_as
    graph = 0 if args.eager else 1
    t_su = time.perf_counter()
    G.setup(theta=0.25, level_smoother=LEVEL_SMOOTHER, precond_precision=1, use_graph=graph)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_su
    nh, nc = G.nh, wl["ncols"]
    config["n_h"] = nh
    Bh = rhs_normal(nh, nc, wl["rhs_seed"])
    B = torch.tensor(Bh, device="cuda")
    X = torch.zeros_like(B)
    stream = torch.cuda.current_stream()

    def step():
        X.zero_()
        _, st = G.solve(B, X)
        return st

    for _ in range(args.warmup):
        st = step()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    col_iters, launches = [], 0
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("timed_solves")
        e0.record(stream)
        for _ in range(args.steps):
            st = step()
            col_iters.append(sum(st["iters"]))
            launches += st["kernel_launches"]
            assert st["rc"] == 0 and all(v == 0 for v in st["status"]), st
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    if ws > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    ms, work = replica_totals(ms, nh * sum(col_iters))
    value = work / (ms / 1e3) / 1e6
    sol_s = ms / 1e3 / args.steps
    info = G.info
    max_true_rel = max(st["true_rel"])

    # end to end through the C ABI with pinned host blocks: H2D of B, D2H of X (from
    # X0 = 0 through pkasp_solve_from_zero: no X0 is uploaded)
    bh = torch.empty((nh, nc), dtype=torch.float64, pin_memory=True)
    bh.copy_(torch.from_numpy(Bh))
    xh = torch.zeros((nh, nc), dtype=torch.float64, pin_memory=True)
    bnp, xnp = bh.numpy(), xh.numpy()
    for _ in range(2):
        G.solve(bnp, xnp, from_zero=True)
    torch.cuda.synchronize()
    e_iters, e_dev = [], []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _, st = G.solve(bnp, xnp, from_zero=True)
        e_dev.append(st["solve_ms"])
        e_iters.append(sum(st["iters"]))
    e2e_s = time.perf_counter() - t0
    e2e_ms, e2e_work = replica_totals(e2e_s * 1e3, nh * sum(e_iters))
    e2e_value = e2e_work / (e2e_ms / 1e3) / 1e6

    # roofline of the dominant kernel, the blocked FP64 SpMM Q = A_h P with its per-column
    # dot (P, Q): 48 FP64 FMA per stored entry and column, so it is bound by the FP64 pipe
    # (algorithmic flops 2 nnz NC + 2 n NC), not by HBM (12 nnz + 24 n NC bytes)
    nnz = int(info.nnz_h)
    spmm_ms = G.time_kernel(4, 10)
    flops = 2.0 * nnz * nc + 2.0 * nh * nc
    ach = flops / (spmm_ms / 1e3) / 1e12
    roof = {"bound": "alu", "kernel": "kb_spmv_pq<48> (blocked FP64 SpMM + per-column dot)",
            "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS,
            "traffic": None, "peak_source": "derived: 152 SMs x 2.07 GHz x 4 FP64 flop/clk/SM",
            "flops_per_launch": flops, "ms_per_launch": spmm_ms,
            "hbm_bytes_per_launch": 12 * nnz + 20 * nh + 16 * nh * nc}
    # the blocked FP32 fine smoother (all colour phases of one S_k application on 48
    # columns): algorithmic bytes 8 per off-diagonal entry (FP32 value + int32 column),
    # per row 20 B of indices/inverse diagonal and per row and column 8 B of r (FP64),
    # 4 B of y written forward, 8 B of y read and rewritten backward
    sm_ms = G.time_kernel(5, 5)
    layout = (int(G.info.block_width), int(G.info.block_group), int(G.info.block_lanes))
    sm_bytes = 8 * (nnz - nh) + 20 * nh + 20 * nh * nc
    pk = peaks()
    hbm = pk.get("hbm_gbs") or 6800.0
    roof_sm = {"bound": "hbm", "kernel": "kb_gs_phase<*, float> (blocked FP32 fine SGS)",
               "achieved": sm_bytes / (sm_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
               "frac": sm_bytes / (sm_ms / 1e3) / 1e9 / hbm, "traffic": None,
               "frac_of_nominal_8000": sm_bytes / (sm_ms / 1e3) / 1e9 / NOMINAL_HBM_GBS,
               "ms_per_application": sm_ms, "bytes_per_application": sm_bytes,
               "column_group": layout[1], "lanes_per_row": layout[2]}
    prec_ms = G.time_kernel(6, 5)

    # the same block with an FP64 preconditioner, and one column solved alone
    G.setup(theta=0.25, level_smoother=LEVEL_SMOOTHER, precond_precision=0, use_graph=graph)
    for _ in range(2):
        st64 = step()
    ms64 = min(step()["solve_ms"] for _ in range(3))
    G.setup(theta=0.25, level_smoother=LEVEL_SMOOTHER, precond_precision=1, use_graph=graph)
    b1 = B[:, 0].contiguous()
    x1 = torch.zeros_like(b1)
    for _ in range(2):
        x1.zero_()
        G.solve(b1, x1)
    one = []
    for _ in range(3):
        x1.zero_()
        one.append(G.solve(b1, x1)[1]["solve_ms"])
    extra = {"time_to_solution_s": sol_s, "column_iterations_min": min(st["iters"]),
             "column_iterations_max": max(st["iters"]), "max_true_rel_residual": max_true_rel,
             "setup_s": setup_s, "assemble_s": assemble_s, "levels": int(info.levels),
             "fine_colours": int(info.fine_colours), "block_width": layout[0],
             "preconditioner_ms": prec_ms,
             "fp64_precond_time_to_solution_s": ms64 / 1e3,
             "single_column_time_to_solution_s": min(one) / 1e3,
             "speedup_vs_48_single_column_solves": 48 * min(one) / 1e3 / sol_s}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        try:
            _, cpu = run_cpu_oracle(1, 0, sample_iters=6, batched=True, mesh_n=args.mesh_n)
            cpu.pop("seconds", None)
        except Exception as e:
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {e}"}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": config, "clocks": clk.summary(),
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * nh * nc,
                        "d2h_bytes_per_step": 8 * nh * nc, "ms_per_step": e2e_ms / args.steps,
                        "solve_ms_per_step": sum(e_dev) / len(e_dev)},
                "gpu_launches": launches, "roofline": roof, "roofline_smoother": roof_sm,
                "cpu_baseline": cpu}
        line.update(extra)
        print(json.dumps(line))


def run_adjoint(args, ws, rank, local):
    """One step = forward solve, adjoint solve and dL/dkappa (the backward pass of the
    differentiable solve for L = 0.5 ||u - u_obs||^2), inputs resident on the device.
    value = n_h * (forward + adjoint iterations) / time. e2e: the same through the public
    differentiable API (autograd.solve + loss.backward()) with kappa uploaded from pinned
    host memory and dL/dkappa read back every step; that path also re-assembles A_h for
    kappa and rebuilds the preconditioner inside every forward call."""
    import torch

    from paper_1204_2586_gb300 import Problem
    from paper_1204_2586_gb300 import autograd as pag
    from paper_1204_2586_gb300.inputs import kappa_lognormal, kuhn_mesh

    wl = ADJOINT
    prec = dict(theta=0.25, level_smoother=LEVEL_SMOOTHER, precond_precision=1,
                use_graph=0 if args.eager else 1)
    t_as = time.perf_counter()
    xyz, tets = kuhn_mesh(wl["n"], wl["jitter"], wl["mesh_seed"])
    nt = tets.shape[0]
    kap_obs = kappa_lognormal(nt, wl["obs_kappa_seed"])
    kap = kappa_lognormal(nt, wl["kappa_seed"])
    G = Problem(xyz, tets, wl["k"], kap_obs)
    torch.cuda.synchronize()
    assemble_s = time.perf_counter() - t_as
    G.setup(**prec)
    b = G.rhs()
    u_obs, st_obs = G.solve(b)
    assert st_obs["status"][0] == 0, st_obs
    G.set_kappa(kap)
    t_su = time.perf_counter()
    G.setup(**prec)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_su
    nh = G.nh
    u = torch.zeros_like(b)
    lam = torch.zeros_like(b)
    stream = torch.cuda.current_stream()

    def step():
        u.zero_()
        _, st = G.solve(b, u)
        g = u - u_obs
        lam.zero_()
        _, sta = G.solve_adjoint(g, lam)
        dk = G.grad_kappa(u, lam)
        assert st["status"][0] == 0 and sta["status"][0] == 0, (st, sta)
        return st["iters"][0] + sta["iters"][0], st, sta, dk

    launches = 0

    for _ in range(args.warmup):
        step()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    its = []
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("timed_solves")
        e0.record(stream)
        for _ in range(args.steps):
            n_it, st, sta, dk = step()
            its.append(n_it)
            launches += st["kernel_launches"] + sta["kernel_launches"] + 1  # + k_grad_kappa
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    if ws > 1:
        torch.distributed.barrier()
    ms, work = replica_totals(e0.elapsed_time(e1), nh * sum(its))
    value = work / (ms / 1e3) / 1e6

    # end to end through torch.autograd: kappa from pinned host memory, dL/dkappa back
    kh = torch.tensor(kap, dtype=torch.float64).pin_memory()
    gh = torch.empty(nt, dtype=torch.float64).pin_memory()
    e_its = []

    def e2e_step():
        kd = kh.to("cuda", non_blocking=True).requires_grad_(True)
        uu = pag.solve(kd, b, G, **prec)
        loss = 0.5 * torch.sum((uu - u_obs) ** 2)
        loss.backward()
        gh.copy_(kd.grad)
        return uu

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
        e_its.append(its[-1])
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_ms, e2e_work = replica_totals(e2e_s * 1e3, nh * sum(e_its))
    e2e_value = e2e_work / (e2e_ms / 1e3) / 1e6
    extra = {"time_per_step_s": ms / 1e3 / args.steps, "forward_iterations": st["iters"][0],
             "adjoint_iterations": sta["iters"][0], "forward_true_rel_residual": st["true_rel"][0],
             "adjoint_true_rel_residual": sta["true_rel"][0], "setup_s": setup_s, "assemble_s": assemble_s,
             "grad_kappa_norm": float(torch.linalg.norm(dk))}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        try:
            _, cpu = run_cpu_oracle(1, 0)
            cpu.pop("seconds", None)
        except Exception as e:
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {e}"}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": CONFIG_ADJOINT, "clocks": clk.summary(),
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * nt,
                        "d2h_bytes_per_step": 8 * nt, "ms_per_step": e2e_ms / args.steps,
                        "includes": "re-assembly of A_h for kappa and the preconditioner setup in every "
                                    "forward call of the differentiable solve"},
                "gpu_launches": launches, "cpu_baseline": cpu}
        line.update(extra)
        print(json.dumps(line))


if __name__ == "__main__":
    main()
