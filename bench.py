"""Benchmark of the QTT fractional step (arXiv:2507.05222, Sec. III.C) on GB300.

Workload (the headline configuration): stationary cylinder, log-polar O-grid
r in [0.5, 20] D (R = 40), 2^10 x 2^10 cells (20 interleaved quantics bits), Re = 200,
dt = 8e-4, chi = 64, FP64.  Synthetic seeded state: uniform inflow plus a Gaussian
perturbation of amplitude 1e-3 on u and v, pressure zero padded with 1e-8 noise.
A step = one full fractional step: four MPO-MPS products with rounding, two fused
variational right-hand sides, two momentum ALS solves, one Poisson ALS solve, two
projection fits.

Output: one JSON line on rank 0 (see the build contract): steps/s over K device-timed steps
(L2 flushed between steps), end-to-end steps/s through host buffers, roofline of the FP64
GEMM (the dominant kernel class), clocks during the timed region, kernel launches, and the
FP64 oracle timed on the host cores as a baseline.

--impl reference times the FP64 oracle (the CPU program the GPU path is checked against)
on the same workload.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(workload="cylinder_qtt_step_2^20_chi64", n_eta=10, n_xi=10, ordering="interleaved", R=40.0,
                Re=200.0, dt=8e-4, chi=64, fit_sweeps=1, mom=(1, 8, 1e-10), poi=(2, 20, 1e-10), seed=0)
METRIC = "QTT fractional steps/s at 2^20 cells, chi=64, fixed oracle error; % TC/HBM roof"
FP64_PEAK_TFLOPS = 1.012   # FP64 FMA throughput measured on GB300 (independent FMA chains on all SMs)


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(values, world, device):
    """Per-rank timings reduced to their element-wise maximum over the job's ranks (every rank
    receives it); the identity on one rank.  device: "cuda" under NCCL, "cpu" under gloo."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def job_throughput(world, seconds_per_step):
    """Whole-job steps/s of `world` independent replicas whose slowest rank takes
    seconds_per_step per step (weak scaling: each rank advances its own case)."""
    return world / seconds_per_step


def initial_fields(cfg):
    from paper_2507_05222_gb300 import inputs
    ne, nx, chi, s = cfg["n_eta"], cfg["n_xi"], cfg["chi"], cfg["seed"]
    u0 = 1.0 + inputs.gaussian_field(ne, nx, s + 1, 1e-3)
    v0 = inputs.gaussian_field(ne, nx, s + 2, 1e-3)
    pad = inputs.random_cores(ne + nx, chi, s + 3, scale=1e-8)
    return u0, v0, pad


class Clocks:
    """nvidia-smi sampling during the timed region (SM clock, throttle reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device, self.samples, self.proc = device, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm = [float(s[1]) for s in self.samples if len(s) >= 9 and s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if len(s) >= 9 and s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples if len(s) >= 9 for i in range(4) if s[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def oracle_steps(cfg, k_steps, budget_s=None):
    """Time the FP64 oracle (L1 QTT step, numpy) on the host cores; returns (steps/s, steps, s, cores)."""
    from oracle import qtt_ops as Q, step as S
    import numpy as np
    u0, v0, pad = initial_fields(cfg)
    ops = Q.Ops(cfg["n_eta"], cfg["n_xi"], cfg["R"], cfg["Re"], cfg["dt"], cfg["ordering"])
    u, v = ops.encode(u0, cfg["chi"]), ops.encode(v0, cfg["chi"])
    p = S.padded([np.zeros((1, 2, 1))] * (cfg["n_eta"] + cfg["n_xi"]), cfg["chi"], pad)
    o = S.StepOpts(chi=cfg["chi"], fit_sweeps=cfg["fit_sweeps"], mom_sweeps=cfg["mom"][0], mom_cg=cfg["mom"][1],
                   poi_sweeps=cfg["poi"][0], poi_cg=cfg["poi"][1], cg_tol=cfg["poi"][2])
    t0 = time.perf_counter()
    done = 0
    for _ in range(k_steps):
        u, v, p, _ = S.step(ops, u, v, p, o)
        done += 1
        if budget_s is not None and time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return done / dt, done, dt, len(os.sched_getaffinity(0))


def run_reference(args, cfg):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    for _ in range(args.warmup):
        pass  # the oracle has no warm-up state; its warm-up steps would only repeat the timed work
    sps, done, dt, cores = oracle_steps(cfg, args.steps)
    line = {"impl": "reference", "metric": METRIC, "value": sps, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": done, "warmup": args.warmup, "ms_per_step": 1e3 * dt / done, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {k: cfg[k] for k in ("workload", "n_eta", "n_xi", "chi", "Re", "dt", "R", "ordering")},
            "cpu_baseline": {"value": sps, "unit": "steps/s", "cores": cores, "kind": "oracle",
                             "sample": f"{done} full fractional steps of the workload (numpy FP64 oracle)"},
            "e2e": {"value": sps, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_ours(args, cfg):
    import torch
    import torch.distributed as dist
    from paper_2507_05222_gb300 import qtt
    rank, world, local = env_rank()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    ctx = qtt.Context(local)
    if args.gemm_mode is not None:
        ctx.set_gemm_mode(args.gemm_mode)
    if args.cg_mode is not None:
        ctx.set_cg_mode(args.cg_mode)
    ne, nx, chi = cfg["n_eta"], cfg["n_xi"], cfg["chi"]
    case = qtt.Case(ctx, ne, nx, cfg["R"], cfg["Re"], cfg["dt"], chi, cfg["ordering"], fit_sweeps=cfg["fit_sweeps"],
                    mom=cfg["mom"], poi=cfg["poi"])
    u0, v0, pad = initial_fields(cfg)
    gu = qtt.qtt_encode(ctx, qtt.qtt_field_to_vector(ctx, u0, cfg["ordering"]), ne + nx, chi)
    gv = qtt.qtt_encode(ctx, qtt.qtt_field_to_vector(ctx, v0, cfg["ordering"]), ne + nx, chi)
    gp = qtt.MPS.from_cores(ctx, pad)
    case.set_state(gu, gv, gp)
    if args.kernel_probe:
        Dx = case.operator(0)
        u, _, _ = case.get_state()
        qtt.mpo_apply_round(ctx, Dx, u, chi)
        ctx.sync()
        qtt.profiler_range(True)
        qtt.mpo_apply_round(ctx, Dx, u, chi)
        ctx.sync()
        qtt.profiler_range(False)
        return
    if args.phase_breakdown:
        # kernel-class time by step phase, kernels launched one by one (eager), next to the
        # phase wall times of a replayed graph step
        for _ in range(2):
            qtt.fractional_step(ctx, case, 1, info=False)
        ctx.sync()
        graph_phases = case.phase_ms()
        case.use_graph(False)
        qtt.fractional_step(ctx, case, 1, info=False)
        ctx.sync()
        ctx.profile(True)
        qtt.fractional_step(ctx, case, 1, info=False)
        ctx.profile(False)
        print(json.dumps({"graph_phase_ms": graph_phases, "eager_phase_ms": case.phase_ms(),
                          "eager_kernel_ms_by_phase": ctx.profile_phases()}))
        return
    if args.profile_one_step:
        qtt.fractional_step(ctx, case, 1, info=False)
        ctx.sync()
        qtt.profiler_range(True)
        qtt.fractional_step(ctx, case, 1, info=False)
        ctx.sync()
        qtt.profiler_range(False)
        return
    flush = torch.empty(int(256 * 2 ** 20 // 4), dtype=torch.float32, device="cuda")  # 256 MB > L2 (129 MB)
    stream = ctx.stream
    for _ in range(args.warmup):
        qtt.fractional_step(ctx, case, 1, info=False)
    ctx.sync()
    # ---- timed region: K device-timed steps, L2 flushed between steps (outside the events)
    clocks = Clocks(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    n0 = ctx.kernel_launches()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            qtt.fractional_step(ctx, case, 1, info=False)
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    launches = ctx.kernel_launches() - n0
    phases = case.phase_ms()
    ms = [a.elapsed_time(b) for a, b in ev]
    clk = clocks.stop()
    step_ms = sum(ms) / len(ms)
    # ---- per-class kernel timing (roofline of the dominant class): the same kernels launched one
    # by one (timing events cannot sit inside the captured graph), L2 flushed between steps
    case.use_graph(False)
    ctx.profile(True)
    for k in range(min(args.steps, 2)):
        flush.fill_(float(k))
        qtt.fractional_step(ctx, case, 1, info=False)
    prof = ctx.profile(False)
    case.use_graph(True)
    nprof = min(args.steps, 2)
    g = prof["gemm_f64"]
    achieved = g["flops"] / (g["ms"] * 1e-3) / 1e12 if g["ms"] > 0 else 0.0
    # ---- end to end through the C ABI with host buffers: state cores in from pinned host
    # memory, one step, state cores and force coefficients back to the host
    state = case.get_state()
    bonds = [x.bonds() for x in state]
    sizes = [int(sum(b[k] * 2 * b[k + 1] for k in range(len(b) - 1))) for b in bonds]
    pin_in = [torch.empty(sz, dtype=torch.float64).pin_memory() for sz in sizes]
    pin_out = [torch.empty(sz, dtype=torch.float64).pin_memory() for sz in sizes]
    for x, t in zip(state, pin_in):
        x.get_flat(t.data_ptr())
    h2d = sum(sizes) * 8
    d2h = sum(sizes) * 8 + 40

    def e2e_step():
        fields = [qtt.MPS.from_flat(ctx, b, 2, t.data_ptr()) for b, t in zip(bonds, pin_in)]
        case.set_state(*fields)
        info = qtt.fractional_step(ctx, case, 1, with_forces=True)
        for x, t in zip(case.get_state(), pin_out):
            x.get_flat(t.data_ptr())
        return info

    e2e_step()   # untimed: captures the step's graph with the force read-out once
    t0 = time.perf_counter()
    for k in range(args.steps):
        info = e2e_step()
    e2e_s = (time.perf_counter() - t0) / args.steps
    step_ms, e2e_s = max_over_ranks([step_ms, e2e_s], world, "cuda")   # the slowest rank
    # ---- CPU baseline: the FP64 oracle on the host cores, one step of the same workload
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        sps, done, dt, cores = oracle_steps(cfg, 2, budget_s=20.0)
        cpu = {"value": sps, "unit": "steps/s", "cores": cores, "kind": "oracle",
               "sample": f"{done} full fractional step(s) of the workload, numpy FP64 oracle, {dt:.1f} s"}
    if rank == 0:
        line = {"metric": METRIC, "value": job_throughput(world, step_ms * 1e-3), "unit": "steps/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {k: cfg[k] for k in ("workload", "n_eta", "n_xi", "chi", "Re", "dt", "R", "ordering")}
                | {"mom_solve": list(cfg["mom"]), "poisson_solve": list(cfg["poi"]), "fit_sweeps": cfg["fit_sweeps"],
                   "l2": "256 MB buffer written between timed steps", "replicas": world,
                   **({"gemm_mode": args.gemm_mode} if args.gemm_mode is not None else {}),
                   **({"cg_mode": args.cg_mode} if args.cg_mode is not None else {})},
                "e2e": {"value": job_throughput(world, e2e_s), "unit": "steps/s", "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "gpu_launches": int(launches),
                "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                             "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                             "kernel": "core contractions: k_gemm + k_contract_direct (FP64 pipe) + k_oz_gemm (digit-split FP64 on "
                                       "the tensor cores), FP64-equivalent flops",
                             "share_of_step": g["ms"] / nprof / step_ms if step_ms > 0 else None},
                "kernel_classes_ms_per_step": {k: v["ms"] / nprof for k, v in prof.items() if not k.startswith("phase")},
                "phase_ms_last_timed_step": phases,
                "clocks": clk, "cpu_baseline": cpu,
                "last_step": {"cd": info[0]["cd"], "cl": info[0]["cl"]}}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=None, help="bits per direction (smaller test case)")
    ap.add_argument("--chi", type=int, default=None)
    ap.add_argument("--profile-one-step", action="store_true",
                    help="set up, one warm-up step, then one step between cudaProfilerStart/Stop (for ncu)")
    ap.add_argument("--gemm-mode", type=int, default=None, choices=(0, 1),
                    help="0: large products on the tensor cores (digit-split FP64); 1: FP64 pipe")
    ap.add_argument("--cg-mode", type=int, default=None, choices=(0, 1, 2, 3),
                    help="ALS local solves: 0 one cooperative kernel, tensor-core contractions at full-bond sites "
                         "(default); 1 one kernel per stage; 2 one FP64 cooperative kernel; 3 tensor cores wherever "
                         "the cooperative kernel fits")
    ap.add_argument("--phase-breakdown", action="store_true",
                    help="print kernel-class time by step phase (diagnostic; no bench line)")
    ap.add_argument("--kernel-probe", action="store_true",
                    help="set up, then one D_x u product with rounding between cudaProfilerStart/Stop (for ncu)")
    args = ap.parse_args()
    cfg = dict(WORKLOAD)
    if args.n is not None:
        cfg.update(n_eta=args.n, n_xi=args.n, workload=f"cylinder_qtt_step_2^{2 * args.n}_chi{args.chi or cfg['chi']}")
    if args.chi is not None:
        cfg.update(chi=args.chi, workload=f"cylinder_qtt_step_2^{cfg['n_eta'] + cfg['n_xi']}_chi{args.chi}")
    if args.impl == "reference":
        run_reference(args, cfg)
    else:
        run_ours(args, cfg)


if __name__ == "__main__":
    main()
