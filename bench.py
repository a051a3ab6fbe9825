#!/usr/bin/env python
"""Benchmark of the iterative polarizability solve on one GB300 (or N, each
solving its own share of the frequencies).

One step = one group of frequencies x 3 field directions solved to the
workload's tolerance through the whole hot path (RHS formation chi0 . d,
then GMRES with A z = z - chi0 (K z) until every right-hand side meets
||b - A x|| / ||b|| <= tol, then P = d . X).  The metric is omega-points/s
(an omega-point counts once all three directions converged).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload medium64]
    python bench.py --impl reference     # the CPU oracle on the host cores

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1005_5340_gb300 import synth  # noqa: E402

METRIC = "omega-points/s at 1e-6 rel. residual"
FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64 (DFMA) nominal rate; no tensor path for FP64
# FP32 CUDA-core peak from unit counts: 152 SMs x 128 lanes x 2 flops x 2.07 GHz
FP32_UNIT_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# kernel launches behind one timed scope (the others launch one kernel each)
KERNELS_PER_SCOPE = {"rhs_formation": 7, "emu_gemm_K": 2, "emu_gemm_T1": 2, "emu_gemm_T2": 2,
                     "emu_alpha_beta": 2, "emu_alpha_dot": 3, "tc_alpha_dot": 2}
# emulated right-hand-side formation: dipole rows, slice + step 2, slice + T1,
# expand, slice + T2, slice + step 5, combine
KERNELS_PER_SCOPE_EMU = dict(KERNELS_PER_SCOPE, rhs_formation=11)
# slice pairs of one emulated float64 product (s slices: pairs with i + j <= s + 1)
EMU_PAIRS = {"fp64emu": 21, "bf16x3emu": 15}

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the tensor-core products, from one-pass ncu captures of the default bench
# command (64-atom molecule, full batch of 192 right-hand sides):
#   T1 + D(omega) (gemm_tc_kernel<1, 256>): 168.1 + 91.4 MB for the algorithmic
#     2 n_virt n_orb N1 = 57.58 GFLOP (N1 = 49152); the B operand and the
#     output scale with N1, so the traffic is taken proportional to the flops;
#   K z (gemm_tc_kernel<0, 128>, clusters of 3 with split K): 388.2 + 17.9 MB,
#     the split kernel matrix read about once whatever the batch: per launch.
TRAFFIC = {"tc_gemm_T1_dscale": ("per_flop", (168.1e6 + 91.4e6) / 57.58e9),
           "tc_gemm_K": ("per_launch", 388.2e6 + 17.9e6)}


def traffic_of(name: str, flops_per_launch: float):
    if name not in TRAFFIC:
        return None
    kind, v = TRAFFIC[name]
    return v * flops_per_launch if kind == "per_flop" else v


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=4)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="medium64")
    p.add_argument("--omega-per-step", type=int, default=64)
    p.add_argument("--e2e-steps", type=int, default=1)
    p.add_argument("--cpu-sample", type=int, default=0,
                   help="omega-points in the CPU-oracle sample (0: one per 3 host cores)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--prec", choices=["fp64", "fp64emu", "bf16x3", "bf16x3emu"],
                   default="bf16x3emu")
    p.add_argument("--no-fp64-compare", action="store_true",
                   help="skip timing the plain float64 form on one step for the speedup")
    p.add_argument("--inner-tol", type=float, default=1e-4)
    p.add_argument("--graph", action="store_true",
                   help="replay each GMRES iteration as a captured CUDA graph")
    return p.parse_args()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []   # (host time, csv line)
        self.t0 = None

    def start(self):
        """Start sampling every 50 ms and wait (at most 5 s) for the first
        sample, so that the timed region that follows is covered."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            deadline = time.perf_counter() + 5.0
            while not self.lines and time.perf_counter() < deadline and self.proc.poll() is None:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        self.t0 = time.perf_counter()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def stop(self):
        t1 = time.perf_counter()
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        # the samples taken between start() returning and stop() (all of them if none)
        inside = [ln for t, ln in self.lines if self.t0 <= t <= t1]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in inside or [ln for _, ln in self.lines]:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# algorithmic work
# ---------------------------------------------------------------------------
def chi0_flops_per_rhs(s) -> float:
    """Algorithmic flops of one chi0 . v for one complex vector (same count for
    every form): the two transforms, the block-sparse beta and G contractions
    over the nonzero orbital blocks (mirrors included), the vertex sums and
    the D(omega) scaling."""
    n_orb, n_occ = s.n_orb, s.n_occ
    n_virt = n_orb - n_occ
    pairs = {(int(a), int(b)) for a, b in s.prod_atoms}
    nb = sum(1 if a == b else 2 for a, b in pairs)
    blk = 13 * 13
    return (8.0 * n_orb * n_virt * n_occ + 8.0 * blk * n_occ * nb + 8.0 * blk * s.n_prod
            + 6.0 * n_occ * n_virt)


def omega_schedule(n_omega: int, rank: int, world: int, per_step: int):
    """Round-robin share of the frequency grid for this rank (the paper's
    distribution of frequencies over processes), cut into step groups."""
    mine = np.arange(rank, n_omega, world)
    groups = [mine[i:i + per_step] for i in range(0, mine.size, per_step)]
    return [g for g in groups if g.size]


# ---------------------------------------------------------------------------
# CPU oracle timing (baseline leg and reference arm)
# ---------------------------------------------------------------------------
def cpu_oracle_run(workload: str, n_points: int, cores: int, pool_state: dict | None = None):
    import oracle.tddft_oracle as O
    w = synth.WORKLOADS[workload]
    om = synth.omega_grid(w["n_omega"], w["w_hi"])
    pick = om[np.linspace(0, om.size - 1, n_points).round().astype(int)]
    t0 = time.perf_counter()
    P, infos = O.polarizability_gmres_parallel((synth.workload_system, (workload,)), pick,
                                               w["eps"], w["restart"], w["tol"], workers=cores)
    dt = time.perf_counter() - t0
    conv = all(i["converged"] for i in infos)
    return n_points / dt, dt, conv, pick


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = host_cores()
    w = synth.WORKLOADS[args.workload]
    per_step = max(1, math.ceil(cores / 3))
    for _ in range(args.warmup):
        cpu_oracle_run(args.workload, per_step, cores)
    times = []
    for _ in range(args.steps):
        _, dt, conv, pick = cpu_oracle_run(args.workload, per_step, cores)
        times.append(dt)
    total = sum(times)
    value = per_step * args.steps / total
    sample = (f"{per_step} omega-points x 3 directions per step (evenly spread over the "
              f"{w['n_omega']}-point grid), oracle GMRES(m={w['restart']}) to tol {w['tol']}")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "omega-points/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(args.workload, "oracle on host cores"),
        "cpu_baseline": {"value": value, "unit": "omega-points/s", "cores": cores,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "omega-points/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


FORM_NOTE = {
    "fp64": "plain float64 GMRES, device resident",
    "fp64emu": "float64 GMRES whose dense products are float64 emulated on the bf16 tensor "
               "cores (6 integer slices per operand, exact sums)",
    "bf16x3": "GMRES cycles with split-bf16 tensor-core products (steps 2 and 5 on the "
              "stored transition vertex), each cycle closed by a float64 residual (iterative "
              "refinement); RHS in float64; float32 basis, float64 Arnoldi scalars and Givens",
    "bf16x3emu": "GMRES cycles with split-bf16 tensor-core products (steps 2 and 5 on the "
                 "stored transition vertex), each cycle closed by a float64 residual whose "
                 "products are float64 emulated on the tensor cores (5 integer slices, exact "
                 "sums); RHS formation likewise; float32 basis, float64 Arnoldi scalars and "
                 "Givens",
}
DTYPE = {"fp64": "f64", "fp64emu": "f64 (emulated on bf16 tensor cores)",
         "bf16x3": "bf16x3+f64", "bf16x3emu": "bf16x3+f64 (emulated on bf16 tensor cores)"}


def roofline_of(timing: dict, step_ms: float, prec: str = "bf16x3emu") -> dict:
    """Roofline entry of the kernel class with the largest device time."""
    peaks, src = measured_peaks()
    name, d = max(timing.items(), key=lambda kv: kv[1]["ms"])
    launches = max(1, d["launches"])
    per_launch_s = d["ms"] / launches / 1e3
    achieved = (d["flops"] / launches) / per_launch_s / 1e12 if d["flops"] else None
    if not d["flops"] and d.get("bytes"):
        # memory-bound class with device-counted algorithmic bytes
        achieved = (d["bytes"] / launches) / per_launch_s / 1e9
        peak = peaks["hbm_gbs"]
        return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                "peak_source": f"{src} HBM copy bandwidth",
                "algorithmic_bytes_per_launch": d["bytes"] / launches,
                "share_of_step": d["ms"] / step_ms, "launches": d["launches"],
                "ms_per_launch": d["ms"] / launches}
    if name.startswith("tc_"):
        peak = peaks["bf16_tflops_sustained"] / 3.0
        bound, note = "tensor", (f"split bf16: 3 bf16 products per algorithmic product; peak = "
                                 f"{src} sustained bf16 {peaks['bf16_tflops_sustained']} / 3")
    elif name.startswith("emu_gemm") or name.startswith("emu_alpha"):
        pairs = EMU_PAIRS.get(prec, 21)
        peak = peaks["bf16_tflops_sustained"] / pairs
        bound, note = "tensor", (f"float64 emulated with {pairs} bf16 slice products per "
                                 f"algorithmic product; peak = {src} sustained bf16 "
                                 f"{peaks['bf16_tflops_sustained']} / {pairs}")
    elif name.startswith("f64_"):
        peak, bound = FP64_NOMINAL_TFLOPS, "alu"
        note = "GB300 FP64 nominal 1.25 TFLOP/s (no FP64 entry among the measured peaks)"
    else:
        peak, bound = FP32_UNIT_TFLOPS, "alu"
        note = "FP32 CUDA cores: 152 SMs x 128 lanes x 2 flops x 2.07 GHz"
    return {"kernel": name, "bound": bound, "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": (achieved / peak) if achieved else None,
            "traffic": traffic_of(name, d["flops"] / launches),
            "traffic_unit": "bytes per launch (ncu, scaled to this class's mean launch)",
            "peak_source": note, "share_of_step": d["ms"] / step_ms,
            "launches": d["launches"], "ms_per_launch": d["ms"] / launches}


def config_of(workload: str, extra: str):
    w = synth.WORKLOADS[workload]
    return {"workload": f"{workload}: {w['n_atoms']} atoms, 13 orbitals/atom, "
                        f"{w['n_omega']} omegas in [0,{w['w_hi']}] Ha x 3 directions, "
                        f"eps {w['eps']} Ha, GMRES({w['restart']}) tol {w['tol']}",
            "l2": "operator inputs (K alone) larger than L2",
            "note": extra}


# ---------------------------------------------------------------------------
# the GPU path
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    from paper_1005_5340_gb300 import tddft

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)

    s, w = synth.workload(args.workload)
    omega = w["omega"]
    groups = omega_schedule(omega.size, rank, world, args.omega_per_step)
    per_step = len(groups[0])
    ctx = tddft.Context(s, batch=3 * per_step, restart=w["restart"], tol=w["tol"],
                        max_restarts=200, stream=stream.cuda_stream, prec=args.prec,
                        inner_tol=args.inner_tol, graph=args.graph)
    dev_groups = [torch.tensor(omega[g], dtype=torch.float64, device=dev) for g in groups]

    def step(i):
        g = dev_groups[i % len(dev_groups)]
        P, info = ctx.polarizability(g, w["eps"])
        return int(np.sum(info["matvecs"])), int(g.numel()), int(np.sum(info["cycles"]))

    with torch.cuda.stream(stream):
        for i in range(args.warmup):
            step(i)
    torch.cuda.synchronize()

    # timed region: device-resident inputs, device events on the library stream
    # the timed steps run uninstrumented; the per-kernel split comes from the
    # same steps run again with CUDA events around every kernel class
    clk = ClockSampler(local)
    ctx.timing_enable(False)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    points = 0
    matvecs = 0
    cycles = 0
    with torch.cuda.stream(stream):
        e0.record(stream)
        for i in range(args.steps):
            mv, n, cy = step(args.warmup + i)
            points += n
            matvecs += mv
            cycles += cy
        e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    # the same steps again, instrumented (non-graph), for the kernel split
    ctx.timing_enable(True)
    torch.cuda.synchronize()
    i0, i1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        i0.record(stream)
        for i in range(args.steps):
            step(args.warmup + i)
        i1.record(stream)
    torch.cuda.synchronize()
    timing_ms = i0.elapsed_time(i1)
    timing = ctx.timing()
    ctx.timing_enable(False)
    t = torch.tensor([ms, float(points)], dtype=torch.float64, device=dev)
    if dist:
        tm = t[:1].clone()
        dist.all_reduce(tm, op=dist.ReduceOp.MAX)
        tp = t[1:].clone()
        dist.all_reduce(tp, op=dist.ReduceOp.SUM)
        ms_max, total_points = float(tm.item()), float(tp.item())
    else:
        ms_max, total_points = ms, float(points)
    value = total_points / (ms_max / 1e3)

    # end to end through the public API with host buffers
    # the same groups as the timed steps, from pinned host memory through the
    # public call (omega in, P out), host wall clock
    e2e_steps = args.e2e_steps or args.steps
    host_groups = [torch.tensor(omega[g], dtype=torch.float64).pin_memory() for g in groups]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_points = 0
    for i in range(e2e_steps):
        g = host_groups[(args.warmup + i) % len(host_groups)]
        P, info = ctx.polarizability(g, w["eps"])
        e2e_points += g.numel()
    dt = time.perf_counter() - t0
    e2e = {"value": world * e2e_points / dt, "unit": "omega-points/s",
           "h2d_bytes_per_step": int(8 * per_step),
           "d2h_bytes_per_step": int(16 * 9 * per_step + 24 * 3 * per_step)}

    if rank != 0:
        ctx.close()
        if dist:
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel class
    roofline = roofline_of(timing, timing_ms, args.prec)
    roofline["timing"] = ("per-launch CUDA-event durations from the same steps run again, "
                          "instrumented, after the (uninstrumented) timed region")
    per_scope = KERNELS_PER_SCOPE_EMU if args.prec.endswith("emu") else KERNELS_PER_SCOPE
    gpu_launches = int(sum(v["launches"] * per_scope.get(k, 1) for k, v in timing.items()))
    chi_cls = ["f64_vertex", "f64_beta", "f64_gemm_T1", "f64_dscale", "f64_gemm_T2",
               "f64_block_dot", "tc_gemm_T1_dscale", "tc_gemm_T2", "emu_gemm_T1", "emu_gemm_T2", "alpha_gather", "tc_alpha_beta",
               "tc_alpha_dot", "emu_alpha_beta", "emu_alpha_dot"]
    chi_ms = sum(timing[c]["ms"] for c in chi_cls)
    n_virt = s.n_orb - s.n_occ
    t1_flops = (timing["f64_gemm_T1"]["flops"] + timing["tc_gemm_T1_dscale"]["flops"]
                + timing["emu_gemm_T1"]["flops"])
    chi_applies = t1_flops / (4.0 * n_virt * s.n_orb * s.n_occ)
    chi0_tflops = chi_applies * chi0_flops_per_rhs(s) / (chi_ms / 1e3) / 1e12 if chi_ms else None

    plain = None
    if args.prec != "fp64" and not args.no_fp64_compare:
        # the plain float64 form on the same frequency groups (one warm-up, one timed step)
        ctx64 = tddft.Context(s, batch=3 * per_step, restart=w["restart"], tol=w["tol"],
                              max_restarts=200, stream=stream.cuda_stream, prec="fp64")
        with torch.cuda.stream(stream):
            ctx64.polarizability(dev_groups[0], w["eps"])
            torch.cuda.synchronize()
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            P64, info64 = ctx64.polarizability(dev_groups[1 % len(dev_groups)], w["eps"])
            f1.record(stream)
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1)
        pts64 = int(dev_groups[1 % len(dev_groups)].numel())
        ctx64.close()
        rate64 = pts64 / (ms64 / 1e3)
        plain = {"value": rate64, "unit": "omega-points/s", "steps": 1,
                 "matvecs_per_rhs": float(np.mean(info64["matvecs"])),
                 "speedup_of_chosen_form": value / rate64}

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cores = host_cores()
        npts = args.cpu_sample or max(1, math.ceil(cores / 3))
        v, dt_cpu, conv, pick = cpu_oracle_run(args.workload, npts, cores)
        cpu = {"value": v, "unit": "omega-points/s", "cores": cores, "kind": "oracle",
               "sample": f"{npts} omega-points x 3 directions spread over the grid "
                         f"({dt_cpu:.1f} s wall, converged={conv})"}

    out = {
        "metric": METRIC, "value": value, "unit": "omega-points/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[args.prec],
        "data": "synthetic",
        "config": dict(config_of(args.workload, FORM_NOTE[args.prec]),
                       precision=args.prec, inner_tol=args.inner_tol,
                       omega_per_step=per_step, parallelism=f"frequency shards x{world}"),
        "chi0_tflops": chi0_tflops,
        "matvecs_per_rhs": matvecs / max(1, 3 * points),
        "cycles_per_rhs": cycles / max(1, 3 * points),
        "plain_fp64": plain,
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
        "gpu_launches": gpu_launches,
        "kernel_ms": {k: round(v["ms"], 3) for k, v in timing.items() if v["launches"]},
        "kernel_launches": {k: v["launches"] for k, v in timing.items() if v["launches"]},
        "tc_n_tiles": list(ctx.tuning()),
    }
    print(json.dumps(out), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


def run_batch(args):
    """The uneven batch: 32 molecules of 8-128 atoms solved together (one graph
    per round with a branch per molecule); a step is omega_per_step frequencies
    x 3 directions for every molecule.  Also times the molecules one after the
    other through single contexts on one step for comparison."""
    import torch
    from paper_1005_5340_gb300 import tddft
    torch.cuda.set_device(0)
    mols = synth.batch_molecules()
    eps, tol, restart = 0.005, 1e-6, 40
    per = args.omega_per_step
    omega = synth.omega_grid(per * max(1, args.steps), 1.5)
    groups = [omega[i::max(1, args.steps)] for i in range(max(1, args.steps))]
    b = tddft.Batch(mols, batch=3 * per, restart=restart, tol=tol, prec=args.prec,
                    inner_tol=args.inner_tol)
    for i in range(args.warmup):
        b.polarizability(groups[i % len(groups)], eps)
    torch.cuda.synchronize()
    clk = ClockSampler(0)
    clk.start()
    t0 = time.perf_counter()
    mv = 0
    for i in range(args.steps):
        P, st = b.polarizability(groups[i], eps)
        mv += int(st["matvecs"].sum())
    dt = time.perf_counter() - t0
    clocks = clk.stop()
    b.close()
    points = len(mols) * per * args.steps
    # the same molecules one at a time (single contexts, host-driven), one step
    seq_time = 0.0
    for s in mols:
        with tddft.Context(s, batch=3 * per, restart=restart, tol=tol, prec=args.prec,
                           inner_tol=args.inner_tol) as ctx:
            ctx.polarizability(groups[0][:1], eps)       # warm the context
            torch.cuda.synchronize()
            a = time.perf_counter()
            ctx.polarizability(groups[0], eps)
            seq_time += time.perf_counter() - a
    seq_rate = len(mols) * per / seq_time
    print(json.dumps({
        "metric": METRIC, "value": points / dt, "unit": "omega-points/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[args.prec], "data": "synthetic",
        "config": {"workload": f"batch32: 32 molecules of {min(x.n_atoms for x in mols)}-"
                               f"{max(x.n_atoms for x in mols)} atoms (sizes log-uniform 8-128), "
                               f"{per} omega x 3 directions each per step, eps {eps}, "
                               f"GMRES({restart}) tol {tol}",
                   "precision": args.prec, "parallelism": "one graph per round, a branch per molecule"},
        "matvecs_per_rhs": mv / (3 * points), "clocks": clocks,
        "one_molecule_at_a_time": {"value": seq_rate, "unit": "omega-points/s",
                                   "speedup_of_batch": (points / dt) / seq_rate},
        "roofline": None, "e2e": None, "cpu_baseline": None,
    }), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch32":
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
