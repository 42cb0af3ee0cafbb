#!/usr/bin/env python
"""Forward+adjoint throughput of the LKS / moving-design-grid / discrete-adjoint path on one GB300.

Workload (default): the 3D D3Q15 256^3 duct with a 96^3 design grid rotating about the flow
axis and translating sinusoidally, 20000 time steps, FP32 state with FP64 objective and
sensitivity accumulation, binomial checkpointing with forward recomputation.  One bench "step"
is one full pass of the path: set_design -> forward (Alg. 1, J) -> adjoint (dJ/dgamma).
MLUPS counts analysis node updates once per time step (nodes * time steps / s / 1e6).

Also reported: the forward-only rate; the plain FP64 GPU path on the same workload at the full
horizon (one pass) with the FP32-vs-FP64 errors on J and dJ/dgamma, and its fraction of the
measured FP64 FMA rate; the forward and adjoint stencil steps against the measured HBM copy
bandwidth (the "roofline" object names the one with the larger share of the pass); the transfer
kernels from the committed ncu summary; the end-to-end rate through the public API with host
buffers; the other named workloads (the 512^2 channel in both precisions, with its FP32 errors);
the single-thread FP64 CPU oracle on a bounded sample; and SM clocks during the timed region.

`--impl reference` times the CPU oracle (the method's plain FP64 restatement) as the
reference arm on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "forward+adjoint MLUPS and % HBM roofline, FP32 vs FP64, at <=1e-4 sensitivity err"
UNIT = "MLUPS"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--horizon", type=int, default=None,
                    help="time steps per pass (default: the workload's full horizon)")
    ap.add_argument("--fp64-horizon", type=int, default=None,
                    help="time steps of the plain FP64 pass (default: the full horizon)")
    ap.add_argument("--fp64-workload", type=int, choices=[3, 4], default=4,
                    help="named workload of the plain FP64 pass and its FP32 comparison: 4, "
                         "the metric's 256^3 duct (default), or 3, the 128^3 duct (small "
                         "profiling runs)")
    ap.add_argument("--e2e-passes", type=int, default=3,
                    help="passes of the end-to-end leg (at most --steps)")
    ap.add_argument("--timing-stride", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched 2D workload leg")
    ap.add_argument("--batch-horizon", type=int, default=5000)
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other named workloads (128^2 FP64, 512^2 FP32, 128^3 FP32)")
    ap.add_argument("--fd-check", type=int, default=0, metavar="CELLS",
                    help="instead of the benchmark: the 512^2 channel workload at its full "
                         "horizon, dJ/dgamma of the GPU FP64 path against central differences "
                         "(eps = 1e-4) at CELLS seeded design cells, one JSON line")
    ap.add_argument("--step-variant", type=int, choices=[0, 1, 2], default=None,
                    help="fused 3D forward-step variant of the 256^3 leg (default: the "
                         "library's, 1)")
    ap.add_argument("--workload", choices=["cfg4", "batch2d"], default="cfg4",
                    help="cfg4: the 256^3 3D line (default); batch2d: the batched 2D workload")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, ws, device="cpu"):
    """Largest value of x over all ranks (the slowest rank sets the job time)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(node_steps_per_pass, passes, ws, seconds):
    """Whole-job MLUPS of ws independent replicas that each ran `passes` passes in `seconds`
    (the max over ranks)."""
    return node_steps_per_pass * passes * ws / seconds / 1e6


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# Source files each timed stencil step is built from; committed ncu counters count only
# while these files are unchanged.
STEP_SOURCES = {
    "forward_step": ("lks_fused3d.cu", "lks_device.cuh", "lks_tma.cuh", "lks_internal.h"),
    "adjoint_step": ("lks_fused3d_adj.cu", "lks_plain.cu", "lks_units.cuh", "lks_device.cuh",
                     "lks_tma.cuh", "lks_internal.h"),
}


def kernel_sources_sha1(names):
    """SHA-1 over the source files a kernel is built from (to tell stale counters)."""
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2506_23895_gb300", "csrc")
    for name in names:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def committed_ncu(name, sources):
    """A committed ncu summary (profiles/<name>.json) if the kernels it describes are built from
    the same sources today, else None."""
    p = os.path.join(ROOT, "profiles", name + ".json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("sources_sha1") != kernel_sources_sha1(sources):
        return None
    return d


TRANSFER_SOURCES = ("lks_transfer.cu", "lks_device.cuh", "lks_internal.h")
FP64_SOURCES = ("lks_plain.cu", "lks_units.cuh", "lks_device.cuh", "lks_internal.h")


def ncu_traffic(step):
    """DRAM bytes per launch of a stencil step (sum over its kernels) from the committed ncu
    figures (profiles/ncu_traffic.json), or None when its sources changed since."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f).get(step)
    if not d or d.get("sources_sha1") != kernel_sources_sha1(STEP_SOURCES[step]):
        return None
    v = d.get("dram_bytes_per_launch")
    return None if v is None else float(v)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.idx)],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(workload_idx, n_steps=2):
    """The FP64 oracle, single thread, on a bounded sample of the workload."""
    import oracle
    from paper_2506_23895_gb300 import workloads as W

    oracle.build()
    w = W.config(workload_idx, n_steps=n_steps)
    t0 = time.perf_counter()
    oracle.gradient(w.problem, w.gamma, w.motion)
    dt = time.perf_counter() - t0
    nodes = w.problem.nodes
    return {"value": nodes * n_steps / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{w.problem.name}: full {w.problem.n[0]}x{w.problem.n[1]}x{w.problem.n[2]}"
                      f" grid and design, {n_steps} time steps forward + exact adjoint,"
                      f" single-thread FP64 C++ (-O2), {dt:.1f} s"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_2506_23895_gb300 import workloads as W

    oracle.build()
    w = W.config(4, n_steps=1)
    nodes = w.problem.nodes
    for _ in range(args.warmup):
        oracle.gradient(w.problem, w.gamma, w.motion)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.gradient(w.problem, w.gamma, w.motion)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    v = nodes * len(times) / tot / 1e6
    sample = (f"{w.problem.name}: full grid and design, 1 time step forward + exact adjoint"
              f" per bench step, single-thread FP64 C++ oracle")
    out = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1000 * tot / len(times),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "impl": "reference",
           "config": {"workload": "cfg4_3d_256: D3Q15 256^3 duct, 96^3 design rotating about z "
                                  "+ transverse sinusoid, 20000-step horizon (1-step samples)"},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def batch2d_leg(args, lks, W, stream, passes=1, warmup=1, clocks=None):
    """The batched 2D workload: 64 channels of side 128..512 (design side 0.4 N, own gamma and
    rotation rate), FP32 forward + adjoint in lock step through lks_batch_*: every phase one
    persistent launch over all instances, runs of steps replayed from CUDA graphs, tile
    shapes from the autotuner."""
    import math
    import torch

    H = args.batch_horizon
    ws = W.batch_config2(n_inst=64, n_steps=H)
    K = math.ceil(math.sqrt(H))
    slots = K + math.ceil(H / K)           # every segment start stored: one recomputation
    b = lks.Batch([w.problem for w in ws], slots, stream=stream)
    for s, w in zip(b.solvers, ws):
        s.set_design(w.gamma)
        s.set_motion(w.motion)
    nodes = sum(w.problem.nodes for w in ws)
    for _ in range(max(1, warmup)):        # warm-up passes: autotune, graph capture
        b.forward()
        b.adjoint()
    torch.cuda.synchronize()
    if clocks is not None:
        clocks.start()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2 * passes + 1)]
    launches = 0
    e[0].record()
    for k in range(passes):
        J = b.forward()
        launches += b.stats()["launches"]
        e[1 + 2 * k].record()
        b.adjoint()
        launches += b.stats()["launches"]
        e[2 + 2 * k].record()
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks is not None else None
    tun = b.tuning()
    t_all = e[0].elapsed_time(e[-1]) / passes
    t_fwd = sum((e[2 * k] if k else e[0]).elapsed_time(e[1 + 2 * k]) for k in range(passes)) / passes
    peak, peak_kind = peaks()
    shapes = lks.tile_shapes()
    ms_step = tun["step_ms"][tun["step"]]
    ms_adj = tun["adjoint_ms"][tun["adjoint"]]
    res = {"value": nodes * H / (t_all / 1000.0) / 1e6, "unit": UNIT,
           "forward_mlups": nodes * H / (t_fwd / 1000.0) / 1e6,
           "ms_per_pass": t_all, "instances": len(ws), "nodes_per_step": nodes,
           "time_steps": H, "dtype": "f32",
           "workload": "batch2d: 64 D2Q9 channels, sides 128..512, design 0.4 N, rim speed "
                       f"0.025..0.1, {H} steps, J1 over the last 10 %, FP32 forward+adjoint",
           "snapshot_slots": slots, "graphs": b.stats()["graphs"],
           "gpu_launches": launches // passes,
           "tiles": {"step": shapes[tun["step"]], "adjoint": shapes[tun["adjoint"]],
                     "step_ms_per_shape": tun["step_ms"],
                     "adjoint_ms_per_shape": tun["adjoint_ms"]},
           # autotuner timings of the chosen shapes (5 back-to-back launches over all instances)
           "roofline_step": {"bound": "hbm", "achieved": 24.0 * nodes / (ms_step / 1000) / 1e9,
                             "peak": peak, "unit": "GB/s",
                             "frac": 24.0 * nodes / (ms_step / 1000) / 1e9 / peak,
                             "algorithmic_bytes_per_launch": 24.0 * nodes,
                             "avg_launch_ms": ms_step, "peak_kind": f"{peak_kind} hbm_gbs",
                             "note": "state 117 MB in + out per launch, near the 129 MB L2"},
           "roofline_adjoint": {"bound": "hbm", "achieved": 32.0 * nodes / (ms_adj / 1000) / 1e9,
                                "peak": peak, "unit": "GB/s",
                                "frac": 32.0 * nodes / (ms_adj / 1000) / 1e9 / peak,
                                "algorithmic_bytes_per_launch": 32.0 * nodes,
                                "avg_launch_ms": ms_adj, "peak_kind": f"{peak_kind} hbm_gbs"},
           "J_first": float(J[0]), "passes": passes, "clocks": clk}
    b.close()
    del b
    torch.cuda.empty_cache()
    return res


def config_leg(lks, W, idx, prec, stream):
    """One full forward + adjoint pass of named workload idx (after one untimed pass), timed with
    CUDA events on the solver's stream: forward and forward+adjoint MLUPS."""
    import torch

    w = W.config(idx)
    p = w.problem
    s = lks.Solver(p, prec, stream=stream)
    s.set_motion(w.motion)
    dev = torch.device("cuda", torch.cuda.current_device())
    g_dev = torch.from_numpy(w.gamma).to(dev)
    out = torch.empty(w.gamma.shape, dtype=torch.float64, device=dev)
    s.set_design(g_dev)
    s.forward()
    s.adjoint(out=out)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record()
    s.set_design(g_dev)
    J = s.forward()
    e[1].record()
    s.adjoint(out=out)
    e[2].record()
    torch.cuda.synchronize()
    st = s.stats()
    grad = out.cpu().numpy()
    s.close()
    del s
    torch.cuda.empty_cache()
    node_steps = p.nodes * p.n_steps
    return grad, {"workload": f"{p.name}: {'D2Q9' if p.dim == 2 else 'D3Q15'} "
                        f"{'x'.join(str(n) for n in p.n[:p.dim])}, design "
                        f"{'x'.join(str(l) for l in p.L[:p.dim])}, {p.n_steps} steps",
            "dtype": "f64" if prec == lks.FP64 else "f32", "unit": UNIT,
            "value": node_steps / (e[0].elapsed_time(e[2]) / 1000.0) / 1e6,
            "forward_mlups": node_steps / (e[0].elapsed_time(e[1]) / 1000.0) / 1e6,
            "ms_per_pass": e[0].elapsed_time(e[2]), "J": J,
            "recomputed_steps": st["recomputed_steps"], "snapshot_slots": st["snapshot_slots"]}


def run_batch_line(args, lks, W, ws, rank, local, dev):
    """--workload batch2d: the batched 2D workload as the measured line (replicas for N > 1)."""
    import torch

    stream = torch.cuda.current_stream()
    r = batch2d_leg(args, lks, W, stream, passes=args.steps, warmup=args.warmup,
                    clocks=ClockSampler(local))
    t_ms = max_over_ranks(r["ms_per_pass"], ws, dev)
    node_steps = r["nodes_per_step"] * r["time_steps"]
    # the dominant kernel per pass: the step kernel runs twice per step (record and
    # recomputation), the adjoint kernel once
    dom = ("roofline_step" if 2 * r["roofline_step"]["avg_launch_ms"] >=
           r["roofline_adjoint"]["avg_launch_ms"] else "roofline_adjoint")
    out = {"metric": METRIC, "value": replica_rate(node_steps, 1, ws, t_ms / 1000.0), "unit": UNIT,
           "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic",
           "config": {"workload": r["workload"], "instances": r["instances"],
                      "nodes_per_step": r["nodes_per_step"], "time_steps": r["time_steps"],
                      "parallelism": f"replicas x{ws}",
                      "l2": "state 121 MB per level over all instances, about the 129 MB L2; "
                            "no flush"},
           "forward_mlups": r["forward_mlups"], "roofline": dict(r[dom], kernel=dom[9:]),
           "roofline_step": r["roofline_step"], "roofline_adjoint": r["roofline_adjoint"],
           "tiles": r["tiles"], "graphs": r["graphs"], "gpu_launches": r["gpu_launches"],
           "clocks": r["clocks"]}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


# kernel of each fused 3D forward-step variant (lks_step_variant)
STEP3D_KERNELS = {0: "k_fused_step3d", 1: "k_zstep3d<8> + k_bc_shell3d",
                  2: "k_zpair3d + k_bc_shell3d"}


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__

    __graft_entry__.build()
    from paper_2506_23895_gb300 import lks
    from paper_2506_23895_gb300 import workloads as W

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if ws > 1:
            dist.barrier()

    if args.workload == "batch2d":
        return run_batch_line(args, lks, W, ws, rank, local, dev)

    w = W.config(4, n_steps=args.horizon)
    p = w.problem
    H = p.n_steps
    nodes = p.nodes
    stream = torch.cuda.current_stream()
    solver = lks.Solver(p, lks.FP32, stream=stream)
    if args.step_variant is not None:
        solver.step_variant(args.step_variant)
    solver.set_motion(w.motion)
    gamma_dev = torch.from_numpy(w.gamma).to(dev)
    g_dev = torch.empty(w.gamma.shape, dtype=torch.float64, device=dev)

    def one_pass():
        solver.set_design(gamma_dev)
        J = solver.forward()
        solver.adjoint(out=g_dev)
        return J

    for _ in range(args.warmup):
        one_pass()
    torch.cuda.synchronize()
    barrier()

    clocks = ClockSampler(local)
    clocks.start()
    solver.set_timing(max(1, min(args.timing_stride, H // 2)))
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps + 2)]
    launches = 0
    torch.cuda.synchronize()
    barrier()
    ev[0].record()
    for k in range(args.steps):
        solver.set_design(gamma_dev)
        J = solver.forward()
        ev[1 + 2 * k].record()
        solver.adjoint(out=g_dev)
        ev[2 + 2 * k].record()
        launches += solver.stats()["launches"] + 2  # + the two design-prep kernels
    ev[-1].record()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    tm = solver.read_timing()
    t_ms = ev[0].elapsed_time(ev[-1])
    fwd_ms = 0.0
    prev = ev[0]
    for k in range(args.steps):
        fwd_ms += prev.elapsed_time(ev[1 + 2 * k])
        prev = ev[2 + 2 * k]
    t_ms = max_over_ranks(t_ms, ws, dev)
    node_steps = nodes * H
    value = replica_rate(node_steps, args.steps, ws, t_ms / 1000.0)
    fwd_mlups = node_steps * args.steps / (fwd_ms / 1000.0) / 1e6

    peak, peak_kind = peaks()
    bytes_fwd = 32.0 * nodes     # read + write (rho - rho0, u) in FP32: 2 x 16 B per node
    bytes_adj = 44.0 * nodes     # lam^n in, u^{n-1} in (12 B), lam^{n-1} out
    fwd_step_ms = tm["fwd_ms"] / max(tm["fwd_n"], 1)
    adj_step_ms = tm["adj_ms"] / max(tm["adj_n"], 1)
    ach = bytes_fwd / (fwd_step_ms / 1000.0) / 1e9
    ach_adj = bytes_adj / (adj_step_ms / 1000.0) / 1e9
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"cfg4_3d_256: D3Q15 {p.n[0]}x{p.n[1]}x{p.n[2]} duct, "
                                  f"{p.L[0]}^3 design rotating about z + transverse sinusoid "
                                  f"(amp 20, period 2000), {H} time steps, FP32 forward+adjoint",
                      "time_steps": H, "nodes": nodes, "parallelism": f"replicas x{ws}",
                      "l2": "state 268 MB per level > 129 MB L2; no flush needed",
                      "checkpointing": solver.stats()},
           "forward_mlups": fwd_mlups,
           "gpu_launches": launches, "clocks": clk, "J": J}
    # share of the pass in each stencil step: the forward step runs for every time step and
    # again for every recomputed one, the adjoint step once per time step
    ck = solver.stats()
    pass_ms = t_ms / args.steps
    share_fwd = fwd_step_ms * (H + ck["recomputed_steps"]) / pass_ms
    share_adj = adj_step_ms * H / pass_ms
    rf = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
          "frac": ach / peak, "traffic": ncu_traffic("forward_step"),
          "kernel": "forward stencil step: " + STEP3D_KERNELS.get(solver.step_variant(), "?"),
          "variant": solver.step_variant(), "share_of_pass": share_fwd,
          "launches_per_pass": H + ck["recomputed_steps"],
          "concurrent": "the next step's transfer runs beside it on a side stream",
          "peak_kind": f"{peak_kind} hbm_gbs (copy)",
          "algorithmic_bytes_per_launch": bytes_fwd,
          "avg_launch_ms": fwd_step_ms, "samples": tm["fwd_n"]}
    ra = {"bound": "hbm", "achieved": ach_adj, "peak": peak, "unit": "GB/s",
          "frac": ach_adj / peak, "traffic": ncu_traffic("adjoint_step"),
          "kernel": "adjoint stencil step: k_adj_bcT + k_fused_adj3d + k_adj_bcorr",
          "share_of_pass": share_adj, "launches_per_pass": H,
          "concurrent": "the next step's transfer and the sensitivity gather run beside it on a "
                        "side stream",
          "peak_kind": f"{peak_kind} hbm_gbs (copy)",
          "algorithmic_bytes_per_launch": bytes_adj,
          "avg_launch_ms": adj_step_ms, "samples": tm["adj_n"]}
    # the roofline line names the kernel with the larger share of the pass
    out["roofline"] = dict(rf if share_fwd >= share_adj else ra)
    out["roofline_forward"] = rf
    out["roofline_adjoint"] = ra
    J_last = J
    g_last = g_dev.cpu().numpy()
    solver.set_timing(0)

    # end to end through the public API with pinned host buffers
    if not args.no_e2e:
        gamma_pin = torch.from_numpy(w.gamma).pin_memory()
        g_pin = torch.empty(w.gamma.shape, dtype=torch.float64).pin_memory()
        n_e2e = max(1, min(args.steps, args.e2e_passes))
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            solver.set_design(gamma_pin)
            solver.forward()
            solver.adjoint(out=g_pin)
        torch.cuda.synchronize()
        dt = max_over_ranks(time.perf_counter() - t0, ws, dev)
        barrier()
        out["e2e"] = {"value": replica_rate(node_steps, n_e2e, ws, dt), "unit": UNIT,
                      "h2d_bytes_per_step": int(w.gamma.nbytes),
                      "d2h_bytes_per_step": int(w.gamma.nbytes) + 8, "passes": n_e2e}
    solver.close()
    del solver
    torch.cuda.empty_cache()

    # measured FMA rates: the arithmetic roofline of the plain FP64 path
    if rank == 0 and not args.no_fp64:
        out["alu_peaks"] = {"fp64_tflops": lks.fma_rate(lks.FP64, stream) / 1e12,
                            "fp32_tflops": lks.fma_rate(lks.FP32, stream) / 1e12,
                            "how": "lks_fma_rate: independent FMA chains over whole waves of "
                                   "every SM, CUDA events, 5 launches after a warm-up"}
    # plain FP64 GPU path on the same workload (the full horizon unless shortened), with the
    # FP32 errors against it: the FP32 result of the last timed pass when the horizons agree
    if rank == 0 and not args.no_fp64:
        if args.fp64_workload == 4:
            Hf = H if args.fp64_horizon is None else min(args.fp64_horizon, H)
            same = Hf == H
            wh = w if same else W.config(4, n_steps=Hf)
        else:
            same = False
            wh = W.config(args.fp64_workload, n_steps=args.fp64_horizon)
        Hf = wh.problem.n_steps
        nodes_h = wh.problem.nodes
        res = {}
        precs = (lks.FP64,) if same else (lks.FP64, lks.FP32)
        for prec in precs:
            s = lks.Solver(wh.problem, prec, stream=stream)
            s.set_motion(wh.motion)
            s.set_design(torch.from_numpy(wh.gamma).to(dev))
            gout = torch.empty(wh.gamma.shape, dtype=torch.float64, device=dev)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            Jh = s.forward()
            s.adjoint(out=gout)
            e1.record()
            torch.cuda.synchronize()
            res[prec] = (Jh, gout.cpu().numpy(), e0.elapsed_time(e1), s.stats())
            s.close()
            del s
            torch.cuda.empty_cache()
        if same:
            res[lks.FP32] = (J_last, g_last, pass_ms, ck)
        J64, g64, ms64, st64 = res[lks.FP64]
        J32, g32, ms32, _ = res[lks.FP32]
        out["fp64_plain"] = {
            "workload": wh.problem.name,
            "value": nodes_h * Hf / (ms64 / 1000.0) / 1e6, "unit": UNIT,
            "time_steps": Hf, "ms_per_pass": ms64,
            "recomputed_steps": st64["recomputed_steps"],
            "fp32_same_horizon": nodes_h * Hf / (ms32 / 1000.0) / 1e6,
            "passes": 1}
        alu = committed_ncu("ncu_fp64_plain", FP64_SOURCES)
        if alu and alu.get("forward_flop_per_node") and alu.get("adjoint_flop_per_node"):
            # FP64 flops of the pass: every forward step (recorded and recomputed) and every
            # adjoint step, per analysis node, from the committed ncu op counts
            fwd_steps = Hf + st64["recomputed_steps"]
            flops = (alu["forward_flop_per_node"] * fwd_steps +
                     alu["adjoint_flop_per_node"] * Hf) * nodes_h
            peak64 = out["alu_peaks"]["fp64_tflops"] * 1e12
            out["fp64_plain"]["roofline"] = {
                "bound": "alu", "achieved": flops / (ms64 / 1000.0) / 1e12,
                "peak": peak64 / 1e12, "unit": "TFLOP/s",
                "frac": flops / (ms64 / 1000.0) / peak64,
                "flop_per_node": {"forward": alu["forward_flop_per_node"],
                                  "adjoint": alu["adjoint_flop_per_node"]},
                "peak_kind": "measured FMA rate (lks_fma_rate, this run)",
                "flop_source": "profiles/ncu_fp64_plain.json (ncu FP64 op counts of the plain "
                               "stencil kernels)"}
        out["accuracy_fp32_vs_fp64"] = {
            "workload": wh.problem.name, "time_steps": Hf, "window": list(wh.problem.win),
            "J_fp64": J64, "J_fp32": J32,
            "J_rel": abs(J32 - J64) / abs(J64),
            "dJdgamma_rel_l2": float(np.linalg.norm(g32 - g64) / np.linalg.norm(g64)),
            "tolerance": {"J_rel": 1e-5, "dJdgamma_rel_l2": 1e-4}}
    tr = committed_ncu("ncu_transfer", TRANSFER_SOURCES)
    if rank == 0 and tr:
        # each transfer kernel against the two ceilings that could bind it: DRAM bytes over the
        # measured copy bandwidth, and executed warp instructions over the SMs' issue rate
        # (152 SMs x 4 schedulers x 2070 MHz); both well below 1 means latency-bound
        issue_rate = 152 * 4 * 2.07e9
        kern = {}
        for name, k in tr.get("kernels", {}).items():
            t = k["us"] * 1e-6
            kern[name] = dict(k, dram_frac=k["dram_mb"] * 1e6 / t / (peak * 1e9),
                              issue_frac=k["warp_inst"] / t / issue_rate)
        out["transfer"] = {"kernels": kern, "per_step": tr.get("per_step"),
                           "note": tr.get("note"), "source": "profiles/ncu_transfer.json"}
    if rank == 0 and not args.no_batch:
        out["batch2d"] = batch2d_leg(args, lks, W, stream)
    if rank == 0 and not args.no_configs:
        # the other named workloads, one pass each (not the metric's configuration); the 512^2
        # channel in both precisions, with the FP32 errors against FP64 at its full horizon
        _, c0 = config_leg(lks, W, 0, lks.FP64, stream)
        g1_32, c1_32 = config_leg(lks, W, 1, lks.FP32, stream)
        g1_64, c1_64 = config_leg(lks, W, 1, lks.FP64, stream)
        _, c3 = config_leg(lks, W, 3, lks.FP32, stream)
        out["other_configs"] = {"cfg0_2d_128_fp64": c0, "cfg1_2d_512_fp32": c1_32,
                                "cfg1_2d_512_fp64": c1_64, "cfg3_3d_128_fp32": c3}
        w1 = W.config(1)
        out["accuracy_fp32_vs_fp64_cfg1"] = {
            "workload": w1.problem.name, "time_steps": w1.problem.n_steps,
            "window": list(w1.problem.win),
            "J_rel": abs(c1_32["J"] - c1_64["J"]) / abs(c1_64["J"]),
            "dJdgamma_rel_l2": float(np.linalg.norm(g1_32 - g1_64) / np.linalg.norm(g1_64)),
            "tolerance": {"J_rel": 1e-5, "dJdgamma_rel_l2": 1e-4}}
    if rank == 0:
        if ws == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(4, n_steps=2)
        print(json.dumps(out), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def fd_check(args):
    """Sec. 2.6's verification on the 512^2 rotating and translating channel at its full
    20000-step horizon: the exact discrete adjoint of the GPU FP64 path (through the
    torch.autograd.Function, binomial checkpointing with recomputation) against central
    differences of J (eps = 1e-4) at seeded design cells with gamma in [0.2, 0.8] among the
    largest sensitivities."""
    import numpy as np
    import torch
    import __graft_entry__

    __graft_entry__.build()
    from paper_2506_23895_gb300 import autograd as ag
    from paper_2506_23895_gb300 import lks
    from paper_2506_23895_gb300 import workloads as W

    w = W.config(1)
    p = w.problem
    t0 = time.perf_counter()
    s = lks.Solver(p, lks.FP64)
    s.set_motion(w.motion)
    gam = torch.tensor(w.gamma, device="cuda", requires_grad=True)
    J = ag.objective(gam, s)
    J.backward()
    g = gam.grad.cpu().numpy().reshape(-1)
    rec = s.stats()["recomputed_steps"]
    gflat = w.gamma.reshape(-1)
    thr = np.quantile(np.abs(g), 0.99)
    cand = np.where((gflat > 0.2) & (gflat < 0.8) & (np.abs(g) >= thr))[0]
    cells = np.random.default_rng(1).choice(cand, size=min(args.fd_check, cand.size),
                                            replace=False)
    eps = 1e-4
    rows = []
    for c in cells:
        gp = gflat.copy()
        gm = gflat.copy()
        gp[c] += eps
        gm[c] -= eps
        s.set_design(gp.reshape(w.gamma.shape))
        Jp = s.forward()
        s.set_design(gm.reshape(w.gamma.shape))
        Jm = s.forward()
        fd = (Jp - Jm) / (2 * eps)
        rows.append({"cell": int(c), "gamma": float(gflat[c]), "adjoint": float(g[c]),
                     "fd": fd, "rel": abs(fd - g[c]) / abs(g[c])})
    s.close()
    out = {"check": "central FD vs exact discrete adjoint", "workload": p.name,
           "time_steps": p.n_steps, "window": list(p.win), "dtype": "f64", "eps": eps,
           "J": J.item(), "recomputed_steps": rec, "cells": rows,
           "max_rel": max(r["rel"] for r in rows), "seconds": time.perf_counter() - t0}
    print(json.dumps(out), flush=True)
    return 0


def main():
    args = parse()
    if args.fd_check:
        return fd_check(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
