#!/usr/bin/env python3
"""Benchmark: leaf cell-updates/s of the MRLT/NERK3 solve on GB300.

Workload (one "step"): a full solve of the 2D compressible Euler four-quadrant
Riemann problem (Table 8 states, seed 0) on [0,1]^2 with walls, finest level
L = 10 (1024^2), eps = 1e-3, MUSCL + HLL, RK3 with natural continuous
extension and local time-stepping, from t = 0 to t_end = 0.25, FP64.
A leaf cell-update is one leaf advanced one step of its own level.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun every rank solves its own
replica (the path has no data exchange; scaling is weak).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "leaf cell-updates/s & HBM roofline frac, MRLT vs MR-GTS; p50/p99 solve latency"
UNIT = "leaf-updates/s"
WORKLOAD = "euler2d_quadrants_L10_eps1e-3_rk3_nerk_lt_tend0.25_fp64"
T_END = 0.25

# Algorithmic work of one leaf-stage of the 2D Euler MUSCL-HLL update, each
# face flux and each cell's primitive state counted once (derivation in the
# design notes): FP64 operations, and bytes of the state arrays (m = 4).
FLOP_PER_LEAF_STAGE = 260.0
BYTES_PER_LEAF_STAGE = {1: 16 * 4, 2: 24 * 4, 3: 24 * 4}
NOMINAL_FP64_TFLOPS = 1.25


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--t-end", type=float, default=T_END)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-run", action="store_true",
                    help="only the timed LT solves (no e2e / GTS / peaks); for ncu captures")
    ap.add_argument("--level", type=int, default=10, help="finest level (profiling runs)")
    ap.add_argument("--eps", type=float, default=1e-3, help="threshold (profiling runs)")
    ap.add_argument("--min-level", type=int, default=3, help="coarsest leaf level (profiling runs)")
    return ap.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for ln in open(self.path):
            f = [x.strip() for x in ln.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


def _fp64_peak_tflops(torch) -> float:
    """measured FP64 throughput of cuBLAS DGEMM (best of 3, 4096^3)"""
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = 1e9
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    return 2.0 * n ** 3 / best / 1e12


def _traffic_per_leaf_stage():
    """DRAM bytes per leaf-stage of the stage kernel from the committed ncu
    summary (None if absent or taken on another kernel version)."""
    path = os.path.join(ROOT, "profiles", "stage_kernel_euler2d_L10.md")
    if not os.path.exists(path):
        return None
    for ln in open(path):
        if ln.startswith("dram_bytes_per_leaf_stage:"):
            try:
                return float(ln.split(":")[1].split()[0])
            except ValueError:
                return None
    return None


def _cpu_baseline(seconds: float = 12.0) -> dict:
    """The FP64 oracle, as it stands, on the first fine iterations of the same
    solve (single host thread), until ~`seconds` of CPU work."""
    import oracle
    from paper_1905_08717_gb300 import inputs
    p, q = inputs.euler_2d_quadrants(L=10, eps=1e-3, seed=0)
    o = oracle.Oracle(p, q)
    dt = 0.5 / 1024 / 3.7
    u0 = o.stats()["updates"]
    n = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds or n == 0:
        o.iterate(dt, 1)
        n += 1
    el = time.perf_counter() - t0
    upd = o.stats()["updates"] - u0
    return {"value": upd / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {n} fine iterations ({upd} leaf updates) of the same L=10 solve, "
                      f"one host thread, {el:.1f} s"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    from paper_1905_08717_gb300 import inputs
    p, q = inputs.euler_2d_quadrants(L=10, eps=1e-3, seed=0)
    o = oracle.Oracle(p, q)
    dt = 0.5 / 1024 / 3.7
    per_step = 4  # fine iterations per reference step (bounded sample)
    for _ in range(args.warmup):
        o.iterate(dt, per_step)
    u0 = o.stats()["updates"]
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.iterate(dt, per_step)
    el = time.perf_counter() - t0
    upd = o.stats()["updates"] - u0
    val = upd / el
    sample = (f"{args.steps} steps x {per_step} fine iterations of the L=10 solve after "
              f"{args.warmup * per_step} warm-up iterations, one host thread")
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    import paper_1905_08717_gb300 as pkg
    from paper_1905_08717_gb300 import inputs

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.current_stream()
    if args.profile_run:
        p, q = inputs.euler_2d_quadrants(L=args.level, eps=args.eps, seed=0, min_level=args.min_level)
    else:
        p, q = inputs.euler_2d_quadrants(L=10, eps=1e-3, seed=0)
    q_pin = torch.from_numpy(q).pin_memory()
    qn = q_pin.numpy()
    n = 1 << p.max_level
    uni_pin = torch.empty(p.nvars() * n * n, dtype=torch.float64).pin_memory().numpy()
    solver = pkg.Solver(p, qn, stream=stream)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        solver.reset(qn)
        solver.step(args.t_end)
    barrier()

    # ---- device-timed region: inputs resident in HBM, L2 flushed per step
    clocks = Clocks(local)
    clocks.start()
    if args.profile_run:
        solver.profile(True)
    total_s, updates, launches = 0.0, 0, 0
    lat = []
    for _ in range(args.steps):
        solver.reset(qn)
        flush.fill_(1.0)
        barrier()
        l0 = solver.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solver.step(args.t_end)
        e1.record(stream)
        torch.cuda.synchronize()
        s = e0.elapsed_time(e1) / 1e3
        lat.append(s)
        total_s += s
        updates += solver.stats()["updates"]
        launches += solver.launch_count() - l0
    clk = clocks.stop()
    st = solver.stats()
    if args.profile_run:
        prof = solver.profile_read()
        solver.profile(False)
        if rank == 0:
            ls = prof["leaf_stages_per_level"]
            print(json.dumps({"profile_run": True, "ms_per_step": 1e3 * total_s / args.steps,
                              "updates": updates, "stage_ms": prof["stage_ms"],
                              "stage_launches": prof["stage_launches"], "launches": launches,
                              "level": args.level, "eps": args.eps, "min_level": args.min_level,
                              "leaf_stages_per_level": [int(x) for x in ls],
                              "stage_ms_per_level": [round(float(x), 3) for x in prof["stage_ms_per_level"]]}))
        return

    # ---- end to end through the C-ABI with host buffers: H2D of q0 from pinned
    # memory, the solve, D2H of the finest-level reconstruction
    e2e_s = 0.0
    for _ in range(args.steps):
        flush.fill_(1.0)
        barrier()
        t0 = time.perf_counter()
        solver.reset(qn)
        solver.step(args.t_end)
        solver._read(pkg.MR_READ_UNIFORM, np.float64, out=uni_pin)
        e2e_s += time.perf_counter() - t0

    tmax = total_s
    if dist is not None:
        t = torch.tensor([total_s, e2e_s], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tmax, e2e_s = float(t[0]), float(t[1])
    value = ws * updates / tmax
    e2e_value = ws * updates / e2e_s

    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel (the tiled stage kernel): one more
    # solve, outside the timed region, with a CUDA-event pair on the solver's
    # stream around every stage launch
    solver.reset(qn)
    flush.fill_(1.0)
    torch.cuda.synchronize()
    solver.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    solver.step(args.t_end)
    e1.record(stream)
    torch.cuda.synchronize()
    prof_solve_s = e0.elapsed_time(e1) / 1e3
    prof = solver.profile_read()
    solver.profile(False)
    leaf_stages = prof["leaf_stages"]
    stage_s = prof["stage_ms"] / 1e3
    flops = float(leaf_stages.sum()) * FLOP_PER_LEAF_STAGE
    nbytes = sum(float(leaf_stages[s - 1]) * BYTES_PER_LEAF_STAGE[s] for s in (1, 2, 3))
    per_launch = float(leaf_stages.sum()) / max(prof["stage_launches"], 1)
    peak = _fp64_peak_tflops(torch)
    achieved = flops / stage_s / 1e12
    tpl = _traffic_per_leaf_stage()
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"hbm_gbs": 6800.0}
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": (tpl * per_launch) if tpl else None,
            "kernel": "mrlt::k_stage_tile<2,2,double> (all levels, all stages)",
            "peak_source": "measured cuBLAS DGEMM (FP64 units; nominal 1.25)",
            "launches": prof["stage_launches"], "leaf_stages_per_launch": per_launch,
            "stage_share_of_step": stage_s / prof_solve_s,
            "timing": "CUDA events around each stage launch in one extra (profiled) solve",
            "hbm_view": {"achieved_gbs": nbytes / stage_s / 1e9, "peak_gbs": peaks["hbm_gbs"],
                         "frac": nbytes / stage_s / 1e9 / peaks["hbm_gbs"]}}

    # ---- the same solve with one global time step (MR/RK3), same GPU
    g_p = p.replace(time_mode=inputs.TIME_GTS)
    gts = pkg.Solver(g_p, qn, stream=stream)
    gts.step(min(args.t_end, 0.02))  # warm-up
    gts.reset(qn)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    gts.step(args.t_end)
    e1.record(stream)
    torch.cuda.synchronize()
    gts_s = e0.elapsed_time(e1) / 1e3
    gst = gts.stats()
    gts.close()

    # ---- the same solve in the mixed-precision mode (FP32 face fluxes), and
    # its relative L1 distance from the FP64 result at t_end
    mx = pkg.Solver(p.replace(precision=inputs.PREC_MIXED), qn, stream=stream)
    mx.step(min(args.t_end, 0.02))  # warm-up
    mx_ms = []
    for _ in range(2):
        mx.reset(qn)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mx.step(args.t_end)
        e1.record(stream)
        torch.cuda.synchronize()
        mx_ms.append(e0.elapsed_time(e1))
    mst = mx.stats()
    u_mx = mx.uniform()
    mx.close()
    u_64 = uni_pin.reshape(u_mx.shape)
    rel_l1 = (np.abs(u_mx - u_64).reshape(u_mx.shape[0], -1).sum(axis=1)
              / np.abs(u_64).reshape(u_64.shape[0], -1).sum(axis=1))
    mixed = {"ms_per_solve": min(mx_ms), "leaf_updates": mst["updates"],
             "updates_per_s": mst["updates"] / (min(mx_ms) / 1e3), "leaves_at_t_end": mst["leaves"],
             "rel_l1_vs_fp64": [float(x) for x in rel_l1],
             "arithmetic": "FP32 reconstruction + face fluxes; FP64 state, RK update, registers, adaptation"}

    lat_ms = sorted(1e3 * x for x in lat)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * tmax / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "finest": "1024x1024", "eps": 1e-3, "min_level": 3,
                      "t_end": args.t_end, "leaf_updates_per_step": updates // max(args.steps, 1),
                      "leaves_at_t_end": st["leaves"], "fine_iterations": st["iters"],
                      "l2": "256 MB buffer written between steps",
                      "parallelism": f"replicas x{ws}"},
           "clocks": clk, "gpu_launches": launches,
           "e2e": {"value": e2e_value, "unit": UNIT,
                   "h2d_bytes_per_step": int(qn.nbytes), "d2h_bytes_per_step": int(uni_pin.nbytes)},
           "roofline": roof,
           "latency_ms": {"p50": lat_ms[len(lat_ms) // 2], "p99": lat_ms[-1]},
           "gts": {"ms_per_solve": 1e3 * gts_s, "leaf_updates": gst["updates"],
                   "updates_per_s": gst["updates"] / gts_s},
           "lt_speedup_vs_gts": gts_s / (tmax / args.steps),
           "precision_mode": mixed}
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = _cpu_baseline()
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
