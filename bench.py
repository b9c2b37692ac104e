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

# 32 hardware work queues instead of the default 8, so that the batched and
# served instances (one stream each) run concurrently; must be set before
# the CUDA context exists, and does not affect single-stream work
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

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
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched-instances, serving and paper-experiment measurements")
    ap.add_argument("--profile-run", action="store_true",
                    help="only the timed LT solves (no e2e / GTS / peaks); for ncu captures")
    ap.add_argument("--level", type=int, default=10, help="finest level (profiling runs)")
    ap.add_argument("--eps", type=float, default=1e-3, help="threshold (profiling runs)")
    ap.add_argument("--min-level", type=int, default=3, help="coarsest leaf level (profiling runs)")
    ap.add_argument("--case", choices=["quadrants2d", "blast3d"], default="quadrants2d",
                    help="profiling runs: the 2D Euler quadrants (default) or the 3D Euler blast")
    ap.add_argument("--mixed", action="store_true", help="profiling runs: mixed precision")
    ap.add_argument("--window", type=float, nargs=2, metavar=("T0", "K"), default=None,
                    help="profiling run: solve to T0, then K fine iterations; prints how many stage launches "
                         "come before those K iterations and the launches and leaf-stages within them "
                         "(the launch window of a small ncu capture)")
    return ap.parse_args()


def replica_aggregate(dist, ws: int, total_s: float, e2e_s: float, updates: int, device: str = "cuda"):
    """Whole-job figures of N independent replicas: the slowest rank's
    device time and end-to-end time (all-reduce MAX over ranks) and the units
    of all ranks over that time.  Every rank solves the same workload, so the
    job's units are ws x the local count.  Returns (tmax, e2e_max, value,
    e2e_value)."""
    import torch
    tmax = total_s
    if dist is not None and ws > 1:
        t = torch.tensor([total_s, e2e_s], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tmax, e2e_s = float(t[0]), float(t[1])
    return tmax, e2e_s, ws * updates / tmax, ws * updates / e2e_s


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


STAGE_SOURCES = ("mrlt_impl.cuh", "mrlt_stage.cuh")


def stage_kernel_hash() -> str:
    """sha256 (first 16 hex digits) of the stage kernel's sources: a DRAM figure
    recorded under profiles/ applies only to the kernel it was measured on"""
    import hashlib
    h = hashlib.sha256()
    for f in STAGE_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_1905_08717_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def _traffic_per_leaf_stage():
    """DRAM bytes per leaf-stage of the stage kernel from the committed ncu
    summary; None if absent or recorded for another version of the kernel
    (its `kernel_sha16:` line differs from the sources built here)."""
    path = os.path.join(ROOT, "profiles", "stage_kernel_dram_euler2d_L10.md")
    if not os.path.exists(path):
        return None
    val, sha = None, None
    for ln in open(path):
        if ln.startswith("dram_bytes_per_leaf_stage:"):
            try:
                val = float(ln.split(":")[1].split()[0])
            except ValueError:
                return None
        elif ln.startswith("kernel_sha16:"):
            sha = ln.split(":")[1].strip()
    return val if sha == stage_kernel_hash() else None


def _uniform_roofline(pkg, inputs, torch, peak: float, iters: int = 20) -> dict:
    """The stage kernel on large launches: the same 2D Euler problem with
    eps = 0 (all 1024^2 cells are leaves) and the global step, so that every
    stage launch holds about a million leaves; CUDA events around each stage
    launch, FP64 and mixed precision."""
    out = {"workload": f"euler2d quadrants L=10, eps=0 (1,048,576 leaves), global step, {iters} fine iterations"}
    for prec, key in ((inputs.PREC_FP64, "fp64"), (inputs.PREC_MIXED, "mixed")):
        p, q = inputs.euler_2d_quadrants(L=10, eps=0.0, seed=0, time_mode=inputs.TIME_GTS)
        s = pkg.Solver(p.replace(precision=prec), q)
        dt = 0.5 / 1024 / 3.7
        s.iterate(dt, 3)
        torch.cuda.synchronize()
        s.profile(True)
        s.iterate(dt, iters)
        pr = s.profile_read()
        s.profile(False)
        s.close()
        ls = float(pr["leaf_stages"].sum())
        sec = pr["stage_ms"] / 1e3
        ach = ls * FLOP_PER_LEAF_STAGE / sec / 1e12
        out[key] = {"achieved": ach, "unit": "TFLOP/s", "frac": ach / peak, "leaf_stages": int(ls),
                    "stage_launches": pr["stage_launches"], "us_per_launch": 1e6 * sec / max(pr["stage_launches"], 1)}
    out["peak"] = peak
    out["note"] = "mixed: fluxes in FP32, so its FP64-based fraction is not a utilisation"
    return out


def _timed_solve(pkg, torch, p, q, t_end):
    s = pkg.Solver(p, q)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    s.step(t_end)
    e1.record()
    torch.cuda.synchronize()
    out = (e0.elapsed_time(e1) / 1e3, s.uniform(), s.stats()["leaves"])
    s.close()
    return out


def _paper_rows(pkg, inputs, torch, make, t_end, paper, var=None, eps_list=(1e-2,)) -> dict:
    """MR (global step) and MRLT/NERK (local step) against the finite-volume
    solution on the same finest grid (eps = 0, global step, no adaptation), for
    RK2 and RK3: L1 error (of component `var` when the state has several), time
    in % of the finite-volume run, memory (leaves) in % of its cells, and the
    paper's gain lambda = mu_MR / mu_MRLT with mu = error x time (Sec. 5).  The
    first threshold of `eps_list` fills the top-level rows; each further one
    adds a block keyed by its value, against the same finite-volume runs."""
    import numpy as np
    out = {}
    for rk in (2, 3):
        p, q = make(rk)
        t_fv, u_fv, n_fv = _timed_solve(pkg, torch, p.replace(eps=0.0, time_mode=inputs.TIME_GTS,
                                                               adapt_mode=inputs.ADAPT_NEVER), q, t_end)
        if var is not None:
            u_fv = u_fv[var]
        for e_i, eps in enumerate(eps_list):
            row = {"fv_s": t_fv}
            for key, mode in (("mr", inputs.TIME_GTS), ("lt", inputs.TIME_LT)):
                t, u, leaves = _timed_solve(pkg, torch, p.replace(eps=eps, time_mode=mode), q, t_end)
                if var is not None:
                    u = u[var]
                row[key] = {"l1": float(np.abs(u - u_fv).mean()), "time_pct_fv": 100.0 * t / t_fv,
                            "memory_pct_fv": 100.0 * leaves / n_fv, "s": t}
            row["lambda"] = (row["mr"]["l1"] * row["mr"]["s"]) / (row["lt"]["l1"] * row["lt"]["s"])
            row["time_ratio_mr_over_lt"] = row["mr"]["s"] / row["lt"]["s"]
            row["paper"] = {"mr": dict(zip(("l1", "time_pct_fv", "memory_pct_fv"), paper[rk]["mr"])),
                            "lt": dict(zip(("l1", "time_pct_fv", "memory_pct_fv"), paper[rk]["lt"])),
                            "lambda": paper[rk]["lambda"]}
            (out if e_i == 0 else out.setdefault(f"eps_{eps:g}", {}))[f"rk{rk}"] = row
    return out


def _paper_burgers2d(pkg, inputs, torch, L: int = 10) -> dict:
    """The paper's 2D Burgers experiment (Sec. 5.1: sin 2 pi x sin 2 pi y, u = 0
    on the walls, sigma = 0.5, eps = 1e-2, t_f = 0.9) on this GPU.  The paper's
    own figures (its CPU, its L = 12 reference) are quoted beside as context."""
    paper = {2: {"mr": (1.2890e-2, 14.7, 4.1), "lt": (1.0740e-2, 6.7, 4.4), "lambda": 2.63},
             3: {"mr": (1.2893e-2, 15.3, 4.1), "lt": (1.0699e-2, 6.4, 4.4), "lambda": 2.88}}
    out = {"workload": f"paper 2D Burgers, L={L}, eps=1e-2, sigma=0.5, t=0.9, zero-Dirichlet walls"}
    out.update(_paper_rows(pkg, inputs, torch, lambda rk: inputs.burgers_2d_paper(
        L=L, eps=1e-2, min_level=3, rk_order=rk), 0.9, paper))
    return out


def _paper_euler2d(pkg, inputs, torch, L: int = 10) -> dict:
    """The paper's 2D Euler experiment (Sec. 5.4: four-quadrant Riemann problem,
    AUSM+ flux, homogeneous Neumann walls, sigma = 0.5, eps = 1e-2, t_f = 0.25)
    on this GPU; errors of the density.  The paper's own figures (its CPU, its
    L = 12 reference; lambda against MR with the same RK order) are quoted
    beside as context.  With this library's detail norm (the largest child
    detail over the variable's largest magnitude) eps = 1e-2 keeps far fewer
    cells than the paper reports; eps = 1e-3 keeps about the paper's share
    (in the oracle: 25.7% and 11.7% of the cells at L = 8 and 9, against its
    26.4% and 14.0%), so it is run as well."""
    paper = {2: {"mr": (0.5835e-1, 14.7, 7.2), "lt": (0.5821e-1, 4.1, 7.3), "lambda": 3.59},
             3: {"mr": (0.5834e-1, 11.2, 7.2), "lt": (0.5821e-1, 3.6, 7.3), "lambda": 3.11}}
    out = {"workload": f"paper 2D Euler quadrants, L={L}, AUSM+, eps=1e-2, sigma=0.5, t=0.25, Neumann walls"}
    out.update(_paper_rows(pkg, inputs, torch, lambda rk: (lambda pq: (pq[0].replace(flux=inputs.FLUX_AUSM_PLUS),
                                                                        pq[1]))(
        inputs.euler_2d_quadrants(L=L, eps=1e-2, seed=0, min_level=3, rk_order=rk)), 0.25, paper, var=0,
        eps_list=(1e-2, 1e-3)))
    return out


def _batched(pkg, inputs, torch, n: int = 256, t1: float = 0.005, span: float = 0.02) -> dict:
    """Batched instances: n 2D reaction-diffusion problems of uneven size (L
    ~ U{7..10}, eps in {1e-3, 1e-4}, RK2 LT/NERK) advanced from t1 to
    t1 + span in one mr_batch_step, against the same instances solved one
    after another over the same span (host wall clock, both synchronised)."""
    probs, qs = inputs.rd_batch(n=n, seed=0, t_end=0.2)
    b = pkg.Batch(probs, qs)
    b.step(t1)  # captures every instance's macro-step graph
    u0 = sum(v.stats()["updates"] for v in b.instances)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.step(t1 + span)
    t_batch = time.perf_counter() - t0
    u1 = sum(v.stats()["updates"] for v in b.instances)
    b.close()
    t_seq = 0.0
    for p, q in zip(probs, qs):
        s = pkg.Solver(p, q)
        s.step(t1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.step(t1 + span)
        t_seq += time.perf_counter() - t0
        s.close()
    # launch shape chosen by the package's tuner on a short span, then timed
    # over the same span as the default batch
    from paper_1905_08717_gb300 import autotune
    tune = autotune.tune_batch(probs, qs, t1, span / 4)
    best = tune["best"]
    t_tuned = t_batch
    if best != 0:
        b = pkg.Batch(probs, qs, grid_cap=best)
        b.step(t1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.step(t1 + span)
        t_tuned = time.perf_counter() - t0
        b.close()
    return {"workload": f"rd2d x{n}, L~U{{7..10}}, eps in {{1e-3,1e-4}}, rk2 lt/nerk, t {t1}->{t1 + span}",
            "leaf_updates": u1 - u0, "batch_s": t_batch, "updates_per_s": (u1 - u0) / t_batch,
            "one_by_one_s": t_seq, "one_by_one_updates_per_s": (u1 - u0) / t_seq,
            "speedup": t_seq / t_batch,
            "autotuned": {"grid_cap": best, "batch_s": t_tuned, "updates_per_s": (u1 - u0) / t_tuned,
                          "speedup_vs_default": t_batch / t_tuned, "speedup_vs_one_by_one": t_seq / t_tuned,
                          "tuning_span": span / 4,
                          "tuning_s": {str(k): v for k, v in tune["seconds"].items()}},
            "timing": "host wall clock around synchronous calls"}


def _serve(pkg, torch, reqs, grid_cap: int = 0) -> dict:
    """Replay (arrival_s, problem, q0, t_end) requests against a fresh
    mr_server in real time (host clock); latency = completion seen by poll -
    arrival.  grid_cap: stage-launch block cap of every request (0: default)."""
    n = len(reqs)
    srv = pkg.Server(mem_budget_bytes=64 << 30, max_active=96)
    srv.set_grid_cap(grid_cap)
    arrival, done_at, updates = {}, {}, 0
    k = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    while len(done_at) < n:
        now = time.perf_counter() - t0
        while k < n and reqs[k][0] <= now:
            a, p, q, t_end = reqs[k]
            arrival[srv.submit(p, q, t_end)] = a
            k += 1
        active, queued = srv.advance()
        got = srv.poll()
        for rid in got:
            done_at[rid] = time.perf_counter() - t0
            if srv.status(rid) != 0:
                raise RuntimeError(f"request {rid} failed")
            updates += srv.result(rid).stats()["updates"]
            srv.release(rid)
        if active == 0 and queued == 0 and k < n:
            time.sleep(max(0.0, reqs[k][0] - (time.perf_counter() - t0)))
        elif not got:
            time.sleep(5e-5)  # advance() never waits: pause briefly between polls
    wall = time.perf_counter() - t0
    srv.close()
    lat = sorted(1e3 * (done_at[r] - arrival[r]) for r in done_at)
    return {"latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                           "max": lat[-1]},
            "requests_per_s": n / wall, "leaf_updates_per_s": updates / wall, "wall_s": wall}


def _serving(pkg, inputs, torch, n: int = 200, rate: float = 200.0) -> dict:
    """Continuous batching on the request mix of a Poisson stream: first the
    capacity (every request submitted at t = 0), then latency with the same
    requests arriving as a Poisson process at half that capacity, then at the
    configured rate when the GPU can sustain it."""
    reqs = inputs.serving_requests(n=n, seed=0, rate=rate)
    sat = _serve(pkg, torch, [(0.0,) + r[1:] for r in reqs])
    # the same capacity run with one stage-kernel block per SM per launch
    # (the cap the tuner picks for the batched workload); latency is measured
    # with whichever launch shape gave the higher capacity
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    sat_cap = _serve(pkg, torch, [(0.0,) + r[1:] for r in reqs], grid_cap=sms)
    gcap = sms if sat_cap["requests_per_s"] > sat["requests_per_s"] else 0
    best = sat_cap if gcap else sat
    cap = best["requests_per_s"]
    rng = __import__("numpy").random.default_rng(1)
    arr = list(__import__("itertools").accumulate(rng.exponential(1.0 / (0.5 * cap), n)))
    half = _serve(pkg, torch, [(a,) + r[1:] for a, r in zip(arr, reqs)], grid_cap=gcap)
    out = {"workload": f"{n} requests: 1D Burgers L10-14 (32-128 fine steps), 2D RD L8-10 (16-64), "
                       "3D blast L6-8 (8-24); eps log-U[1e-4,1e-2]; mixed precision",
           "capacity": best, "capacity_default_launch": sat, "capacity_one_block_per_sm": sat_cap,
           "grid_cap": gcap, "at_half_capacity": dict(half, rate_per_s=0.5 * cap),
           "configured_rate_per_s": rate, "timing": "host wall clock"}
    if rate <= cap:
        out["at_configured_rate"] = _serve(pkg, torch, reqs, grid_cap=gcap)
    return out


def _mixed_vs_oracle(pkg, inputs, case: str, L: int, t_end: float) -> dict:
    """L1 error of rho of the mixed-precision GPU solve (and of the FP64 GPU
    solve) against the FP64 oracle over a whole solve at a size the oracle
    finishes in seconds, relative to the oracle's L1 norm of rho."""
    import numpy as np
    import oracle
    if case == "euler2d":
        p, q = inputs.euler_2d_quadrants(L=L, eps=1e-3, seed=0)
    else:
        p, q = inputs.euler_3d_blast(L=L, eps=1e-3, min_level=3, precision=inputs.PREC_FP64)
    p = p.replace(precision=inputs.PREC_FP64)
    ref = oracle.Oracle(p, q)
    ref.step(t_end)
    u_o = ref.uniform()[0]
    out = {"workload": f"{case} L={L} eps=1e-3 t={t_end}", "oracle_iters": ref.stats()["iters"]}
    ref.close()
    for key, prec in (("mixed", inputs.PREC_MIXED), ("fp64", inputs.PREC_FP64)):
        g = pkg.Solver(p.replace(precision=prec), q)
        g.step(t_end)
        u = g.uniform()[0]
        g.close()
        out[f"rel_l1_rho_{key}"] = float(np.abs(u - u_o).sum() / np.abs(u_o).sum())
    return out


def _precision_3d(pkg, inputs, torch, L: int = 8, t_end: float = 0.1) -> dict:
    """The 3D Euler blast (rho = 1, p = 1, p = 10 inside r < 0.1, walls), L = 8
    (256^3 finest), eps = 1e-3, RK3 LT/NERK to t = 0.1, in FP64 and in the
    mixed mode: solve time, leaf updates/s, the stage kernel's algorithmic HBM
    rate (state bytes of every leaf-stage / summed CUDA-event time of the stage
    launches), the mixed-vs-FP64 L1 distance of rho, and both against the
    FP64 oracle at L = 6 (whole solve)."""
    import numpy as np
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"hbm_gbs": 6800.0}
    p, q = inputs.euler_3d_blast(L=L, eps=1e-3, min_level=3)
    out = {"workload": f"euler3d blast L={L} (256^3), eps=1e-3, rk3 lt/nerk, t=0..{t_end}"}
    u = {}
    for key, prec, esz in (("fp64", inputs.PREC_FP64, 8), ("mixed", inputs.PREC_MIXED, 4)):
        s = pkg.Solver(p.replace(precision=prec), q)
        s.step(0.005)  # warm-up (graph capture)
        ts = []
        for _ in range(2):
            s.reset(q)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            s.step(t_end)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        st = s.stats()
        u[key] = s.uniform()[0]
        # stage kernel: one more profiled solve (CUDA events around each stage launch)
        s.reset(q)
        s.profile(True)
        s.step(t_end)
        pr = s.profile_read()
        s.profile(False)
        s.close()
        ls = pr["leaf_stages"]
        nbytes = (2 * float(ls[0]) + 3 * float(ls[1] + ls[2])) * 5 * esz
        sec = pr["stage_ms"] / 1e3
        out[key] = {"ms_per_solve": 1e3 * min(ts), "leaf_updates": st["updates"],
                    "updates_per_s": st["updates"] / min(ts), "leaves_at_t_end": st["leaves"],
                    "stage_kernel": {"achieved_gbs": nbytes / sec / 1e9, "peak_gbs": peaks["hbm_gbs"],
                                     "frac": nbytes / sec / 1e9 / peaks["hbm_gbs"],
                                     "launches": pr["stage_launches"],
                                     "leaf_stages_per_launch": float(ls.sum()) / max(pr["stage_launches"], 1),
                                     "bytes_per_leaf_stage": f"stage 1: 2 x 5 x {esz}, stages 2-3: 3 x 5 x {esz}"}}
    out["rel_l1_rho_mixed_vs_fp64_gpu"] = float(np.abs(u["mixed"] - u["fp64"]).sum() / np.abs(u["fp64"]).sum())
    out["speedup_mixed_vs_fp64"] = out["fp64"]["ms_per_solve"] / out["mixed"]["ms_per_solve"]
    out["vs_oracle_L6"] = _mixed_vs_oracle(pkg, inputs, "euler3d", 6, t_end)
    return out


def _persistent(pkg, torch, p, qn, t_end: float) -> dict:
    """The same solve in the persistent launch mode (one cooperative kernel per
    macro step): time and kernel launches per solve, beside the default."""
    s = pkg.Solver(p, qn)
    s.set_launch_mode(pkg.MR_LAUNCH_PERSISTENT)
    s.step(0.005)
    s.reset(qn)
    torch.cuda.synchronize()
    l0 = s.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    s.step(t_end)
    e1.record()
    torch.cuda.synchronize()
    out = {"ms_per_solve": e0.elapsed_time(e1), "launches_per_solve": s.launch_count() - l0,
           "launch_mode": "MR_LAUNCH_PERSISTENT (cooperative macro-step kernel, bounded grid barriers)"}
    s.close()
    return out


def _profile_problem(inputs, args):
    """the problem of a profiling run: --case at --level, --eps, --min-level"""
    prec = inputs.PREC_MIXED if args.mixed else inputs.PREC_FP64
    if args.case == "blast3d":
        return inputs.euler_3d_blast(L=args.level, eps=args.eps, min_level=args.min_level, precision=prec)
    p, q = inputs.euler_2d_quadrants(L=args.level, eps=args.eps, seed=0, min_level=args.min_level)
    return p.replace(precision=prec), q


def _profile_window(pkg, inputs, args, stream, rank):
    """A window of K fine iterations of the profiling solve, after solving to
    T0: the stage launches before the window (ncu -s), the stage launches and
    leaf-stages within it (ncu -c, and the divisor of its DRAM bytes).  Every
    stage launch is counted in profiling mode, which launches directly."""
    p, q = _profile_problem(inputs, args)
    s = pkg.Solver(p, q, stream=stream)
    s.profile(True)
    t0, k = args.window[0], int(args.window[1])
    s.step(t0)
    a = s.profile_read()
    s.iterate(s.stats()["dt"], k)
    b = s.profile_read()
    s.profile(False)
    if rank == 0:
        print(json.dumps({"profile_window": True, "level": args.level, "eps": args.eps, "t0": t0, "iterations": k,
                          "stage_launches_before": a["stage_launches"],
                          "stage_launches": b["stage_launches"] - a["stage_launches"],
                          "leaf_stages": int(b["leaf_stages"].sum() - a["leaf_stages"].sum()),
                          "leaves": s.stats()["leaves"]}))
    s.close()


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
    if args.profile_run and args.window is not None:
        _profile_window(pkg, inputs, args, stream, rank)
        return
    if args.profile_run:
        p, q = _profile_problem(inputs, args)
    else:
        p, q = inputs.euler_2d_quadrants(L=10, eps=1e-3, seed=0)
    q_pin = torch.from_numpy(q).pin_memory()
    qn = q_pin.numpy()
    n = 1 << p.max_level
    uni_pin = torch.empty(p.nvars() * n ** p.dim, dtype=torch.float64).pin_memory().numpy()
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
                              "case": args.case, "mixed": args.mixed,
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

    tmax, e2e_s, value, e2e_value = replica_aggregate(dist, ws, total_s, e2e_s, updates)

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
            "peak_source": "bench-measured cuBLAS DGEMM, 4096^3 FP64, best of 3 (MEASURED_PEAKS.json "
                           "has no FP64 entry; nominal 1.25 TFLOP/s)",
            "traffic_source": "profiles/stage_kernel_dram_euler2d_L10.md x leaf-stages per launch"
                              if tpl else "no DRAM capture of this kernel version",
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
    u_gts = gts.uniform()
    gts.close()

    # ---- equal accuracy: both adaptive solutions against the finite-volume
    # solution on the finest grid (eps = 0, global step, no adaptation: every
    # cell of level L is a leaf), L1 norm as the paper's (mean over the finest
    # cells), per variable
    fv = pkg.Solver(p.replace(eps=0.0, time_mode=inputs.TIME_GTS, adapt_mode=inputs.ADAPT_NEVER), qn,
                    stream=stream)
    fv.step(args.t_end)
    u_fv = fv.uniform()
    fv.close()
    u_lt = uni_pin.reshape(u_fv.shape)
    l1 = lambda u: [float(x) for x in np.abs(u - u_fv).reshape(u_fv.shape[0], -1).mean(axis=1)]
    e_lt, e_gts = l1(u_lt), l1(u_gts)
    t_lt = tmax / args.steps
    accuracy = {"reference": "finite volumes on the finest grid (eps = 0, global step)",
                "l1_lt_nerk": e_lt, "l1_gts": e_gts, "lt_speedup_vs_gts": gts_s / t_lt,
                # the paper's cost mu = L1 error x time; lambda = mu_GTS / mu_LT > 1
                # favours MRLT/NERK (density error)
                "cost_ratio_lambda": (e_gts[0] * gts_s) / (e_lt[0] * t_lt)}

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
             "rel_l1_vs_fp64_gpu": [float(x) for x in rel_l1],
             "vs_oracle_L6": _mixed_vs_oracle(pkg, inputs, "euler2d", 6, 0.25),
             "arithmetic": "FP32 state, exposures, reconstruction, fluxes and RK updates; "
                           "FP64 flux registers and detail-norm threshold test"}

    uniform = _uniform_roofline(pkg, inputs, torch, peak)
    precision_3d = _precision_3d(pkg, inputs, torch)
    persistent = _persistent(pkg, torch, p, qn, args.t_end)
    paper_b2d = _paper_burgers2d(pkg, inputs, torch) if not args.no_batch else None
    paper_e2d = _paper_euler2d(pkg, inputs, torch) if not args.no_batch else None
    batched = _batched(pkg, inputs, torch) if not args.no_batch else None
    serving = _serving(pkg, inputs, torch) if not args.no_batch else None

    lat_ms = sorted(1e3 * x for x in lat)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * tmax / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "finest": "1024x1024", "eps": 1e-3, "min_level": 3,
                      "t_end": args.t_end, "leaf_updates_per_step": updates // max(args.steps, 1),
                      "leaves_at_t_end": st["leaves"], "fine_iterations": st["iters"],
                      "l2": "256 MB buffer written between steps",
                      "parallelism": f"replicas x{ws}"},
           "clocks": clk, "gpu_launches": launches, "launches_per_solve": launches // max(args.steps, 1),
           "launch_mode": "MR_LAUNCH_GRAPH (one kernel per phase, macro steps as CUDA graphs)",
           "e2e": {"value": e2e_value, "unit": UNIT,
                   "h2d_bytes_per_step": int(qn.nbytes), "d2h_bytes_per_step": int(uni_pin.nbytes)},
           "roofline": roof,
           "latency_ms": {"p50": lat_ms[len(lat_ms) // 2], "p99": lat_ms[-1]},
           "gts": {"ms_per_solve": 1e3 * gts_s, "leaf_updates": gst["updates"],
                   "updates_per_s": gst["updates"] / gts_s},
           "lt_speedup_vs_gts": gts_s / (tmax / args.steps),
           "equal_accuracy": accuracy,
           "precision_mode": mixed,
           "precision_mode_3d": precision_3d,
           "persistent_launch": persistent,
           "roofline_uniform": uniform}
    if batched is not None:
        out["batched"] = batched
    if serving is not None:
        out["serving"] = serving
    if paper_b2d is not None:
        out["paper_burgers2d"] = paper_b2d
    if paper_e2d is not None:
        out["paper_euler2d"] = paper_e2d
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
