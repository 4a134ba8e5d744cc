#!/usr/bin/env python
"""Benchmark of the multistep BSDE solve: grid-point time steps per second.

Default workload (config3, the largest single-GPU configuration): the call
with different lending and borrowing rates (r = .04, R = .06, mu = .06,
sigma = .2, T = .5, strike 100) in log price, Nx = 2^20, N = 1024, L = 16,
solved once per step for the configuration's k = 4 and for k = 2.  A solve
counts towards the value only when it passes the gate (see GATE_TEXT): on
this grid the scheme itself diverges at k = 4 (the FP64 oracle too), so that
solve is timed but reported as excluded.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32c|fp64]
                  [--workload config3|config2|config4|config5|ex4_2d|general|decomp]
  python bench.py --impl reference ...   (the FP64 CPU oracle on the host cores)

Prints one JSON line (rank 0).  Under torchrun each rank solves its own copy
of the workload (independent instances, weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grid-point·steps/s at max|err|≤tol vs FP64 oracle; served solves/s + p99 ms"
UNIT = "grid-point·steps/s"
KS = (1, 2, 3, 4, 5, 6)
# Algorithmic FP operations per grid-point time step of the Black-Scholes
# driver: per Gauss-Hermite node two spline values (7 each: 4 products, 3
# sums), the linear driver (3) and three quadrature sums (2 each), plus E[y]
# at j = k; then the z and y combinations (4 per j) and ~3 Picard iterations.
FLOP_NODE = 7 + 7 + 3 + 6


# Algorithmic L2 -> SM bytes per point and node of the FP32C step kernel: the
# value record (y_hi, z_hi, y_lo, z_lo) and the second derivatives (M_y, M_z)
# of the node's cell's left end.
L2_BYTES_NODE = 16 + 8


def flops_per_gp_step(k: int, L: int) -> float:
    return k * L * FLOP_NODE + 2 * L + 4 * k + 12


# The per-node count of the method's arithmetic used for the rooflines of the
# 1-D step kernels: per node the y and z spline values (8 each), the driver
# (4-8) and the quadrature sums (6-10), about 30, and 42 once the sums carry
# their compensation (the FP32C kernels); per point ~3 per step j for z and
# ~6 per Picard iteration.  The narrower count above (23 per node: the
# Black-Scholes driver, plain sums) is reported beside it.
FLOP_NODE_PLAIN, FLOP_NODE_COMP = 30, 42


def flops_per_gp_step_method(k: int, L: int, compensated: bool, picard_iters: int) -> float:
    return k * L * (FLOP_NODE_COMP if compensated else FLOP_NODE_PLAIN) + 3 * k + 6 * picard_iters


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def _traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary."""
    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as fh:
            t = json.load(fh)[kernel]
        return int(t["dram_bytes_read"]) + int(t["dram_bytes_write"])
    except (OSError, KeyError, ValueError):
        return None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.rows = []
        self.proc = None
        self.thread = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        cmd = ["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.uuid:
            cmd.insert(1, f"--id={self.uuid}")
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return self

        def pump():
            for line in self.proc.stdout:
                self.rows.append([c.strip() for c in line.split(",")])
        self.thread = threading.Thread(target=pump, daemon=True)
        self.thread.start()
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _gold_num(v):
    # non-finite oracle values are stored as text ("nan", "inf", "-inf")
    return float(v)


def _golden(workload: str = "config2"):
    """The FP64 oracle's stored (y0, z0) per k for a single-solve workload
    (tests/golden/<workload>_oracle.json, written by the script beside it,
    which calls only the oracle)."""
    try:
        with open(os.path.join(ROOT, "tests", "golden", f"{workload}_oracle.json")) as fh:
            rows = json.load(fh)["rows"]
    except OSError:
        return {}
    out = {}
    for r in rows:
        r = dict(r)
        for f in ("y0", "z0"):
            r[f] = _gold_num(r[f])
        out[int(r["k"])] = r
    return out


# The bench gate.  A solve is counted when (1) the scheme itself converges
# on this grid -- the stored FP64 oracle's y0 and z0 lie within CONV_REL of
# the closed form -- and (2) its y0 and z0 agree with that oracle within the
# precision's tolerance, relative to max(1, |value|).
CONV_REL = 1e-2
PARITY_REL = {"fp32c": 1e-6, "fp64": 1e-12}


def gate(y0: float, z0: float, oracle_y0: float, oracle_z0: float, exact_y0: float,
         exact_z0: float, precision: str) -> dict:
    conv = (math.isfinite(oracle_y0) and math.isfinite(oracle_z0)
            and abs(oracle_y0 - exact_y0) <= CONV_REL * max(1.0, abs(exact_y0))
            and abs(oracle_z0 - exact_z0) <= CONV_REL * max(1.0, abs(exact_z0)))
    tol = PARITY_REL[precision]
    ey, ez = abs(y0 - oracle_y0), abs(z0 - oracle_z0)
    par = (math.isfinite(y0) and math.isfinite(z0)
           and ey <= tol * max(1.0, abs(oracle_y0)) and ez <= tol * max(1.0, abs(oracle_z0)))
    return {"scheme_converges": conv, "within_tol": par, "counted": conv and par,
            "err_y0_vs_oracle": ey, "err_z0_vs_oracle": ez,
            "err_y0_vs_exact": abs(y0 - exact_y0), "err_z0_vs_exact": abs(z0 - exact_z0)}


GATE_TEXT = ("a solve counts when the stored FP64 oracle's y0 and z0 are within 1% of the "
             "closed form (the scheme converges on this grid) and the solve's y0 and z0 are "
             "within 1e-6 (FP32C) or 1e-12 (FP64) x max(1, |value|) of that oracle")


def _golden_variants():
    try:
        with open(os.path.join(ROOT, "tests", "golden", "config2_oracle.json")) as fh:
            return json.load(fh).get("variants", [])
    except OSError:
        return []


def measure_variants(args, dev, stream, flush):
    """The scheme's variants on the config2 workload (K_z != K_y, the E[y dW]
    z form, the one-step start-up), each solve timed alone with CUDA events
    (L2 flushed before each, outside the events) and compared with the FP64
    oracle's value stored for it."""
    import torch
    from paper_1909_13560_gb300 import bsde as B
    from paper_1909_13560_gb300 import workloads as W
    sp = stream.cuda_stream
    rows = []
    for g in _golden_variants():
        f = dict(g["fields"])
        p = W.config2(k=f.pop("k"))
        p.update(f)
        s = B.Solver(p, args.precision, device=dev)
        for _ in range(3):
            flush.zero_()
            B.bsde_solve(s.plan, sp, want_result=False)
        torch.cuda.synchronize(dev)
        ms = 0.0
        for _ in range(max(1, args.steps)):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            B.bsde_solve(s.plan, sp, want_result=False)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms += e0.elapsed_time(e1)
        ms /= max(1, args.steps)
        r = B.bsde_result_fetch(s.plan, sp)
        K = W.levels_K(p)
        startup = p["Nx"] * (K - 1) * int(p.get("init_substeps", 0)) if p.get("init_mode") else 0
        tol = (1e-12 if args.precision == "fp64" else 1e-6) * max(1.0, abs(g["y0"]))
        rows.append({"name": g["name"], "fields": g["fields"], "ms_per_solve": ms,
                     "gp_steps_per_s": W.gp_steps(p) / (ms / 1000.0),
                     "startup_gp_steps": startup, "launches": s.launches,
                     "y0": r.y0, "z0": r.z0, "err_y0_vs_oracle": abs(r.y0 - g["y0"]),
                     "err_z0_vs_oracle": abs(r.z0 - g["z0"]),
                     "within_tol": abs(r.y0 - g["y0"]) <= tol,
                     "err_y0_vs_exact": abs(r.y0 - g["exact_y0"]),
                     "err_z0_vs_exact": abs(r.z0 - g["exact_z0"])})
        s.close()
    return rows


def _dist_init(world):
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        return dist
    return None


def _max_over_ranks(dist, v: float) -> float:
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(dist):
    if dist is not None:
        dist.barrier()


C3_KS = (2, 4)


def _single_problems(workload: str, ks=None):
    """The solves of one step of a single-solve workload: config2 (k = 1..6)
    or config3 at full size (the configuration's k = 4 beside k = 2)."""
    from paper_1909_13560_gb300 import workloads as W
    if workload == "config3":
        return [(k, W.config3(k=k)) for k in (ks or C3_KS)]
    return [(k, W.config2(k=k)) for k in (ks or KS)]


def _workload_text(workload: str, ks) -> str:
    if workload == "config3":
        return ("config3: call with lending/borrowing rates (r=.04, R=.06, mu=.06, sigma=.2, "
                "T=.5, K=100, x in ln100 +- 6 sigma sqrt T), Nx=2^20, N=1024, L=16; one solve "
                f"per k in {{{','.join(map(str, ks))}}} per step (the configuration's k=4 beside "
                "k=2)")
    return ("config2: Black-Scholes call in log price (S0=K=100, r=.03, mu=.05, sigma=.2, T=1, "
            f"x in ln100 +- 6 sigma), Nx=65536, N=256, L=16; one solve per k in "
            f"{{{','.join(map(str, ks))}}} per step")


def cpu_baseline(levels: int, threads: int, workload: str = "config3") -> dict:
    """The FP64 oracle as it stands, on a bounded sample of the workload: its
    solves, first `levels` backward levels each, `threads` host threads."""
    from oracle import oracle as O
    from paper_1909_13560_gb300 import workloads as W
    probs = _single_problems(workload)
    t0 = time.perf_counter()
    units = 0
    for _, p in probs:
        r = O.solve(p, levels=levels, threads=threads)
        units += int(p["Nx"]) * int(r["levels_done"])
    dt = time.perf_counter() - t0
    ks = ",".join(str(k) for k, _ in probs)
    return {"value": units / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{workload} (k={ks}, full grid), first {levels} backward levels of each "
                      f"solve, {threads} host threads; {units} grid-point steps in {dt:.2f} s"}


def run_reference(args, rank, world):
    """The FP64 CPU oracle on the host cores, on the same workload, metric and
    unit as our arm; each step a bounded sample (the first --ref-levels
    backward levels of each of the workload's solves)."""
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    wl = args.workload if args.workload in ("config2", "config3") else "config3"
    levels = args.ref_levels if args.ref_levels else (4 if wl == "config3" else 12)
    for _ in range(args.warmup):
        cpu_baseline(levels, threads, wl)
    t0 = time.perf_counter()
    tot = 0.0
    for _ in range(args.steps):
        r = cpu_baseline(levels, threads, wl)
        tot += r["value"]
    wall = time.perf_counter() - t0
    value = tot / args.steps
    probs = _single_problems(wl)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "devices": "host cores only (rank 0)",
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * wall / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": _workload_text(wl, [k for k, _ in probs]),
                       "Nx": probs[0][1]["Nx"], "N": probs[0][1]["N"],
                       "k": [k for k, _ in probs], "L": 16, "sample_levels_per_solve": levels},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": r["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def measured_peaks(dev) -> dict:
    """FMA-pipe rates measured now by bsde_fma_probe (FP32: the better of the
    scalar and packed FP32x2 forms; FP64) and the L2 -> SM read bandwidth by
    bsde_l2_read_probe."""
    from paper_1909_13560_gb300 import bsde as B
    f32 = B.fma_peak_tflops("fp32", device=dev)
    f32x2 = B.fma_peak_tflops("fp32x2", device=dev)
    return {"fp32_tflops": max(f32, f32x2), "fp32_scalar_tflops": f32, "fp32x2_tflops": f32x2,
            "fp64_tflops": B.fma_peak_tflops("fp64", device=dev),
            "l2_read_gbs": B.l2_read_bandwidth(device=dev),
            "how": "bsde_fma_probe: 8 CTAs x 256 threads per SM, 8 independent FMA chains per "
                   "thread, best of 5 launches (CUDA events); bsde_l2_read_probe: 48 MiB "
                   "L2-resident buffer read 40 times with 16-byte loads, best of 5"}


def _gpu_uuid(dev):
    import torch
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        return uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        return None


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_1909_13560_gb300 import bsde as B
    from paper_1909_13560_gb300 import workloads as W

    dist = _dist_init(world)
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    wl = args.workload
    c3 = wl == "config3"
    ks_arg = None if tuple(args.ks) == KS else tuple(args.ks)
    probs_k = _single_problems(wl, ks_arg)
    ks = tuple(k for k, _ in probs_k)
    probs = [p for _, p in probs_k]
    # config2's six solves run concurrently: together they fill the GPU, and
    # the flat FP32C step kernel (no shared-memory partial sums, no barrier,
    # uniform table reads; bitwise the grouped kernel's results) then beats
    # the grouped one that the library picks for a 65536-point grid alone
    flat2 = (wl == "config2" and args.precision == "fp32c"
             and (not args.sequential or args.step_kernel == "FLAT"))
    if flat2:
        probs = [dict(p, step_kernel="FLAT") for p in probs]
    solvers = [B.Solver(p, args.precision, device=dev) for p in probs]
    units = [W.gp_steps(p) for p in probs]
    units_per_step = sum(units)
    launches_per_step = sum(s.launches for s in solvers)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    # the solves of a step are independent: each runs on its own stream,
    # forked from and joined to the timing stream, so their dependent launch
    # chains overlap (--sequential: one after another on the timing stream)
    conc = B.ConcurrentSolves(solvers, dev)

    def one_step():
        if args.sequential:
            for s in solvers:
                B.bsde_solve(s.plan, sp, want_result=False)
        else:
            conc.enqueue(stream)

    for _ in range(args.warmup):
        flush.zero_()
        one_step()
    torch.cuda.synchronize(dev)

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    _barrier(dist)
    torch.cuda.synchronize(dev)
    with ClockSampler(_gpu_uuid(dev)) as clk:
        w0 = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()  # L2 flush between steps, outside the events
            starts[i].record(stream)
            one_step()
            ends[i].record(stream)
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - w0
    _barrier(dist)
    ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    ms_max = _max_over_ranks(dist, ms)

    # the gate: results of the last step against the stored FP64 oracle values
    gold = _golden(wl)
    rows, counted = [], []
    for k, p, s, u in zip(ks, probs, solvers, units):
        r = B.bsde_result_fetch(s.plan, sp)
        g = gold.get(k)
        row = {"k": k, "y0": r.y0, "z0": r.z0, "picard_iters_max": r.picard_iters_max,
               "gp_steps": u}
        if g:
            row.update({"oracle_y0": g["y0"], "oracle_z0": g["z0"], "exact_y0": g["exact_y0"],
                        "exact_z0": g["exact_z0"]})
            row.update(gate(r.y0, r.z0, g["y0"], g["z0"], g["exact_y0"], g["exact_z0"],
                            args.precision))
        else:
            row.update({"counted": False, "why": "no stored oracle value for this k"})
        rows.append(row)
        counted.append(bool(row["counted"]))
    counted_units = sum(u for u, c in zip(units, counted) if c)
    value = world * counted_units * args.steps / (ms_max / 1000.0)
    excluded = [{"k": r["k"], "gp_steps": r["gp_steps"],
                 "reason": (r.get("why") or
                            ("the scheme diverges on this grid: the FP64 oracle's "
                             f"y0 = {r['oracle_y0']:.6g}, z0 = {r['oracle_z0']:.6g} against the "
                             f"closed form {r['exact_y0']:.6g}, {r['exact_z0']:.6g}"
                             if not r["scheme_converges"] else
                             "outside the parity tolerance of the FP64 oracle"))}
                for r in rows if not r["counted"]]

    # each solve alone (context for the concurrent step)
    alone_ms = {}
    for k, s in zip(ks, solvers):
        tot = 0.0
        for _ in range(3):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            B.bsde_solve(s.plan, sp, want_result=False)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            tot += e0.elapsed_time(e1)
        alone_ms[str(k)] = tot / 3

    # dominant kernel: the step kernel, re-running level 0 of each plan (its
    # input levels 1..k are resident after the solve).  The repeats are
    # captured in a CUDA graph, so the host's launch overhead does not starve
    # the device; the graph is replayed on the timing stream between events.
    reps = 20
    fp64 = args.precision == "fp64"
    iters = {r["k"]: max(1, int(r["picard_iters_max"])) for r in rows}
    kern_ms, kern_flops, kern_l2, step_us, levels_total = 0.0, 0.0, 0.0, {}, 0
    kern_flops_min = 0.0
    for k, p, s in zip(ks, probs, solvers):
        B.bsde_enqueue_level(s.plan, sp, 0, 1)
        torch.cuda.synchronize(dev)
        graph = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream(dev)
        with torch.cuda.graph(graph, stream=cap):
            for _ in range(reps):
                B.bsde_enqueue_level(s.plan, cap.cuda_stream, 0, 1)
        graph.replay()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        graph.replay()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        avg = e0.elapsed_time(e1) / reps
        step_us[str(k)] = round(1000.0 * avg, 3)
        nlev = p["N"] - k + 1
        levels_total += nlev
        kern_ms += avg * nlev
        kern_flops += flops_per_gp_step_method(k, p["L"], not fp64, iters[k]) * p["Nx"] * nlev
        kern_flops_min += flops_per_gp_step(k, p["L"]) * p["Nx"] * nlev
        kern_l2 += L2_BYTES_NODE * p["Nx"] * k * p["L"] * nlev
        del graph
    pk = measured_peaks(dev)
    peak = pk["fp64_tflops"] if fp64 else pk["fp32_tflops"]
    achieved = kern_flops / (kern_ms / 1000.0) / 1e12
    achieved_min = kern_flops_min / (kern_ms / 1000.0) / 1e12
    # the FP32C step kernel reads, per point and node, the value record
    # (16 B) and the second derivatives (8 B) of its cell's left node from L2
    # (the right node's are the next lane's, an L1 hit): its L2 -> SM rate
    # against the L2 read bandwidth measured now by a plain streaming kernel
    l2 = None
    if not fp64:
        l2_gbs = kern_l2 / (kern_ms / 1000.0) / 1e9
        l2 = {"achieved": l2_gbs, "peak": pk["l2_read_gbs"], "unit": "GB/s",
              "frac": l2_gbs / pk["l2_read_gbs"], "bytes_per_point_node": L2_BYTES_NODE,
              "peak_source": "measured in this run (bsde_l2_read_probe)"}

    # end to end through the C ABI with host buffers: bsde_solve takes the
    # pinned host initial levels and writes level 0 into pinned host memory,
    # copies included; the solves of a step run concurrently, one host thread
    # (and stream) each, and the step ends when every result is on the host
    import threading
    host_in, host_out = [], []
    h2d = d2h = 0
    for p in probs:
        iy, iz = W.initial_levels(p)
        ty = torch.from_numpy(iy).pin_memory()
        tz = torch.from_numpy(iz).pin_memory()
        oy = torch.empty(p["Nx"], dtype=torch.float64).pin_memory()
        oz = torch.empty(p["Nx"], dtype=torch.float64).pin_memory()
        host_in.append((ty, tz))
        host_out.append((oy, oz))
        h2d += ty.numel() * 8 + tz.numel() * 8
        d2h += oy.numel() * 8 + oz.numel() * 8 + 40
    e2e_res = [None] * len(solvers)

    def e2e_one(i, st):
        (ty, tz), (oy, oz) = host_in[i], host_out[i]
        e2e_res[i] = B.bsde_solve(solvers[i].plan, st.cuda_stream, ty.data_ptr(), tz.data_ptr(),
                                  True, oy.data_ptr(), oz.data_ptr(), True)

    def e2e_step():
        if args.sequential:
            for i in range(len(solvers)):
                e2e_one(i, stream)
            return
        th = [threading.Thread(target=e2e_one, args=(i, st))
              for i, st in enumerate(conc.streams)]
        for t in th:
            t.start()
        for t in th:
            t.join()

    torch.cuda.synchronize(dev)
    e2e_step()
    _barrier(dist)
    e_t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    e_dt = _max_over_ranks(dist, time.perf_counter() - e_t0)
    e2e_counted = 0
    for k, u, r in zip(ks, units, e2e_res):
        g = gold.get(k)
        if g and gate(r.y0, r.z0, g["y0"], g["z0"], g["exact_y0"], g["exact_z0"],
                      args.precision)["counted"]:
            e2e_counted += u
    e2e_value = world * e2e_counted * args.steps / e_dt

    variants = None
    if not c3 and not args.no_variants:
        variants = measure_variants(args, dev, stream, flush)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # about 10 s of oracle work on 16 host threads at either size
        lv = max(1, args.cpu_levels // (2 if c3 else 1))
        cpu = cpu_baseline(lv, os.cpu_count() or 1, wl)
        one = cpu_baseline(max(1, lv // 8), 1, wl)
        cpu["single_thread"] = {"value": one["value"], "cores": 1, "sample": one["sample"]}

    if rank == 0:
        # FP32C at config3's size runs the flat step kernel (the grid fills
        # the resident threads more than twice); config2 too when its solves
        # run concurrently (flat2), the grouped one when they run in turn
        kname = "k_step64" if fp64 else ("k_step32f" if (c3 or flat2) else "k_step32")
        tkey = f"{kname}_{wl}"
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if fp64 else "f32",
            "data": "synthetic",
            "config": {"workload": _workload_text(wl, ks),
                       "Nx": probs[0]["Nx"], "N": probs[0]["N"], "k": list(ks), "L": 16,
                       "precision": args.precision,
                       "l2": ("flushed between steps (256 MiB write, outside the timed events); "
                              "inputs of the timed steps are the level rings, "
                              + ("210 MB at k = 4, larger than L2" if c3 else
                                 "<= 18 MB per solve, L2-resident within a solve by design")),
                       "step_kernel": ("FP64" if fp64 else
                                       "flat FP32C (chosen by the library for this grid)" if c3
                                       else ("flat FP32C (step_kernel = FLAT, asked for with "
                                             "--step-kernel)" if args.sequential else
                                             "flat FP32C (step_kernel = FLAT: the concurrent "
                                             "solves fill the GPU together)") if flat2
                                       else "grouped FP32C (chosen by the library for this grid)"),
                       "schedule": ("the step's solves one after another on one stream"
                                    if args.sequential else
                                    "the step's solves concurrently, one stream each "
                                    "(forked from and joined to the timing stream)"),
                       "parallelism": f"{world} independent replica(s)"},
            "accuracy": {"gate": GATE_TEXT, "oracle": f"tests/golden/{wl}_oracle.json",
                         "counted_gp_steps_per_step": counted_units,
                         "all_gp_steps_per_step": units_per_step, "rows": rows},
            "excluded": excluded,
            "ungated": {"value": world * units_per_step * args.steps / (ms_max / 1000.0),
                        "note": "every solve of the step counted, diverged ones included "
                                "(not the metric)"},
            "solve_alone_ms": alone_ms,
            "roofline": {"kernel": kname, "bound": "alu", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": _traffic(tkey),
                         "traffic_source": f"profiles/dram_traffic.json[{tkey}] (ncu)",
                         "peak_source": ("measured in this run: bsde_fma_probe, "
                                         + ("FP64 FMA" if fp64 else
                                            "FP32 FMA (better of scalar and packed FP32x2)")
                                         + " (of measured)"),
                         "flop_per_gp_step": {str(k): flops_per_gp_step_method(k, 16, not fp64,
                                                                               iters[k])
                                              for k in ks},
                         "flop_count": (f"{FLOP_NODE_COMP if not fp64 else FLOP_NODE_PLAIN} per "
                                        "node (spline values, driver, "
                                        + ("compensated " if not fp64 else "") +
                                        "sums), 3 per step j, 6 per Picard iteration "
                                        "(the solve's maximum count)"),
                         "minimal": {"flop_per_gp_step": {str(k): flops_per_gp_step(k, 16)
                                                          for k in ks},
                                     "achieved": achieved_min, "frac": achieved_min / peak,
                                     "flop_count": "23 per node (two spline values, the "
                                                   "Black-Scholes driver, three plain sums), "
                                                   "2L + 4k + 12 per point"},
                         "avg_launch_ms": kern_ms / levels_total,
                         "step_launch_us": step_us,
                         "l2": l2},
            "peaks": pk,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h,
                    "how": "bsde_solve with pinned host initial levels in and level 0 out, one "
                           "host thread and stream per solve, gated like value"},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clk.summary(),
            "wall_s_timed_region": wall,
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        if variants is not None:
            line["variants"] = {
                "workload": "config2 with the scheme's variants (Eq. 16 K_z != K_y; the "
                            "E[y dW]/dt z form; the one-step start-up of Section 3.1 step 2)",
                "gate": "|y0 - stored FP64 oracle| <= 1e-6 max(1, |y0|) (FP32C), "
                        "1e-12 max(1, |y0|) (FP64)",
                "rows": variants}
        print(json.dumps(line), flush=True)
    for s in solvers:
        s.close()
    if dist is not None:
        dist.destroy_process_group()


def _golden4():
    """The FP64 oracle's (y0, z0) and the closed form for every config4
    instance (tests/golden/config4_oracle.json, in the order of
    workloads.config4())."""
    try:
        with open(os.path.join(ROOT, "tests", "golden", "config4_oracle.json")) as fh:
            d = json.load(fh)
    except OSError:
        return None
    return [[_gold_num(v) for v in r[:4]] for r in d["rows"]]


def run_batch(args, rank, world, local_rank):
    """config4: 4096 Black-Scholes problems of uneven Nx, N, k.  The value is
    the FP32C batch (one persistent launch per step); beside it the plain
    FP64 form, one bsde_solve per instance launched concurrently over a pool
    of streams.  Both are gated per instance against the stored FP64 oracle
    values, and only the instances that pass in both arms are counted."""
    # more hardware work queues for the FP64 arm's many concurrent streams
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    import torch
    from paper_1909_13560_gb300 import bsde as B
    from paper_1909_13560_gb300 import workloads as W

    dist = _dist_init(world)
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    probs = W.config4()
    # --instances n: the first n instances (a small case for profiling; the
    # workload is all 4096)
    n_inst = len(probs) if args.instances <= 0 else min(args.instances, len(probs))
    probs = probs[:n_inst]
    units = [W.gp_steps(p) for p in probs]
    units_per_step = sum(units)
    flops_per_step = sum(flops_per_gp_step(p["k"], p["L"]) * u for p, u in zip(probs, units))
    t0 = time.perf_counter()
    bs = B.BatchSolver(probs, device=dev)
    plan_s = time.perf_counter() - t0
    # the batch configuration by timing (bsde_batch_autotune, outside the timed
    # region) unless a fixed one is asked for
    fixed = (1, 4, 0) if args.no_autotune else args.batch_config
    cfg = (bs.set_config(*fixed) or bs.config()) if fixed else bs.autotune()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        flush.zero_()
        bs.solve(want_results=False)
    torch.cuda.synchronize(dev)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    _barrier(dist)
    torch.cuda.synchronize(dev)
    with ClockSampler(_gpu_uuid(dev)) as clk:
        for i in range(args.steps):
            flush.zero_()
            starts[i].record(stream)
            bs.solve(want_results=False)
            ends[i].record(stream)
        torch.cuda.synchronize(dev)
    _barrier(dist)
    ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends))
    ms_max = _max_over_ranks(dist, ms)
    res32 = bs.solve()

    gold = _golden4()
    if gold is None or len(gold) != len(W.config4()):
        raise RuntimeError("tests/golden/config4_oracle.json is missing or stale")
    gold = gold[:len(probs)]
    g32 = [gate(r["y0"], r["z0"], *g, "fp32c") for r, g in zip(res32, gold)]

    # the plain FP64 per-instance form: one plan per instance, its solves
    # launched round robin over a pool of streams forked from the timing
    # stream and joined back
    fp64 = None
    if not args.no_fp64_arm:
        solvers = [B.Solver(p, "fp64", device=dev) for p in probs]
        pool = [torch.cuda.Stream(dev) for _ in range(32)]
        fork, joins = torch.cuda.Event(), [torch.cuda.Event() for _ in pool]

        def fp64_step():
            fork.record(stream)
            for st in pool:
                st.wait_event(fork)
            for i, s in enumerate(solvers):
                B.bsde_solve(s.plan, pool[i % len(pool)].cuda_stream, want_result=False)
            for st, ev in zip(pool, joins):
                ev.record(st)
                stream.wait_event(ev)

        for _ in range(args.warmup):  # the first one also captures each plan's graph
            flush.zero_()
            fp64_step()
        torch.cuda.synchronize(dev)
        steps64 = max(1, args.fp64_steps)
        e_ms = 0.0
        for _ in range(steps64):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fp64_step()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            e_ms += e0.elapsed_time(e1)
        e_ms = _max_over_ranks(dist, e_ms)
        res64 = [B.bsde_result_fetch(s.plan, sp) for s in solvers]
        g64 = [gate(r.y0, r.z0, *g, "fp64") for r, g in zip(res64, gold)]
        for s in solvers:
            s.close()
        del solvers
        fp64 = {"ms_per_step": e_ms / steps64, "steps": steps64, "g": g64,
                "launches_per_step": None}

    both = [a["counted"] and (fp64 is None or b["counted"])
            for a, b in zip(g32, fp64["g"] if fp64 else g32)]
    counted_units = sum(u for u, c in zip(units, both) if c)
    value = world * counted_units * args.steps / (ms_max / 1000.0)
    diverged = sum(1 for a in g32 if not a["scheme_converges"])
    e32 = sorted(a["err_y0_vs_oracle"] / max(1.0, abs(g[0]))
                 for a, g in zip(g32, gold) if a["scheme_converges"])
    ex = sorted(a["err_y0_vs_exact"] for a in g32 if a["scheme_converges"])

    # end to end: plan the batch from host problem descriptions (tables and
    # descriptors copied in), solve, read every result back
    e_t0 = time.perf_counter()
    for _ in range(args.steps):
        bs.close()
        bs = B.BatchSolver(probs, device=dev)
        bs.set_config(cfg["cluster"], cfg["target_groups"], cfg.get("flat_tiles", 0))
        eres = bs.solve()
    torch.cuda.synchronize(dev)
    e_dt = _max_over_ranks(dist, time.perf_counter() - e_t0)
    e_counted = sum(u for u, r, g, b in zip(units, eres, gold, both)
                    if b and gate(r["y0"], r["z0"], *g, "fp32c")["counted"])
    h2d = sum(1024 + 64 * p["k"] * ((p["L"] + 1) // 2) for p in probs) + 4 * len(probs)
    d2h = 32 * len(probs)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import oracle as O
        threads = os.cpu_count() or 1
        c0 = time.perf_counter()
        cu = 0
        for p in probs[:: max(1, len(probs) // 24)]:
            O.solve(p, threads=threads)
            cu += W.gp_steps(p)
        cdt = time.perf_counter() - c0
        cpu = {"value": cu / cdt, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"every {max(1, len(probs) // 24)}th problem of config4 "
                         f"({cu} grid-point steps, {cdt:.1f} s)"}
    if rank == 0:
        pk = measured_peaks(dev)
        achieved_min = flops_per_step / (ms_max / args.steps / 1000.0) / 1e12
        # the method's count (compensated sums) with each instance's Picard count
        flops_method = sum(flops_per_gp_step_method(p["k"], p["L"], True,
                                                    max(1, int(r["picard_iters_max"]))) * u
                           for p, u, r in zip(probs, units, res32))
        achieved = flops_method / (ms_max / args.steps / 1000.0) / 1e12
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": ("config4: 4096 Black-Scholes calls" if n_inst == 4096 else
                                    f"config4 (first {n_inst} of its 4096 Black-Scholes calls)")
                                   + ", seed 13560, K~U[70,130], "
                                   "sigma~U[.1,.5], T~U[.25,2], r~U[0,.05], Nx in 2^10..2^14, "
                                   "N in 32..256, k~U{1..6}, L=16; FP32C, one persistent launch",
                       "instances": len(probs), "batch_config": cfg, "plan_s": plan_s,
                       "l2": "flushed between steps (256 MiB write)",
                       "parallelism": f"{world} independent replica(s)"},
            "accuracy": {"gate": GATE_TEXT + "; an instance counts only when it passes in both "
                                             "the FP32C batch and the FP64 per-instance arm",
                         "oracle": "tests/golden/config4_oracle.json",
                         "instances_counted": sum(both),
                         "instances_diverged": diverged,
                         "instances_fp32c_outside_tol": sum(1 for a in g32 if a["scheme_converges"]
                                                            and not a["within_tol"]),
                         "counted_gp_steps_per_step": counted_units,
                         "all_gp_steps_per_step": units_per_step,
                         "fp32c_rel_err_y0_vs_oracle": {"median": e32[len(e32) // 2],
                                                        "max": e32[-1]} if e32 else None,
                         "err_y0_vs_exact": {"median": ex[len(ex) // 2],
                                             "p90": ex[int(0.9 * len(ex))],
                                             "max": ex[-1]} if ex else None},
            "ungated": {"value": world * units_per_step * args.steps / (ms_max / 1000.0),
                        "note": "every instance counted, diverged ones included (not the metric)"},
            "roofline": {"kernel": "k_batch32", "bound": "alu", "achieved": achieved,
                         "peak": pk["fp32_tflops"], "unit": "TFLOP/s",
                         "frac": achieved / pk["fp32_tflops"], "traffic": None,
                         "traffic_note": "one launch runs the whole batch (about 0.5 s), too "
                                         "long for a multi-pass capture; the DRAM bytes of "
                                         "512-instance launches (profiles/k_batch32_config4.md) "
                                         "do not scale by instance count, since how many rings "
                                         "stay in L2 depends on how many run at once",
                         "flop_count": f"{FLOP_NODE_COMP} per node (compensated sums), 3 per "
                                       "step j, 6 per Picard iteration; whole batch over the "
                                       "step time",
                         "minimal": {"achieved": achieved_min,
                                     "frac": achieved_min / pk["fp32_tflops"],
                                     "flop_count": "23 per node, 2L + 4k + 12 per point"},
                         "peak_source": "measured in this run: bsde_fma_probe, FP32 FMA (of "
                                        "measured)"},
            "peaks": pk,
            "e2e": {"value": world * e_counted * args.steps / e_dt, "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": 2 * args.steps,
            "clocks": clk.summary(),
        }
        if fp64 is not None:
            fv = world * counted_units * fp64["steps"] / (fp64["ms_per_step"] * fp64["steps"] / 1000.0)
            line["fp64_per_instance"] = {
                "value": fv, "unit": UNIT, "ms_per_step": fp64["ms_per_step"],
                "steps": fp64["steps"],
                "how": "one FP64 plan per instance (bsde_plan/bsde_solve, one CUDA graph per "
                       "solve), the 4096 solves launched round robin over 32 streams, CUDA "
                       "events around the whole set; same instances counted as the FP32C value",
                "instances_within_tol": sum(1 for b in fp64["g"] if b["counted"]),
                "fp32c_batch_over_fp64": value / fv if fv > 0 else None}
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    bs.close()
    if dist is not None:
        dist.destroy_process_group()


def flops_per_gp_step_2d32(k: int, L: int) -> float:
    """FP32C 2-D: per tensor node 15 weight products, per field three value
    increments (3 ops each) and 15 FMA, a compensated accumulation (~10) for
    the three fields, the driver (3) and the three driver sums (3); counted as
    operations (an FMA as 2 flop); per point the group sums and Picard."""
    per_node = 15 + 3 * (9 + 15 * 2) + 3 * 10 + 3 * 2 + 3 * 2
    return k * L * L * per_node + 9 * 6 + 10 * 6


def flops_per_gp_step_2d(k: int, L: int) -> float:
    """Algorithmic FP64 flops of one 2-D grid-point step: per tensor node three
    bicubic values (12 FMA each), the linear driver (2 FMA + 1 mul) and the
    three weighted sums (2 FMA each); per point the group sums and ~10
    Picard iterations."""
    per_node = 3 * 12 * 2 + 5 + 3 * 2 * 2
    return k * L * L * per_node + 3 * 6 + 10 * 6


def flops_per_gp_step_tp(k: int, L: int, precision: str) -> dict:
    """Algorithmic flops of one 2-D grid-point step in the tensor-product form,
    per pass (an FMA as 2 flop).  FP64: the x2 pass takes per (j, l2) and
    field the two x2 interpolants R, S (1 mul + 3 FMA each) and four weighted
    sums (4 FMA): 66 per (j, l2); the x1 pass per (j, l1) and field the two x1
    interpolants and three sums: 60, per j the driver combinations and the
    z, A updates (27), per point ~10 Picard iterations (80).  FP32C, per
    mirror pair of nodes: the x2 pass two interpolant sets (48 ops each) and
    per field the exact pair sum, one compensated product and the plain
    slope and difference sums (33 ops): 195; the x1 pass two interpolant sets
    (96), the drivers of both nodes and their difference (40), the z sums by
    compensated products (44) and the driver sums (13): 193."""
    if precision == "fp64":
        return {"x2": k * L * 66.0, "x1": k * L * 60.0 + k * 27.0 + 80.0}
    pairs = (L + 1) // 2
    return {"x2": k * pairs * 195.0, "x1": k * pairs * 193.0 + 80.0}


def run_2d(args, rank, world, local_rank):
    """Example 4 (Eq. 34-35) at the paper's largest configuration (Table 9:
    K = 6, N = 64, M = 1024 intervals per dimension on [-8, 8]^2, L = 8 per
    dimension), in --precision (FP32C by default, FP64 on request); one step =
    one whole solve."""
    import torch
    from paper_1909_13560_gb300 import bsde as B
    from paper_1909_13560_gb300 import workloads as W
    dist = _dist_init(world)
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    K, N, M, L = 6, 64, 1024, 8
    p = dict(W.ex4_problem(M=M, N=N, k=K, L=L), step_form=args.step_form)
    prec = args.precision
    # AUTO takes the tensor-product passes for Example 4 (b21 = 0)
    tensor = args.step_form == "TENSOR" or (args.step_form == "AUTO" and p["b21"] == 0.0)
    s = B.Solver2(p, device=dev, precision=prec)
    np_ = p["Nx1"] * p["Nx2"]
    units = np_ * (N - K + 1)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        flush.zero_()
        s.enqueue(sp)
    torch.cuda.synchronize(dev)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        if not uuid.startswith("GPU-"):
            uuid = "GPU-" + uuid
    except Exception:
        uuid = None
    _barrier(dist)
    torch.cuda.synchronize(dev)
    with ClockSampler(uuid) as clk:
        w0 = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()
            starts[i].record(stream)
            s.enqueue(sp)
            ends[i].record(stream)
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - w0
    _barrier(dist)
    ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends))
    ms_max = _max_over_ranks(dist, ms)
    value = world * units * args.steps / (ms_max / 1000.0)
    r = s.fetch(sp)
    ey = abs(r["y0"])
    ez = math.hypot(r["z0"][0] - 1.0, r["z0"][1] - 1.0)

    # the step and derivative kernels of one level, replayed from a graph
    # (the tensor form's two passes one by one)
    reps = 10
    times = {}
    parts = ((4, "x2"), (8, "x1"), (1, "k2_step"), (2, "k2_deriv")) if tensor else \
        ((1, "k2_step"), (2, "k2_deriv"))
    for part, name in parts:
        s.enqueue_level(sp, 0, part)
        torch.cuda.synchronize(dev)
        g = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream(dev)
        with torch.cuda.graph(g, stream=cap):
            for _ in range(reps):
                s.enqueue_level(cap.cuda_stream, 0, part)
        g.replay()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.replay()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        times[name] = e0.elapsed_time(e1) / reps
        del g
    peaks = _peaks()
    pk = measured_peaks(dev)
    peak = pk["fp64_tflops"] if prec == "fp64" else pk["fp32_tflops"]
    rec = 96 if prec == "fp64" else 64
    if tensor:
        fp = flops_per_gp_step_tp(K, L, prec)
        dom = max(("x2", "x1"), key=lambda q: times[q])
        kname = {("x2", "fp64"): "k2_tp1", ("x1", "fp64"): "k2_tp2",
                 ("x2", "fp32c"): "k2_tp1_32", ("x1", "fp32c"): "k2_tp2_32"}[(dom, prec)]
        fpg = fp[dom]
        step_ms = times[dom]
        # L1 data per point: two records per node and field set; HBM: the x2
        # pass reads the k ring levels and writes k buffer records, the x1
        # pass reads them back and writes the new values (24 B)
        l1b = K * L * 2 * rec
        hbm_b = {"x2": 2 * K * rec, "x1": K * rec + (32 if prec == "fp64" else 16) + 24}[dom]
    else:
        fpg = flops_per_gp_step_2d(K, L) if prec == "fp64" else flops_per_gp_step_2d32(K, L)
        kname = "k2_step" if prec == "fp64" else "k2_step32p"
        step_ms = times["k2_step"]
        l1b = K * L * L * (384 if prec == "fp64" else 256)
        hbm_b = K * rec + 24
    achieved = fpg * np_ / (step_ms / 1000.0) / 1e12
    # derivative kernel: reads the new values (24 B: doubles, or float pairs
    # in FP32C) and writes the ring records (96 B FP64, 64 B FP32C) per point
    der_b = 24 + rec
    der_gbs = der_b * np_ / (times["k2_deriv"] / 1000.0) / 1e9
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    hbm_gbs = hbm_b * np_ / (step_ms / 1000.0) / 1e9

    # end to end: caller levels from pinned host memory, level 0 back
    init = [torch.from_numpy(a).pin_memory() for a in _ex4_levels(p)]
    outs = [torch.empty((p["Nx2"], p["Nx1"]), dtype=torch.float64).pin_memory() for _ in range(3)]
    lib = B.load()
    import ctypes
    res = B.bsde2_result()

    def e2e_once():
        rc = lib.bsde2_solve(ctypes.c_void_p(s.plan), ctypes.c_void_p(sp),
                             *[ctypes.c_void_p(t.data_ptr()) for t in init], 1,
                             *[ctypes.c_void_p(t.data_ptr()) for t in outs], 1, ctypes.byref(res))
        if rc < 0:
            raise B.BsdeError(rc, "bsde2_solve")
    e2e_once()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_once()
    torch.cuda.synchronize(dev)
    e_dt = _max_over_ranks(dist, time.perf_counter() - t0)
    h2d = sum(t.numel() * 8 for t in init)
    d2h = sum(t.numel() * 8 for t in outs) + 64

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import oracle as O
        threads = os.cpu_count() or 1
        lv = 2
        c0 = time.perf_counter()
        O.solve2(p, levels=lv, threads=threads)
        cdt = time.perf_counter() - c0
        cpu = {"value": np_ * lv / cdt, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"Example 4 at M=1024, K=6: closed-form start and the first {lv} "
                         f"backward levels, {threads} host threads, {cdt:.1f} s"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == "fp64" else "f32", "data": "synthetic",
            "config": {"workload": "ex4_2d: two-dimensional Example 4 (f = y - (z1+z2)/2, "
                                   "g = sin(x1+x2+T), X = W), x in [-8,8]^2, M=1024 intervals "
                                   "per dimension (1025^2 points), N=64, K=6, L=8 per dimension "
                                   f"(64 tensor nodes), {prec.upper()}; one solve per step",
                       "precision": prec,
                       "step_form": ("tensor-product passes (x2 pass, x1 pass)" if tensor
                                     else "node-wise step kernel"),
                       "Nx1": p["Nx1"], "Nx2": p["Nx2"], "N": N, "k": K, "L": L,
                       "l2": "flushed between steps (256 MiB write, outside the timed events); "
                             "the level ring (700 MB) is HBM-resident",
                       "parallelism": f"{world} independent replica(s)"},
            "accuracy": {"gate": "errors against the closed form equal the paper's Table 9 row "
                                 "(K=6, N=64, M=1024: 8.00e-7, 2.32e-6) to 2%",
                         "err_y0": ey, "err_z0_norm": ez,
                         "within_tol": abs(ey - 8.00e-7) <= 0.02 * 8.00e-7
                         and abs(ez - 2.32e-6) <= 0.02 * 2.32e-6},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": _traffic(kname) if (tensor or prec != "fp64") else None,
                         # node-wise, K = 6, L = 8: the 192-entry pair table
                         # fits the FP32C step's parameters (k2_step32p)
                         "kernel": kname,
                         "hbm": {"achieved": hbm_gbs, "peak": hbm, "unit": "GB/s",
                                 "frac": hbm_gbs / hbm, "bytes_per_point": hbm_b},
                         "pass_ms": ({"k2_tp1": times["x2"], "k2_tp2": times["x1"]}
                                     if tensor else None),
                         "peak_source": "measured in this run: bsde_fma_probe, "
                                        + ("FP64 FMA" if prec == "fp64" else
                                           "FP32 FMA (better of scalar and packed FP32x2)")
                                        + " (of measured)",
                         "flop_per_gp_step": fpg,
                         "l1_bytes_per_gp_step": l1b,
                         "step_launch_ms": times["k2_step"],
                         "deriv": {"kernel": "k2_deriv" if prec == "fp64" else "k2_deriv32",
                                   "bound": "hbm", "achieved": der_gbs,
                                   "peak": hbm, "unit": "GB/s", "frac": der_gbs / hbm,
                                   "launch_ms": times["k2_deriv"],
                                   "bytes_per_point": der_b}},
            "e2e": {"value": world * units * args.steps / e_dt, "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": s.launches * args.steps,
            "clocks": clk.summary(),
            "wall_s_timed_region": wall,
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    s.close()
    if dist is not None:
        dist.destroy_process_group()


def _ex4_levels(p):
    """Closed-form initial levels of Example 4 as host arrays (y, z1, z2),
    each (k, Nx2, Nx1): input data for the end-to-end leg."""
    import numpy as np
    x1 = np.linspace(p["x1_min"], p["x1_max"], p["Nx1"])
    x2 = np.linspace(p["x2_min"], p["x2_max"], p["Nx2"])
    X1, X2 = np.meshgrid(x1, x2)
    dt = p["T"] / p["N"]
    ys = np.array([np.sin(X1 + X2 + (p["N"] - m) * dt) for m in range(p["k"])])
    zs = np.array([np.cos(X1 + X2 + (p["N"] - m) * dt) for m in range(p["k"])])
    return ys, zs, zs.copy()


def flops_per_gp_step_general(k: int, L: int) -> float:
    """Algorithmic FP64 flops of one grid-point step on the general forward
    path: per node the Euler position (2 FMA), cell and theta (sub, div,
    floor, sub), the four spline weights (~8), the two spline values (2 x 6),
    the driver (~3) and the weighted sums (~6); per point ~10 Picard
    iterations."""
    return k * L * (4 + 4 + 8 + 12 + 3 + 6) + 10 * 6


def flops_per_gp_step_general32(k: int, L: int) -> float:
    """FP32C general path, per node (half a pair): the double-float offset
    (~10), floor and theta (~6), kappa (3), the spline value (3 packed FMA on
    the (y, z) lanes = 6 lane ops x 2), the driver (~4), and the pair's share
    of the compensated sums and driver terms (~12); per point ~10 Picard
    iterations.  Operations, an FMA counted as 2 flop."""
    return k * L * (10 + 6 + 3 + 12 + 4 + 12) * 2 + 10 * 6


def run_general(args, rank, world, local_rank):
    """The general forward path (affine coefficients, Euler) in --precision
    (FP32C by default) at the benchmark's grid size: the Vasicek bond (short-rate driver f = -x y,
    K_y = 2, K_z = 1 with the E[y dW]/dt z form) and the Black-Scholes call in
    the price (geometric Brownian motion, K = 3); Nx = 65536, N = 256, L = 16.
    One step = one solve of each."""
    import torch
    from paper_1909_13560_gb300 import bsde as B
    from paper_1909_13560_gb300 import workloads as W
    dist = _dist_init(world)
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    probs = {"vasicek_k2_kz1_ydw": dict(W.vasicek_problem(Nx=65536, N=256, k=2), kz=1, zform=1),
             "gbm_price_call_k3": W.gbm_call_problem(Nx=65536, N=256, k=3)}
    prec = args.precision
    solvers = {n: B.Solver(p, prec, device=dev) for n, p in probs.items()}
    units = sum(W.gp_steps(p) for p in probs.values())
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def one_step():
        for s in solvers.values():
            B.bsde_solve(s.plan, sp, want_result=False)

    for _ in range(args.warmup):
        flush.zero_()
        one_step()
    torch.cuda.synchronize(dev)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        if not uuid.startswith("GPU-"):
            uuid = "GPU-" + uuid
    except Exception:
        uuid = None
    _barrier(dist)
    torch.cuda.synchronize(dev)
    with ClockSampler(uuid) as clk:
        w0 = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()
            starts[i].record(stream)
            one_step()
            ends[i].record(stream)
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - w0
    _barrier(dist)
    ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends))
    ms_max = _max_over_ranks(dist, ms)
    value = world * units * args.steps / (ms_max / 1000.0)
    rows = []
    kern_ms = kern_flops = 0.0
    for name, p in probs.items():
        s = solvers[name]
        r = B.bsde_result_fetch(s.plan, sp)
        if p["terminal"] == "ONE":
            u, ux = W.vasicek_bond(p, 0.0, p["x0"])
        else:
            u, ux = W.price_call(p, 0.0, p["x0"])
        u, z = float(u), float((p["b_x"] + p["b_1"] * p["x0"]) * ux)
        # the step kernel of level 0, replayed from a graph
        B.bsde_enqueue_level(s.plan, sp, 0, 1)
        torch.cuda.synchronize(dev)
        g = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream(dev)
        with torch.cuda.graph(g, stream=cap):
            for _ in range(20):
                B.bsde_enqueue_level(s.plan, cap.cuda_stream, 0, 1)
        g.replay()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.replay()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        avg = e0.elapsed_time(e1) / 20
        del g
        K = W.levels_K(p)
        nlev = p["N"] - K + 1
        kern_ms += avg * nlev
        fpg = flops_per_gp_step_general if prec == "fp64" else flops_per_gp_step_general32
        kern_flops += fpg(K, p["L"]) * p["Nx"] * nlev
        rows.append({"name": name, "y0": r.y0, "z0": r.z0, "exact_y0": u, "exact_z0": z,
                     "err_y0_vs_exact": abs(r.y0 - u), "err_z0_vs_exact": abs(r.z0 - z),
                     "step_launch_us": 1000.0 * avg, "launches": s.launches})
    pk = measured_peaks(dev)
    peak = pk["fp64_tflops"] if prec == "fp64" else pk["fp32_tflops"]
    achieved = kern_flops / (kern_ms / 1000.0) / 1e12

    # end to end: caller levels from pinned host memory, level 0 and the
    # result back, every step
    host = {}
    h2d = d2h = 0
    for name, p in probs.items():
        iy, iz = W.initial_levels(p)
        ty, tz = torch.from_numpy(iy).pin_memory(), torch.from_numpy(iz).pin_memory()
        oy = torch.empty(p["Nx"], dtype=torch.float64).pin_memory()
        oz = torch.empty(p["Nx"], dtype=torch.float64).pin_memory()
        host[name] = (ty, tz, oy, oz)
        h2d += (ty.numel() + tz.numel()) * 8
        d2h += (oy.numel() + oz.numel()) * 8 + 40
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for name, s in solvers.items():
            ty, tz, oy, oz = host[name]
            B.bsde_solve(s.plan, sp, ty.data_ptr(), tz.data_ptr(), True, oy.data_ptr(),
                         oz.data_ptr(), True)
    torch.cuda.synchronize(dev)
    e_dt = _max_over_ranks(dist, time.perf_counter() - t0)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import oracle as O
        threads = os.cpu_count() or 1
        lv = 32
        c0 = time.perf_counter()
        cu = 0
        for p in probs.values():
            rr = O.solve(p, levels=lv, threads=threads)
            cu += p["Nx"] * rr["levels_done"]
        cdt = time.perf_counter() - c0
        cpu = {"value": cu / cdt, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"both problems, first {lv} backward levels each, {threads} host "
                         f"threads, {cdt:.1f} s"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == "fp64" else "f32", "data": "synthetic",
            "config": {"workload": "general: forward process by Euler with affine a(x), b(x); "
                                   "Vasicek bond (kappa=.8, theta=.04, sigma=.02, r0=.03, T=2, "
                                   "f = -x y, K_y=2, K_z=1, E[y dW]/dt z form) and the call in "
                                   "the price under GBM (S0=K=100, r=.03, mu=.05, sigma=.2, "
                                   f"T=1, K=3); Nx=65536, N=256, L=16, {prec.upper()}; one solve "
                                   "each per step", "precision": prec,
                       "Nx": 65536, "N": 256, "L": 16,
                       "l2": "flushed between steps (256 MiB write, outside the timed events)",
                       "parallelism": f"{world} independent replica(s)"},
            "accuracy": {"gate": "errors against the closed forms (Euler forward: first "
                                 "order in dt)", "rows": rows},
            "roofline": {"kernel": "k_step64_gen" if prec == "fp64" else "k_step32_gen",
                         "bound": "alu", "achieved": achieved,
                         "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": None,
                         "traffic_note": ("the step launches of the two problems differ; one "
                                          "captured Vasicek launch read 3.16 MB "
                                          "(profiles/k_step32_gen_general.md), its input "
                                          "levels once") if prec != "fp64" else
                                         "no DRAM capture of the FP64 general kernel",
                         "peak_source": "measured in this run: bsde_fma_probe, "
                                        + ("FP64 FMA" if prec == "fp64" else
                                           "FP32 FMA (better of scalar and packed FP32x2)")
                                        + " (of measured)",
                         "flop_per_gp_step": {n: (flops_per_gp_step_general if prec == "fp64"
                                                  else flops_per_gp_step_general32)(W.levels_K(p), p["L"])
                                              for n, p in probs.items()}},
            "e2e": {"value": world * units * args.steps / e_dt, "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": sum(s.launches for s in solvers.values()) * args.steps,
            "clocks": clk.summary(),
            "wall_s_timed_region": wall,
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    for s in solvers.values():
        s.close()
    if dist is not None:
        dist.destroy_process_group()


def run_decomp(args, rank, world, local_rank):
    """One large problem decomposed into slabs (the lending/borrowing call of
    config3 at full size, Nx = 2^20, N = 1024, K = 2, FP32C): solved as one
    plan and as 2, 4 and 8 slabs with halo exchange after every step, all
    slabs on this GPU (LocalTransport).  Reports each layout's time, the halo
    overhead (extra points computed) and the exchange volume per level, and
    the agreement of y0 with the one-plan solve.  One step = one solve of the
    largest layout."""
    import torch
    from paper_1909_13560_gb300 import bsde as B
    from paper_1909_13560_gb300 import decomp
    from paper_1909_13560_gb300 import workloads as W
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    p = W.config3(k=2)
    units = W.gp_steps(p)
    halo = decomp.halo_width(p)
    ref = B.solve(p, "fp32c")
    rows = []
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        if not uuid.startswith("GPU-"):
            uuid = "GPU-" + uuid
    except Exception:
        uuid = None
    parts_list = (2, 4, 8)
    with ClockSampler(uuid) as clk:
        for parts in parts_list:
            ss = decomp.ShardedSolver(p, parts, "fp32c", device=dev)  # plans made once
            ss.replay(stream)  # captures the level loop into a graph, then runs it
            torch.cuda.synchronize(dev)
            ms = 0.0
            steps = min(max(1, args.steps), 5)
            for _ in range(steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ss.replay(stream)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                ms += e0.elapsed_time(e1)
            ms /= steps
            got = ss.result(stream)
            ss.close()
            lay = got["slabs"]
            extra = sum(sl["local"][1] - sl["local"][0] for sl in lay) - p["Nx"]
            rows.append({"parts": parts, "ms_per_solve": ms, "gp_steps_per_s": units / (ms / 1000.0),
                         "halo": halo, "extra_points_frac": extra / p["Nx"],
                         "exchange_bytes_per_level": 2 * (parts - 1) * halo * 16,
                         "y0": got["y0"], "dy0_vs_one_plan": abs(got["y0"] - ref["y0"])})
    s1 = B.Solver(p, "fp32c", device=dev)
    s1.solve()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    B.bsde_solve(s1.plan, stream.cuda_stream, want_result=False)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    one_ms = e0.elapsed_time(e1)
    launches = s1.launches
    s1.close()
    if rank == 0:
        last = rows[-1]
        line = {
            "metric": METRIC, "value": last["gp_steps_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": 1, "ms_per_step": last["ms_per_solve"],
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "decomp: lending/borrowing call (config3 parameters) at full "
                                   "size Nx=2^20, N=1024, K=2, L=16, FP32C, one problem as 8 "
                                   "slabs with halo exchange every level, all slabs on one GPU "
                                   "(the level loop captured once into a CUDA graph)",
                       "Nx": p["Nx"], "N": p["N"], "k": 2, "halo": halo},
            "one_plan": {"ms_per_solve": one_ms, "gp_steps_per_s": units / (one_ms / 1000.0),
                         "y0": ref["y0"], "launches": launches},
            "layouts": rows,
            "accuracy": {"gate": "|y0(slabs) - y0(one plan)| <= 1e-6 max(1, |y0|)",
                         "within_tol": all(r["dy0_vs_one_plan"] <= 1e-6 * max(1.0, abs(ref["y0"]))
                                           for r in rows)},
            "gpu_launches": None,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)


def _closed_form_call(p):
    """Closed-form price and z of a config5 request at t = 0 (Black-Scholes;
    the lending/borrowing driver at the rate r - s (R - r), since its min()
    is active everywhere for a call)."""
    r = p["r"] - (p["lb_sign"] * (p["R"] - p["r"]) if p["driver"] == "LB" else 0.0)
    S0, K, sig, T = math.exp(p["x0"]), p["strike"], p["sigma"], p["T"]
    sq = sig * math.sqrt(T)
    d1 = (math.log(S0 / K) + (r + 0.5 * sig * sig) * T) / sq
    ncdf = lambda x: 0.5 * math.erfc(-x / math.sqrt(2.0))
    price = S0 * ncdf(d1) - K * math.exp(-r * T) * ncdf(d1 - sq)
    return price, sig * S0 * ncdf(d1)


def _served_ok(p, res) -> bool:
    """A served result counts when its y0 and z0 are within CONV_REL (1%) x
    max(1, |value|) of the closed form, the accuracy the scheme reaches where
    it converges on the request's grid."""
    u, z = _closed_form_call(p)
    return (math.isfinite(res["y0"]) and math.isfinite(res["z0"])
            and abs(res["y0"] - u) <= CONV_REL * max(1.0, abs(u))
            and abs(res["z0"] - z) <= CONV_REL * max(1.0, abs(z)))


def run_serving(args, rank, world, local_rank):
    """config5: Poisson arrivals of pricing requests served by the persistent
    continuous-batching kernel; one step = the whole arrival sequence.  The
    value counts the served results that pass the accuracy gate; a sweep of
    lower rates finds the highest one the device sustains with p99 under
    --p99-bound-ms."""
    import torch
    from paper_1909_13560_gb300 import bsde as B
    from paper_1909_13560_gb300 import serve
    from paper_1909_13560_gb300 import workloads as W

    dist = _dist_init(world)
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    arrivals = W.config5_arrivals(rate=args.rate, duration=args.duration)
    units = sum(W.gp_steps(p) for _, p in arrivals)
    srv = B.Server(slots=1024, pool_bytes=8 << 30, device=dev)
    srv.start(cluster=args.server_cluster, idle_ms=60000)
    sweep = []
    try:
        # warm-up: a short burst through the same server
        serve.serve(srv, [(0.0, p) for _, p in arrivals[:64]])
        _barrier(dist)
        with ClockSampler(_gpu_uuid(dev)) as clk:
            records, summary = serve.serve(srv, arrivals)
        _barrier(dist)
        if not args.no_sweep:
            for rate in (1500.0, 1000.0, 750.0, 500.0, 250.0):
                arr = W.config5_arrivals(rate=rate, duration=args.sweep_duration)
                _, sm = serve.serve(srv, arr)
                sweep.append({"rate": rate, "requests": sm["requests"],
                              "solves_per_s": sm["solves_per_s"], "p50_ms": sm["p50_ms"],
                              "p99_ms": sm["p99_ms"]})
    finally:
        srv.stop()
        srv.close()
    t = _max_over_ranks(dist, summary["duration_s"])
    ok = [_served_ok(p, r["result"]) for (_, p), r in zip(arrivals, records)]
    lb4 = [(p["driver"] == "LB") for _, p in arrivals]
    if rank == 0:
        sustained = [r for r in sweep if r["p99_ms"] <= args.p99_bound_ms]
        line = {
            "metric": METRIC, "value": world * sum(ok) / t, "unit": "solves/s",
            "n_gpus": world, "steps": 1, "warmup": 1, "ms_per_step": 1000.0 * t,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"config5: Poisson arrivals at {args.rate:g}/s for "
                                   f"{args.duration:g} s (seed 1909), 70% Black-Scholes "
                                   "(Nx=2^12, N=64, k=3), 30% lending/borrowing calls "
                                   "(Nx=2^16, N=256, k=4), L=16; admission by device memory "
                                   "(8 GiB pool, 1024 slots); persistent continuous-batching kernel, "
                                   f"{args.server_cluster} CTA(s) per request",
                       "requests": summary["requests"]},
            "accuracy": {"gate": "a served result counts when y0 and z0 are within 1% x max(1, "
                                 "|value|) of the closed form (Black-Scholes; the lending/"
                                 "borrowing call at r - (R - r))",
                         "served": summary["requests"], "counted": sum(ok),
                         "black_scholes_counted": sum(1 for o, l in zip(ok, lb4) if o and not l),
                         "black_scholes_served": sum(1 for l in lb4 if not l),
                         "lending_borrowing_counted": sum(1 for o, l in zip(ok, lb4) if o and l),
                         "lending_borrowing_served": sum(lb4),
                         "note": "the lending/borrowing requests (k=4 at Nx=2^16, N=256) are the "
                                 "grid on which the scheme diverges (the FP64 oracle of config3 at "
                                 "this size too): served and timed, not counted"},
            "serving": {"p50_ms": summary["p50_ms"], "p99_ms": summary["p99_ms"],
                        "solves_per_s_all": world * summary["requests"] / t,
                        "max_inflight": summary["max_inflight"],
                        "admit_wait_p99_ms": summary["admit_wait_p99_ms"],
                        "grid_point_steps_per_s": world * units / t},
            "sustained": {"p99_bound_ms": args.p99_bound_ms,
                          "highest_rate_within_bound": (max(r["rate"] for r in sustained)
                                                        if sustained else None),
                          "sweep": sweep,
                          "how": f"the same mix at lower Poisson rates, {args.sweep_duration:g} s "
                                 "of arrivals each, through the same server"},
            "e2e": {"value": world * sum(ok) / t, "unit": "solves/s",
                    "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 40 * summary["requests"]},
            "gpu_launches": 1,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 20 for config3, 100 for config2, whose step "
                         "is ~16 ms, so that the clock samples cover the timed region; 40 "
                         "otherwise; 10 for the reference arm)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32c", "fp64"], default="fp32c")
    ap.add_argument("--step-form", choices=["AUTO", "NODEWISE", "TENSOR"], default="AUTO",
                    help="ex4_2d: form of the 2-D step kernels")
    ap.add_argument("--workload", choices=["config2", "config3", "config4", "config5", "ex4_2d",
                                           "general", "decomp"],
                    default="config3",
                    help="config3: the lending/borrowing call at Nx=2^20, N=1024 (k=4 and "
                         "k=2; the default); config2: the Black-Scholes solves k = 1..6; "
                         "config4: the 4096-instance batch in one persistent launch; "
                         "config5: the serving run (Poisson arrivals, continuous batching)")
    ap.add_argument("--duration", type=float, default=10.0, help="config5: seconds of arrivals")
    ap.add_argument("--rate", type=float, default=2000.0, help="config5: arrivals per second")
    ap.add_argument("--no-sweep", action="store_true", help="config5: skip the rate sweep")
    ap.add_argument("--server-cluster", type=int, default=8, choices=(1, 2, 4, 8),
                    help="config5: CTAs per cluster of the serving kernel (one request each)")
    ap.add_argument("--sweep-duration", type=float, default=3.0,
                    help="config5: seconds of arrivals per rate of the sweep")
    ap.add_argument("--p99-bound-ms", type=float, default=500.0,
                    help="config5: the p99 latency a sustained rate must stay under")
    ap.add_argument("--ks", type=lambda v: [int(t) for t in v.split(",")], default=list(KS),
                    help="config2: the step counts k to solve (default 1,2,3,4,5,6; a subset "
                         "is for profiling one kernel shape, not a bench line)")
    ap.add_argument("--cpu-levels", type=int, default=64)
    ap.add_argument("--ref-levels", type=int, default=0,
                    help="reference arm: backward levels per solve in each step's sample "
                         "(default 4 for config3, 12 for config2)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sequential", action="store_true",
                    help="config2/3: run a step's solves one after another on one stream "
                         "(default: concurrently, one stream each)")
    ap.add_argument("--no-variants", action="store_true",
                    help="config2: skip the timing of the scheme's variants")
    ap.add_argument("--no-fp64-arm", action="store_true",
                    help="config4: skip the FP64 per-instance comparison")
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="config4: timed steps of the FP64 per-instance arm (~7 s each)")
    ap.add_argument("--step-kernel", choices=["AUTO", "FLAT"], default="AUTO",
                    help="config2 FP32C: FLAT also with --sequential (the concurrent default "
                         "takes it anyway)")
    ap.add_argument("--instances", type=int, default=0,
                    help="config4: only the first n instances (a small case for profiling; "
                         "0 = all 4096)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="config4: a fixed batch configuration (cluster 1, 4 groups) instead "
                         "of the autotuned one")
    ap.add_argument("--batch-config", default=None,
                    type=lambda v: tuple(int(t) for t in v.split(",")),
                    help="config4: a fixed batch configuration 'cluster,groups,flat' "
                         "(e.g. 1,1,1) instead of the autotuned one")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = _env_int("RANK", 0)
    if args.steps is None:
        args.steps = {"config2": 100, "config3": 20}.get(args.workload, 40) \
            if args.impl == "ours" else 10
    world = _env_int("WORLD_SIZE", 1)
    local_rank = _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "config4":
        run_batch(args, rank, world, local_rank)
    elif args.workload == "config5":
        run_serving(args, rank, world, local_rank)
    elif args.workload == "ex4_2d":
        run_2d(args, rank, world, local_rank)
    elif args.workload == "general":
        run_general(args, rank, world, local_rank)
    elif args.workload == "decomp":
        run_decomp(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
