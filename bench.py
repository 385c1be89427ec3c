#!/usr/bin/env python3
"""Benchmark of the CSPH-TVD time step (arXiv 1912.04855, Sec. 2.2-3) on B300.

Workload (default): supersonic flow through a gravitational potential well on
a 256^3 grid, FP32 state and arithmetic, inflow/outflow in x and periodic in
y/z, CFL 0.4 (the paper's 3D performance problem of Sec. 3).  One "step" is
one full CSPH-TVD update of the grid: dt reduction, ghost layers, Lagrangian
predictor and corrector, Eulerian fluxes and update.

Prints ONE JSON line.  ``value`` is whole-job cell-updates per second (in
G/s) over K timed steps with the state resident in HBM (the 335 MB FP32
state and its scratch exceed the 126 MB L2, so no flush is needed between
steps).  ``e2e`` repeats the measurement through the C ABI with pinned host
buffers: each step uploads the full FP64 state, advances one step and
downloads it.  ``roofline`` rates the dominant kernel from its own CUDA-event
durations inside this run.  ``cpu_baseline`` times the FP64 CPU oracle on a
bounded window of the same workload.

Multi-GPU: ``--gpus N`` under torchrun runs N independent replicas (one grid
per GPU, no collective in the data path; the method's steps are not sharded
here), a barrier and a max-over-ranks time around the timed region.

``--impl reference`` times the FP64 CPU oracle as the reference arm.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FALLBACK = {"hbm_gbs": 6400.0, "sm_max_mhz": 2032.0}
# Algorithmic DRAM bytes per cell-update of one full step: read U (5 words)
# and psi (1), write U (5).
WORDS_PER_CELL = 11
# Algorithmic floating-point operations per cell of each fused kernel (an FMA
# counts 2), counted from the method's per-cell formulas with constants
# folded: the Lagrangian kernel holds primitive recovery (13), the predictor
# force (186) and update (28), the corrector force over 26 displaced pairs
# (782) and update (41); the Euler kernel the slopes (90), half-step state and
# reconstruction (83), Riemann fluxes (105), update (35) and the signal speed
# (17).  The plain path splits the same work over more kernels.
FLOPS_PER_CELL = {"lagrange": 1050, "euler": 330}
# ALU peaks from the unit counts: 148 SMs x 128 FP32 lanes x 2 flops x clock;
# FP64 dense rate of this part, nominal.
FP32_LANES = 148 * 128
FP64_TFLOPS_NOMINAL = 1.25
KERNEL_SOURCES = ["paper_1912_04855_b300/csrc/fast.cuh", "paper_1912_04855_b300/csrc/common.cuh",
                  "paper_1912_04855_b300/csrc/tma.cuh"]


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def recorded_counts(kernel, prec):
    """Per-cell counters of `kernel` from the committed ncu capture summary
    (DRAM bytes, thread instructions, shared-memory wavefronts), or {} when
    the kernels changed since it was taken."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(p):
        return {}
    d = json.load(open(p))
    if d.get("source_hash") != kernel_source_hash():
        return {}
    return d.get("kernels", {}).get(f"{kernel}_fp{prec}") or {}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def init_dist(world, use_cuda):
    if world <= 1:
        return None
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group("nccl" if use_cuda else "gloo")
    return dist


def max_over_ranks(dist, value, device=None):
    """Max of a float over all ranks (identity without a process group)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_workload(name):
    from paper_1912_04855_b300 import workloads as wl
    if name == "well256":
        return wl.potential_well(n=256), "supersonic flow through a potential well, 256^3, psi0=2, sigma=0.1, Mach 3, gamma=5/3"
    if name == "well128":
        return wl.potential_well(n=128), "supersonic flow through a potential well, 128^3"
    if name == "well192":
        return wl.potential_well(n=192), "supersonic flow through a potential well, 192^3"
    if name == "sod":
        return wl.shock_tube(), "Sod shock tube 128x16x16"
    if name == "hydro128":
        return wl.hydrostatic(n=128), "hydrostatic isothermal atmosphere 128^3 with vacuum above z=0.8"
    if name == "blast512":
        return wl.blast(n=512), "point blast 512^3"
    if name.startswith("well") and name[4:].isdigit():  # the same flow on an n^3 grid
        n = int(name[4:])
        return wl.potential_well(n=n), f"supersonic flow through a potential well, {n}^3"
    raise SystemExit(f"unknown workload {name}")


# ----------------------------------------------------------------- CPU side

def cpu_oracle_rate(w, budget_s=15.0, max_windows=64):
    """Times the FP64 CPU oracle on windows of the workload (bounded CPU time).
    Returns (cell-updates per second, description, threads)."""
    from oracle import oracle as O
    O.build()
    P = O.Problem(w.shape, w.h, w.gamma, w.bc, inflow=w.inflow)
    U = P.prim_to_cons(w.W)
    dt = P.dt(U, w.cfl)
    nz, ny, nx = w.shape
    edge = min(64, nx, ny, nz)
    cells = 0
    t0 = time.perf_counter()
    nwin = 0
    while nwin < max_windows and (time.perf_counter() - t0) < budget_s:
        z0 = (nwin * edge) % max(nz - edge + 1, 1)
        box = ((0, edge), (0, edge), (z0, z0 + edge))
        P.step(w.psi, U, dt, box=box)
        cells += edge ** 3
        nwin += 1
    el = time.perf_counter() - t0
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return cells / el, f"{nwin} one-step windows of {edge}^3 cells of the same workload ({el:.1f} s)", threads


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    w, desc = make_workload(args.workload)
    from oracle import oracle as O
    O.build()
    P = O.Problem(w.shape, w.h, w.gamma, w.bc, inflow=w.inflow)
    U = P.prim_to_cons(w.W)
    dt = P.dt(U, w.cfl)
    nz, ny, nx = w.shape
    edge = min(32, nx, ny, nz)
    box = ((0, edge), (0, edge), (0, edge))
    for _ in range(args.warmup):
        P.step(w.psi, U, dt, box=box)
    t0 = time.perf_counter()
    for s in range(args.steps):
        z0 = (s * edge) % max(nz - edge + 1, 1)
        P.step(w.psi, U, dt, box=((0, edge), (0, edge), (z0, z0 + edge)))
    el = time.perf_counter() - t0
    rate = args.steps * edge ** 3 / el / 1e9
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {
        "impl": "reference", "metric": "cell_updates_per_s", "value": rate, "unit": "Gcell/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "precision": "fp64 CPU oracle", "sample": f"{edge}^3 window per step"},
        "cpu_baseline": {"value": rate, "unit": "Gcell/s", "cores": threads, "kind": "oracle",
                         "sample": f"one-step {edge}^3 windows of the {nx}x{ny}x{nz} grid"},
        "e2e": {"value": rate, "unit": "Gcell/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- GPU side

def run_ours(args):
    import torch
    from paper_1912_04855_b300 import cspht

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (no CPU fallback)")
    torch.cuda.set_device(local)
    dist = init_dist(world, True)
    dev = torch.device("cuda", local)
    w, desc = make_workload(args.workload)
    prec = args.precision
    path = cspht.PATH_PLAIN if args.path == "plain" else cspht.PATH_FAST
    N = w.cells
    stream = torch.cuda.Stream(device=dev)
    sim = cspht.Sim.from_workload(w, precision=prec, path=path)
    sim.set_stream(stream)
    W = np.ascontiguousarray(w.W)
    sim.set_primitive(W)
    # develop the flow a little so the timed steps see shocks, not a uniform state
    sim.advance(args.develop, w.cfl)
    sim.sync()
    # tile depth of the fused kernels, timed on this state (which it restores)
    zchunk = sim.autotune(steps=args.tune_steps, cfl=w.cfl) if args.tune_steps > 0 else None
    U0 = sim.get_state()

    def barrier():
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()

    # ---- value: K graph-replayed steps, state resident in HBM
    sim.advance(args.warmup, w.cfl)
    sim.sync()
    l0 = sim.launch_count()
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            ev0.record(stream)
            sim.advance(args.steps, w.cfl)
            ev1.record(stream)
        barrier()
    sim.sync()
    launches = sim.launch_count() - l0
    ms = ev0.elapsed_time(ev1)
    ms_max = max_over_ranks(dist, ms, dev)
    value = world * N * args.steps / (ms_max * 1e-3) / 1e9

    # ---- dominant kernel: per-kernel CUDA events over K steps
    sim.profile(True)
    sim.advance(args.steps, w.cfl)
    prof = sim.profile_read()
    sim.profile(False)
    total_ms = sum(v[0] for v in prof.values())
    top = max(prof.items(), key=lambda kv: kv[1][0])
    top_name, (top_ms, top_n) = top
    per_launch_ms = top_ms / top_n
    bytes_per_cell = WORDS_PER_CELL * (4 if prec == 32 else 8)
    peaks, peak_kind = load_peaks()
    step_ms = total_ms / args.steps
    flops_cell = FLOPS_PER_CELL.get(top_name)
    if prec == 32:
        peak_tf = FP32_LANES * 2 * peaks.get("sm_max_mhz", 2032.0) * 1e6 / 1e12
        peak_note = "FP32: 148 SMs x 128 lanes x 2 flops x %.0f MHz (%s max SM clock)" % (
            peaks.get("sm_max_mhz", 2032.0), peak_kind)
    else:
        peak_tf = FP64_TFLOPS_NOMINAL
        peak_note = "FP64: nominal dense rate of the part"
    achieved_tf = (flops_cell * N / (per_launch_ms * 1e-3) / 1e12) if flops_cell else None
    counts = recorded_counts(top_name, prec)
    traffic_cell, inst_cell = counts.get("dram_bytes_per_cell"), counts.get("thread_inst_per_cell")
    wave_cell = counts.get("smem_wavefronts_per_cell")
    # issue roofline: the kernels are bound by instruction issue (one warp
    # instruction per scheduler per clock: 148 SMs x 4 x 32 thread instructions)
    issue_peak = 148 * 4 * 32 * peaks.get("sm_max_mhz", 2032.0) * 1e6 / 1e12
    issue = None
    if inst_cell:
        got = inst_cell * N / (per_launch_ms * 1e-3) / 1e12
        issue = {"thread_inst_per_cell": inst_cell, "achieved": got, "peak": issue_peak,
                 "unit": "T thread-inst/s", "frac": got / issue_peak,
                 "peak_source": "148 SMs x 4 schedulers x 32 lanes x max SM clock; instructions per cell "
                                "from the committed ncu capture (profiles/dram_traffic.json)"}
    # shared-memory roofline: one 128-byte wavefront per SM per clock
    smem = None
    if wave_cell:
        smem_peak = 148 * peaks.get("sm_max_mhz", 2032.0) * 1e6 / 1e9
        got = wave_cell * N / (per_launch_ms * 1e-3) / 1e9
        smem = {"wavefronts_per_cell": wave_cell,
                "conflict_wavefronts_per_cell": counts.get("smem_conflict_wavefronts_per_cell"),
                "achieved": got, "peak": smem_peak, "unit": "G wavefronts/s", "frac": got / smem_peak,
                "peak_source": "148 SMs x one 128-byte shared-memory wavefront per clock x max SM clock; "
                               "wavefronts per cell from the committed ncu capture (profiles/dram_traffic.json)"}
    step_gbs = N * bytes_per_cell / (step_ms * 1e-3) / 1e9
    roofline = {
        "bound": "alu", "kernel": top_name,
        "achieved": achieved_tf, "peak": peak_tf, "unit": "TFLOP/s",
        "frac": (achieved_tf / peak_tf) if achieved_tf else None,
        "traffic": (traffic_cell * N) if traffic_cell else None,
        "peak_source": peak_note,
        "algorithmic_flops_per_launch": (flops_cell * N) if flops_cell else None,
        "kernel_ms_per_launch": per_launch_ms,
        "kernel_share": top_ms / total_ms,
        "kernels": {k: {"ms": v[0] / args.steps, "launches_per_step": v[1] / args.steps} for k, v in prof.items()},
        "hbm": {"algorithmic_bytes_per_step": N * bytes_per_cell, "achieved": step_gbs,
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": step_gbs / peaks["hbm_gbs"],
                "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json)" if peak_kind == "measured" else "fallback"},
        "issue": issue,
        "smem": smem,
        "traffic_source": "profiles/dram_traffic.json (ncu dram__bytes_read.sum + write.sum, scaled per cell)"
                          if traffic_cell else "null: kernels changed since the last ncu capture",
    }

    # ---- e2e: through the C ABI with pinned host buffers, copies inside the timing
    e2e = None
    if args.e2e_steps > 0:
        # host state in the handle's precision (the API takes float32 or float64)
        hin = torch.from_numpy(U0.astype(np.float32) if prec == 32 else U0).pin_memory()
        hout = torch.empty_like(hin).pin_memory()
        # FP32 host arrays go through the asynchronous calls: one step's download
        # overlaps the next upload (the bus is full duplex) and the upload the
        # previous step's kernels; FP64 arrays through the synchronous ones
        pipelined = prec == 32

        def e2e_step():
            if pipelined:
                sim.upload_async(hin)
                sim.advance(1, w.cfl)
                sim.download_async(hout)
            else:
                sim.set_state(hin)
                sim.step(w.cfl)
                sim.get_state(hout)

        e2e_step()
        sim.sync()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            e2e_step()
        sim.sync()  # every download has landed in host memory
        barrier()
        el = max_over_ranks(dist, time.perf_counter() - t0, dev)
        e2e = {"value": world * N * args.e2e_steps / el / 1e9, "unit": "Gcell/s",
               "h2d_bytes_per_step": int(hin.numel() * hin.element_size()),
               # the synchronous step also reads the 64-byte status word back
               "d2h_bytes_per_step": int(hout.numel() * hout.element_size() + (0 if pipelined else 64)),
               "host_dtype": str(hin.dtype).replace("torch.", ""),
               "pipelined": pipelined,
               "steps": args.e2e_steps}

    # ---- FP64 steps beside the FP32 one (the comparison the method asks for):
    # the unfused path and the fused kernels instantiated in FP64
    fp64 = {}
    if args.compare_fp64 and rank == 0:
        for name, path64 in (("plain", cspht.PATH_PLAIN), ("fused", cspht.PATH_FAST)):
            s64 = cspht.Sim.from_workload(w, precision=64, path=path64)
            s64.set_stream(stream)
            s64.set_state(U0)
            s64.advance(2, w.cfl)
            s64.sync()
            k = max(2, args.steps // 4)
            with torch.cuda.stream(stream):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                s64.advance(k, w.cfl)
                b.record(stream)
            s64.sync()
            m64 = a.elapsed_time(b)
            fp64[name] = {"value": N * k / (m64 * 1e-3) / 1e9, "unit": "Gcell/s", "steps": k,
                          "ms_per_step": m64 / k}
            s64.close()
    fp64_plain, fp64_fused = fp64.get("plain"), fp64.get("fused")

    status = sim.last_error()
    sim.close()

    # ---- serving: the C5 request stream through the continuous-batching loop:
    # per-request streams with priorities by size (the server's default), the
    # same without priorities, and one captured batch graph per tick
    serving = serving_batched = serving_streams = None
    if args.serve_requests > 0:
        from paper_1912_04855_b300 import serve
        from paper_1912_04855_b300 import workloads as wlm
        reqs = wlm.serving_stream(n_requests=args.serve_requests, seed=2024)
        out = {}
        for mode in ("priorities", "streams", "graph"):
            srv = serve.Server(budget_bytes=int(args.serve_budget_gb * 2**30), max_active=32, chunk=20,
                               batched=mode == "graph", priorities=mode == "priorities")
            srv.run(reqs)
            m = srv.metrics()
            m["workload"] = ("Poisson arrivals (mean 20 ms), edges {32,64,96,128,192}^3, half Riemann "
                             "problems, half potential wells, 200 steps each, FP32 fused path")
            m["aggregate_gcell_s_x_ranks"] = m["aggregate_gcell_s"] * world
            out[mode] = m
        serving, serving_streams, serving_batched = out["priorities"], out["streams"], out["graph"]

    if dist is not None:
        dist.barrier()
    if rank != 0:
        return 0

    cpu = None
    if args.cpu_baseline:
        rate, sample, threads = cpu_oracle_rate(w)
        cpu = {"value": rate / 1e9, "unit": "Gcell/s", "cores": threads, "kind": "oracle", "sample": sample}

    line = {
        "metric": "cell_updates_per_s",
        "value": value,
        "unit": "Gcell/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if prec == 32 else "f64",
        "data": "synthetic",
        "config": {"workload": desc, "grid": list(w.shape[::-1]), "cells": N, "precision": f"fp{prec}",
                   "path": args.path, "cfl": w.cfl, "develop_steps": args.develop,
                   "tile": {"xy": [32, 8], "z_planes": zchunk, "autotuned": zchunk is not None},
                   "l2": "inputs larger than L2 (state 5 x N x 4 B = %.0f MB per buffer)" % (5 * N * (4 if prec == 32 else 8) / 1e6),
                   "parallelism": f"replicas x{world}"},
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "roofline": roofline,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "fp64_plain": fp64_plain,
        "fp64_fused": fp64_fused,
        "fp32_over_fp64": (value / world / fp64_fused["value"]) if fp64_fused else None,
        "serving": serving,
        "serving_no_priorities": serving_streams,
        "serving_batch_graph": serving_batched,
        "status": status,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="well256")
    ap.add_argument("--precision", type=int, default=32, choices=[32, 64])
    ap.add_argument("--path", choices=["fast", "plain"], default="fast")
    ap.add_argument("--develop", type=int, default=20)
    ap.add_argument("--tune-steps", type=int, default=5,
                    help="steps timed per candidate tile depth before the run (0: keep the default depth)")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-fp64", dest="compare_fp64", action="store_false")
    ap.add_argument("--serve-requests", type=int, default=64)
    ap.add_argument("--serve-budget-gb", type=float, default=16.0)
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
