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

# more hardware work queues than the driver's default 8: the serving runs keep
# one stream per active request, and with 8 queues a request's setup and result
# kernels wait behind other streams' work sharing its queue (set before CUDA
# starts in this process)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FALLBACK = {"hbm_gbs": 6400.0, "sm_max_mhz": 2032.0}
# Algorithmic DRAM bytes per cell-update of one full step: read U (5 words)
# and psi (1), write U (5).
WORDS_PER_CELL = 11
FLOP_COUNT = os.path.join(ROOT, "profiles", "flop_count.json")
KERNEL_SOURCES = ["paper_1912_04855_b300/csrc/fast.cuh", "paper_1912_04855_b300/csrc/lagrange_pair.cuh",
                  "paper_1912_04855_b300/csrc/common.cuh", "paper_1912_04855_b300/csrc/tma.cuh"]


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


def flop_counts():
    """Algorithmic floating-point operations per cell of the fused kernels,
    counted by running the oracle's own code with a counting number type
    (profiles/flop_count.json, written by ``python oracle/opcount.py``): the
    Lagrangian kernel holds primitive recovery, predictor and corrector; the
    Euler kernel the slopes, face fluxes, update and the signal speed."""
    d = json.load(open(FLOP_COUNT))
    s = d["states"][d["bench_uses"]]
    return ({"lagrange": s["lagrange_kernel"]["flops"], "euler": s["euler_kernel"]["flops"]},
            f"profiles/flop_count.json (oracle code with a counting number type, state "
            f"'{d['bench_uses']}': {s['note']})")


def measure_alu_peaks(local):
    """Measured multiply-add throughput of this GPU from the library's own
    probe kernels (cspht_probe_fma), best of three, with the SM clocks sampled
    while they run."""
    from paper_1912_04855_b300 import cspht
    out = {}
    with ClockSampler(local) as clk:
        for name, kind, trips in (("fp32", cspht.PROBE_FP32, 200000), ("fp32x2", cspht.PROBE_FP32X2, 100000),
                                  ("fp64", cspht.PROBE_FP64, 4000)):
            out[name] = max(cspht.probe_fma(kind, trips)[0] for _ in range(3))
    out["clocks"] = clk.summary()
    return out


def measure_bus(nbytes, reps=8):
    """Measured host-device copy bandwidth for nbytes between page-locked
    host memory and the device (torch copies, CUDA events): upload alone,
    download alone, and both at once on two streams (GB/s per direction)."""
    import torch
    h_in = torch.empty(nbytes // 4, dtype=torch.float32).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    d_a = torch.empty(nbytes // 4, dtype=torch.float32, device="cuda")
    d_b = torch.empty_like(d_a)
    s_up, s_down = torch.cuda.Stream(), torch.cuda.Stream()

    def timed(up, down):
        best = float("inf")
        for _ in range(reps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            s_up.wait_event(e0)
            s_down.wait_event(e0)
            if up:
                with torch.cuda.stream(s_up):
                    d_a.copy_(h_in, non_blocking=True)
            if down:
                with torch.cuda.stream(s_down):
                    h_out.copy_(d_b, non_blocking=True)
            torch.cuda.current_stream().wait_stream(s_up)
            torch.cuda.current_stream().wait_stream(s_down)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) * 1e-3)
        return nbytes / best / 1e9

    out = {"h2d_gbs": timed(True, False), "d2h_gbs": timed(False, True),
           "both_gbs_per_direction": timed(True, True), "bytes": int(nbytes), "reps": reps,
           "source": "torch copies between page-locked host memory and the device, best of the reps"}
    del h_in, h_out, d_a, d_b
    torch.cuda.empty_cache()
    return out


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

def oracle_state(name):
    """The state the oracle is timed on: for the potential-well workloads the
    seeded developed-like flow on the same grid (workloads.developed_well), so
    that the windows see compressions, a shock surface and transverse
    velocities rather than the uniform initial inflow; else the workload's
    initial state."""
    from paper_1912_04855_b300 import workloads as wl
    w, desc = make_workload(name)
    if w.name == "potential_well":
        nz, ny, nx = w.shape
        w = wl.developed_well(n=nx, ny=ny, nz=nz)
    return w, desc


class OracleSampler:
    """Times the FP64 CPU oracle stepping the workload's grid in one-step
    windows of edge^3 cells that march through the grid (x fastest); each
    window's result is written back, so the state advances, and dt is taken
    from the whole grid at the start of every sweep (the oracle's CFL rule)."""

    def __init__(self, name, edge=64):
        from oracle import oracle as O
        O.build()
        self.O = O
        self.w, self.desc = oracle_state(name)
        w = self.w
        self.P = O.Problem(w.shape, w.h, w.gamma, w.bc, inflow=w.inflow)
        self.U = self.P.prim_to_cons(w.W)
        self.buf = self.U.copy()
        nz, ny, nx = w.shape
        self.edge = min(edge, nx, ny, nz)
        e = self.edge
        self.boxes = [((x, x + e), (y, y + e), (z, z + e)) for z in range(0, nz - e + 1, e)
                      for y in range(0, ny - e + 1, e) for x in range(0, nx - e + 1, e)]
        self.k = 0
        self.dt = None

    def window(self):
        """One window step (and the sweep's dt when a sweep starts)."""
        if self.k % len(self.boxes) == 0:
            self.dt = self.P.dt(self.U, self.w.cfl)
        box = self.boxes[self.k % len(self.boxes)]
        self.k += 1
        self.P.step(self.w.psi, self.U, self.dt, box=box, out=self.buf)
        sl = (slice(None), slice(*box[2]), slice(*box[1]), slice(*box[0]))
        self.U[sl] = self.buf[sl]
        return self.edge ** 3

    def rate(self, budget_s=None, windows=None, threads=None):
        """Cell-updates per second over `windows` windows or `budget_s`
        seconds, with `threads` OpenMP threads (None: all cores)."""
        O = self.O
        before = O.max_threads()
        if threads is not None:
            O.set_threads(threads)
        used = O.max_threads()
        cells, n, t0 = 0, 0, time.perf_counter()
        try:
            while (windows is None or n < windows) and (budget_s is None or time.perf_counter() - t0 < budget_s):
                cells += self.window()
                n += 1
        finally:
            O.set_threads(before)
        el = time.perf_counter() - t0
        return cells / el, n, el, used


def cpu_oracle_rate(name, budget_s=15.0, one_thread_windows=2):
    """The FP64 oracle as it stands on the machine's host cores: all cores for
    about budget_s seconds, then one thread (its plain definition) on a few
    windows.  Returns the cpu_baseline record."""
    S = OracleSampler(name)
    S.window()  # warm-up: first touch of the arrays
    rate, n, el, threads = S.rate(budget_s=budget_s)
    r1, n1, el1, _ = S.rate(windows=one_thread_windows, threads=1)
    nz, ny, nx = S.w.shape
    return {"value": rate / 1e9, "unit": "Gcell/s", "cores": threads, "kind": "oracle",
            "sample": f"{n} one-step {S.edge}^3 windows ({el:.1f} s) marching through the {nx}x{ny}x{nz} "
                      f"grid from the developed-like state, each written back so the state advances",
            "one_thread": {"value": r1 / 1e9, "unit": "Gcell/s", "cores": 1,
                           "sample": f"{n1} more windows of the same sweep ({el1:.1f} s)"}}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    S = OracleSampler(args.workload)
    for _ in range(args.warmup):
        S.window()
    rate, n, el, threads = S.rate(windows=args.steps)
    r1, n1, el1, _ = S.rate(windows=2, threads=1)
    nz, ny, nx = S.w.shape
    value = rate / 1e9
    line = {
        "impl": "reference", "metric": "cell_updates_per_s", "value": value, "unit": "Gcell/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el / n * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": S.desc, "precision": "fp64 CPU oracle",
                   "sample": f"one {S.edge}^3 window of the grid per step"},
        "cpu_baseline": {"value": value, "unit": "Gcell/s", "cores": threads, "kind": "oracle",
                         "sample": f"{n} one-step {S.edge}^3 windows ({el:.1f} s) marching through the "
                                   f"{nx}x{ny}x{nz} grid from the developed-like state, each written back",
                         "one_thread": {"value": r1 / 1e9, "unit": "Gcell/s", "cores": 1,
                                        "sample": f"{n1} more windows ({el1:.1f} s)"}},
        "e2e": {"value": value, "unit": "Gcell/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
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
    flops, flops_source = flop_counts()
    flops_cell = flops.get(top_name)
    alu = measure_alu_peaks(local)
    if prec == 32:
        # the FP32 FMA peak of the part: the faster of the scalar and the packed
        # two-lane instruction (the kernels use the scalar one)
        peak_tf = max(alu["fp32"], alu["fp32x2"])
        peak_note = ("measured: the library's FMA-throughput probe in this run (cspht_probe_fma), "
                     "FP32 scalar %.1f, packed f32x2 %.1f TFLOP/s" % (alu["fp32"], alu["fp32x2"]))
    else:
        peak_tf = alu["fp64"]
        peak_note = "measured: the library's FMA-throughput probe in this run (cspht_probe_fma), FP64"
    achieved_tf = (flops_cell * N / (per_launch_ms * 1e-3) / 1e12) if flops_cell else None
    counts = recorded_counts(top_name, prec)
    traffic_cell, inst_cell = counts.get("dram_bytes_per_cell"), counts.get("thread_inst_per_cell")
    wave_cell = counts.get("smem_wavefronts_per_cell")
    # issue roofline: the kernels are bound by instruction issue.  The scalar
    # FP32 probe issues one FFMA (one thread instruction, 2 flops) per lane per
    # slot, so its rate / 2 is the measured thread-instruction issue peak
    issue_peak = alu["fp32"] / 2.0
    issue = None
    if inst_cell:
        got = inst_cell * N / (per_launch_ms * 1e-3) / 1e12
        issue = {"thread_inst_per_cell": inst_cell, "achieved": got, "peak": issue_peak,
                 "unit": "T thread-inst/s", "frac": got / issue_peak,
                 "peak_source": "measured: scalar FP32 FMA probe rate / 2 (one instruction per FMA); "
                                "instructions per cell from the committed ncu capture "
                                "(profiles/dram_traffic.json)"}
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
        "alu_probe": alu,
        "algorithmic_flops_per_cell": flops_cell,
        "algorithmic_flops_source": flops_source,
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
        # the bus's own rate for the same transfers: the e2e step's ceiling
        bus = measure_bus(int(hin.numel() * hin.element_size()))
        moved = 2 * hin.numel() * hin.element_size() * args.e2e_steps / el / 1e9  # GB/s, both directions
        bus["e2e_achieved_gbs_both_directions"] = moved
        bus["frac"] = moved / (2 * bus["both_gbs_per_direction"])
        e2e = {"value": world * N * args.e2e_steps / el / 1e9, "unit": "Gcell/s",
               "bus": bus,
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
    # same without priorities, every active request in one launch per step
    # kernel (lockstep), and the adaptive mode that takes the lockstep batch
    # while requests wait and per-request streams otherwise; then a sweep of
    # offered load below capacity
    serving = serving_batched = serving_streams = serving_adaptive = None
    if args.serve_requests > 0:
        from paper_1912_04855_b300 import serve
        from paper_1912_04855_b300 import workloads as wlm
        reqs = wlm.serving_stream(n_requests=args.serve_requests, seed=2024)
        # the requests' payloads (initial state and potential) stand for the
        # data the clients send with them, in page-locked transfer buffers:
        # built before the replays, once (the load sweep's streams draw the
        # same requests at other arrival times)
        payloads = {r["id"]: serve.pinned(wlm.request_workload(r)) for r in reqs}
        out = {}
        for mode in ("priorities", "streams", "graph", "adaptive"):
            srv = serve.Server(budget_bytes=int(args.serve_budget_gb * 2**30), max_active=32, chunk=20,
                               batched=mode == "graph", priorities=mode != "streams", adaptive=mode == "adaptive")
            srv.run(reqs, payloads=payloads)
            m = srv.metrics()
            m["workload"] = ("Poisson arrivals (mean 20 ms), edges {32,64,96,128,192}^3, half Riemann "
                             "problems, half potential wells, 200 steps each, FP32 fused path; payloads "
                             "(initial states) built in page-locked host memory before the replay, "
                             "uploaded at admission")
            m["aggregate_gcell_s_x_ranks"] = m["aggregate_gcell_s"] * world
            out[mode] = m
        serving, serving_streams, serving_batched = out["priorities"], out["streams"], out["graph"]
        serving_adaptive = out["adaptive"]
        # latency at sustained load: the same request mix with the arrival rate
        # scaled to a fraction of the capacity measured above (the saturated
        # stream's aggregate rate), so that the queue stays bounded
        # capacity: the best saturated rate of the modes above
        cap = max(m["aggregate_gcell_s"] for m in out.values() if "adaptive" not in m["mode"])
        mean_work = float(np.mean([r["edge"] ** 3 * r["steps"] for r in reqs]))
        sweep = []
        for frac in args.serve_load:
            gap = mean_work / (frac * cap * 1e9)
            rq = wlm.serving_stream(n_requests=args.serve_requests, seed=2024, mean_gap_s=gap)
            assert all({k: v for k, v in a.items() if k != "arrival"} == {k: v for k, v in b.items() if k != "arrival"}
                       for a, b in zip(rq, reqs)), "the sweep's requests must be the same as the payloads'"

            for mode in ("priorities", "graph", "adaptive"):
                srv = serve.Server(budget_bytes=int(args.serve_budget_gb * 2**30), max_active=32, chunk=20,
                                   batched=mode == "graph", priorities=True, adaptive=mode == "adaptive")
                srv.run(rq, payloads=payloads)
                m = srv.metrics()
                sweep.append({"mode": m["mode"], "target_fraction_of_capacity": frac, "mean_gap_ms": gap * 1e3,
                              "offered_gcell_s": m["offered_gcell_s"],
                              "utilisation": m["offered_gcell_s"] / cap,
                              "aggregate_gcell_s": m["aggregate_gcell_s"],
                              "p50_ms": m["p50_ms"], "p99_ms": m["p99_ms"], "mean_ms": m["mean_ms"],
                              "max_waiting": m["max_waiting"], "makespan_s": m["makespan_s"]})
        serving["capacity_gcell_s"] = cap
        serving["load_sweep"] = sweep

    if dist is not None:
        dist.barrier()
    if rank != 0:
        return 0

    cpu = cpu_oracle_rate(args.workload) if args.cpu_baseline else None

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
        "serving_adaptive": serving_adaptive,
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
    ap.add_argument("--serve-load", type=float, nargs="*", default=[0.5, 0.75, 0.9],
                    help="offered load of the latency sweep, as fractions of the measured capacity")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
