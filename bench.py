#!/usr/bin/env python
"""Throughput benchmark of multilevel summation for r^-6 dispersion on GB300.

One step = one full ``mls6_eval`` (bin, local pair part, anterpolation,
restriction, level stencils, coarsest level, prolongation, interpolation,
energy/virial reduction) of the 65,536-atom liquid/vacuum slab (40x40x51.2
slab at rho=0.8 in a periodic 40x40x120 box, C6 in [0.8,1.2], a=3, h=1.25,
4 levels, FP32 with FP64 energy/virial).  Metric: atom-evals/s (atoms whose
energy contribution and force one evaluation produces, per second).

  --impl ours        (default) the CUDA library through its C ABI
  --impl reference   the FP64 CPU oracle on the host cores (bounded sample)

Under torchrun each rank evaluates an independent replica (different seed)
on its own GPU; value = atoms of all ranks / max-over-ranks time.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

FP32_LANES_PER_SM = 128
FP64_LANES_PER_SM = 2   # GB300 FP64 issue rate per SM per clock (FMA lanes)
SMS = 152
# Floating-point operations counted per unit of algorithmic work (fixed
# tallies, see the design notes):
FLOP_PAIR = 42          # one pair inside the cutoff: energy + force
FLOP_PAIR_VIR = 12      # ... plus the six virial products
FLOP_TAP = 2            # one stencil tap (multiply-add) per node
FLOP_TAP_VIR = 12       # ... plus six virial multiply-adds


# DRAM bytes (read + write) per launch of a kernel, from one ncu capture of
# it on the named workload and precision (virial on); a kernel changed since
# its capture has no entry and reports null.
TRAFFIC = {("slab65536", "fp32", "pair"): 1.190144e6,
           ("cube1m", "fp32", "stencil"): 6.509568e6,
           ("cube1m", "fp32", "pair"): 1.8241792e7,
           ("cube1m", "mixed", "pair"): 1.8241792e7}

# arithmetic of each precision mode (pair/grid transfers; level stencils)
DTYPE = {"fp64": "f64", "fp32": "f32", "mixed": "f32+bf16x3"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="slab65536")
    ap.add_argument("--precision", choices=["fp32", "fp64", "mixed"], default="fp32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-virial", action="store_true",
                    help="evaluate energy and forces only (no virial arithmetic)")
    ap.add_argument("--no-tune", action="store_true",
                    help="batched workloads: keep the seeded configuration")
    ap.add_argument("--dwell", type=float, default=1.5,
                    help="seconds of untimed back-to-back evaluations before timing")
    return ap.parse_args()


# ---------------------------------------------------------------- clocks

_REASON_BITS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap",
                0x8: "hw_slowdown", 0x10: "sync_boost", 0x20: "sw_thermal_slowdown",
                0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown",
                0x100: "display_clock_setting"}


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons (read only)."""

    FIELDS = ("clocks.sm,clocks.max.sm,utilization.gpu,power.draw,clocks_event_reasons.active")

    def __init__(self, gpu_id):
        self.samples = []
        self.err = None
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(gpu_id)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception as e:  # nvidia-smi missing
            self.p = None
            self.err = repr(e)
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.p.stdout:
            parts = [s.strip() for s in line.split(",")]
            if len(parts) < 5:
                continue
            try:
                sm, smax, util = float(parts[0]), float(parts[1]), float(parts[2])
                reasons = int(parts[4], 16)
            except ValueError:
                continue
            self.samples.append((time.time(), sm, smax, util, reasons))

    def stop(self):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self, t0, t1):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "note": self.err}
        win = [s for s in self.samples if t0 <= s[0] <= t1]
        load = [s for s in win if s[3] > 0] or win
        if not load:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        reasons = set()
        for s in load:
            for bit, name in _REASON_BITS.items():
                if s[4] & bit and name != "gpu_idle":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(s[1] for s in load),
                "sm_max_mhz": max(s[2] for s in load),
                "reasons": sorted(reasons), "samples": len(load)}


def gpu_smi_id(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        return vis.split(",")[dev] if vis else str(dev)


# ---------------------------------------------------------- distributed

def dist_setup(torch):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def reduce_max(torch, value, world, device):
    if world == 1:
        return value
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(torch, local_total_ms, atoms_per_rank, steps, world, device):
    """Whole-job atom-evals/s: atoms of all ranks over the slowest rank's
    time (max over ranks of the summed step times)."""
    total_ms = reduce_max(torch, local_total_ms, world, device)
    return world * atoms_per_rank * steps / (total_ms / 1e3), total_ms


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


# ------------------------------------------------------------- workload

def workload_arrays(name, rank, precision):
    import numpy as np

    from paper_1308_4005_gb300 import inputs as I

    w = I.workload(name)
    if rank:
        import dataclasses

        w = dataclasses.replace(w, seed=w.seed + 1000 * rank)
    x, c = I.generate(w)
    dt = np.float64 if precision == "fp64" else np.float32
    return w, x.astype(dt), c.astype(dt)


def count_pairs(x, box, a):
    """Ordered pairs (i, j) with periodic distance < a (the pair kernel's
    algorithmic work)."""
    import numpy as np
    from scipy.spatial import cKDTree

    xx = np.mod(np.asarray(x, dtype=np.float64), box)
    p = cKDTree(xx, boxsize=box).query_pairs(a, output_type="ndarray")
    return 2 * int(p.shape[0])


# ------------------------------------------------------------ CPU oracle

def _oracle_parts(O, w, xd, cd, S, rng):
    """Seconds for the oracle's grid part (all atoms) and for its local part
    over S random atoms."""
    import numpy as np

    n = O.grid_dims(w.box, w.h, w.levels)
    t0 = time.perf_counter()
    O.evaluate_sample(w.box, w.a, n, w.levels, xd, cd, np.zeros(0, np.int64))
    t_grid = time.perf_counter() - t0
    idx = rng.choice(w.N, S, replace=False)
    t0 = time.perf_counter()
    O.local(w.box, w.a, xd, cd, idx)
    t_loc = time.perf_counter() - t0
    return t_grid, t_loc


def oracle_baseline(w, x, c, budget_s=15.0):
    """Time the FP64 oracle on the host cores on a bounded sample: the whole
    grid part (anterpolation .. interpolation, all atoms) once, and the local
    part for a random sample of S atoms; the full-evaluation time is
    t_grid + t_local(S) * N / S."""
    import numpy as np

    from oracle import oracle as O

    O.build()
    O.set_threads(os.cpu_count() or 1)
    xd, cd = np.asarray(x, np.float64), np.asarray(c, np.float64)
    rng = np.random.default_rng(7)
    S = min(w.N, 256)
    t_grid, t_loc = _oracle_parts(O, w, xd, cd, S, rng)
    S2 = int(min(w.N, max(S, S * max(budget_s - t_grid, 1.0) / max(t_loc, 1e-6))))
    t_grid, t_loc2 = _oracle_parts(O, w, xd, cd, S2, rng)
    t_full = t_grid + t_loc2 * w.N / S2
    return {"value": w.N / t_full, "unit": "atom-evals/s", "cores": O.threads(),
            "kind": "oracle",
            "sample": (f"FP64 oracle, {w.name}: grid part for all {w.N} atoms "
                       f"({t_grid:.2f} s) + local part for {S2} random atoms ({t_loc2:.2f} s), "
                       f"full evaluation extrapolated to {t_full:.1f} s")}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np

    from oracle import oracle as O

    w, x, c = workload_arrays(args.workload, 0, args.precision)
    O.build()
    O.set_threads(os.cpu_count() or 1)
    xd, cd = np.asarray(x, np.float64), np.asarray(c, np.float64)
    rng = np.random.default_rng(11)
    S = min(w.N, max(1, w.N // 32))
    for _ in range(args.warmup):
        _oracle_parts(O, w, xd, cd, S, rng)
    full, tg = [], []
    for _ in range(args.steps):
        t_grid, t_loc = _oracle_parts(O, w, xd, cd, S, rng)
        tg.append(t_grid)
        full.append(t_grid + t_loc * w.N / S)
    ms = 1e3 * statistics.mean(full)
    value = w.N / (ms / 1e3)
    line = {"metric": "atom-evals/s", "value": value, "unit": "atom-evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": config_of(w, args, world),
            "cpu_baseline": {"value": value, "unit": "atom-evals/s", "cores": O.threads(),
                             "kind": "oracle",
                             "sample": (f"each step: FP64 oracle grid part for all {w.N} atoms "
                                        f"(mean {statistics.mean(tg):.2f} s) + local part for "
                                        f"{S} random atoms, extrapolated to all {w.N}")},
            "e2e": {"value": value, "unit": "atom-evals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_reference_batch(args):
    """Oracle arm of the batched workload: each step times the FP64 oracle on
    one replica (cycling through the replicas by size rank), grid part in full
    and local part on a 1/32 sample, and reports atoms per second."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import dataclasses

    import numpy as np

    from oracle import oracle as O
    from paper_1308_4005_gb300 import inputs as I

    nrep = 256 if args.workload == "batch256" else 16
    ws = I.batch_workloads(B=nrep)
    O.build()
    O.set_threads(os.cpu_count() or 1)
    rng = np.random.default_rng(11)
    order = sorted(range(nrep), key=lambda r: ws[r].N)
    picks = [order[(k * nrep) // max(1, args.steps + args.warmup)]
             for k in range(args.steps + args.warmup)]
    atoms = secs = 0.0
    for k, r in enumerate(picks):
        w = ws[r]
        w = dataclasses.replace(w, levels=I_auto_levels(w))
        x, c = I.generate(w)
        S = min(w.N, max(1, w.N // 32))
        t_grid, t_loc = _oracle_parts(O, w, x, c, S, rng)
        if k >= args.warmup:
            atoms += w.N
            secs += t_grid + t_loc * w.N / S
    value = atoms / secs
    line = {"metric": "atom-evals/s", "value": value, "unit": "atom-evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "replicas": nrep, "a": ws[0].a,
                       "h": ws[0].h, "levels": "auto per replica"},
            "cpu_baseline": {"value": value, "unit": "atom-evals/s", "cores": O.threads(),
                             "kind": "oracle",
                             "sample": (f"each step: one replica (spread over the size range), "
                                        "FP64 oracle grid part in full + local part for 1/32 "
                                        "of its atoms, extrapolated")},
            "e2e": {"value": value, "unit": "atom-evals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def I_auto_levels(w):
    from paper_1308_4005_gb300 import mls6

    return mls6.mls6_auto_levels(w.box, w.h)


def config_of(w, args, world):
    return {"workload": w.name, "N_per_gpu": w.N, "box": list(w.box), "a": w.a, "h": w.h,
            "levels": w.levels, "order": 3, "precision": args.precision,
            "virial": not getattr(args, "no_virial", False),
            "parallelism": f"replicas{world}" if world > 1 else "single",
            "l2": "flushed between timed steps (256 MiB write)"}


# ------------------------------------------------------------------ ours

def run_ours(args):
    import numpy as np
    import torch

    from paper_1308_4005_gb300 import build as B
    from paper_1308_4005_gb300 import mls6

    world, rank, local = dist_setup(torch)
    assert torch.cuda.is_available(), "bench.py --impl ours needs a GPU"
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.build()
    mls6.load()
    w, x, c = workload_arrays(args.workload, rank, args.precision)
    dt = torch.float64 if args.precision == "fp64" else torch.float32
    esz = 8 if args.precision == "fp64" else 4
    N = w.N
    stream = torch.cuda.Stream(device=dev)
    plan = mls6.Plan(w.box, N, w.a, w.h, w.levels, precision=args.precision,
                     stream=stream.cuda_stream)
    info = plan.info()
    pos_h = torch.tensor(np.c_[x, c], dtype=dt).pin_memory()
    pos = torch.empty((N, 4), dtype=dt, device=dev)
    F = torch.empty((N, 3), dtype=dt, device=dev)
    F_h = torch.empty((N, 3), dtype=dt).pin_memory()
    out = torch.zeros(8, dtype=torch.float64, device=dev)
    out_h = torch.zeros(8, dtype=torch.float64).pin_memory()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    with torch.cuda.stream(stream):
        pos.copy_(pos_h, non_blocking=True)
    stream.synchronize()

    vir_ptr = 0 if args.no_virial else out.data_ptr() + 8

    def step():
        rc = mls6.mls6_eval(plan.handle, pos.data_ptr(), 0, F.data_ptr(), out.data_ptr(),
                            vir_ptr)
        if rc:
            raise mls6.MLS6Error(rc, "mls6_eval")

    sampler = ClockSampler(gpu_smi_id(torch, local))
    t_dwell0 = time.time()
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.fill_(1)
            step()
        stream.synchronize()
        t_end = time.time() + args.dwell
        while time.time() < t_end:
            for _ in range(50):
                step()
            stream.synchronize()
    rc = mls6.mls6_last_error(plan.handle)
    if rc:
        raise mls6.MLS6Error(rc, "warmup")

    # ------------------------------------------------ timed region (device)
    # Production path: captured graph, pair sum concurrent with the grid
    # chain, no per-stage events.  L2 flushed before every step.
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize(dev)
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    _, launches_per_step = mls6.mls6_stage_times(plan.handle)
    launches = launches_per_step * args.steps
    value, total_ms = job_throughput(torch, sum(a.elapsed_time(b) for a, b in ev), N,
                                     args.steps, world, dev)
    ms_per_step = total_ms / args.steps
    E_dev = float(out[0].item())

    # ------------------------------------- per-kernel times (serialised pass)
    # Same steps with per-stage CUDA events on the launching stream; stages
    # run one after another so each event pair times one stage alone.
    mls6.mls6_profile(plan.handle, True)
    stage_acc = {}
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            step()
            st, _ = mls6.mls6_stage_times(plan.handle)  # waits for this step
            for name, ms in st.items():
                stage_acc[name] = stage_acc.get(name, 0.0) + ms
    mls6.mls6_profile(plan.handle, False)
    stage_ms = {k: v / args.steps for k, v in stage_acc.items()}

    # --------------------------------------------- end-to-end (host buffers)
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize(dev)
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            ev2[k][0].record(stream)
            pos.copy_(pos_h, non_blocking=True)
            step()
            F_h.copy_(F, non_blocking=True)
            out_h.copy_(out, non_blocking=True)
            ev2[k][1].record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    e2e_value, _ = job_throughput(torch, sum(a.elapsed_time(b) for a, b in ev2), N, args.steps,
                                  world, dev)
    t_e2e1 = time.time()
    sampler.stop()
    clocks = sampler.summary(t_dwell0, t_e2e1)
    clocks["window"] = "warm-up dwell + timed steps (the timed region alone is shorter than the sampling period)"

    # ------------------------------------------------------------- roofline
    n_pairs = count_pairs(x, np.array(w.box), w.a)
    lv = info["n_grid"]
    nodes_lt = sum(n[0] * n[1] * n[2] for n in lv[:-1])
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    fp32_peak = SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12  # TFLOP/s
    fp_pair = FLOP_PAIR + (0 if args.no_virial else FLOP_PAIR_VIR)
    fp_tap = FLOP_TAP + (0 if args.no_virial else FLOP_TAP_VIR)
    work = {
        "pair": ("alu", n_pairs * fp_pair / 1e12, "TFLOP/s",
                 f"{n_pairs} ordered pairs inside a x {fp_pair} flop"),
        "stencil": ("alu", nodes_lt * info["ntaps"] * fp_tap / 1e12,
                    "TFLOP/s", f"{nodes_lt} nodes on levels < l x {info['ntaps']} taps x "
                               f"{fp_tap} flop"),
        "interpolate": ("hbm", (N * (16 + 4 + esz + 3 * esz + 3 * esz) + lv[0][0] * lv[0][1] *
                                lv[0][2] * esz) / 1e9, "GB/s",
                        "per atom: sorted record, index, e0, local force in, force out; grid once"),
        "anterpolate": ("hbm", (N * 16 + lv[0][0] * lv[0][1] * lv[0][2] * esz) / 1e9, "GB/s",
                        "per atom: sorted record; finest grid written once"),
        "bin": ("hbm", N * (16 + 16 + 4 + 4 + 16 + 4 + 16 + 4) / 1e9, "GB/s",
                "read input, write wrapped record + cell id, scatter read/write, sort"),
    }
    dom = max(stage_ms, key=lambda k: stage_ms[k])
    roof = None
    if dom in work:
        bound, amount, unit, note = work[dom]
        ach = amount / (stage_ms[dom] / 1e3)
        if dom == "stencil" and info.get("stencil_kind") == 2:
            bound, peak = "tensor", tensor_peak()
            peak_note = ("MEASURED_PEAKS.json bf16_tflops (of measured; cuBLAS bf16 burst): the "
                         "stencil runs as BF16 mma with split operands")
        if bound == "tensor":
            pass
        elif bound == "alu":
            peak, peak_note = fp32_peak, (f"FP32 FMA peak derived: {SMS} SMs x "
                                          f"{FP32_LANES_PER_SM} lanes x 2 flop x {sm_mhz:.0f} MHz "
                                          "(median sampled SM clock)")
        else:
            peak, peak_note = hbm_peak(), "MEASURED_PEAKS.json hbm_gbs (of measured)"
        traffic = None if args.no_virial else TRAFFIC.get((w.name, args.precision, dom))
        roof = {"kernel": dom, "bound": bound, "achieved": ach, "peak": peak, "unit": unit,
                "frac": ach / peak, "traffic": traffic, "work": note, "peak_source": peak_note,
                "avg_launch_ms": stage_ms[dom],
                "timing": ("CUDA events on the launching stream around the stage, averaged over "
                           "a serialised pass of the same steps right after the timed region")}
    line = {"metric": "atom-evals/s", "value": value, "unit": "atom-evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": config_of(w, args, world),
            "e2e": {"value": e2e_value, "unit": "atom-evals/s",
                    "h2d_bytes_per_step": int(pos_h.numel() * pos_h.element_size()),
                    "d2h_bytes_per_step": int(F_h.numel() * F_h.element_size() + 8 * 8)},
            "gpu_launches": int(launches),
            "roofline": roof, "stages_ms": stage_ms, "clocks": clocks,
            "energy": E_dev}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_baseline(w, x, c)
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


# ------------------------------------------------------- batched replicas

def run_batch(args):
    """Batched replicas (256 uneven systems, about 5.0M atoms): one graph
    launch per step over all replicas; value = atoms of all replicas per
    second.  Autotuned (branch count, kernel shapes) before the timed
    region unless --no-tune."""
    import numpy as np
    import torch

    from paper_1308_4005_gb300 import build as B
    from paper_1308_4005_gb300 import inputs as I
    from paper_1308_4005_gb300 import mls6

    world, rank, local = dist_setup(torch)
    assert torch.cuda.is_available(), "bench.py --impl ours needs a GPU"
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.build()
    mls6.load()
    nrep = 256 if args.workload == "batch256" else 16
    ws = I.batch_workloads(B=nrep, seed=I.SEED_BASE + 3 + 1000 * rank)
    t0 = time.time()
    x, c, off = I.generate_batch(ws, processes=min(16, os.cpu_count() or 1))
    t_gen = time.time() - t0
    dt = torch.float64 if args.precision == "fp64" else torch.float32
    Ntot = int(off[-1])
    stream = torch.cuda.Stream(device=dev)
    t0 = time.time()
    bt = mls6.Batch([w.box for w in ws], [w.N for w in ws], ws[0].a, ws[0].h, 0,
                    precision=args.precision)
    t_plan = time.time() - t0
    mls6.mls6_batch_set_stream(bt.handle, stream.cuda_stream)
    pos_h = torch.tensor(np.c_[x, c], dtype=dt).pin_memory()
    pos = torch.empty((Ntot, 4), dtype=dt, device=dev)
    F = torch.empty((Ntot, 3), dtype=dt, device=dev)
    F_h = torch.empty((Ntot, 3), dtype=dt).pin_memory()
    E = torch.zeros(nrep, dtype=torch.float64, device=dev)
    W = torch.zeros((nrep, 6), dtype=torch.float64, device=dev)
    E_h = torch.zeros(nrep, dtype=torch.float64).pin_memory()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    with torch.cuda.stream(stream):
        pos.copy_(pos_h, non_blocking=True)
    stream.synchronize()
    seed_info = bt.info()
    t_tune = None
    if not args.no_tune:
        t0 = time.time()
        with torch.cuda.stream(stream):
            bt.tune(pos, reps=3)
        t_tune = time.time() - t0
    info = bt.info()

    def step():
        rc = mls6.mls6_batch_eval(bt.handle, pos.data_ptr(), 0, F.data_ptr(), E.data_ptr(),
                                  W.data_ptr())
        if rc:
            raise mls6.MLS6Error(rc, "mls6_batch_eval")

    sampler = ClockSampler(gpu_smi_id(torch, local))
    t_dwell0 = time.time()
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.fill_(1)
            step()
        stream.synchronize()
    info = bt.info()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize(dev)
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    value, total_ms = job_throughput(torch, sum(a.elapsed_time(b) for a, b in ev), Ntot,
                                     args.steps, world, dev)
    ms_per_step = total_ms / args.steps
    # end to end: positions in from pinned host memory, forces and energies out
    ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize(dev)
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            ev2[k][0].record(stream)
            pos.copy_(pos_h, non_blocking=True)
            step()
            F_h.copy_(F, non_blocking=True)
            E_h.copy_(E, non_blocking=True)
            ev2[k][1].record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    e2e_value, _ = job_throughput(torch, sum(a.elapsed_time(b) for a, b in ev2), Ntot,
                                  args.steps, world, dev)
    sampler.stop()
    clocks = sampler.summary(t_dwell0, time.time())

    # per-replica stage times: each replica's plan alone, stages serialised
    stage_acc = {}
    work_pair = work_sten = 0.0
    esz = 8 if args.precision == "fp64" else 4
    for r, w in enumerate(ws):
        ph = mls6.mls6_batch_replica(bt.handle, r)
        pinfo = mls6.mls6_plan_info(ph)
        mls6.mls6_profile(ph, True)
        sl = slice(int(off[r]), int(off[r + 1]))
        with torch.cuda.stream(stream):
            mls6.mls6_set_stream(ph, stream.cuda_stream)
            for _ in range(2):
                rc = mls6.mls6_eval(ph, pos[sl].data_ptr(), 0, F[sl].data_ptr(), 0,
                                    W[r].data_ptr())
                if rc:
                    raise mls6.MLS6Error(rc, "replica eval")
            st, _ = mls6.mls6_stage_times(ph)
        mls6.mls6_profile(ph, False)
        for name, ms in st.items():
            stage_acc[name] = stage_acc.get(name, 0.0) + ms
        lv = pinfo["n_grid"]
        work_pair += count_pairs(x[sl], np.array(w.box), w.a) * (FLOP_PAIR + FLOP_PAIR_VIR)
        work_sten += sum(n[0] * n[1] * n[2] for n in lv[:-1]) * pinfo["ntaps"] * \
            (FLOP_TAP + FLOP_TAP_VIR)
    dom = max(stage_acc, key=lambda k: stage_acc[k])
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    fp32_peak = SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    roof = None
    if dom in ("pair", "stencil"):
        amount = (work_pair if dom == "pair" else work_sten) / 1e12
        ach = amount / (stage_acc[dom] / 1e3)
        roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": fp32_peak,
                "unit": "TFLOP/s", "frac": ach / fp32_peak, "traffic": None,
                "work": f"sum over the {nrep} replicas of the {dom} kernel's algorithmic flops",
                "peak_source": (f"FP32 FMA peak derived: {SMS} SMs x {FP32_LANES_PER_SM} lanes "
                                f"x 2 flop x {sm_mhz:.0f} MHz (median sampled SM clock)"),
                "avg_launch_ms": stage_acc[dom] / nrep,
                "timing": ("CUDA events around the stage, each replica's plan evaluated alone "
                           "with serialised stages after the timed region")}
    line = {"metric": "atom-evals/s", "value": value, "unit": "atom-evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": {"workload": args.workload, "replicas": nrep, "atoms_per_gpu": Ntot,
                       "N_min": int(min(w.N for w in ws)), "N_max": int(max(w.N for w in ws)),
                       "a": ws[0].a, "h": ws[0].h, "levels": "auto per replica",
                       "precision": args.precision,
                       "parallelism": f"replicas{world}" if world > 1 else "single",
                       "branches": info["branches"], "seed_branches": seed_info["branches"],
                       "autotune_s": t_tune, "plan_s": t_plan, "generate_s": t_gen,
                       "l2": "flushed between timed steps (256 MiB write)"},
            "e2e": {"value": e2e_value, "unit": "atom-evals/s",
                    "h2d_bytes_per_step": int(pos_h.numel() * pos_h.element_size()),
                    "d2h_bytes_per_step": int(F_h.numel() * F_h.element_size() + 8 * nrep)},
            "gpu_launches": int(info["launches"]) * args.steps,
            "roofline": roof,
            "stages_ms_sum_over_replicas": stage_acc, "clocks": clocks}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        mid = sorted(range(nrep), key=lambda r: ws[r].N)[nrep // 2]
        sl = slice(int(off[mid]), int(off[mid + 1]))
        wm = ws[mid]
        import dataclasses

        wm = dataclasses.replace(wm, levels=info["levels"][mid])
        cb = oracle_baseline(wm, x[sl], c[sl])
        cb["sample"] = f"median-size replica {mid} (N={wm.N}): " + cb["sample"]
        line["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(line), flush=True)
    bt.close()
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


# ------------------------------------------- throughput at equal accuracy

def _timed_evals(fn, steps, warmup, stream):
    import torch

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            fn()
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def run_accuracy(args):
    """Force error against a converged reference and throughput of the plain
    FP32, mixed-precision and learned forms over a cutoff sweep on a held-out
    slab (proportions of the 4,194,304-atom slab), and the throughput of
    each form interpolated (log-log) at eps_F = 1e-4."""
    import numpy as np
    import torch

    from paper_1308_4005_gb300 import build as B
    from paper_1308_4005_gb300 import learn
    from paper_1308_4005_gb300 import mls6

    world, rank, local = dist_setup(torch)
    torch.cuda.set_device(local)
    B.build()
    mls6.load()
    N = 1048576 if args.workload == "accuracy" else 65536
    box, x, c = learn.slab_system(N, 7000 + rank)
    stream = torch.cuda.Stream()
    ref = learn.Setup()
    _, _, Fref = learn._forces(box, x, c, ref.a_ref, ref.h_ref, "fp32")
    cuts = [3.0, 3.5, 4.0] if args.workload == "accuracy" else [3.0, 3.5]
    res = {"fp32": [], "mixed": [], "learned": []}
    pos32 = torch.tensor(np.c_[x, c], dtype=torch.float32, device="cuda")
    F = torch.empty((N, 3), dtype=torch.float32, device="cuda")
    for a in cuts:
        for form in ("fp32", "mixed"):
            plan = mls6.Plan(box, N, a, 1.0, 0, precision=form, stream=stream.cuda_stream)
            r = plan.evaluate(pos32, virial=False)
            torch.cuda.synchronize()
            eps = learn.eps_F(r["F"], Fref)
            ms = _timed_evals(lambda: mls6.mls6_eval(plan.handle, pos32.data_ptr(), 0,
                                                     F.data_ptr(), 0, 0), 20, 3, stream)
            res[form].append({"a": a, "h": 1.0, "eps_F": eps, "ms": ms, "value": N / (ms / 1e3)})
            plan.close()
        st = learn.Setup(a=a)
        train = [learn.slab_system(32768, 9000 + 10 * int(4 * a) + s) for s in range(2)]
        model, hist = learn.build_model(st, train, steps=800, batch=16384, lr=2e-3)
        plan = mls6.Plan(box, N, a, st.h_coarse, 0, precision="fp32", stream=stream.cuda_stream)
        r = plan.evaluate(pos32, virial=False)
        torch.cuda.synchronize()  # the plan runs on its own stream
        Fl = r["F"].clone()
        torch.cuda.synchronize()
        model.apply(plan, Fl)
        torch.cuda.synchronize()
        eps_c = learn.eps_F(r["F"], Fref)
        eps = learn.eps_F(Fl, Fref)

        def learned_step():
            mls6.mls6_eval(plan.handle, pos32.data_ptr(), 0, F.data_ptr(), 0, 0)
            model.apply(plan, F)

        ms = _timed_evals(learned_step, 20, 3, stream)
        res["learned"].append({"a": a, "h": st.h_coarse, "eps_F": eps, "eps_F_coarse": eps_c,
                               "ms": ms, "value": N / (ms / 1e3), "train_loss": hist[-1]})
        model.close()
        plan.close()

    def at(points, target=1e-4):
        pts = sorted(points, key=lambda p: p["eps_F"])
        le = np.log([p["eps_F"] for p in pts])
        lv = np.log([p["value"] for p in pts])
        t = np.log(target)
        if len(pts) < 2:
            return None, "one point"
        j = int(np.clip(np.searchsorted(le, t), 1, len(pts) - 1))
        f = (t - le[j - 1]) / (le[j] - le[j - 1])
        how = "interpolated" if le[0] <= t <= le[-1] else "extrapolated"
        return float(np.exp(lv[j - 1] + f * (lv[j] - lv[j - 1]))), how

    at_target = {k: at(v) for k, v in res.items()}
    line = {"metric": "atom-evals/s at eps_F = 1e-4", "value": at_target["mixed"][0],
            "unit": "atom-evals/s", "n_gpus": world, "steps": 20, "warmup": 3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+bf16x3", "data": "synthetic",
            "config": {"workload": f"slab{N} (proportions of the 4,194,304-atom slab)",
                       "reference": f"FP32 MLS a={ref.a_ref}, h={ref.h_ref}",
                       "virial": False, "cutoffs": cuts,
                       "learned": "coarse h=2 + network trained on h=1 targets per cutoff"},
            "at_1e-4": {k: {"value": v[0], "how": v[1]} for k, v in at_target.items()},
            "sweep": res}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_learned(args):
    """The 4,194,304-atom slab (160 x 160 x 240, a = 3): throughput of the fine
    evaluation (h = 1), the coarse one (h = 2) and the coarse one plus the
    learned correction (network trained first on two 32,768-atom slabs of the
    same proportions).  Forces only (no virial), FP32."""
    import numpy as np
    import torch

    from paper_1308_4005_gb300 import build as B
    from paper_1308_4005_gb300 import learn
    from paper_1308_4005_gb300 import mls6

    world, rank, local = dist_setup(torch)
    torch.cuda.set_device(local)
    B.build()
    mls6.load()
    st = learn.Setup()
    t0 = time.time()
    train = [learn.slab_system(32768, 9100 + s) for s in range(2)]
    model, hist = learn.build_model(st, train, steps=800, batch=16384, lr=2e-3)
    t_train = time.time() - t0
    N = 4194304 if args.workload == "learned4m" else 262144
    t0 = time.time()
    box, x, c = learn.slab_system(N, 9200 + rank)
    t_gen = time.time() - t0
    stream = torch.cuda.Stream()
    pos = torch.tensor(np.c_[x, c], dtype=torch.float32, device="cuda")
    F = torch.empty((N, 3), dtype=torch.float32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    out = {}
    for name, h, learned in (("fine", st.h_fine, False), ("coarse", st.h_coarse, False),
                             ("learned", st.h_coarse, True)):
        plan = mls6.Plan(box, N, st.a, h, 0, precision="fp32", stream=stream.cuda_stream)

        def step():
            flush.fill_(1)
            rc = mls6.mls6_eval(plan.handle, pos.data_ptr(), 0, F.data_ptr(), 0, 0)
            if rc:
                raise mls6.MLS6Error(rc, "mls6_eval")
            if learned:
                model.apply(plan, F)

        ev = []
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                step()
            stream.synchronize()
            for _ in range(args.steps):
                a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                flush.fill_(2)
                a_.record(stream)
                rc = mls6.mls6_eval(plan.handle, pos.data_ptr(), 0, F.data_ptr(), 0, 0)
                if learned:
                    model.apply(plan, F)
                b_.record(stream)
                ev.append((a_, b_))
        torch.cuda.synchronize()
        ms = sum(a_.elapsed_time(b_) for a_, b_ in ev) / len(ev)
        out[name] = {"h": h, "ms": ms, "value": N / (ms / 1e3),
                     "levels": plan.info()["levels"], "grid": plan.info()["n_grid"][0]}
        plan.close()
    line = {"metric": "atom-evals/s", "value": out["learned"]["value"], "unit": "atom-evals/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": out["learned"]["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+bf16", "data": "synthetic",
            "config": {"workload": f"slab{N} (160x160x240 proportions)", "a": st.a,
                       "virial": False, "train_s": t_train, "generate_s": t_gen,
                       "train_loss": [hist[0], hist[-1]],
                       "l2": "flushed between timed steps (256 MiB write)"},
            "forms": out}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def tensor_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except Exception:
        return 1900.0


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except Exception:
        return 6800.0


def main():
    args = parse()
    if args.workload.startswith("accuracy"):
        return run_accuracy(args)
    if args.workload.startswith("learned"):
        return run_learned(args)
    if args.workload.startswith("batch"):
        if args.impl == "reference":
            return run_reference_batch(args)
        return run_batch(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
