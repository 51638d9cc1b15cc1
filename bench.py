#!/usr/bin/env python
"""Throughput benchmark of multilevel summation for r^-6 dispersion on GB300.

One step = one full ``mls6_eval`` (bin, local pair part, anterpolation,
restriction, level stencils, coarsest level, prolongation, interpolation,
energy/virial reduction).  Metric: atom-evals/s (atoms whose energy
contribution and force one evaluation produces, per second).

Default workload: the 1,048,576-atom fluid cube (rho = 0.85, C6 in
[0.5, 1.5], a = 3, h = 1 -> 112^3, 5 levels) in mixed precision (FP32 pair
kernel and transfers, tensor-core level stencils with BF16 hi+lo operands,
FP64 coarsest level, energy and virial).  The same run also measures the
plain FP32 form on the same system, the relative force error eps_F of each
form against exact forces (direct periodic r^-6 sums on sampled atoms), a
cutoff sweep giving each form's throughput at eps_F = 1e-4, the learned
correction (coarse grid plus network) and the batched replicas, and a
roofline entry for every stage.

  --impl ours        (default) the CUDA library through its C ABI
  --impl reference   the FP64 CPU oracle on the host cores (full evaluations)

Under torchrun each rank evaluates an independent replica (different seed)
on its own GPU; value = atoms of all ranks / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import itertools
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

# Floating-point operations counted per unit of algorithmic work (fixed
# tallies, independent of how a kernel organises the work):
FLOP_PAIR = 42          # one ordered pair (i, j) inside the cutoff: e0_i and F_i terms
FLOP_PAIR_VIR = 12      # ... plus the six virial products
FLOP_TAP = 2            # one stencil tap (multiply-add) per node
FLOP_TAP_VIR = 12       # ... plus six virial multiply-adds
TARGET_EPS = 1e-4       # equal-accuracy point of the metric
EXACT_R = 20.0          # radius of the direct sums behind the exact sampled forces


# DRAM bytes (read + write) per step of each stage's kernels (all launches
# of the stage in one evaluation, L2 flushed before the step), from one ncu
# launch-list capture (dram__bytes_read.sum + dram__bytes_write.sum) of the
# named workload and precision, virial on; a kernel changed since its
# capture has no entry and reports null.
TRAFFIC = {
    ("cube1m", "mixed", "bin"): 84425728,          # k_bin, scans, k_scatter, k_cellsort
    ("cube1m", "mixed", "anterpolate"): 28061184,  # k_anterp + k_from_fixed
    ("cube1m", "mixed", "restrict"): 6534656,      # k_restrict, 4 levels
    ("cube1m", "mixed", "stencil"): 8270080,       # k_stencil_mma<1>: q of levels 1-4
    ("cube1m", "mixed", "prolongate"): 7336960,    # k_prolong, 4 levels
    ("cube1m", "mixed", "interpolate"): 45970688,  # k_interp (+ final reduction)
}

# arithmetic of each precision mode (pair/grid transfers; level stencils)
DTYPE = {"fp64": "f64", "fp32": "f32", "mixed": "f32+bf16x3"}
DEFAULT_PREC = {"cube1m": "mixed", "slab4m": "fp32"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="cube1m")
    ap.add_argument("--precision", choices=["fp32", "fp64", "mixed"], default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-virial", action="store_true",
                    help="evaluate energy and forces only (no virial arithmetic)")
    ap.add_argument("--no-tune", action="store_true",
                    help="batched workloads: keep the seeded configuration")
    ap.add_argument("--quick", action="store_true",
                    help="main line only: no other forms, sweep, learned or batched runs")
    ap.add_argument("--dwell", type=float, default=1.0,
                    help="seconds of untimed back-to-back evaluations before timing")
    a = ap.parse_args()
    if a.precision is None:
        a.precision = DEFAULT_PREC.get(a.workload, "fp32")
    return a


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
    """Ordered pairs (i, j), i != j, with periodic distance < a (the pair
    kernel's algorithmic work)."""
    import numpy as np
    from scipy.spatial import cKDTree

    boxv = np.asarray(box, dtype=np.float64)
    xx = np.mod(np.asarray(x, dtype=np.float64), boxv)
    t = cKDTree(xx, boxsize=boxv)
    r = np.nextafter(a, 0.0)  # count_neighbors counts distance <= r
    return int(t.count_neighbors(t, r)) - xx.shape[0]


def exact_forces(x, c, box, idx, R=EXACT_R):
    """Forces on the atoms idx of the exact periodic r^-6 energy
    E = -1/2 sum_i sum_{j,n}' c_i c_j |x_j - x_i + nL|^-6, summed directly
    over every image within R.  The neglected remainder beyond R is the
    field of the density fluctuations there (a uniform medium exerts no
    net force): of order 6 c^2 (4 pi rho / (11 R^11))^(1/2) ~ 1e-6 at
    R = 20 for a fluid, and of order 1.5 pi rho R^-4 ~ 2e-5 near a slab
    surface, both far below the 1e-4 force errors measured with it."""
    import numpy as np
    from scipy.spatial import cKDTree

    L = np.asarray(box, dtype=np.float64)
    xw = np.mod(np.asarray(x, dtype=np.float64), L)
    c = np.asarray(c, dtype=np.float64)
    idx = np.asarray(idx)
    if np.all(L > 2.0 * R):  # one image at most: periodic tree, minimum image
        tree, src, pts = cKDTree(xw, boxsize=L), None, xw
    else:  # replicate the box so every image within R is an explicit point
        reps = [range(-int(math.ceil(R / l)), int(math.ceil(R / l)) + 1) for l in L]
        sh = np.array(list(itertools.product(*reps)), dtype=np.float64) * L
        pts = (xw[None, :, :] + sh[:, None, :]).reshape(-1, 3)
        src = np.tile(np.arange(xw.shape[0]), sh.shape[0])
        tree = cKDTree(pts)
    F = np.zeros((idx.size, 3))
    for s in range(0, idx.size, 128):
        ii = idx[s:s + 128]
        nb = tree.query_ball_point(xw[ii], R, return_sorted=False)
        cnt = np.array([len(v) for v in nb])
        jj = np.concatenate([np.asarray(v, dtype=np.int64) for v in nb])
        owner = np.repeat(np.arange(ii.size), cnt)
        d = pts[jj] - xw[ii][owner]
        if src is None:
            d -= L * np.round(d / L)
            cj = c[jj]
        else:
            cj = c[src[jj]]
        r2 = np.sum(d * d, axis=1)
        keep = r2 > 1e-20  # the atom itself
        w = np.where(keep, 6.0 * cj / np.where(keep, r2, 1.0) ** 4, 0.0)
        for k in range(3):
            F[s:s + ii.size, k] = np.bincount(owner, weights=w * d[:, k], minlength=ii.size)
        F[s:s + ii.size] *= c[ii][:, None]
    return F


def eps_F(F, Fex):
    import numpy as np

    F = np.asarray(F, dtype=np.float64)
    return float(np.sqrt(np.sum((F - Fex) ** 2) / np.sum(Fex ** 2)))


def best_at_target(points, target=TARGET_EPS):
    """The form's throughput at eps_F = target, choosing the grid spacing:
    at_target along the cutoff sweep of each h, the best interpolated one
    (extrapolated ones only when no h brackets the target)."""
    by_h = {}
    for p in points:
        if p.get("eps_F"):
            by_h.setdefault(p["h"], []).append(p)
    best = None
    for h, pts in by_h.items():
        r = at_target(pts, target)
        if r["value"] is None:
            continue
        r = dict(r, h=h)
        rank = (r["how"] == "interpolated", r["value"])
        if best is None or rank > (best["how"] == "interpolated", best["value"]):
            best = r
    return best or {"value": None, "how": "fewer than two points"}


def at_target(points, target=TARGET_EPS):
    """Throughput at eps_F = target by log-log interpolation between the
    bracketing points of a cutoff sweep (extrapolated from the nearest two
    when the sweep does not bracket it)."""
    import numpy as np

    pts = sorted([p for p in points if p.get("eps_F")], key=lambda p: p["eps_F"])
    if len(pts) < 2:
        return {"value": None, "how": "fewer than two points"}
    le = np.log([p["eps_F"] for p in pts])
    lv = np.log([p["value"] for p in pts])
    t = math.log(target)
    j = int(np.clip(np.searchsorted(le, t), 1, len(pts) - 1))
    f = (t - le[j - 1]) / (le[j] - le[j - 1])
    how = "interpolated" if le[0] <= t <= le[-1] else "extrapolated"
    return {"value": float(math.exp(lv[j - 1] + f * (lv[j] - lv[j - 1]))), "how": how}


# ------------------------------------------------------------ CPU oracle

def oracle_full(O, w, xd, cd):
    """Seconds of one full FP64 oracle evaluation on the current threads."""
    n = O.grid_dims(w.box, w.h, w.levels)
    t0 = time.perf_counter()
    O.evaluate(w.box, w.a, n, w.levels, xd, cd)
    return time.perf_counter() - t0


def oracle_single_thread(O, w, xd, cd, frac=0):
    """Single-thread oracle time of a full evaluation from a bounded sample:
    the whole grid part once and the local part of 1/frac of the atoms."""
    import numpy as np

    n = O.grid_dims(w.box, w.h, w.levels)
    frac = frac or max(16, w.N // 65536)  # the local part of about 65,536 atoms
    O.set_threads(1)
    try:
        t0 = time.perf_counter()
        O.evaluate_sample(w.box, w.a, n, w.levels, xd, cd, np.zeros(0, np.int64))
        t_grid = time.perf_counter() - t0
        idx = np.random.default_rng(7).choice(w.N, max(1, w.N // frac), replace=False)
        t0 = time.perf_counter()
        O.local(w.box, w.a, xd, cd, idx)
        t_loc = (time.perf_counter() - t0) * w.N / idx.size
    finally:
        O.set_threads(os.cpu_count() or 1)
    return t_grid + t_loc, (f"grid part for all {w.N} atoms ({t_grid:.1f} s) + local part for "
                            f"{idx.size} random atoms, scaled to all ({t_loc:.1f} s)")


def oracle_baseline(w, x, c):
    """The FP64 oracle on the host cores: one full evaluation on all cores
    (value), and a single-thread figure from a bounded sample."""
    import numpy as np

    from oracle import oracle as O

    O.build()
    O.set_threads(os.cpu_count() or 1)
    xd, cd = np.asarray(x, np.float64), np.asarray(c, np.float64)
    t_all = oracle_full(O, w, xd, cd)
    t_one, how = oracle_single_thread(O, w, xd, cd)
    return {"value": w.N / t_all, "unit": "atom-evals/s", "cores": O.threads(), "kind": "oracle",
            "sample": f"one full FP64 oracle evaluation of {w.name} on all cores ({t_all:.1f} s)",
            "single_thread": {"value": w.N / t_one, "cores": 1, "sample": how}}


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
    for _ in range(args.warmup):
        oracle_full(O, w, xd, cd)
    secs = [oracle_full(O, w, xd, cd) for _ in range(args.steps)]
    ms = 1e3 * statistics.mean(secs)
    value = w.N / (ms / 1e3)
    t_one, how = oracle_single_thread(O, w, xd, cd)
    line = {"metric": "atom-evals/s", "value": value, "unit": "atom-evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": config_of(w, args, world),
            "cpu_baseline": {"value": value, "unit": "atom-evals/s", "cores": O.threads(),
                             "kind": "oracle",
                             "sample": (f"each step one full FP64 oracle evaluation of all "
                                        f"{w.N} atoms on all cores"),
                             "single_thread": {"value": w.N / t_one, "cores": 1,
                                               "sample": how}},
            "e2e": {"value": value, "unit": "atom-evals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_reference_batch(args):
    """Oracle arm of the batched workload: each step is one full FP64 oracle
    evaluation of one replica (cycling through the replicas by size rank)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import dataclasses

    from oracle import oracle as O
    from paper_1308_4005_gb300 import inputs as I

    nrep = 256 if args.workload == "batch256" else 16
    ws = I.batch_workloads(B=nrep)
    O.build()
    O.set_threads(os.cpu_count() or 1)
    order = sorted(range(nrep), key=lambda r: ws[r].N)
    picks = [order[(k * nrep) // max(1, args.steps + args.warmup)]
             for k in range(args.steps + args.warmup)]
    atoms = secs = 0.0
    for k, r in enumerate(picks):
        w = dataclasses.replace(ws[r], levels=I_auto_levels(ws[r]))
        x, c = I.generate(w)
        t = oracle_full(O, w, x, c)
        if k >= args.warmup:
            atoms += w.N
            secs += t
    value = atoms / secs
    line = {"metric": "atom-evals/s", "value": value, "unit": "atom-evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "replicas": nrep, "a": ws[0].a,
                       "h": ws[0].h, "levels": "auto per replica"},
            "cpu_baseline": {"value": value, "unit": "atom-evals/s", "cores": O.threads(),
                             "kind": "oracle",
                             "sample": ("each step one full FP64 oracle evaluation of one "
                                        "replica (spread over the size range)")},
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


# ----------------------------------------------------------- roofline

def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "of measured (MEASURED_PEAKS.json)"
    except Exception:
        return 6800.0, 1900.0, "of fallback"


def stage_work(info, N, n_pairs, prec, vir):
    """Algorithmic work of one launch of every stage: (bound, amount, unit,
    what is counted).  Bytes are the data each stage must move at least
    once; flops follow the fixed tallies above."""
    esz = 8 if prec == "fp64" else 4
    lv = info["n_grid"]
    np_ = [n[0] * n[1] * n[2] for n in lv]
    l = len(lv)
    fp_pair = FLOP_PAIR + (FLOP_PAIR_VIR if vir else 0)
    fp_tap = FLOP_TAP + (FLOP_TAP_VIR if vir else 0)
    fx = 8 if prec == "fp64" else 4  # fixed-point sums
    w = {
        "bin": ("hbm", N * 80.0, "B", "per atom: input 16 B read, record 16 B + cell 4 B "
                "written, scatter 20 B read + 20 B written, order 4 B"),
        "pair": ("alu", n_pairs * float(fp_pair), "flop",
                 f"{n_pairs} ordered pairs inside a x {fp_pair} flop"),
        "anterpolate": ("hbm", N * 16.0 + np_[0] * (2.0 * fx + esz), "B",
                        "per atom: sorted record; finest grid: fixed-point sums written and "
                        "read once, q^1 written"),
        "restrict": ("hbm", sum((np_[k] + np_[k + 1]) * esz for k in range(l - 1)) * 1.0, "B",
                     "every level k < l read once, level k+1 written"),
        "stencil": ("alu", sum(np_[:-1]) * float(info["ntaps"]) * fp_tap, "flop",
                    f"{sum(np_[:-1])} nodes on levels < l x {info['ntaps']} taps x {fp_tap} flop"),
        "coarsest": ("alu64", np_[-1] ** 2 * float(2 + (12 if vir else 0)), "flop",
                     f"{np_[-1]}^2 node pairs of the coarsest table"),
        "prolongate": ("hbm", sum((np_[k + 1] + 2 * np_[k]) * esz for k in range(l - 1)) * 1.0,
                       "B", "e^{k+1,tot} and e^k read, e^{k,tot} written per level"),
        "interpolate": ("hbm", N * (16.0 + 4 + 7 * esz) + np_[0] * esz, "B",
                        "per atom: sorted record, index, e0 + local force in, force out; "
                        "finest grid once"),
    }
    return w


def rooflines(stage_ms, work, peaks, prec, stencil_kind, workload, vir):
    """One entry per stage: achieved rate (algorithmic work / stage time)
    against the stage's peak."""
    hbm, bf16, hbm_src = peaks["hbm"], peaks["bf16"], peaks["src"]
    out = {}
    for st, (bound, amount, unit, note) in work.items():
        ms = stage_ms.get(st)
        if not ms:
            continue
        if bound == "hbm":
            ach, pk, u, src = amount / (ms * 1e-3) / 1e9, hbm, "GB/s", f"hbm_gbs {hbm_src}"
        elif bound == "alu64" or (bound == "alu" and prec == "fp64"):
            ach, pk, u, src = (amount / (ms * 1e-3) / 1e12, peaks["fp64"], "TFLOP/s",
                               "FP64 FMA rate measured in this run (mls6_fma_peak)")
            bound = "alu"
        elif st == "stencil" and stencil_kind in (2, 3):
            ach, pk, u, src = (amount / (ms * 1e-3) / 1e12, bf16, "TFLOP/s",
                               f"bf16_tflops {hbm_src}: useful flops of BF16 split products")
            bound = "tensor"
        else:
            ach, pk, u, src = (amount / (ms * 1e-3) / 1e12, peaks["fp32"], "TFLOP/s",
                               "FP32 FMA rate measured in this run (mls6_fma_peak)")
        tr = None if not vir else TRAFFIC.get((workload, prec, st))
        out[st] = {"bound": bound, "achieved": ach, "peak": pk, "unit": u, "frac": ach / pk,
                   "traffic": tr, "work": note, "peak_source": src, "avg_launch_ms": ms}
    return out


# ------------------------------------------------------------------ ours

def timed_steps(torch, stream, step, steps, flush, world=1):
    """CUDA-event time (ms) of each of `steps` calls of step(), the L2
    flushed (256 MiB write) before each."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    barrier(world)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for k in range(steps):
            flush.fill_(k & 0xFF)
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    return [a.elapsed_time(b) for a, b in ev]


class Bench:
    """Device buffers and one plan of a workload."""

    def __init__(self, torch, mls6, dev, stream, box, N, a, h, levels, prec, x, c, vir=True,
                 order=3):
        import numpy as np

        self.torch, self.mls6, self.stream = torch, mls6, stream
        dt = torch.float64 if prec == "fp64" else torch.float32
        self.N, self.prec = N, prec
        self.plan = mls6.Plan(box, N, a, h, levels, precision=prec, order=order,
                              stream=stream.cuda_stream)
        self.info = self.plan.info()
        self.pos_h = torch.tensor(np.c_[x, c], dtype=dt).pin_memory()
        self.pos = torch.empty((N, 4), dtype=dt, device=dev)
        self.F = torch.empty((N, 3), dtype=dt, device=dev)
        self.F_h = torch.empty((N, 3), dtype=dt).pin_memory()
        self.out = torch.zeros(8, dtype=torch.float64, device=dev)
        self.out_h = torch.zeros(8, dtype=torch.float64).pin_memory()
        with torch.cuda.stream(stream):
            self.pos.copy_(self.pos_h, non_blocking=True)
        stream.synchronize()
        self.vir_ptr = self.out.data_ptr() + 8 if vir else 0

    def step(self):
        rc = self.mls6.mls6_eval(self.plan.handle, self.pos.data_ptr(), 0, self.F.data_ptr(),
                                 self.out.data_ptr(), self.vir_ptr)
        if rc:
            raise self.mls6.MLS6Error(rc, "mls6_eval")

    def e2e_step(self):
        """End to end with host buffers: the positions stay in page-locked
        host memory and the binning kernel reads them over the host link
        (mls6_eval accepts such pointers); forces and the energy/virial
        words are copied back to page-locked host memory."""
        rc = self.mls6.mls6_eval(self.plan.handle, self.pos_h.data_ptr(), 0, self.F.data_ptr(),
                                 self.out.data_ptr(), self.vir_ptr)
        if rc:
            raise self.mls6.MLS6Error(rc, "mls6_eval")
        self.F_h.copy_(self.F, non_blocking=True)
        self.out_h.copy_(self.out, non_blocking=True)

    def e2e_copy_step(self):
        """End to end with an explicit host-to-device copy of the positions
        before the evaluation."""
        self.pos.copy_(self.pos_h, non_blocking=True)
        self.step()
        self.F_h.copy_(self.F, non_blocking=True)
        self.out_h.copy_(self.out, non_blocking=True)

    def warm(self, n, dwell=0.0):
        with self.torch.cuda.stream(self.stream):
            for _ in range(n):
                self.step()
            self.stream.synchronize()
            t_end = time.time() + dwell
            while time.time() < t_end:
                for _ in range(20):
                    self.step()
                self.stream.synchronize()
        rc = self.mls6.mls6_last_error(self.plan.handle)
        if rc:
            raise self.mls6.MLS6Error(rc, "warm-up")

    def stages(self, steps, flush):
        """Per-stage CUDA-event times (ms), stages serialised."""
        mls6 = self.mls6
        mls6.mls6_profile(self.plan.handle, True)
        acc = {}
        with self.torch.cuda.stream(self.stream):
            for k in range(steps):
                flush.fill_(k & 0xFF)
                self.step()
                st, _ = mls6.mls6_stage_times(self.plan.handle)
                for name, ms in st.items():
                    acc[name] = acc.get(name, 0.0) + ms
        mls6.mls6_profile(self.plan.handle, False)
        return {k: v / steps for k, v in acc.items()}

    def forces(self):
        self.torch.cuda.synchronize()
        return self.F.double().cpu().numpy()

    def close(self):
        self.plan.close()


def form_point(torch, mls6, dev, stream, flush, w, x, c, prec, a, h, levels, idx, Fex, steps,
               order=3):
    """Throughput and eps_F of one form at one (a, h, interpolation order)."""
    b = Bench(torch, mls6, dev, stream, w.box, w.N, a, h, levels, prec, x, c, order=order)
    try:
        b.warm(3)
        ms = statistics.mean(timed_steps(torch, stream, b.step, steps, flush))
        e = eps_F(b.forces()[idx], Fex)
        return {"a": a, "h": h, "order": order, "levels": b.info["levels"], "ms": ms,
                "value": w.N / (ms / 1e3), "eps_F": e, "stencil_kind": b.info["stencil_kind"]}
    finally:
        b.close()


def learned_point(torch, mls6, dev, stream, flush, w, x, c, a, idx, Fex, steps, log,
                  slabs=False):
    """The learned correction at cutoff a: coarse evaluation (h = 2) plus the
    network, trained on two 32,768-atom systems against the fine (h = 1)
    evaluation -- cubes of the workload's density, or (slabs) slabs with the
    proportions of the 4,194,304-atom slab; eps_F, throughput, and the
    measured floor (network time per atom against the grid time the coarse
    grid saves)."""
    from paper_1308_4005_gb300 import inputs as I
    from paper_1308_4005_gb300 import learn

    st = learn.Setup(a=a)
    t0 = time.time()
    rho = w.N / (w.box[0] * w.box[1] * w.box[2])
    train = []
    for s in range(2):
        if slabs:
            train.append(learn.slab_system(32768, 9300 + s))
            continue
        tw = I.scaled_cube(32768, rho, a, 1.0, 0, 9300 + s)
        tx, tc = I.generate(tw)
        train.append((tw.box, tx, tc))
    model, hist = learn.build_model(st, train, steps=800, batch=16384, lr=2e-3)
    t_train = time.time() - t0
    b = Bench(torch, mls6, dev, stream, w.box, w.N, a, st.h_coarse, 0, "fp32", x, c)
    try:
        b.warm(2)
        ms_coarse = statistics.mean(timed_steps(torch, stream, b.step, steps, flush))

        def step():
            b.step()
            model.apply(b.plan, b.F)

        with torch.cuda.stream(stream):
            step()
        Fl = b.forces()
        ms = statistics.mean(timed_steps(torch, stream, step, steps, flush))
        net = statistics.mean(timed_steps(torch, stream, lambda: model.apply(b.plan, b.F),
                                          steps, flush))
        e = eps_F(Fl[idx], Fex)
        with torch.cuda.stream(stream):
            b.step()
        e_c = eps_F(b.forces()[idx], Fex)
        return {"a": a, "h": st.h_coarse, "ms": ms, "value": w.N / (ms / 1e3), "eps_F": e,
                "eps_F_coarse_alone": e_c, "ms_coarse_alone": ms_coarse,
                "ms_network": net, "train_s": t_train,
                "train_loss": [float(hist[0]), float(hist[-1])]}
    finally:
        b.close()
        model.close()


def batch_point(torch, mls6, dev, stream, flush, ws, x, c, off, a, steps, tune):
    """The batched replicas at cutoff a (h = 1, levels by the automatic
    rule): one graph launch per step over every replica; eps_F on sampled
    atoms of two cube and two slab replicas against exact forces."""
    import numpy as np

    Ntot = int(off[-1])
    t0 = time.time()
    bt = mls6.Batch([w.box for w in ws], [w.N for w in ws], a, ws[0].h, 0, precision="fp32")
    t_plan = time.time() - t0
    try:
        mls6.mls6_batch_set_stream(bt.handle, stream.cuda_stream)
        pos = torch.tensor(np.c_[x, c], dtype=torch.float32, device=dev)
        F = torch.empty((Ntot, 3), dtype=torch.float32, device=dev)
        E = torch.zeros(len(ws), dtype=torch.float64, device=dev)
        W = torch.zeros((len(ws), 6), dtype=torch.float64, device=dev)
        t_tune = None
        if tune:
            t0 = time.time()
            with torch.cuda.stream(stream):
                bt.tune(pos, reps=3)
            t_tune = time.time() - t0

        def step():
            rc = mls6.mls6_batch_eval(bt.handle, pos.data_ptr(), 0, F.data_ptr(), E.data_ptr(),
                                      W.data_ptr())
            if rc:
                raise mls6.MLS6Error(rc, "mls6_batch_eval")

        with torch.cuda.stream(stream):
            for _ in range(3):
                step()
        ms = statistics.mean(timed_steps(torch, stream, step, steps, flush))
        torch.cuda.synchronize()
        Fb = F.double().cpu().numpy()
        info = bt.info()
        # the other launch form (graph of kernel chains / one persistent
        # kernel), timed for the record with the tuned shapes
        mode = mls6.mls6_batch_mode(bt.handle)
        forms = {("persistent" if mode else "chains"): ms}
        mls6.mls6_batch_set_mode(bt.handle, not mode)
        with torch.cuda.stream(stream):
            for _ in range(3):
                step()
        other = "persistent" if mls6.mls6_batch_mode(bt.handle) else "chains"
        if other not in forms:
            forms[other] = statistics.mean(timed_steps(torch, stream, step, steps, flush))
        mls6.mls6_batch_set_mode(bt.handle, mode)
        rng = np.random.default_rng(17)
        picks = [r for r in range(0, len(ws), 2)][:2] + [r for r in range(1, len(ws), 2)][:2]
        num = den = 0.0
        for r in picks:
            sl = slice(int(off[r]), int(off[r + 1]))
            ii = rng.choice(ws[r].N, min(256, ws[r].N), replace=False)
            Fex = exact_forces(x[sl], c[sl], ws[r].box, ii)
            num += float(np.sum((Fb[sl][ii] - Fex) ** 2))
            den += float(np.sum(Fex ** 2))
        return {"a": a, "h": ws[0].h, "ms": ms, "value": Ntot / (ms / 1e3),
                "eps_F": math.sqrt(num / den), "replicas": len(ws), "atoms": Ntot,
                "launches_per_step": int(info["launches"]), "branches": info["branches"],
                "form": "persistent" if mode else "chains", "ms_by_form": forms,
                "plan_s": t_plan, "autotune_s": t_tune,
                "eps_F_sample": "256 atoms of each of replicas " + ", ".join(map(str, picks))}
    finally:
        bt.close()


def lb_point(torch, mls6, dev, stream, flush, w, x, steps, prec="fp32"):
    """Lorentz-Berthelot mixing (Sec. II.D, seven grid channels) on the same
    positions: sigma_i ~ U[0.85, 1.15], eps_i ~ U[0.5, 1.5] (seeded), energy
    and forces."""
    import numpy as np

    rng = np.random.default_rng(1308)
    sig = rng.uniform(0.85, 1.15, w.N)
    eps = rng.uniform(0.5, 1.5, w.N)
    dt = torch.float64 if prec == "fp64" else torch.float32
    plan = mls6.Plan(w.box, w.N, w.a, w.h, w.levels, precision=prec, stream=stream.cuda_stream)
    try:
        pos = torch.tensor(np.asarray(x, np.float64), dtype=dt, device=dev).contiguous()
        ds = torch.tensor(sig, dtype=dt, device=dev)
        de = torch.tensor(eps, dtype=dt, device=dev)
        F = torch.empty((w.N, 3), dtype=dt, device=dev)
        E = torch.zeros(1, dtype=torch.float64, device=dev)

        def step():
            rc = mls6.mls6_eval_lb(plan.handle, pos.data_ptr(), ds.data_ptr(), de.data_ptr(),
                                   F.data_ptr(), E.data_ptr())
            if rc:
                raise mls6.MLS6Error(rc, "mls6_eval_lb")

        with torch.cuda.stream(stream):
            for _ in range(2):
                step()
        ms = statistics.mean(timed_steps(torch, stream, step, steps, flush))
        _, launches = mls6.mls6_stage_times(plan.handle)
        return {"precision": prec, "ms": ms, "value": w.N / (ms / 1e3), "channels": 7,
                "launches_per_step": int(launches), "energy": float(E.item()),
                "species": "sigma ~ U[0.85, 1.15], eps ~ U[0.5, 1.5] (seed 1308)"}
    finally:
        plan.close()


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
    log = (lambda m: print(f"[bench] {m}", file=sys.stderr, flush=True)) if rank == 0 else \
        (lambda m: None)
    t_start = time.time()
    w, x, c = workload_arrays(args.workload, rank, args.precision)
    log(f"inputs {w.name} in {time.time() - t_start:.1f} s")
    vir = not args.no_virial
    N = w.N
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    hbm, bf16, src = load_peaks()
    peaks = {"fp32": mls6.mls6_fma_peak("fp32"), "fp64": mls6.mls6_fma_peak("fp64"),
             "hbm": hbm, "bf16": bf16, "src": src}
    log(f"measured FMA peaks: FP32 {peaks['fp32']:.1f}, FP64 {peaks['fp64']:.2f} TFLOP/s")

    b = Bench(torch, mls6, dev, stream, w.box, N, w.a, w.h, w.levels, args.precision, x, c, vir)
    info = b.info
    sampler = ClockSampler(gpu_smi_id(torch, local))
    t_dwell0 = time.time()
    b.warm(args.warmup, args.dwell)

    # ------------------------------------------------ timed region (device)
    # Production path: captured graph, pair sum concurrent with the grid
    # chain, no per-stage events.  L2 flushed before every step.
    ms_list = timed_steps(torch, stream, b.step, args.steps, flush, world)
    _, launches_per_step = mls6.mls6_stage_times(b.plan.handle)
    value, total_ms = job_throughput(torch, sum(ms_list), N, args.steps, world, dev)
    ms_per_step = total_ms / args.steps
    E_dev = float(b.out[0].item())
    # --------------------------------------------- end to end (host buffers)
    # both protocols through mls6_eval (positions read from host memory by
    # the kernel, or copied first), each after untimed warm-up steps (the
    # plan re-captures its graph when the input pointer changes)
    e2e_ms = {}
    for name, fn in (("host_read", b.e2e_step), ("copy_in", b.e2e_copy_step)):
        with torch.cuda.stream(stream):
            for _ in range(3):
                fn()
        torch.cuda.synchronize()
        e2e_ms[name] = sum(timed_steps(torch, stream, fn, args.steps, flush, world))
    e2e_how = min(e2e_ms, key=e2e_ms.get)
    e2e_value, _ = job_throughput(torch, e2e_ms[e2e_how], N, args.steps, world, dev)
    e2e_alt = {k: job_throughput(torch, v, N, args.steps, world, dev)[0] for k, v in e2e_ms.items()}
    t_timed1 = time.time()
    sampler.stop()
    clocks = sampler.summary(t_dwell0, t_timed1)
    clocks["window"] = "warm-up dwell + timed steps"
    # ------------------------------------- per-kernel times (serialised pass)
    stage_ms = b.stages(args.steps, flush)
    F_main = b.forces()
    b.close()

    # ------------------------------------------------------------- roofline
    n_pairs = count_pairs(x, w.box, w.a)
    work = stage_work(info, N, n_pairs, args.precision, vir)
    roofs = rooflines(stage_ms, work, peaks, args.precision, info["stencil_kind"], w.name, vir)
    dom = max(roofs, key=lambda k: roofs[k]["avg_launch_ms"])
    roof = dict(roofs[dom], kernel=dom,
                timing=("CUDA events on the launching stream around the stage, averaged over a "
                        "serialised pass of the same steps right after the timed region"))
    if dom == "stencil" and info["stencil_kind"] in (2, 3):
        roof["issued_over_useful"] = "32/13 Toeplitz band x 3 split products (energy channel)"
    line = {"metric": "atom-evals/s", "value": value, "unit": "atom-evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": config_of(w, args, world),
            "e2e": {"value": e2e_value, "unit": "atom-evals/s",
                    "h2d_bytes_per_step": int(b.pos_h.numel() * b.pos_h.element_size()),
                    "d2h_bytes_per_step": int(b.F_h.numel() * b.F_h.element_size() + 8 * 8),
                    "how": {"host_read": "positions read from page-locked host memory by the "
                                         "binning kernel",
                            "copy_in": "positions copied host to device before the call"}[e2e_how]
                           + "; forces and energy/virial copied device to host",
                    "by_protocol": e2e_alt},
            "gpu_launches": int(launches_per_step) * args.steps,
            "roofline": roof, "roofline_stages": roofs, "stages_ms": stage_ms,
            "peaks": {k: v for k, v in peaks.items()}, "clocks": clocks, "energy": E_dev}

    extras = rank == 0 and world == 1 and not args.quick and w.name == "cube1m"
    if extras:
        rng = np.random.default_rng(5)
        idx = rng.choice(N, 2048, replace=False)
        t0 = time.time()
        Fex = exact_forces(x, c, w.box, idx)
        log(f"exact forces on {idx.size} sampled atoms in {time.time() - t0:.1f} s")
        line["eps_F"] = eps_F(F_main[idx], Fex)
        line["accuracy"] = {
            "eps_F": "||F - F_exact|| / ||F_exact|| over all components of 2048 sampled atoms",
            "F_exact": (f"direct periodic sum of c_i c_j r^-6 over every image within "
                        f"{EXACT_R} sigma"),
            "target": TARGET_EPS}
        # accuracy sweep over the cutoff a and the finest spacing h (the
        # workload's h with its levels first; coarser h with the automatic
        # level count): each form's throughput at eps_F = 1e-4 is taken on
        # the h that reaches it fastest (the paper trades a against h for a
        # given accuracy, Sec. IV)
        sweep = {"fp32": [], "mixed": []}
        for h in (w.h, 1.25 * w.h, 1.5 * w.h, 2.0 * w.h):
            for a in (3.0, 3.5, 4.0):
                for prec in ("fp32", "mixed"):
                    lev = w.levels if h == w.h else 0
                    try:
                        sweep[prec].append(form_point(torch, mls6, dev, stream, flush, w, x, c,
                                                      prec, a, h, lev, idx, Fex, 10))
                    except Exception as e:  # report, keep the main line
                        sweep[prec].append({"a": a, "h": h, "error": repr(e)})
        # the quintic basis (order 5, Sec. III.B's comparison): smaller
        # interpolation error at a given h/a for 216 instead of 64 nodes per atom
        sweep["fp32_order5"] = []
        for h in (1.5 * w.h, 2.0 * w.h):
            for a in (2.5, 3.0, 3.5):
                try:
                    sweep["fp32_order5"].append(form_point(torch, mls6, dev, stream, flush, w, x,
                                                           c, "fp32", a, h, 0, idx, Fex, 10,
                                                           order=5))
                except Exception as e:
                    sweep["fp32_order5"].append({"a": a, "h": h, "order": 5, "error": repr(e)})
        log(f"sweep done at {time.time() - t_start:.0f} s")
        line["forms"] = {p: dict(v[0]) for p, v in sweep.items()
                         if p in ("fp32", "mixed") and v and "value" in v[0]}
        line["sweep"] = sweep
        # best over h, and along the workload's own h
        at = {p: dict(best_at_target(v),
                      at_workload_h=at_target([q for q in v if q.get("h") == w.h]))
              for p, v in sweep.items() if p in ("fp32", "mixed")}
        at["fp32_order5"] = best_at_target(sweep["fp32_order5"])
        try:
            lp = [learned_point(torch, mls6, dev, stream, flush, w, x, c, a, idx, Fex, 10, log)
                  for a in (3.0, 3.5)]
            line["learned"] = lp
            at["learned"] = best_at_target(lp)
        except Exception as e:
            line["learned"] = {"error": repr(e)}
        log(f"learned done at {time.time() - t_start:.0f} s")
        try:
            from paper_1308_4005_gb300 import inputs as I

            ws = I.batch_workloads(B=256)
            t0 = time.time()
            bx, bc, off = I.generate_batch(ws, processes=min(16, os.cpu_count() or 1))
            bx, bc = bx.astype(np.float32), bc.astype(np.float32)
            t_gen = time.time() - t0
            bp = [batch_point(torch, mls6, dev, stream, flush, ws, bx, bc, off, a, 10,
                              not args.no_tune) for a in (2.5, 3.5)]
            bp[0]["generate_s"] = t_gen
            line["batched"] = bp
            at["batched"] = best_at_target(bp)
        except Exception as e:
            line["batched"] = {"error": repr(e)}
        log(f"batched done at {time.time() - t_start:.0f} s")
        try:
            line["lorentz_berthelot"] = lb_point(torch, mls6, dev, stream, flush, w, x, 5)
        except Exception as e:
            line["lorentz_berthelot"] = {"error": repr(e)}
        log(f"Lorentz-Berthelot done at {time.time() - t_start:.0f} s")
        line["at_1e-4"] = at
    if rank == 0 and world == 1 and not args.quick and w.name == "slab4m":
        # the learned-correction configuration: the coarse grid of the main
        # line (h = 2), the same plus the network (trained on 32,768-atom
        # slabs of the same proportions), and the fine grid (h = 1) that
        # supplies the training targets and the accuracy check of the correction
        rng = np.random.default_rng(5)
        idx = rng.choice(N, 2048, replace=False)
        t0 = time.time()
        Fex = exact_forces(x, c, w.box, idx)
        log(f"exact forces on {idx.size} sampled atoms in {time.time() - t0:.1f} s")
        line["eps_F"] = eps_F(F_main[idx], Fex)
        try:
            line["learned"] = learned_point(torch, mls6, dev, stream, flush, w, x, c, w.a, idx,
                                            Fex, 10, log, slabs=True)
        except Exception as e:
            line["learned"] = {"error": repr(e)}
        log(f"learned done at {time.time() - t_start:.0f} s")
        try:
            line["fine_grid"] = form_point(torch, mls6, dev, stream, flush, w, x, c, "fp32",
                                            w.a, 1.0, 0, idx, Fex, 10)
        except Exception as e:
            line["fine_grid"] = {"error": repr(e)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t0 = time.time()
        line["cpu_baseline"] = oracle_baseline(w, x, c)
        log(f"oracle baseline in {time.time() - t0:.1f} s")
    line["wall_s"] = time.time() - t_start
    if rank == 0:
        print(json.dumps(line), flush=True)
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
    fp32_peak = mls6.mls6_fma_peak("fp32")
    roof = None
    if dom in ("pair", "stencil"):
        amount = (work_pair if dom == "pair" else work_sten) / 1e12
        ach = amount / (stage_acc[dom] / 1e3)
        roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": fp32_peak,
                "unit": "TFLOP/s", "frac": ach / fp32_peak, "traffic": None,
                "work": f"sum over the {nrep} replicas of the {dom} kernel's algorithmic flops",
                "peak_source": "FP32 FMA rate measured in this run (mls6_fma_peak)",
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


def main():
    args = parse()
    if args.workload.startswith("batch"):
        if args.impl == "reference":
            return run_reference_batch(args)
        return run_batch(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
