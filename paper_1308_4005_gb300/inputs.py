"""Seeded synthetic inputs for the dispersion workloads.

This module only places atoms and draws coefficients; it holds none of the
multilevel-summation arithmetic and is shared by the GPU tests, the benchmark
and the CPU oracle's tests.

The paper's systems (Sec. III.A) are energy-minimised Lennard-Jones slabs and
cubes that need repulsion and an external MD code to prepare.  They are
replaced here by random sequential addition (RSA): uniform random trial points,
accepted when no accepted atom lies closer than ``dmin`` (periodic distance),
which keeps every r^-6 term finite.  Trial points are drawn in batches; within
a batch they are accepted greedily in draw order, so the result is the RSA
sequence of that draw order.  Dispersion coefficients follow geometric mixing
(Sec. II.D): C6_i ~ U[lo, hi] and c_i = sqrt(C6_i).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 13084005


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic system plus the MLS parameters it is evaluated with."""
    name: str
    N: int
    box: tuple            # (Lx, Ly, Lz), periodic
    region: tuple         # ((x0, x1), (y0, y1), (z0, z1)) where atoms are placed
    c6: tuple             # (lo, hi) of the uniform C6 draw
    a: float              # local cutoff
    h: float              # requested finest-grid spacing
    levels: int
    seed: int
    dmin: float = 0.8


def _cube(L):
    return ((0.0, L), (0.0, L), (0.0, L))


def workload(name: str) -> Workload:
    """The named workloads.

    ``cube1000``     N=1000 in a periodic cube L=10 (rho=1), C6 in [0.5,1.5],
                     a=2.5, h=1, 3 levels (FP64 parity case).
    ``slab65536``    N=65,536 liquid slab, rho=0.8, 40x40x51.2 slab centred in
                     a periodic 40x40x120 box, C6 in [0.8,1.2], a=3, h=1.25,
                     4 levels (top grid 4x4x12).
    ``cube1m``       N=1,048,576 uniform fluid at rho=0.85 in a periodic cube,
                     C6 in [0.5,1.5], a=3, h=1, 5 levels.
    ``slab4m``       N=4,194,304 liquid slab at rho=0.8 in a periodic
                     160x160x240 box, centred, N/(rho 160^2) = 204.8 thick (N and
                     rho fixed), C6 in [0.5,1.5]; a=3 and the coarse grid of the
                     learned correction, h=2, 5 levels (the automatic rule:
                     80x80x128 finest grid).
    """
    if name == "cube1000":
        return Workload(name, 1000, (10.0, 10.0, 10.0), _cube(10.0), (0.5, 1.5), 2.5, 1.0, 3,
                        SEED_BASE + 0)
    if name == "slab65536":
        N, rho, Lx, Lz = 65536, 0.8, 40.0, 120.0
        t = N / (rho * Lx * Lx)
        z0 = 0.5 * (Lz - t)
        return Workload(name, N, (Lx, Lx, Lz), ((0.0, Lx), (0.0, Lx), (z0, z0 + t)), (0.8, 1.2),
                        3.0, 1.25, 4, SEED_BASE + 1)
    if name == "cube1m":
        N, rho = 1 << 20, 0.85
        L = (N / rho) ** (1.0 / 3.0)
        return Workload(name, N, (L, L, L), _cube(L), (0.5, 1.5), 3.0, 1.0, 5, SEED_BASE + 2)
    if name == "slab4m":
        N, rho, Lx, Lz = 1 << 22, 0.8, 160.0, 240.0
        t = N / (rho * Lx * Lx)
        z0 = 0.5 * (Lz - t)
        return Workload(name, N, (Lx, Lx, Lz), ((0.0, Lx), (0.0, Lx), (z0, z0 + t)), (0.5, 1.5),
                        3.0, 2.0, 5, SEED_BASE + 4)
    raise KeyError(name)


def batch_workloads(B: int = 256, nmin: int = 2048, nmax: int = 65536, rho: float = 0.8,
                    a: float = 2.5, h: float = 1.0, seed: int = SEED_BASE + 3,
                    c6=(0.5, 1.5)) -> list:
    """Independent replicas of uneven size (the batched workload): N drawn
    log-uniform in [nmin, nmax]; even replicas are periodic cubes at density
    rho, odd ones liquid slabs of the 65,536-atom slab's proportions (box
    Lx = Ly, Lz = 3 Lx, slab 0.4267 Lz thick, centred, density rho inside).
    Grid levels are left to the library's automatic rule (levels = 0)."""
    rng = np.random.default_rng(seed)
    sizes = np.floor(np.exp(rng.uniform(math.log(nmin), math.log(nmax), B))).astype(np.int64)
    seeds = rng.integers(1, 2**31 - 1, B)
    out = []
    for r in range(B):
        N = int(sizes[r])
        if r % 2 == 0:
            L = (N / rho) ** (1.0 / 3.0)
            out.append(Workload(f"rep{r}_cube{N}", N, (L, L, L), _cube(L), tuple(c6), a, h, 0,
                                int(seeds[r])))
        else:
            f = 51.2 / 120.0
            Lx = (N / (rho * 3.0 * f)) ** (1.0 / 3.0)
            Lz = 3.0 * Lx
            t = f * Lz
            z0 = 0.5 * (Lz - t)
            out.append(Workload(f"rep{r}_slab{N}", N, (Lx, Lx, Lz),
                                ((0.0, Lx), (0.0, Lx), (z0, z0 + t)), tuple(c6), a, h, 0,
                                int(seeds[r])))
    return out


def generate_batch(ws, processes: int = 0):
    """Concatenated (x[sum N, 3], c[sum N]) and the B+1 row offsets; replicas
    are generated independently (in a spawned process pool if processes>1)."""
    if processes and processes > 1:
        import multiprocessing as mp

        with mp.get_context("spawn").Pool(processes) as pool:
            parts = pool.map(generate, ws)
    else:
        parts = [generate(w) for w in ws]
    off = np.zeros(len(ws) + 1, dtype=np.int64)
    off[1:] = np.cumsum([w.N for w in ws])
    x = np.concatenate([p[0] for p in parts]) if parts else np.zeros((0, 3))
    c = np.concatenate([p[1] for p in parts]) if parts else np.zeros(0)
    return x, c, off


def scaled_cube(N: int, rho: float, a: float, h: float, levels: int, seed: int,
                c6=(0.5, 1.5), dmin: float = 0.8) -> Workload:
    """A uniform periodic cube of N atoms at density rho."""
    L = (N / rho) ** (1.0 / 3.0)
    return Workload(f"cube{N}", N, (L, L, L), _cube(L), tuple(c6), a, h, levels, seed, dmin)


def rsa_positions(rng: np.random.Generator, N: int, region, box, dmin: float) -> np.ndarray:
    """N points in the axis-aligned ``region`` with pairwise periodic
    separation >= dmin (periodic in ``box``)."""
    from scipy.spatial import cKDTree

    lo = np.array([r[0] for r in region], dtype=np.float64)
    hi = np.array([r[1] for r in region], dtype=np.float64)
    boxv = np.asarray(box, dtype=np.float64)
    acc = np.zeros((0, 3))
    stall = 0
    while acc.shape[0] < N:
        need = N - acc.shape[0]
        m = max(2 * need, 65536)
        cand = lo + (hi - lo) * rng.random((m, 3))
        cand = np.mod(cand, boxv)
        if acc.shape[0]:
            d, _ = cKDTree(acc, boxsize=boxv).query(cand, k=1, distance_upper_bound=dmin,
                                                     workers=-1)
            cand = cand[~(d < dmin)]
        if cand.shape[0]:
            pairs = _close_pairs(cand, boxv, dmin)
            keep = _greedy_in_order(cand.shape[0], pairs)
            cand = cand[keep][:need]
        stall = stall + 1 if cand.shape[0] == 0 else 0
        if stall > 50:
            raise RuntimeError("RSA cannot place more atoms at this density")
        acc = np.concatenate([acc, cand], axis=0)
    return acc


def _close_pairs(pts: np.ndarray, boxv: np.ndarray, dmin: float) -> np.ndarray:
    """All index pairs (i, j), i != j, closer than dmin (periodic)."""
    from scipy.spatial import cKDTree

    tree = cKDTree(pts, boxsize=boxv)
    k = 8
    d, nb = tree.query(pts, k=k, distance_upper_bound=dmin, workers=-1)
    if np.any(d[:, k - 1] < dmin):  # some point has >= k-1 close neighbours
        return tree.query_pairs(dmin, output_type="ndarray")
    src = np.repeat(np.arange(pts.shape[0]), k - 1)
    dst = nb[:, 1:].reshape(-1)
    ok = (d[:, 1:].reshape(-1) < dmin) & (dst != src)
    p = np.stack([src[ok], dst[ok]], axis=1)
    return p[p[:, 0] < p[:, 1]] if p.shape[0] else p.reshape(0, 2)


def _greedy_in_order(m: int, pairs: np.ndarray) -> np.ndarray:
    """Sequential acceptance in draw order for m trial points with the
    conflicting pairs ``pairs``: point j is kept iff no earlier kept point
    conflicts with it.  Resolved in vectorised rounds: a point is rejected
    once an earlier conflicting point is kept, and kept once every earlier
    conflicting point is rejected; the lowest undecided point is always
    decidable, so the rounds terminate."""
    state = np.zeros(m, dtype=np.int8)  # 0 undecided, 1 kept, -1 rejected
    if pairs.shape[0] == 0:
        return np.ones(m, dtype=bool)
    pairs = np.sort(pairs, axis=1)
    i, j = pairs[:, 0], pairs[:, 1]
    while True:
        und = state == 0
        if not und.any():
            break
        rej = np.zeros(m, dtype=bool)
        rej[j[state[i] == 1]] = True
        state[und & rej] = -1
        blocking = np.bincount(j[state[i] != -1], minlength=m)
        state[(state == 0) & (blocking == 0)] = 1
    return state == 1


def coefficients(rng: np.random.Generator, N: int, c6) -> np.ndarray:
    """c_i = sqrt(C6_i) with C6_i ~ U[c6[0], c6[1]]."""
    return np.sqrt(c6[0] + (c6[1] - c6[0]) * rng.random(N))


def generate(w: Workload):
    """(x[N,3] float64, c[N] float64) for a workload, deterministic in w.seed."""
    rng = np.random.default_rng(w.seed)
    x = rsa_positions(rng, w.N, w.region, w.box, w.dmin)
    c = coefficients(rng, w.N, w.c6)
    return x, c


def uniform_atoms(seed: int, N: int, box, dmin: float = 0.8, c6=(0.5, 1.5),
                  region=None):
    """Small RSA systems for parity and pin tests."""
    rng = np.random.default_rng(seed)
    reg = region if region is not None else tuple((0.0, float(L)) for L in box)
    x = rsa_positions(rng, N, reg, box, dmin) if N else np.zeros((0, 3))
    c = coefficients(rng, N, c6)
    return x, c


def lattice_atoms(seed: int, box, nodes, fill: float, c6=(0.5, 1.5)):
    """Atoms on a random subset (fraction ``fill``) of the nodes of a periodic
    nodes[0] x nodes[1] x nodes[2] lattice spanning ``box``."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = (int(v) for v in nodes)
    idx = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"),
                   axis=-1).reshape(-1, 3)
    sel = idx[rng.random(idx.shape[0]) < fill]
    if sel.shape[0] == 0:
        sel = idx[:1]
    x = sel * (np.asarray(box, dtype=np.float64) / np.array([nx, ny, nz]))
    c = coefficients(rng, sel.shape[0], c6)
    return x, c


def c6_mean_sq(c6) -> float:
    """Mean of c^2 = mean C6 (for order-of-magnitude estimates in tests)."""
    return 0.5 * (c6[0] + c6[1])


def cube_side(N: int, rho: float) -> float:
    return (N / rho) ** (1.0 / 3.0) if N else 0.0


__all__ = ["Workload", "workload", "scaled_cube", "rsa_positions", "coefficients", "generate",
           "uniform_atoms", "lattice_atoms", "c6_mean_sq", "cube_side", "SEED_BASE"]

_ = math  # keep the import for users who extend the recipes
