"""ctypes wrapper around the FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).

The oracle is a plain restatement of multilevel summation for r^-6 dispersion
(arXiv 1308.4005, Sec. II); see ``mls6_oracle.h`` for its conventions.  Only
the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this module.  It shares no code with the GPU library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mls6_oracle.c")
_LIB = os.path.join(_HERE, "libmls6_oracle.so")
_lib = None

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_i64p = C.POINTER(C.c_int64)


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/libmls6_oracle.so`` with gcc."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC),
                                              os.path.getmtime(os.path.join(_HERE, "mls6_oracle.h")))):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-D_DEFAULT_SOURCE", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        for name in ("orc_gamma", "orc_dgamma", "orc_Phi", "orc_dPhi"):
            getattr(L, name).restype = C.c_double
            getattr(L, name).argtypes = [C.c_double]
        for name in ("orc_gk", "orc_dgk"):
            getattr(L, name).restype = C.c_double
            getattr(L, name).argtypes = [C.c_int, C.c_int, C.c_double, C.c_double]
        L.orc_grid_dims.restype = C.c_int
        L.orc_grid_dims.argtypes = [_dp, C.c_double, C.c_int, _ip]
        L.orc_eval.restype = C.c_int
        L.orc_eval.argtypes = [_dp, C.c_double, _ip, C.c_int, C.c_double, C.c_int64, _dp, _dp,
                               _dp, _dp, _dp, _dp, _dp]
        L.orc_eval_sample.restype = C.c_int
        L.orc_eval_sample.argtypes = [_dp, C.c_double, _ip, C.c_int, C.c_double, C.c_int64, _dp,
                                      _dp, C.c_int64, _i64p, _dp, _dp, _dp]
        L.orc_local.restype = C.c_int
        L.orc_local.argtypes = [_dp, C.c_double, C.c_int64, _dp, _dp, C.c_int64, _i64p, _dp, _dp]
        for name in ("orc_local_cells", "orc_local_allpairs"):
            getattr(L, name).restype = C.c_int
            getattr(L, name).argtypes = [_dp, C.c_double, C.c_int64, _dp, _dp, C.c_int64, _i64p,
                                         _dp, _dp, _dp]
        L.orc_grids.restype = C.c_int
        L.orc_grids.argtypes = [_dp, C.c_double, _ip, C.c_int, C.c_double, C.c_int64, _dp, _dp, _dp]
        L.orc_top_table.restype = C.c_int
        L.orc_top_table.argtypes = [_dp, C.c_double, _ip, C.c_int, C.c_double, _dp, _dp]
        L.orc_brute.restype = C.c_int
        L.orc_brute.argtypes = [_dp, C.c_double, C.c_int64, _dp, _dp, _dp, _dp, _dp]
        L.orc_set_smoothing.restype = None
        L.orc_set_smoothing.argtypes = [C.c_int]
        L.orc_get_smoothing.restype = C.c_int
        L.orc_get_smoothing.argtypes = []
        L.orc_set_order.restype = None
        L.orc_set_order.argtypes = [C.c_int]
        L.orc_get_order.restype = C.c_int
        L.orc_get_order.argtypes = []
        L.orc_set_threads.restype = None
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_get_threads.restype = C.c_int
        L.orc_get_threads.argtypes = []
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _cell(box):
    box = np.asarray(box, dtype=np.float64)
    if box.shape == (3,):
        return np.ascontiguousarray(np.diag(box))
    assert box.shape == (3, 3)
    return np.ascontiguousarray(box)


def _atoms(x, c):
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1, 3))
    c = np.ascontiguousarray(np.asarray(c, dtype=np.float64).reshape(-1))
    assert x.shape[0] == c.shape[0]
    return x, c


def set_smoothing(n: int) -> None:
    """Continuity C^n (1..4) of the smoothing function gamma (2 = Eq. gamma)."""
    lib().orc_set_smoothing(int(n))


def smoothing() -> int:
    return int(lib().orc_get_smoothing())


class smoothing_order:
    """Context manager: evaluate with the C^n smoothing function."""

    def __init__(self, n):
        self.n = n

    def __enter__(self):
        self.old = smoothing()
        set_smoothing(self.n)
        return self

    def __exit__(self, *exc):
        set_smoothing(self.old)


def set_order(p: int) -> None:
    """Interpolation order p of the nodal basis: 3 (Eq. Phi-Hermite) or 5
    (the C^1 quintic)."""
    lib().orc_set_order(int(p))


def order() -> int:
    return int(lib().orc_get_order())


class interp_order:
    """Context manager: evaluate with the order-p nodal basis."""

    def __init__(self, p):
        self.p = p

    def __enter__(self):
        self.old = order()
        set_order(self.p)
        return self

    def __exit__(self, *exc):
        set_order(self.old)


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def threads() -> int:
    return int(lib().orc_get_threads())


def gamma(rho):
    return lib().orc_gamma(float(rho))


def dgamma(rho):
    return lib().orc_dgamma(float(rho))


def gk(k, l, a, r):
    return lib().orc_gk(int(k), int(l), float(a), float(r))


def dgk(k, l, a, r):
    return lib().orc_dgk(int(k), int(l), float(a), float(r))


def Phi(t):
    return lib().orc_Phi(float(t))


def dPhi(t):
    return lib().orc_dPhi(float(t))


def grid_dims(L, h, levels):
    Lv = np.ascontiguousarray(np.asarray(L, dtype=np.float64))
    n = (C.c_int * 3)()
    rc = lib().orc_grid_dims(_d(Lv), float(h), int(levels), n)
    if rc:
        raise ValueError(f"orc_grid_dims failed ({rc})")
    return tuple(int(v) for v in n)


def evaluate(box, a, n, levels, x, c, r_img=0.0):
    """Full MLS.  Returns dict(E, F, W, eatom, level_energy)."""
    H = _cell(box)
    x, c = _atoms(x, c)
    N = x.shape[0]
    nn = (C.c_int * 3)(*[int(v) for v in n])
    E = np.zeros(1)
    F = np.zeros((N, 3))
    W = np.zeros(6)
    ea = np.zeros(N)
    le = np.zeros(levels + 3)
    rc = lib().orc_eval(_d(H), float(a), nn, int(levels), float(r_img), N, _d(x), _d(c), _d(E),
                        _d(F), _d(W), _d(ea), _d(le))
    if rc:
        raise ValueError(f"orc_eval failed ({rc})")
    return dict(E=float(E[0]), F=F, W=W, eatom=ea, level_energy=le)


def evaluate_sample(box, a, n, levels, x, c, idx, r_img=0.0):
    """MLS forces / per-atom energies for the atoms in idx (any N)."""
    H = _cell(box)
    x, c = _atoms(x, c)
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    nn = (C.c_int * 3)(*[int(v) for v in n])
    F = np.zeros((idx.size, 3))
    ea = np.zeros(idx.size)
    eg = np.zeros(1)
    rc = lib().orc_eval_sample(_d(H), float(a), nn, int(levels), float(r_img), x.shape[0], _d(x),
                               _d(c), idx.size, idx.ctypes.data_as(_i64p), _d(F), _d(ea), _d(eg))
    if rc:
        raise ValueError(f"orc_eval_sample failed ({rc})")
    return dict(F=F, eatom=ea, grid_energy=float(eg[0]))


def local(box, a, x, c, idx):
    """Local part (Eq. g_0) for the atoms in idx: (e0, F)."""
    H = _cell(box)
    x, c = _atoms(x, c)
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    e0 = np.zeros(idx.size)
    F = np.zeros((idx.size, 3))
    rc = lib().orc_local(_d(H), float(a), x.shape[0], _d(x), _d(c), idx.size,
                         idx.ctypes.data_as(_i64p), _d(e0), _d(F))
    if rc:
        raise ValueError(f"orc_local failed ({rc})")
    return e0, F


def local_forms(box, a, x, c, idx, form):
    """Local part for the atoms in idx by one loop form ("cells": linked
    cells, "allpairs": all atoms x all images): (e0, F, W per atom)."""
    H = _cell(box)
    x, c = _atoms(x, c)
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    e0 = np.zeros(idx.size)
    F = np.zeros((idx.size, 3))
    W = np.zeros((idx.size, 6))
    fn = {"cells": lib().orc_local_cells, "allpairs": lib().orc_local_allpairs}[form]
    rc = fn(_d(H), float(a), x.shape[0], _d(x), _d(c), idx.size, idx.ctypes.data_as(_i64p),
            _d(e0), _d(F), _d(W))
    if rc:
        raise ValueError(f"orc_local_{form} failed ({rc})")
    return e0, F, W


def grids(box, a, n, levels, x, c, r_img=0.0):
    """Per-level (q^k, e^k, e^{k,tot}) arrays, each shaped (nz, ny, nx)."""
    H = _cell(box)
    x, c = _atoms(x, c)
    dims = [tuple(int(v) // (1 << (k - 1)) for v in n) for k in range(1, levels + 1)]
    tot = sum(3 * d[0] * d[1] * d[2] for d in dims)
    out = np.zeros(tot)
    nn = (C.c_int * 3)(*[int(v) for v in n])
    rc = lib().orc_grids(_d(H), float(a), nn, int(levels), float(r_img), x.shape[0], _d(x),
                         _d(c), _d(out))
    if rc:
        raise ValueError(f"orc_grids failed ({rc})")
    res, off = [], 0
    for d in dims:
        npk = d[0] * d[1] * d[2]
        shp = (d[2], d[1], d[0])
        res.append(tuple(out[off + i * npk: off + (i + 1) * npk].reshape(shp) for i in range(3)))
        off += 3 * npk
    return res


def top_table(box, a, nl, levels, r_img=0.0):
    H = _cell(box)
    npk = int(nl[0]) * int(nl[1]) * int(nl[2])
    T = np.zeros(npk)
    V = np.zeros(6 * npk)
    nn = (C.c_int * 3)(*[int(v) for v in nl])
    rc = lib().orc_top_table(_d(H), float(a), nn, int(levels), float(r_img), _d(T), _d(V))
    if rc:
        raise ValueError(f"orc_top_table failed ({rc})")
    return T, V.reshape(6, npk)


def brute(box, x, c, r_img):
    """Exact periodic sum (direct images to r_img + continuum tail)."""
    H = _cell(box)
    x, c = _atoms(x, c)
    N = x.shape[0]
    E = np.zeros(1)
    F = np.zeros((N, 3))
    W = np.zeros(6)
    rc = lib().orc_brute(_d(H), float(r_img), N, _d(x), _d(c), _d(E), _d(F), _d(W))
    if rc:
        raise ValueError(f"orc_brute failed ({rc})")
    return dict(E=float(E[0]), F=F, W=W)
