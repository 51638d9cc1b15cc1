"""Thin ctypes binding of ``libmls6.so`` (see ``include/mls6.h``).

The functions carry the C-ABI names and only marshal arguments; every step of
an evaluation runs in the library's CUDA kernels.  Device buffers are passed
as raw pointers (``tensor.data_ptr()``); PyTorch is used by callers only for
device memory and streams.  If the library is missing or fails to load,
``load()`` raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmls6.so")

MLS6_OK = 0
MLS6_ERR_ARG = -1
MLS6_ERR_GRID = -2
MLS6_ERR_BOX = -3
MLS6_ERR_ORDER = -4
MLS6_ERR_CUDA = -5
MLS6_ERR_NOMEM = -6
MLS6_ERR_TIMEOUT = -7
MLS6_ERR_NONFINITE = -8
MLS6_ERR_SIZE = -9

MLS6_FP64 = 0
MLS6_FP32 = 1
MLS6_MIXED = 2
_PREC = {"fp64": MLS6_FP64, "fp32": MLS6_FP32, "mixed": MLS6_MIXED,
         MLS6_FP64: MLS6_FP64, MLS6_FP32: MLS6_FP32, MLS6_MIXED: MLS6_MIXED}

# every symbol declared in include/mls6.h
EXPORTS = ("mls6_grid_dims", "mls6_coarse_tables", "mls6_plan", "mls6_plan_ex",
           "mls6_set_stream",
           "mls6_set_graph", "mls6_eval",
           "mls6_eval_atoms", "mls6_eval_lb", "mls6_last_error", "mls6_plan_info", "mls6_debug_grid",
           "mls6_profile", "mls6_stage_times", "mls6_stage_name", "mls6_auto_levels",
           "mls6_set_tuning", "mls6_get_tuning", "mls6_stencil_kind", "mls6_cost_model", "mls6_lpt_assign",
           "mls6_batch_plan", "mls6_batch_set_stream", "mls6_batch_eval", "mls6_batch_tune",
           "mls6_batch_set_config", "mls6_batch_info", "mls6_batch_size", "mls6_batch_replica",
           "mls6_batch_destroy", "mls6_batch_set_mode", "mls6_batch_mode", "mls6_batch_set_wait",
           "mls6_batch_last_error",
           "mls6_mlp_n_params", "mls6_mlp_create", "mls6_mlp_set_stream", "mls6_mlp_get_params",
           "mls6_mlp_set_params", "mls6_mlp_set_norm", "mls6_mlp_features", "mls6_mlp_forward",
           "mls6_mlp_grad", "mls6_mlp_train_step", "mls6_mlp_apply", "mls6_mlp_destroy",
           "mls6_coarse_apply_noalloc", "mls6_fma_peak", "mls6_destroy", "mls6_status_string")

_lib = None
_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class MLS6Error(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        msg = status_string(code) if _lib is not None else str(code)
        super().__init__(f"{where}: {msg} ({code})" if where else f"{msg} ({code})")


def load(path: str = LIB_PATH):
    """Load the in-tree library (raises if it is absent)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: run paper_1308_4005_gb300/build.py "
                           "(the library has no CPU fallback)")
    L = C.CDLL(path)
    L.mls6_grid_dims.argtypes = [_dp, C.c_double, C.c_int, _ip]
    L.mls6_grid_dims.restype = C.c_int
    L.mls6_coarse_tables.argtypes = [_dp, _ip, C.c_int, C.c_double, _dp, _dp]
    L.mls6_coarse_tables.restype = C.c_int
    L.mls6_plan.argtypes = [C.POINTER(C.c_void_p), _dp, C.c_int64, C.c_double, C.c_double,
                            C.c_int, C.c_int, C.c_int]
    L.mls6_plan.restype = C.c_int
    L.mls6_plan_ex.argtypes = [C.POINTER(C.c_void_p), _dp, C.c_int64, C.c_double, C.c_double,
                               C.c_int, C.c_int, C.c_int, C.POINTER(PlanOptions)]
    L.mls6_plan_ex.restype = C.c_int
    L.mls6_set_stream.argtypes = [C.c_void_p, C.c_void_p]
    L.mls6_set_stream.restype = C.c_int
    L.mls6_set_graph.argtypes = [C.c_void_p, C.c_int]
    L.mls6_set_graph.restype = C.c_int
    L.mls6_eval.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                            C.c_void_p]
    L.mls6_eval.restype = C.c_int
    L.mls6_eval_atoms.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p]
    L.mls6_eval_atoms.restype = C.c_int
    L.mls6_eval_lb.argtypes = [C.c_void_p] * 6
    L.mls6_eval_lb.restype = C.c_int
    L.mls6_last_error.argtypes = [C.c_void_p]
    L.mls6_last_error.restype = C.c_int
    L.mls6_plan_info.argtypes = [C.c_void_p, _ip, _dp, _ip, _ip]
    L.mls6_plan_info.restype = C.c_int
    L.mls6_debug_grid.argtypes = [C.c_void_p, C.c_int, C.c_int, _dp]
    L.mls6_debug_grid.restype = C.c_int
    L.mls6_profile.argtypes = [C.c_void_p, C.c_int]
    L.mls6_profile.restype = C.c_int
    L.mls6_stage_times.argtypes = [C.c_void_p, _dp, C.c_int, _ip]
    L.mls6_stage_times.restype = C.c_int
    L.mls6_stage_name.argtypes = [C.c_int]
    L.mls6_stage_name.restype = C.c_char_p
    L.mls6_coarse_apply_noalloc.argtypes = [C.c_void_p, _ip, C.c_void_p, C.c_void_p, C.c_void_p,
                                            C.c_void_p, C.c_void_p]
    L.mls6_coarse_apply_noalloc.restype = C.c_int
    L.mls6_fma_peak.argtypes = [C.c_int, _dp]
    L.mls6_fma_peak.restype = C.c_int
    L.mls6_destroy.argtypes = [C.c_void_p]
    L.mls6_destroy.restype = None
    L.mls6_auto_levels.argtypes = [_dp, C.c_double]
    L.mls6_auto_levels.restype = C.c_int
    L.mls6_set_tuning.argtypes = [C.c_void_p, C.c_int, C.c_int]
    L.mls6_set_tuning.restype = C.c_int
    L.mls6_stencil_kind.argtypes = [C.c_void_p]
    L.mls6_stencil_kind.restype = C.c_int
    L.mls6_get_tuning.argtypes = [C.c_void_p, _ip, _ip]
    L.mls6_get_tuning.restype = C.c_int
    L.mls6_cost_model.argtypes = [_dp, C.c_int64, C.c_double, C.c_double, C.c_int, _dp, _dp]
    L.mls6_cost_model.restype = C.c_int
    L.mls6_lpt_assign.argtypes = [C.c_int, _dp, C.c_int, _ip, _dp]
    L.mls6_lpt_assign.restype = C.c_int
    L.mls6_batch_plan.argtypes = [C.POINTER(C.c_void_p), C.c_int, _dp, C.POINTER(C.c_int64),
                                  C.c_double, C.c_double, C.c_int, C.c_int, C.c_int]
    L.mls6_batch_plan.restype = C.c_int
    L.mls6_batch_set_stream.argtypes = [C.c_void_p, C.c_void_p]
    L.mls6_batch_set_stream.restype = C.c_int
    L.mls6_batch_eval.argtypes = [C.c_void_p] * 6
    L.mls6_batch_eval.restype = C.c_int
    L.mls6_batch_tune.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, _dp]
    L.mls6_batch_tune.restype = C.c_int
    L.mls6_batch_set_config.argtypes = [C.c_void_p, C.c_int, _ip, _ip]
    L.mls6_batch_set_config.restype = C.c_int
    L.mls6_batch_info.argtypes = [C.c_void_p, _ip, _ip, _ip, _ip, _dp, _ip, _ip]
    L.mls6_batch_info.restype = C.c_int
    L.mls6_batch_size.argtypes = [C.c_void_p, _ip, C.POINTER(C.c_int64)]
    L.mls6_batch_size.restype = C.c_int
    L.mls6_batch_replica.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_void_p)]
    L.mls6_batch_replica.restype = C.c_int
    _fp = C.POINTER(C.c_float)
    L.mls6_mlp_n_params.argtypes = []
    L.mls6_mlp_n_params.restype = C.c_int
    L.mls6_mlp_create.argtypes = [C.POINTER(C.c_void_p), C.c_uint64]
    L.mls6_mlp_set_stream.argtypes = [C.c_void_p, C.c_void_p]
    L.mls6_mlp_get_params.argtypes = [C.c_void_p, _fp, C.c_int]
    L.mls6_mlp_set_params.argtypes = [C.c_void_p, _fp, C.c_int]
    L.mls6_mlp_set_norm.argtypes = [C.c_void_p, _fp, _fp, C.c_float]
    L.mls6_mlp_features.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
    L.mls6_mlp_forward.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]
    L.mls6_mlp_grad.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, _dp]
    L.mls6_mlp_train_step.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_float,
                                      _dp]
    L.mls6_mlp_apply.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    for fn in ("mls6_mlp_create", "mls6_mlp_set_stream", "mls6_mlp_get_params",
               "mls6_mlp_set_params", "mls6_mlp_set_norm", "mls6_mlp_features",
               "mls6_mlp_forward", "mls6_mlp_grad", "mls6_mlp_train_step", "mls6_mlp_apply"):
        getattr(L, fn).restype = C.c_int
    L.mls6_mlp_destroy.argtypes = [C.c_void_p]
    L.mls6_mlp_destroy.restype = None
    L.mls6_batch_set_mode.argtypes = [C.c_void_p, C.c_int]
    L.mls6_batch_set_mode.restype = C.c_int
    L.mls6_batch_mode.argtypes = [C.c_void_p]
    L.mls6_batch_mode.restype = C.c_int
    L.mls6_batch_set_wait.argtypes = [C.c_void_p, C.c_longlong, C.c_longlong]
    L.mls6_batch_set_wait.restype = C.c_int
    L.mls6_batch_last_error.argtypes = [C.c_void_p]
    L.mls6_batch_last_error.restype = C.c_int
    L.mls6_batch_destroy.argtypes = [C.c_void_p]
    L.mls6_batch_destroy.restype = None
    L.mls6_status_string.argtypes = [C.c_int]
    L.mls6_status_string.restype = C.c_char_p
    _lib = L
    return L


def _check(rc, where):
    if rc != MLS6_OK:
        raise MLS6Error(rc, where)


def _darr(vals):
    return (C.c_double * len(vals))(*[float(v) for v in vals])


def mls6_fma_peak(precision):
    """Measured FMA rate of the current device in TFLOP/s."""
    v = C.c_double()
    _check(load().mls6_fma_peak(_PREC[precision], C.byref(v)), "mls6_fma_peak")
    return v.value


def status_string(code: int) -> str:
    return load().mls6_status_string(int(code)).decode()


def mls6_grid_dims(box, h, levels):
    n = (C.c_int * 3)()
    _check(load().mls6_grid_dims(_darr(box), float(h), int(levels), n), "mls6_grid_dims")
    return tuple(n)


def mls6_coarse_tables(box, nl, levels, a):
    import numpy as np

    npk = int(nl[0]) * int(nl[1]) * int(nl[2])
    T = np.zeros(npk)
    V = np.zeros(6 * npk)
    nn = (C.c_int * 3)(*[int(v) for v in nl])
    _check(load().mls6_coarse_tables(_darr(box), nn, int(levels), float(a),
                                     T.ctypes.data_as(_dp), V.ctypes.data_as(_dp)),
           "mls6_coarse_tables")
    return T, V.reshape(6, npk)


def mls6_plan(box, N, a, h, levels, order=3, precision=MLS6_FP64):
    """Returns an opaque plan handle (int)."""
    out = C.c_void_p()
    _check(load().mls6_plan(C.byref(out), _darr(box), int(N), float(a), float(h), int(levels),
                            int(order), int(precision)), "mls6_plan")
    return out.value


class PlanOptions(C.Structure):
    """mls6_plan_options: continuity (0 = 2), stencil (0 auto, 1 CUDA cores,
    2 tcgen05 tensor cores; mixed precision only)."""
    _fields_ = [("continuity", C.c_int), ("stencil", C.c_int)]


_STENCIL = {"auto": 0, "cuda": 1, "tensor": 2, 0: 0, 1: 1, 2: 2}


def mls6_plan_ex(box, N, a, h, levels, order=3, precision=MLS6_FP64, continuity=2,
                 stencil="auto"):
    """As mls6_plan with options (smoothing continuity, stencil kernel)."""
    out = C.c_void_p()
    opt = PlanOptions(int(continuity), _STENCIL[stencil])
    _check(load().mls6_plan_ex(C.byref(out), _darr(box), int(N), float(a), float(h),
                               int(levels), int(order), int(precision), C.byref(opt)),
           "mls6_plan_ex")
    return out.value


def mls6_set_stream(plan, stream_handle):
    _check(load().mls6_set_stream(C.c_void_p(plan), C.c_void_p(stream_handle or 0)),
           "mls6_set_stream")


def mls6_set_graph(plan, enable=True):
    _check(load().mls6_set_graph(C.c_void_p(plan), int(bool(enable))), "mls6_set_graph")


def mls6_eval(plan, pos_ptr, c_ptr, forces_ptr, energy_ptr, virial_ptr):
    """All pointers are integers (0 = NULL); energy/virial may be host or
    device addresses."""
    return load().mls6_eval(C.c_void_p(plan), C.c_void_p(pos_ptr or None),
                            C.c_void_p(c_ptr or None), C.c_void_p(forces_ptr or None),
                            C.c_void_p(energy_ptr or None), C.c_void_p(virial_ptr or None))


def mls6_eval_atoms(plan, pos_ptr, c_ptr, forces_ptr, energy_ptr, virial_ptr, atom_energy_ptr):
    return load().mls6_eval_atoms(C.c_void_p(plan), C.c_void_p(pos_ptr or None),
                                  C.c_void_p(c_ptr or None), C.c_void_p(forces_ptr or None),
                                  C.c_void_p(energy_ptr or None), C.c_void_p(virial_ptr or None),
                                  C.c_void_p(atom_energy_ptr or None))


def mls6_eval_lb(plan, pos_ptr, sigma_ptr, eps_ptr, forces_ptr, energy_ptr):
    return load().mls6_eval_lb(C.c_void_p(plan), C.c_void_p(pos_ptr), C.c_void_p(sigma_ptr),
                               C.c_void_p(eps_ptr), C.c_void_p(forces_ptr),
                               C.c_void_p(energy_ptr))


def mls6_last_error(plan):
    return load().mls6_last_error(C.c_void_p(plan))


def mls6_plan_info(plan):
    L = load()
    lev = C.c_int()
    nt = C.c_int()
    _check(L.mls6_plan_info(C.c_void_p(plan), None, None, C.byref(lev), C.byref(nt)),
           "mls6_plan_info")
    ng = (C.c_int * (3 * lev.value))()
    h = (C.c_double * 3)()
    _check(L.mls6_plan_info(C.c_void_p(plan), ng, h, None, None), "mls6_plan_info")
    dims = [tuple(ng[3 * k: 3 * k + 3]) for k in range(lev.value)]
    return dict(levels=lev.value, n_grid=dims, h=tuple(h), ntaps=nt.value,
                stencil_kind=L.mls6_stencil_kind(C.c_void_p(plan)))


def mls6_debug_grid(plan, level, which):
    """Returns the grid as a numpy array shaped (nz, ny, nx)."""
    import numpy as np

    info = mls6_plan_info(plan)
    n = info["n_grid"][level - 1]
    out = np.zeros(n[0] * n[1] * n[2])
    _check(load().mls6_debug_grid(C.c_void_p(plan), int(level), int(which),
                                  out.ctypes.data_as(_dp)), "mls6_debug_grid")
    return out.reshape(n[2], n[1], n[0])


def mls6_profile(plan, enable=True):
    _check(load().mls6_profile(C.c_void_p(plan), int(bool(enable))), "mls6_profile")


def mls6_stage_times(plan):
    """(dict stage -> ms of the last profiled evaluation, kernels launched)."""
    ms = (C.c_double * 16)()
    nl = C.c_int()
    n = load().mls6_stage_times(C.c_void_p(plan), ms, 16, C.byref(nl))
    if n < 0:
        raise MLS6Error(n, "mls6_stage_times")
    return {mls6_stage_name(i): ms[i] for i in range(n)}, nl.value


def mls6_stage_name(i):
    s = load().mls6_stage_name(int(i))
    return s.decode() if s else None


def mls6_destroy(plan):
    if plan:
        load().mls6_destroy(C.c_void_p(plan))


def mls6_auto_levels(box, h):
    rc = load().mls6_auto_levels(_darr(box), h)
    if rc < 0:
        _check(rc, "mls6_auto_levels")
    return rc


def mls6_set_tuning(plan, pair_split=0, stencil_groups=0):
    _check(load().mls6_set_tuning(C.c_void_p(plan), pair_split, stencil_groups),
           "mls6_set_tuning")


def mls6_stencil_kind(plan):
    return load().mls6_stencil_kind(C.c_void_p(plan))


def mls6_get_tuning(plan):
    s, g = C.c_int(), C.c_int()
    _check(load().mls6_get_tuning(C.c_void_p(plan), C.byref(s), C.byref(g)), "mls6_get_tuning")
    return s.value, g.value


def mls6_cost_model(box, N, a, h, levels, coef=None):
    out = C.c_double()
    cf = _darr(coef) if coef is not None else None
    _check(load().mls6_cost_model(_darr(box), int(N), a, h, levels, cf, C.byref(out)),
           "mls6_cost_model")
    return out.value


def mls6_lpt_assign(cost, K):
    B = len(cost)
    br = (C.c_int * max(B, 1))()
    load_ = (C.c_double * K)()
    _check(load().mls6_lpt_assign(B, _darr(cost) if B else None, K, br, load_),
           "mls6_lpt_assign")
    return list(br)[:B], list(load_)


def mls6_batch_plan(boxes, N, a, h, levels=0, order=3, precision=MLS6_FP64):
    B = len(N)
    flat = [float(v) for b in boxes for v in b]
    handle = C.c_void_p()
    n64 = (C.c_int64 * B)(*[int(n) for n in N])
    _check(load().mls6_batch_plan(C.byref(handle), B, _darr(flat), n64, a, h, levels, order,
                                  precision), "mls6_batch_plan")
    return handle.value


def mls6_batch_set_stream(batch, stream_handle):
    _check(load().mls6_batch_set_stream(C.c_void_p(batch), C.c_void_p(stream_handle)),
           "mls6_batch_set_stream")


def mls6_batch_eval(batch, pos_ptr, c_ptr, forces_ptr, energy_ptr, virial_ptr):
    return load().mls6_batch_eval(C.c_void_p(batch), C.c_void_p(pos_ptr), C.c_void_p(c_ptr),
                                  C.c_void_p(forces_ptr), C.c_void_p(energy_ptr),
                                  C.c_void_p(virial_ptr))


def mls6_batch_tune(batch, pos_ptr, c_ptr, forces_ptr, reps=5):
    best = C.c_double()
    _check(load().mls6_batch_tune(C.c_void_p(batch), C.c_void_p(pos_ptr), C.c_void_p(c_ptr),
                                  C.c_void_p(forces_ptr), reps, C.byref(best)),
           "mls6_batch_tune")
    return best.value


def mls6_batch_set_config(batch, branches=0, pair_split=None, stencil_groups=None):
    sp = (C.c_int * len(pair_split))(*pair_split) if pair_split is not None else None
    sg = (C.c_int * len(stencil_groups))(*stencil_groups) if stencil_groups is not None else None
    _check(load().mls6_batch_set_config(C.c_void_p(batch), branches, sp, sg),
           "mls6_batch_set_config")


def mls6_batch_size(batch):
    B = C.c_int()
    _check(load().mls6_batch_size(C.c_void_p(batch), C.byref(B), None), "mls6_batch_size")
    off = (C.c_int64 * (B.value + 1))()
    _check(load().mls6_batch_size(C.c_void_p(batch), None, off), "mls6_batch_size")
    return B.value, list(off)


def mls6_batch_info(batch):
    B, _ = mls6_batch_size(batch)
    K, nl = C.c_int(), C.c_int()
    sp, sg, br, lv = ((C.c_int * B)() for _ in range(4))
    cost = (C.c_double * B)()
    _check(load().mls6_batch_info(C.c_void_p(batch), C.byref(K), sp, sg, br, cost, lv,
                                  C.byref(nl)), "mls6_batch_info")
    return dict(branches=K.value, pair_split=list(sp), stencil_groups=list(sg),
                branch_of=list(br), cost=list(cost), levels=list(lv), launches=nl.value)


def mls6_batch_replica(batch, r):
    h = C.c_void_p()
    _check(load().mls6_batch_replica(C.c_void_p(batch), r, C.byref(h)), "mls6_batch_replica")
    return h.value


def mls6_batch_set_mode(batch, persistent=True):
    _check(load().mls6_batch_set_mode(C.c_void_p(batch), 1 if persistent else 0),
           "mls6_batch_set_mode")


def mls6_batch_mode(batch):
    return int(load().mls6_batch_mode(C.c_void_p(batch)))


def mls6_batch_set_wait(batch, limit=1 << 22, withhold=-1):
    _check(load().mls6_batch_set_wait(C.c_void_p(batch), int(limit), int(withhold)),
           "mls6_batch_set_wait")


def mls6_batch_last_error(batch):
    return int(load().mls6_batch_last_error(C.c_void_p(batch)))


def mls6_batch_destroy(batch):
    if batch:
        load().mls6_batch_destroy(C.c_void_p(batch))


class Plan:
    """Owns one ``mls6_plan_t``; evaluates torch CUDA tensors in place.

    ``evaluate(pos, c=None)`` takes a CUDA tensor of shape (N, 4) (x, y, z, c)
    or (N, 3) plus c (N,), of the plan's dtype, and returns (E, F, W) with
    F a new (N, 3) CUDA tensor.  Only marshalling happens here.
    """

    def __init__(self, box, N, a, h, levels, precision="fp64", order=3, stream=None,
                 continuity=2, stencil="auto"):
        self.precision = _PREC[precision]
        if continuity == 2 and stencil == "auto":
            self.handle = mls6_plan(box, N, a, h, levels, order, self.precision)
        else:
            self.handle = mls6_plan_ex(box, N, a, h, levels, order, self.precision, continuity,
                                       stencil)
        self.N = int(N)
        self.box = tuple(float(v) for v in box)
        if stream is not None:
            mls6_set_stream(self.handle, stream)

    @property
    def dtype(self):
        import torch

        return torch.float64 if self.precision == MLS6_FP64 else torch.float32

    def info(self):
        return mls6_plan_info(self.handle)

    def evaluate(self, pos, c=None, virial=True, atom_energy=False, forces=None):
        import torch

        dev = pos.device
        F = forces if forces is not None else torch.empty((self.N, 3), dtype=self.dtype,
                                                          device=dev)
        out = torch.zeros(7, dtype=torch.float64, device=dev)
        ea = torch.empty(self.N, dtype=torch.float64, device=dev) if atom_energy else None
        vp = out.data_ptr() + 8 if virial else 0
        if ea is not None:
            rc = mls6_eval_atoms(self.handle, pos.data_ptr(), c.data_ptr() if c is not None else 0,
                                 F.data_ptr(), out.data_ptr(), vp, ea.data_ptr())
        else:
            rc = mls6_eval(self.handle, pos.data_ptr(), c.data_ptr() if c is not None else 0,
                           F.data_ptr(), out.data_ptr(), vp)
        _check(rc, "mls6_eval")
        res = dict(out=out, F=F)
        if ea is not None:
            res["eatom"] = ea
        return res

    def close(self):
        if getattr(self, "handle", None):
            mls6_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Owns one ``mls6_batch_t``: B replicas evaluated by one graph launch.

    ``evaluate(pos, c=None)`` takes the concatenated (sum N, 4) or (sum N, 3)
    CUDA tensor and returns energies (B,), virials (B, 6) and forces
    (sum N, 3); ``offsets`` gives each replica's first row.
    """

    def __init__(self, boxes, N, a, h, levels=0, precision="fp64", order=3):
        self.precision = _PREC[precision]
        self.handle = mls6_batch_plan(boxes, N, a, h, levels, order, self.precision)
        self.B, self.offsets = mls6_batch_size(self.handle)

    @property
    def dtype(self):
        import torch

        return torch.float64 if self.precision == MLS6_FP64 else torch.float32

    def info(self):
        return mls6_batch_info(self.handle)

    def tune(self, pos, c=None, reps=5):
        import torch

        F = torch.empty((self.offsets[-1], 3), dtype=self.dtype, device=pos.device)
        return mls6_batch_tune(self.handle, pos.data_ptr(),
                               c.data_ptr() if c is not None else 0, F.data_ptr(), reps)

    def evaluate(self, pos, c=None, virial=True, forces=None):
        import torch

        dev = pos.device
        F = forces if forces is not None else torch.empty((self.offsets[-1], 3),
                                                          dtype=self.dtype, device=dev)
        E = torch.zeros(self.B, dtype=torch.float64, device=dev)
        W = torch.zeros((self.B, 6), dtype=torch.float64, device=dev)
        rc = mls6_batch_eval(self.handle, pos.data_ptr(), c.data_ptr() if c is not None else 0,
                             F.data_ptr(), E.data_ptr(), W.data_ptr() if virial else 0)
        _check(rc, "mls6_batch_eval")
        return dict(E=E, W=W, F=F)

    def close(self):
        if getattr(self, "handle", None):
            mls6_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MLP:
    """Owns one ``mls6_mlp_t`` (learned force correction; see mls6.h)."""

    def __init__(self, seed=0):
        L = load()
        h = C.c_void_p()
        _check(L.mls6_mlp_create(C.byref(h), seed), "mls6_mlp_create")
        self.handle = h.value
        self.n_params = L.mls6_mlp_n_params()

    def set_stream(self, stream_handle):
        _check(load().mls6_mlp_set_stream(C.c_void_p(self.handle), C.c_void_p(stream_handle)),
               "mls6_mlp_set_stream")

    def get_params(self):
        import numpy as np

        out = np.zeros(self.n_params, dtype=np.float32)
        _check(load().mls6_mlp_get_params(C.c_void_p(self.handle),
                                          out.ctypes.data_as(C.POINTER(C.c_float)),
                                          self.n_params), "mls6_mlp_get_params")
        return out

    def set_params(self, p):
        import numpy as np

        p = np.ascontiguousarray(np.asarray(p, dtype=np.float32))
        _check(load().mls6_mlp_set_params(C.c_void_p(self.handle),
                                          p.ctypes.data_as(C.POINTER(C.c_float)), p.size),
               "mls6_mlp_set_params")

    def set_norm(self, shift, scale, out_scale):
        import numpy as np

        sh = np.ascontiguousarray(np.asarray(shift, dtype=np.float32))
        sc = np.ascontiguousarray(np.asarray(scale, dtype=np.float32))
        fp = C.POINTER(C.c_float)
        _check(load().mls6_mlp_set_norm(C.c_void_p(self.handle), sh.ctypes.data_as(fp),
                                        sc.ctypes.data_as(fp), float(out_scale)),
               "mls6_mlp_set_norm")

    def features(self, plan, fmt="bf16"):
        import torch

        dt = torch.bfloat16 if fmt == "bf16" else torch.float32
        out = torch.empty((plan.N, 128), dtype=dt, device="cuda")
        _check(load().mls6_mlp_features(C.c_void_p(plan.handle), C.c_void_p(self.handle),
                                        C.c_void_p(out.data_ptr()), 0 if fmt == "bf16" else 1),
               "mls6_mlp_features")
        return out

    def forward(self, X):
        import torch

        Y = torch.empty((X.shape[0], 8), dtype=torch.float32, device=X.device)
        _check(load().mls6_mlp_forward(C.c_void_p(self.handle), C.c_void_p(X.data_ptr()),
                                       X.shape[0], C.c_void_p(Y.data_ptr())), "mls6_mlp_forward")
        return Y

    def grad(self, X, T):
        import torch

        g = torch.empty(self.n_params, dtype=torch.float32, device=X.device)
        loss = C.c_double()
        _check(load().mls6_mlp_grad(C.c_void_p(self.handle), C.c_void_p(X.data_ptr()),
                                    C.c_void_p(T.data_ptr()), X.shape[0],
                                    C.c_void_p(g.data_ptr()), C.byref(loss)), "mls6_mlp_grad")
        return loss.value, g

    def train_step(self, X, T, lr):
        loss = C.c_double()
        _check(load().mls6_mlp_train_step(C.c_void_p(self.handle), C.c_void_p(X.data_ptr()),
                                          C.c_void_p(T.data_ptr()), X.shape[0], float(lr),
                                          C.byref(loss)), "mls6_mlp_train_step")
        return loss.value

    def apply(self, plan, forces):
        _check(load().mls6_mlp_apply(C.c_void_p(plan.handle), C.c_void_p(self.handle),
                                     C.c_void_p(forces.data_ptr())), "mls6_mlp_apply")

    def close(self):
        if getattr(self, "handle", None):
            load().mls6_mlp_destroy(C.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
