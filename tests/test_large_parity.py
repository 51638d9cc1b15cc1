"""Full-size parity: the 1,048,576-atom cube in FP32 and in mixed precision
against a full FP64 oracle evaluation (every atom, total energy, virial and
the energy of every grid level), the fixed-point anterpolation of the FP32
path against its stated resolution, and the global-memory level stencil.

Tolerances are those derived in test_gpu_parity.py (FP32) and test_mixed.py
(split-product tensor-core stencils).  Per-level grid energies
-1/2 q^k . e^k (Sec. II.B, Eq. evaluation) are held to 1e-5 (FP32) and 3e-5
(mixed: each stencil product within 3 * 2^-18 of w q) relative.
"""
import numpy as np
import pytest

from paper_1308_4005_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL32 = dict(E=2e-6, F=1e-4, W=2e-5, eatom=2e-5, level=1e-5)
TOLMIX = dict(E=2e-5, F=1e-4, W=5e-5, eatom=5e-5, level=3e-5)


@pytest.fixture(scope="module")
def cube1m(orc):
    """Inputs (rounded to float) and the FP64 oracle's full evaluation."""
    w = I.workload("cube1m")
    x, c = I.generate(w)
    x = x.astype(np.float32).astype(np.float64)
    c = c.astype(np.float32).astype(np.float64)
    n = orc.grid_dims(w.box, w.h, w.levels)
    o = orc.evaluate(w.box, w.a, n, w.levels, x, c)
    return w, x, c, o


def _gpu(gpu_lib, w, x, c, prec):
    import torch

    plan = gpu_lib.Plan(w.box, w.N, w.a, w.h, w.levels, precision=prec)
    pos = torch.tensor(np.c_[x, c], dtype=torch.float32, device="cuda")
    r = plan.evaluate(pos, virial=True, atom_energy=True)
    torch.cuda.synchronize()
    assert gpu_lib.mls6_last_error(plan.handle) == 0
    out = r["out"].cpu().numpy()
    g = dict(E=out[0], W=out[1:7], F=r["F"].cpu().double().numpy(),
             eatom=r["eatom"].cpu().numpy(), plan=plan)
    # grid energy of every level from the grids the evaluation produced
    g["level"] = np.array([
        -0.5 * np.sum(gpu_lib.mls6_debug_grid(plan.handle, k, 0).astype(np.float64) *
                      gpu_lib.mls6_debug_grid(plan.handle, k, 1))
        for k in range(1, w.levels + 1)])
    return g


def _check(g, o, tol, levels, label):
    rms = np.sqrt(np.mean(np.sum(o["F"] ** 2, axis=1)))
    dE = abs(g["E"] - o["E"]) / abs(o["E"])
    dF = np.abs(g["F"] - o["F"]).max() / rms
    dW = np.abs(g["W"] - o["W"]).max() / np.abs(o["W"]).max()
    dea = np.abs(g["eatom"] - o["eatom"]).max() / np.abs(o["eatom"]).max()
    ref_lv = o["level_energy"][2:levels + 2]
    dlv = np.abs(g["level"] - ref_lv) / np.abs(ref_lv)
    msg = f"{label}: dE={dE:.2e} dF={dF:.2e} dW={dW:.2e} deatom={dea:.2e} dlevel={dlv}"
    print(msg)
    assert dE <= tol["E"], msg
    assert dF <= tol["F"], msg
    assert dW <= tol["W"], msg
    assert dea <= tol["eatom"], msg
    assert np.all(dlv <= tol["level"]), msg
    # the grid energy plus the local and self parts is the total
    assert g["eatom"].sum() == pytest.approx(g["E"], rel=1e-8)


@pytest.mark.slow
def test_cube1m_fp32_full(gpu_lib, cube1m):
    """N=1,048,576 cube at rho=0.85, a=3, h=1 (112^3), 5 levels, FP32 with
    FP64 energy/virial: every atom's force and energy, the total energy, the
    virial and each level's grid energy against the FP64 oracle."""
    w, x, c, o = cube1m
    g = _gpu(gpu_lib, w, x, c, "fp32")
    assert g["plan"].info()["stencil_kind"] == 0
    _check(g, o, TOL32, w.levels, "cube1m/fp32")


@pytest.mark.slow
def test_cube1m_mixed_full(gpu_lib, cube1m):
    """The same cube in mixed precision: tensor-core level stencils with BF16
    hi+lo operands (2a/h_1 = 6.3 < 9), everything else as FP32."""
    w, x, c, o = cube1m
    g = _gpu(gpu_lib, w, x, c, "mixed")
    assert g["plan"].info()["stencil_kind"] == 3  # tcgen05 tensor cores
    _check(g, o, TOLMIX, w.levels, "cube1m/mixed")


def test_fp32_anterpolation_fixed_point_resolution(gpu_lib, orc):
    """The FP32 path anterpolates (Eq. anterpolation) with 32-bit fixed-point
    sums: each contribution c_j phi(x_j) is rounded to 2^(e-30), where 2^e
    exceeds the worst-case node sum B = (most atoms in one cell) x (cells a
    4h support box can meet) x max c, so that no sum can overflow.  Against
    the FP64 oracle's q^1, node mu may therefore differ by at most
    n_mu (2^(e-31) + 8 u c_max) + u |q_mu| (n_mu contributions, FP32 weights
    and conversion, u = 2^-24), and the test checks exactly that bound on
    the 65,536-atom slab.  For a typical node sum of ~0.5 the fixed-point
    step is a few parts in 1e6, tens of FP32 rounding units: far below the
    FP32 path's force tolerance (1e-4 of the RMS force), but not below FP32
    rounding."""
    import torch

    w = I.workload("slab65536")
    x, c = I.generate(w)
    x = x.astype(np.float32).astype(np.float64)
    c = c.astype(np.float32).astype(np.float64)
    plan = gpu_lib.Plan(w.box, w.N, w.a, w.h, w.levels, precision="fp32")
    pos = torch.tensor(np.c_[x, c], dtype=torch.float32, device="cuda")
    plan.evaluate(pos, virial=False)
    torch.cuda.synchronize()
    q_gpu = gpu_lib.mls6_debug_grid(plan.handle, 1, 0).astype(np.float64)
    n = orc.grid_dims(w.box, w.h, w.levels)
    q_orc = orc.grids(w.box, w.a, n, w.levels, x, c)[0][0]
    # worst-case node sum as the library bounds it: cells of width
    # L / floor(2L/a), support box of 4 h per axis
    L, h = np.array(w.box), np.array(w.box) / np.array(n)
    nc = np.floor(2.0 * L / w.a).astype(int)
    cw = L / nc
    cell = np.minimum((np.mod(x, L) / cw).astype(int), nc - 1)
    pop = np.bincount(cell[:, 0] + nc[0] * (cell[:, 1] + nc[1] * cell[:, 2])).max()
    span = np.prod(np.ceil(4.0 * h / cw) + 1.0)
    B = pop * span * c.max()
    e = np.frexp(B)[1]
    step = 2.0 ** (e - 30)
    # contributions per node: every atom adds to the 4x4x4 nodes around it
    u = np.mod(x, L) / h
    base = np.floor(u).astype(int) - 1
    cnt = np.zeros(n[0] * n[1] * n[2], dtype=np.int64)
    for dz in range(4):
        for dy in range(4):
            for dx in range(4):
                ix = (base[:, 0] + dx) % n[0]
                iy = (base[:, 1] + dy) % n[1]
                iz = (base[:, 2] + dz) % n[2]
                np.add.at(cnt, ix + n[0] * (iy + n[1] * iz), 1)
    cnt = cnt.reshape(n[2], n[1], n[0])
    uu = 2.0 ** -24
    bound = cnt * (0.5 * step + 8 * uu * c.max()) + uu * np.abs(q_orc)
    err = np.abs(q_gpu - q_orc)
    print(f"fixed-point step {step:.2e}, max err {err.max():.2e}, "
          f"max err / bound {np.max(err / np.maximum(bound, 1e-300)):.3f}, "
          f"median |q| {np.median(np.abs(q_orc[cnt > 0])):.3f}")
    assert np.all(err <= bound)
    # and the step itself is what the library's comment states it is
    assert step <= 1e-5 * np.abs(q_orc).max()


@pytest.mark.parametrize("prec,a,h", [("fp64", 3.0, 0.5), ("fp32", 4.0, 0.5)])
def test_global_memory_stencil(gpu_lib, orc, prec, a, h):
    """Stencils whose tile and halo exceed the shared-memory budget
    (2a/h = 12 in FP64, 16 in FP32) run the global-memory level-stencil
    kernel: results against the oracle at the precision's tolerance."""
    import torch

    box, l, N = (12.0, 12.0, 13.0), 2, 1100
    x, c = I.uniform_atoms(5150 + int(a), N, box)
    if prec == "fp32":
        x = x.astype(np.float32).astype(np.float64)
        c = c.astype(np.float32).astype(np.float64)
    plan = gpu_lib.Plan(box, N, a, h, l, precision=prec)
    assert plan.info()["stencil_kind"] == 1
    dt = torch.float64 if prec == "fp64" else torch.float32
    r = plan.evaluate(torch.tensor(np.c_[x, c], dtype=dt, device="cuda"), virial=True)
    torch.cuda.synchronize()
    out = r["out"].cpu().numpy()
    n = orc.grid_dims(box, h, l)
    o = orc.evaluate(box, a, n, l, x, c)
    rms = np.sqrt(np.mean(np.sum(o["F"] ** 2, axis=1)))
    tol = dict(E=1e-12, F=1e-11, W=1e-11) if prec == "fp64" else dict(E=2e-6, F=1e-4, W=2e-5)
    assert abs(out[0] - o["E"]) <= tol["E"] * abs(o["E"])
    assert np.abs(r["F"].cpu().double().numpy() - o["F"]).max() <= tol["F"] * rms
    assert np.abs(out[1:7] - o["W"]).max() <= tol["W"] * np.abs(o["W"]).max()
    G = orc.grids(box, a, n, l, x, c)
    got = gpu_lib.mls6_debug_grid(plan.handle, 1, 1)
    ref = G[0][1]
    assert np.abs(got - ref).max() <= (1e-12 if prec == "fp64" else 1e-5) * np.abs(ref).max()
