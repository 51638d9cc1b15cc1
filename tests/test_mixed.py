"""Mixed precision (tensor-core level stencils with BF16 hi+lo operands)
against the FP64 oracle.

Error budget.  A tap weight w and a node value q are each split as
x = x_hi + x_lo + d with |d| <= 2^-18 |x| (two round-to-nearest bf16 parts,
8 significant bits each); the tensor cores form w_hi q_hi + w_hi q_lo +
w_lo q_hi, dropping w_lo q_lo (<= 2^-18 |wq|), so each product is within
3 * 2^-18 = 1.1e-5 of wq, and FP32 accumulation adds ~1e-7.  The level
potentials e^k are sums of terms of one sign (g_k > 0, q mostly > 0), so
they carry <= 1.2e-5 relative error; e^1 is held to 2e-5 of its largest
entry.  Energies and forces mix that with the FP32 pair part: |dE|/|E| <=
2e-5, forces 1e-4 of the RMS force, virial 5e-5 of its largest entry.
"""
import numpy as np
import pytest

from paper_1308_4005_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOLMIX = dict(E=2e-5, F=1e-4, W=5e-5)


def run(gpu_lib, box, a, h, l, x, c, prec="mixed", virial=True):
    import torch

    # these grids are small: ask for the tensor-core stencil explicitly
    plan = gpu_lib.Plan(box, len(c), a, h, l, precision=prec, stencil="tensor")
    pos = torch.tensor(np.c_[x, c], dtype=torch.float32, device="cuda")
    r = plan.evaluate(pos, virial=virial)
    torch.cuda.synchronize()
    out = r["out"].cpu().numpy()
    return dict(E=out[0], W=out[1:7], F=r["F"].cpu().double().numpy(), plan=plan)


def errs(g, o):
    rms = np.sqrt(np.mean(np.sum(o["F"] ** 2, axis=1)))
    return (abs(g["E"] - o["E"]) / abs(o["E"]), np.abs(g["F"] - o["F"]).max() / rms,
            np.abs(g["W"] - o["W"]).max() / np.abs(o["W"]).max())


CASES = [
    # name, N, box, a, h, levels  (2a/h < 9 so the tensor-core stencil runs)
    ("cube_l3", 2000, (14.0, 14.0, 14.0), 3.0, 1.0, 3),
    ("slab_l4", 3000, (16.0, 16.0, 48.0), 3.0, 1.25, 4),
    ("aniso_ragged", 700, (9.0, 11.0, 13.0), 2.0, 0.6, 3),
    ("two_levels", 500, (10.0, 10.0, 10.0), 2.5, 0.7, 2),
]


@pytest.mark.parametrize("name,N,box,a,h,l", CASES)
def test_mixed_vs_oracle(gpu_lib, orc, name, N, box, a, h, l):
    region = None
    if name.startswith("slab"):
        region = ((0.0, box[0]), (0.0, box[1]), (0.3 * box[2], 0.7 * box[2]))
    x, c = I.uniform_atoms(97 + N, N, box, region=region)
    x32 = x.astype(np.float32).astype(np.float64)
    c32 = c.astype(np.float32).astype(np.float64)
    n = orc.grid_dims(box, h, l)
    o = orc.evaluate(box, a, n, l, x32, c32)
    g = run(gpu_lib, box, a, h, l, x, c)
    info = g["plan"].info()
    assert info["levels"] == l
    assert info["stencil_kind"] == 3  # tcgen05 tensor cores
    dE, dF, dW = errs(g, o)
    assert dE <= TOLMIX["E"], (name, dE)
    assert dF <= TOLMIX["F"], (name, dF)
    assert dW <= TOLMIX["W"], (name, dW)
    # the level potentials themselves
    G = orc.grids(box, a, n, l, x32, c32)
    for k in range(1, l):
        ref = G[k - 1][1]
        got = gpu_lib.mls6_debug_grid(g["plan"].handle, k, 1)
        assert np.abs(got - ref).max() <= 2e-5 * np.abs(ref).max(), (name, k)


def test_mixed_no_virial_and_repeatable(gpu_lib, orc):
    box, a, h, l = (12.0, 12.0, 12.0), 2.5, 0.8, 3
    x, c = I.uniform_atoms(5, 1200, box)
    g1 = run(gpu_lib, box, a, h, l, x, c, virial=False)
    g2 = run(gpu_lib, box, a, h, l, x, c, virial=False)
    assert g1["E"] == g2["E"] and np.array_equal(g1["F"], g2["F"])
    # with the virial the kernels are other instantiations (different FMA
    # contraction): forces agree to FP32 rounding, not bit for bit
    g3 = run(gpu_lib, box, a, h, l, x, c, virial=True)
    assert g3["E"] == pytest.approx(g1["E"], rel=1e-7)
    assert np.abs(g3["F"] - g1["F"]).max() <= 1e-6 * np.abs(g1["F"]).max()


def test_mixed_wide_stencil_uses_fp32_path(gpu_lib, orc):
    """2a/h >= 9: no tensor-core kernel; the plan keeps the FP32 stencil and
    the FP32 tolerances."""
    box, a, h, l = (12.0, 12.0, 12.0), 3.0, 0.6, 2
    x, c = I.uniform_atoms(8, 800, box)
    x32 = x.astype(np.float32).astype(np.float64)
    c32 = c.astype(np.float32).astype(np.float64)
    n = orc.grid_dims(box, h, l)
    o = orc.evaluate(box, a, n, l, x32, c32)
    gm = run(gpu_lib, box, a, h, l, x, c, prec="mixed")
    gf = run(gpu_lib, box, a, h, l, x, c, prec="fp32")
    assert gm["plan"].info()["stencil_kind"] == 0
    assert gm["E"] == gf["E"] and np.array_equal(gm["F"], gf["F"])
    dE, dF, dW = errs(gm, o)
    assert dE <= 2e-6 and dF <= 1e-4 and dW <= 2e-5


def test_mixed_stencil_choice_by_grid_size(gpu_lib):
    """Automatic choice: the tcgen05 stencil when the levels give at least
    two 16^3 tiles per SM (the 1M-atom cube's 112^3 grid), the FP32 CUDA-core
    stencil for the 65,536-atom slab's 32 x 32 x 96 grid; both on request."""
    w = I.workload("slab65536")
    auto = gpu_lib.Plan(w.box, w.N, w.a, w.h, w.levels, precision="mixed")
    assert auto.info()["stencil_kind"] == 0
    forced = gpu_lib.Plan(w.box, w.N, w.a, w.h, w.levels, precision="mixed", stencil="tensor")
    assert forced.info()["stencil_kind"] == 3
    c = I.workload("cube1m")
    big = gpu_lib.Plan(c.box, 1000, c.a, c.h, c.levels, precision="mixed")
    assert big.info()["stencil_kind"] == 3
    cuda = gpu_lib.Plan(c.box, 1000, c.a, c.h, c.levels, precision="mixed", stencil="cuda")
    assert cuda.info()["stencil_kind"] == 0
