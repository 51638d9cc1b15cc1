"""Smoothing functions of continuity C^1..C^4 (Sec. II.A.3, compared in
Sec. III.B; gamma_n is the order-n Taylor polynomial of u^(-1/2) about u = 1,
u = rho^12, n = 2 being Eq. gamma) on the GPU against the FP64 oracle with the
same smoothing function, in FP64, FP32 and mixed precision."""
import numpy as np
import pytest

from paper_1308_4005_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _run(gpu_lib, box, a, h, l, x, c, prec, n):
    import torch

    plan = gpu_lib.Plan(box, len(c), a, h, l, precision=prec, continuity=n, stencil="tensor")
    dt = torch.float64 if prec == "fp64" else torch.float32
    r = plan.evaluate(torch.tensor(np.c_[x, c], dtype=dt, device="cuda"), virial=True)
    torch.cuda.synchronize()
    assert gpu_lib.mls6_last_error(plan.handle) == 0
    out = r["out"].cpu().numpy()
    return dict(E=out[0], W=out[1:7], F=r["F"].cpu().double().numpy(), plan=plan)


def _errs(g, o):
    rms = np.sqrt(np.mean(np.sum(o["F"] ** 2, axis=1)))
    return (abs(g["E"] - o["E"]) / abs(o["E"]), np.abs(g["F"] - o["F"]).max() / rms,
            np.abs(g["W"] - o["W"]).max() / np.abs(o["W"]).max())


@pytest.mark.parametrize("n", [1, 3, 4])
def test_smoothing_fp64_parity(gpu_lib, orc, n):
    box, a, h, l = (8.0, 9.0, 10.0), 2.0, 0.6, 3
    x, c = I.uniform_atoms(4100 + n, 500, box)
    nn = orc.grid_dims(box, h, l)
    with orc.smoothing_order(n):
        o = orc.evaluate(box, a, nn, l, x, c)
    g = _run(gpu_lib, box, a, h, l, x, c, "fp64", n)
    dE, dF, dW = _errs(g, o)
    assert dE <= 1e-12 and dF <= 1e-11 and dW <= 1e-11, (n, dE, dF, dW)
    # the smoothing function matters: C^2 gives another energy
    o2 = orc.evaluate(box, a, nn, l, x, c)
    assert abs(o2["E"] - o["E"]) > 1e-6 * abs(o["E"])


@pytest.mark.parametrize("n,prec", [(1, "fp32"), (4, "fp32"), (3, "mixed")])
def test_smoothing_single_precision(gpu_lib, orc, n, prec):
    box, a, h, l = (14.0, 14.0, 14.0), 3.0, 1.0, 3
    x, c = I.uniform_atoms(4200 + n, 2000, box)
    x = x.astype(np.float32).astype(np.float64)
    c = c.astype(np.float32).astype(np.float64)
    nn = orc.grid_dims(box, h, l)
    with orc.smoothing_order(n):
        o = orc.evaluate(box, a, nn, l, x, c)
    g = _run(gpu_lib, box, a, h, l, x, c, prec, n)
    if prec == "mixed":
        assert g["plan"].info()["stencil_kind"] == 3
    dE, dF, dW = _errs(g, o)
    tol = (2e-6, 1e-4, 2e-5) if prec == "fp32" else (2e-5, 1e-4, 5e-5)
    assert dE <= tol[0] and dF <= tol[1] and dW <= tol[2], (n, prec, dE, dF, dW)


def test_smoothing_restricts_kernel_forms(gpu_lib):
    """Plans with n != 2 run the per-atom pair kernel only and refuse the
    Lorentz-Berthelot evaluation."""
    import torch

    box = (9.0, 9.0, 9.0)
    plan = gpu_lib.Plan(box, 100, 2.0, 0.75, 2, precision="fp64", continuity=3)
    with pytest.raises(gpu_lib.MLS6Error):
        gpu_lib.mls6_set_tuning(plan.handle, 32, 0)
    assert gpu_lib.mls6_get_tuning(plan.handle)[0] <= 8
    pos = torch.zeros((100, 3), dtype=torch.float64, device="cuda")
    one = torch.ones(100, dtype=torch.float64, device="cuda")
    F = torch.empty((100, 3), dtype=torch.float64, device="cuda")
    rc = gpu_lib.load().mls6_eval_lb(plan.handle, pos.data_ptr(), one.data_ptr(), one.data_ptr(),
                                     F.data_ptr(), None)
    assert rc == gpu_lib.MLS6_ERR_ARG
