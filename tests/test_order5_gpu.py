"""Interpolation order p = 5 (the C^1 quintic, 6 x 6 x 6 nodes per atom) on
the GPU against the oracle at p = 5: FP64 at 1e-12 (energy) / 1e-11 of the
RMS force, FP32 and mixed at their tolerances, every stage grid in FP64,
Lorentz-Berthelot, and a batch of order-5 plans against single plans."""
import numpy as np
import pytest

from paper_1308_4005_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(E=1e-12, F=1e-11, W=1e-11), "fp32": dict(E=2e-6, F=1e-4, W=2e-5),
       "mixed": dict(E=2e-5, F=1e-4, W=5e-5)}

CASES = [
    # name, N, box, a, h, levels
    ("cube_l3", 1500, (12.0, 12.0, 12.0), 2.5, 0.75, 3),
    ("aniso_l2", 700, (9.0, 11.0, 13.0), 2.0, 0.6, 2),
    ("one_level", 400, (8.0, 8.0, 8.0), 2.0, 0.5, 1),
    ("slab_l4", 2000, (16.0, 16.0, 48.0), 3.0, 1.0, 4),
]


def _run(gpu_lib, box, a, h, l, x, c, prec, stencil="auto"):
    import torch

    plan = gpu_lib.Plan(box, len(c), a, h, l, precision=prec, order=5, stencil=stencil)
    dt = torch.float64 if prec == "fp64" else torch.float32
    r = plan.evaluate(torch.tensor(np.c_[x, c], dtype=dt, device="cuda"), virial=True)
    torch.cuda.synchronize()
    out = r["out"].cpu().numpy()
    return dict(E=out[0], W=out[1:7], F=r["F"].cpu().double().numpy(), plan=plan)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed"])
@pytest.mark.parametrize("name,N,box,a,h,l", CASES)
def test_order5_vs_oracle(gpu_lib, orc, name, N, box, a, h, l, prec):
    region = None
    if name.startswith("slab"):
        region = ((0.0, box[0]), (0.0, box[1]), (0.3 * box[2], 0.7 * box[2]))
    x, c = I.uniform_atoms(500 + N, N, box, region=region)
    if prec != "fp64":
        x = x.astype(np.float32).astype(np.float64)
        c = c.astype(np.float32).astype(np.float64)
    n = orc.grid_dims(box, h, l)
    with orc.interp_order(5):
        o = orc.evaluate(box, a, n, l, x, c)
        G = orc.grids(box, a, n, l, x, c) if prec == "fp64" else None
    stencil = "tensor" if prec == "mixed" and l >= 2 and 2 * a / h < 9 else "auto"
    g = _run(gpu_lib, box, a, h, l, x, c, prec, stencil)
    t = TOL[prec]
    rms = np.sqrt(np.mean(np.sum(o["F"] ** 2, axis=1)))
    dE = abs(g["E"] - o["E"]) / abs(o["E"])
    dF = np.abs(g["F"] - o["F"]).max() / rms
    dW = np.abs(g["W"] - o["W"]).max() / np.abs(o["W"]).max()
    assert dE <= t["E"], (name, prec, dE)
    assert dF <= t["F"], (name, prec, dF)
    assert dW <= t["W"], (name, prec, dW)
    if G is not None:  # q^k, e^k and e^{k,tot} of every level
        # 5e-12: the coarsest level is an all-to-all sum over up to 4,096
        # nodes, summed in another order than the oracle's
        for k in range(1, l + 1):
            for which in range(3):
                ref = G[k - 1][which]
                got = gpu_lib.mls6_debug_grid(g["plan"].handle, k, which)
                assert np.abs(got - ref).max() <= 5e-12 * np.abs(ref).max(), (name, k, which)


def test_order5_differs_from_order3(gpu_lib):
    """The order is honoured: p = 3 and p = 5 give different energies that
    agree to the method's accuracy."""
    import torch

    box, a, h, l = (10.0, 10.0, 10.0), 2.5, 0.8, 2
    x, c = I.uniform_atoms(77, 900, box)
    pos = torch.tensor(np.c_[x, c], dtype=torch.float64, device="cuda")
    E = {}
    for p in (3, 5):
        plan = gpu_lib.Plan(box, 900, a, h, l, precision="fp64", order=p)
        E[p] = float(plan.evaluate(pos, virial=False)["out"][0].cpu())
    assert E[3] != E[5]
    assert E[5] == pytest.approx(E[3], rel=1e-2)


def test_order5_lorentz_berthelot(gpu_lib, orc):
    import ctypes as C

    import torch
    from oracle import lb

    box, a, h, l, N = (9.0, 9.0, 9.0), 2.2, 0.75, 3, 500
    x, _ = I.uniform_atoms(571, N, box)
    rng = np.random.default_rng(572)
    s, e = rng.uniform(0.85, 1.15, N), rng.uniform(0.5, 1.5, N)
    n = orc.grid_dims(box, h, l)
    with orc.interp_order(5):
        r = lb.evaluate_lb(box, a, n, l, x, s, e)
    plan = gpu_lib.Plan(box, N, a, h, l, precision="fp64", order=5)
    dev = dict(dtype=torch.float64, device="cuda")
    pos, sg, ep = (torch.tensor(v, **dev).contiguous() for v in (x, s, e))
    F = torch.empty((N, 3), **dev)
    E = C.c_double()
    rc = gpu_lib.mls6_eval_lb(plan.handle, pos.data_ptr(), sg.data_ptr(), ep.data_ptr(),
                              F.data_ptr(), C.addressof(E))
    assert rc == 0, gpu_lib.status_string(rc)
    rms = np.sqrt(np.mean(np.sum(r["F"] ** 2, axis=1)))
    assert abs(E.value - r["E"]) <= 1e-12 * abs(r["E"])
    assert np.abs(F.cpu().numpy() - r["F"]).max() <= 1e-11 * rms


def test_order5_batch_equals_single_plans(gpu_lib):
    """A batch of order-5 plans (chained graph: the persistent kernel takes
    the cubic only) gives each replica's single-plan result bit for bit."""
    import torch

    ws = I.batch_workloads(B=4, nmin=600, nmax=2000, seed=5005)
    xs, cs, off = I.generate_batch(ws)
    pos = torch.tensor(np.c_[xs, cs], dtype=torch.float32, device="cuda")
    bt = gpu_lib.Batch([w.box for w in ws], [w.N for w in ws], ws[0].a, ws[0].h, 0,
                       precision="fp32", order=5)
    res = bt.evaluate(pos, virial=True)
    torch.cuda.synchronize()
    assert gpu_lib.mls6_batch_mode(bt.handle) == 0
    for r, w in enumerate(ws):
        p = gpu_lib.Plan(w.box, w.N, w.a, w.h, 0, precision="fp32", order=5)
        one = p.evaluate(pos[off[r]:off[r + 1]].contiguous(), virial=True)
        torch.cuda.synchronize()
        assert np.array_equal(res["F"][off[r]:off[r + 1]].cpu().numpy(), one["F"].cpu().numpy())
        assert res["E"][r].item() == one["out"][0].item()


def test_order5_refused_by_learned_features(gpu_lib):
    import ctypes as C

    box, a, h, l = (8.0, 8.0, 8.0), 2.0, 0.8, 2
    plan = gpu_lib.Plan(box, 100, a, h, l, precision="fp32", order=5)
    m = gpu_lib.MLP(1)
    rc = gpu_lib.load().mls6_mlp_features(C.c_void_p(plan.handle), C.c_void_p(m.handle), None, 0)
    assert rc == gpu_lib.MLS6_ERR_ORDER
