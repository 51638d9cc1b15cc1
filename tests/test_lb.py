"""Lorentz-Berthelot mixing (Sec. II.D): seven instances of the method.

CPU pins of the oracle form (oracle/lb.py, polarization of single-coefficient
oracle evaluations):
  - the binomial expansion sum_k xi_{i,k} xi_{j,6-k} equals
    2 sqrt(eps_i eps_j) ((sigma_i + sigma_j)/2)^6 (to rounding);
  - with equal sigma the LB result equals geometric mixing with
    c_i = sqrt(2 eps_i) sigma^3;
  - the LB MLS agrees with the exact LB lattice sum within the method's
    approximation error.
GPU parity: mls6_eval_lb against the oracle form (FP64 at the north-star
tolerances, FP32 and mixed at theirs), equal-sigma reduction to mls6_eval.
"""
import numpy as np
import pytest

from paper_1308_4005_gb300 import inputs as I


@pytest.fixture(scope="module")
def lb(orc):
    from oracle import lb

    return lb


def _species(seed, N):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.85, 1.15, N), rng.uniform(0.5, 1.5, N)


def test_lb_expansion_identity(lb):
    s, e = _species(1, 40)
    X = lb.xi(s, e)
    M = sum(np.outer(X[k], X[6 - k]) for k in range(7))
    C = lb.c_lb(s[:, None], s[None, :], e[:, None], e[None, :])
    assert np.abs(M - C).max() <= 4e-15 * C.max()
    # each channel pairing is symmetric in (i, j) only summed: k <-> 6-k
    assert np.allclose(M, M.T, rtol=1e-14)


def test_lb_equal_sigma_is_geometric(orc, lb):
    box, a, h, l = (7.0, 7.5, 8.0), 2.0, 0.7, 2
    x, _ = I.uniform_atoms(3, 60, box)
    _, e = _species(4, 60)
    s = np.full(60, 1.07)
    n = orc.grid_dims(box, h, l)
    r = lb.evaluate_lb(box, a, n, l, x, s, e)
    g = orc.evaluate(box, a, n, l, x, np.sqrt(2 * e) * s ** 3)
    assert r["E"] == pytest.approx(g["E"], rel=1e-12)
    assert np.abs(r["F"] - g["F"]).max() <= 1e-11 * np.abs(g["F"]).max()


def test_lb_mls_vs_exact_sum(orc, lb):
    box, a, h, l = (6.0, 6.0, 6.0), 2.0, 0.5, 2
    x, _ = I.uniform_atoms(5, 40, box)
    s, e = _species(6, 40)
    n = orc.grid_dims(box, h, l)
    r = lb.evaluate_lb(box, a, n, l, x, s, e)
    b = lb.brute_lb(box, x, s, e, r_img=18.0)
    assert abs(r["E"] - b["E"]) <= 5e-3 * abs(b["E"])
    rms = np.sqrt(np.mean(np.sum(b["F"] ** 2, axis=1)))
    assert np.sqrt(np.mean(np.sum((r["F"] - b["F"]) ** 2, axis=1))) <= 2e-2 * rms


# ------------------------------------------------------------------- GPU


def _gpu_lb(gpu_lib, box, a, h, l, x, s, e, prec):
    import ctypes as C

    import torch

    dt = torch.float64 if prec == "fp64" else torch.float32
    N = len(s)
    plan = gpu_lib.Plan(box, N, a, h, l, precision=prec)
    pos = torch.tensor(x, dtype=dt, device="cuda").contiguous()
    sg = torch.tensor(s, dtype=dt, device="cuda")
    ep = torch.tensor(e, dtype=dt, device="cuda")
    F = torch.empty((N, 3), dtype=dt, device="cuda")
    E = C.c_double()
    rc = gpu_lib.mls6_eval_lb(plan.handle, pos.data_ptr(), sg.data_ptr(), ep.data_ptr(),
                              F.data_ptr(), C.addressof(E))
    assert rc == 0, gpu_lib.status_string(rc)
    return E.value, F.cpu().double().numpy(), plan


LBCASES = [
    # name, N, box, a, h, levels
    ("cube_l3", 500, (9.0, 9.0, 9.0), 2.2, 0.75, 3),
    ("aniso_l2", 300, (7.0, 8.0, 10.0), 2.0, 0.6, 2),
]


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed"])
@pytest.mark.parametrize("name,N,box,a,h,l", LBCASES)
def test_lb_gpu_vs_oracle(gpu_lib, orc, lb, name, N, box, a, h, l, prec):
    x, _ = I.uniform_atoms(71 + N, N, box)
    s, e = _species(72 + N, N)
    if prec != "fp64":
        x, s, e = (v.astype(np.float32).astype(np.float64) for v in (x, s, e))
    n = orc.grid_dims(box, h, l)
    r = lb.evaluate_lb(box, a, n, l, x, s, e)
    Eg, Fg, _ = _gpu_lb(gpu_lib, box, a, h, l, x, s, e, prec)
    tol = {"fp64": (1e-12, 1e-11), "fp32": (2e-6, 1e-4), "mixed": (2e-5, 1e-4)}[prec]
    rms = np.sqrt(np.mean(np.sum(r["F"] ** 2, axis=1)))
    assert abs(Eg - r["E"]) / abs(r["E"]) <= tol[0], (name, prec)
    assert np.abs(Fg - r["F"]).max() / rms <= tol[1], (name, prec)


@pytest.mark.gpu
def test_lb_gpu_equal_sigma_and_repeatable(gpu_lib):
    import torch

    box, a, h, l = (8.0, 8.0, 8.0), 2.0, 0.6, 3
    x, _ = I.uniform_atoms(9, 400, box)
    _, e = _species(10, 400)
    s = np.full(400, 0.95)
    E1, F1, _ = _gpu_lb(gpu_lib, box, a, h, l, x, s, e, "fp64")
    E2, F2, _ = _gpu_lb(gpu_lib, box, a, h, l, x, s, e, "fp64")
    assert E1 == E2 and np.array_equal(F1, F2)
    c = np.sqrt(2 * e) * s ** 3
    plan = gpu_lib.Plan(box, 400, a, h, l, precision="fp64")
    r = plan.evaluate(torch.tensor(np.c_[x, c], dtype=torch.float64, device="cuda"),
                      virial=False)
    torch.cuda.synchronize()
    Eg = float(r["out"][0].cpu())
    Fg = r["F"].cpu().numpy()
    assert E1 == pytest.approx(Eg, rel=1e-12)
    assert np.abs(F1 - Fg).max() <= 1e-11 * np.abs(Fg).max()


@pytest.mark.gpu
def test_lb_no_atoms(gpu_lib):
    import ctypes as C

    plan = gpu_lib.Plan((8.0, 8.0, 8.0), 0, 2.0, 0.8, 2, precision="fp64")
    E = C.c_double(1.0)
    rc = gpu_lib.mls6_eval_lb(plan.handle, 0, 0, 0, 0, C.addressof(E))
    assert rc == 0 and E.value == 0.0
