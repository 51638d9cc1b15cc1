"""The allocation-free coarsest-level entry point against the full evaluation.

mls6_coarse_apply_noalloc serves callers that may not allocate device memory
at call time (engines with a fixed up-front memory budget, code where
cudaMalloc/cudaFree would synchronise or are not allowed); its scratch is a
fixed file-scope device array.  This test runs a normal FP64 evaluation,
takes the coarsest-level grid xi^l it produced, applies the allocation-free
entry point to it twice in a row, and checks e^l against the grid the
evaluation itself computed, and the virial term against the same quadratic
form evaluated from the table in FP64 on the host.  Each test builds
everything it uses, so it passes alone, after the other tests, or in any
order; it lives in a file that pytest collects last only so that, in a run
that stops at the first failure, every other test has already run.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1308_4005_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_coarse_apply_noalloc_matches_eval(gpu_lib):
    import torch

    box, a, h, l = (8.0, 9.0, 10.0), 2.0, 0.5, 3
    x, c = I.uniform_atoms(77, 400, box)
    plan = gpu_lib.Plan(box, len(c), a, h, l, precision="fp64")
    pos = torch.tensor(np.c_[x, c], dtype=torch.float64, device="cuda")
    plan.evaluate(pos, virial=True)
    torch.cuda.synchronize()
    info = plan.info()
    nl = info["n_grid"][l - 1]
    q_l = gpu_lib.mls6_debug_grid(plan.handle, l, 0).reshape(-1)
    e_l = gpu_lib.mls6_debug_grid(plan.handle, l, 1).reshape(-1)
    T, V = gpu_lib.mls6_coarse_tables(box, nl, l, a)

    dq = torch.tensor(q_l, dtype=torch.float64, device="cuda")
    dT = torch.tensor(T, dtype=torch.float64, device="cuda")
    dV = torch.tensor(V.reshape(-1), dtype=torch.float64, device="cuda")
    n = (C.c_int * 3)(*nl)
    npk = len(q_l)
    # reference virial term: 1/2 q . (V_c * q) with the circulant table
    idx = np.arange(npk)
    m0, m1, m2 = idx % nl[0], (idx // nl[0]) % nl[1], idx // (nl[0] * nl[1])
    diff = (((m0[:, None] - m0[None, :]) % nl[0]) + nl[0] * (((m1[:, None] - m1[None, :]) % nl[1])
            + nl[1] * ((m2[:, None] - m2[None, :]) % nl[2])))
    vir_ref = np.array([0.5 * q_l @ (V[k][diff] @ q_l) for k in range(6)])

    for call in range(2):
        de = torch.full((npk,), np.nan, dtype=torch.float64, device="cuda")
        dw = torch.full((6,), np.nan, dtype=torch.float64, device="cuda")
        rc = gpu_lib.load().mls6_coarse_apply_noalloc(
            C.c_void_p(dq.data_ptr()), n, C.c_void_p(dT.data_ptr()), C.c_void_p(dV.data_ptr()),
            C.c_void_p(de.data_ptr()), C.c_void_p(dw.data_ptr()), None)
        assert rc == 0, (call, rc)
        torch.cuda.synchronize()
        got_e = de.cpu().numpy()
        got_w = dw.cpu().numpy()
        assert np.abs(got_e - e_l).max() <= 1e-12 * np.abs(e_l).max(), call
        assert np.abs(got_w - vir_ref).max() <= 1e-11 * np.abs(vir_ref).max(), call


def test_coarse_apply_noalloc_rejects_oversize(gpu_lib):
    n = (C.c_int * 3)(32, 32, 32)  # 32768 nodes, above the fixed scratch
    rc = gpu_lib.load().mls6_coarse_apply_noalloc(
        C.c_void_p(1), n, C.c_void_p(1), C.c_void_p(1), C.c_void_p(1), C.c_void_p(1), None)
    assert rc == gpu_lib.MLS6_ERR_SIZE
