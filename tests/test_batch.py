"""Batched replicas: host logic (automatic level count, longest-processing-
time assignment, cost model) on the CPU, and on the GPU per-replica parity of
one graph launch over uneven replicas against single plans (bit for bit, same
kernel shapes) and against the FP64 oracle."""
import itertools
import math

import numpy as np
import pytest

from paper_1308_4005_gb300 import inputs as I
from paper_1308_4005_gb300 import mls6

# ----------------------------------------------------------------- host logic


@pytest.fixture(scope="module")
def lib():
    return mls6.load()


BOXES = [(10.0, 10.0, 10.0), (13.7, 13.7, 13.7), (40.0, 40.0, 120.0), (23.0, 23.0, 69.0),
         (5.0, 6.0, 9.0), (107.25, 107.25, 107.25), (3.0, 3.0, 3.0), (31.0, 47.0, 64.0)]


@pytest.mark.parametrize("box", BOXES)
@pytest.mark.parametrize("h", [0.5, 1.0, 1.25])
def test_auto_levels_rule(lib, box, h):
    """l is the largest level count whose rounded hierarchy keeps >= 4 points
    per axis on the coarsest grid (1 if even 2 levels do not)."""
    l = mls6.mls6_auto_levels(box, h)
    assert 1 <= l <= 12

    def coarsest_min(k):
        n = mls6.mls6_grid_dims(box, h, k)
        return min(n) // 2 ** (k - 1)

    if l > 1:
        for k in range(2, l + 1):
            assert coarsest_min(k) >= 4, (k, coarsest_min(k))
    if l < 12:
        assert coarsest_min(l + 1) < 4


def test_auto_levels_slab_config(lib):
    """The 65,536-atom slab (40x40x120, h=1.25) is specified with a 4x4x12
    top grid, i.e. 4 levels: the rule reproduces it."""
    assert mls6.mls6_auto_levels((40.0, 40.0, 120.0), 1.25) == 4
    assert tuple(mls6.mls6_grid_dims((40.0, 40.0, 120.0), 1.25, 4)) == (32, 32, 96)


def _lpt_ref(cost, K):
    order = sorted(range(len(cost)), key=lambda r: (-cost[r], r))
    load = [0.0] * K
    out = [0] * len(cost)
    for r in order:
        k = min(range(K), key=lambda q: (load[q], q))
        out[r] = k
        load[k] += cost[r]
    return out, load


def test_lpt_assignment(lib):
    rng = np.random.default_rng(5)
    for _ in range(20):
        B = int(rng.integers(1, 40))
        K = int(rng.integers(1, 9))
        cost = list(rng.exponential(1.0, B))
        got, load = mls6.mls6_lpt_assign(cost, K)
        ref, rload = _lpt_ref(cost, K)
        assert got == ref
        assert np.allclose(load, rload)
        assert all(0 <= k < K for k in got)


def test_lpt_graham_bound(lib):
    """LPT makespan <= (4/3 - 1/(3K)) x optimum (Graham 1969), optimum by
    brute force on small instances."""
    rng = np.random.default_rng(9)
    for _ in range(30):
        B = int(rng.integers(2, 8))
        K = int(rng.integers(2, 4))
        cost = list(rng.uniform(0.1, 1.0, B))
        _, load = mls6.mls6_lpt_assign(cost, K)
        opt = min(max(sum(cost[r] for r in range(B) if a[r] == k) for k in range(K))
                  for a in itertools.product(range(K), repeat=B))
        assert max(load) <= (4.0 / 3.0 - 1.0 / (3 * K)) * opt + 1e-12


def test_cost_model_terms(lib):
    """Each term of the model on its own (coefficient vector picks it): the
    local term is (a/d)^3 N with d the mean spacing (V/N)^(1/3) and the grid
    term (a/h)^3 V/h^3 times 8/7 for the level sum (Sec. IV)."""
    box, N, a, h, l = (20.0, 25.0, 30.0), 12000, 2.5, 1.0, 3
    V = 20.0 * 25.0 * 30.0
    d = (V / N) ** (1.0 / 3.0)
    e = [[1, 0, 0, 0, 0], [0, 1, 0, 0, 0], [0, 0, 1, 0, 0], [0, 0, 0, 1, 0], [0, 0, 0, 0, 1]]
    t = [mls6.mls6_cost_model(box, N, a, h, l, coef=c) for c in e]
    assert t[0] == pytest.approx((a / d) ** 3 * N, rel=1e-12)
    assert t[1] == pytest.approx((a / h) ** 3 * (V / h ** 3) * 8 / 7, rel=1e-12)
    assert t[2] == pytest.approx(N, rel=1e-15)
    n_l = V / (h * 2 ** (l - 1)) ** 3
    assert t[3] == pytest.approx(n_l ** 2, rel=1e-12)
    assert t[4] == pytest.approx(8 + 2 * (l - 1), rel=1e-15)
    # defaults: positive and growing with N at fixed box
    c1 = mls6.mls6_cost_model(box, N, a, h, l)
    c2 = mls6.mls6_cost_model(box, 2 * N, a, h, l)
    assert 0 < c1 < c2


def test_batch_workloads_shape():
    ws = I.batch_workloads()
    assert len(ws) == 256
    Ns = np.array([w.N for w in ws])
    assert Ns.min() >= 2048 and Ns.max() <= 65536
    for r, w in enumerate(ws[:8]):
        V = w.box[0] * w.box[1] * w.box[2]
        if r % 2 == 0:
            assert w.N / V == pytest.approx(0.8, rel=1e-9)
        else:
            assert w.box[2] == pytest.approx(3 * w.box[0])
            t = w.region[2][1] - w.region[2][0]
            assert w.N / (w.box[0] * w.box[1] * t) == pytest.approx(0.8, rel=1e-9)
        assert w.levels == 0


# ------------------------------------------------------------------ GPU parity

SMALL = dict(B=6, nmin=300, nmax=3000, a=2.5, h=1.0)


@pytest.fixture(scope="module")
def small_batch():
    ws = I.batch_workloads(B=SMALL["B"], nmin=SMALL["nmin"], nmax=SMALL["nmax"],
                           a=SMALL["a"], h=SMALL["h"], seed=4242)
    x, c, off = I.generate_batch(ws)
    return ws, x, c, off


def _single(gpu_lib, w, x, c, prec, split, groups, virial=True):
    import torch

    dt = torch.float64 if prec == "fp64" else torch.float32
    p = gpu_lib.Plan(w.box, w.N, w.a, w.h, 0, precision=prec)
    gpu_lib.mls6_set_tuning(p.handle, split, groups)
    pos = torch.tensor(np.c_[x, c], dtype=dt, device="cuda")
    r = p.evaluate(pos, virial=virial)
    torch.cuda.synchronize()
    out = r["out"].cpu().numpy()
    return out[0], out[1:7], r["F"].cpu().numpy(), p


def _batch_eval(bt, x, c, prec, virial=True):
    import torch

    dt = torch.float64 if prec == "fp64" else torch.float32
    pos = torch.tensor(np.c_[x, c], dtype=dt, device="cuda")
    r = bt.evaluate(pos, virial=virial)
    torch.cuda.synchronize()
    return r["E"].cpu().numpy(), r["W"].cpu().numpy(), r["F"].cpu().numpy(), pos


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_bitwise_vs_single(gpu_lib, small_batch, prec):
    ws, x, c, off = small_batch
    bt = gpu_lib.Batch([w.box for w in ws], [w.N for w in ws], SMALL["a"], SMALL["h"], 0,
                       precision=prec)
    assert bt.offsets == list(off)
    E, W, F, _ = _batch_eval(bt, x, c, prec)
    info = bt.info()  # the shapes the evaluation ran with
    for r, w in enumerate(ws):
        sl = slice(off[r], off[r + 1])
        e1, w1, f1, p = _single(gpu_lib, w, x[sl], c[sl], prec, info["pair_split"][r],
                                info["stencil_groups"][r])
        assert p.info()["levels"] == info["levels"][r]
        assert E[r] == e1, (r, E[r], e1)
        assert np.array_equal(W[r], w1), r
        assert np.array_equal(F[sl], f1), r


@pytest.mark.gpu
def test_batch_vs_oracle(gpu_lib, orc, small_batch):
    """The smallest replica of the batch against the FP64 oracle."""
    ws, x, c, off = small_batch
    bt = gpu_lib.Batch([w.box for w in ws], [w.N for w in ws], SMALL["a"], SMALL["h"], 0)
    E, W, F, _ = _batch_eval(bt, x, c, "fp64")
    r = int(np.argmin([w.N for w in ws]))
    w = ws[r]
    l = bt.info()["levels"][r]
    n = orc.grid_dims(w.box, w.h, l)
    sl = slice(off[r], off[r + 1])
    o = orc.evaluate(w.box, w.a, n, l, x[sl], c[sl])
    assert abs(E[r] - o["E"]) / abs(o["E"]) <= 1e-12
    rms = np.sqrt(np.mean(np.sum(o["F"] ** 2, axis=1)))
    assert np.abs(F[sl] - o["F"]).max() / rms <= 1e-11
    assert np.abs(W[r] - o["W"]).max() / np.abs(o["W"]).max() <= 1e-11


@pytest.mark.gpu
def test_batch_branches_and_tuning(gpu_lib, small_batch):
    """Results do not depend on the chain count; after autotuning each
    replica still equals a single plan with the tuned shapes."""
    ws, x, c, off = small_batch
    bt = gpu_lib.Batch([w.box for w in ws], [w.N for w in ws], SMALL["a"], SMALL["h"], 0)
    E0, W0, F0, pos = _batch_eval(bt, x, c, "fp64")
    for K in (1, 3, 6):
        gpu_lib.mls6_batch_set_config(bt.handle, branches=K)
        assert bt.info()["branches"] == K
        E, W, F, _ = _batch_eval(bt, x, c, "fp64")
        assert np.array_equal(E, E0) and np.array_equal(W, W0) and np.array_equal(F, F0)
    t = bt.tune(pos, reps=2)
    assert t > 0
    info = bt.info()
    assert 1 <= info["branches"] <= len(ws)
    E, W, F, _ = _batch_eval(bt, x, c, "fp64")
    for r, w in enumerate(ws):
        sl = slice(off[r], off[r + 1])
        e1, w1, f1, _ = _single(gpu_lib, w, x[sl], c[sl], "fp64", info["pair_split"][r],
                                info["stencil_groups"][r])
        assert E[r] == e1 and np.array_equal(W[r], w1) and np.array_equal(F[sl], f1)


@pytest.mark.gpu
def test_batch_host_outputs_and_nonfinite(gpu_lib, small_batch):
    import ctypes as C

    import torch

    ws, x, c, off = small_batch
    bt = gpu_lib.Batch([w.box for w in ws], [w.N for w in ws], SMALL["a"], SMALL["h"], 0)
    E0, W0, F0, pos = _batch_eval(bt, x, c, "fp64")
    B = len(ws)
    Eh = (C.c_double * B)()
    Wh = (C.c_double * (6 * B))()
    Fd = torch.empty((off[-1], 3), dtype=torch.float64, device="cuda")
    rc = gpu_lib.mls6_batch_eval(bt.handle, pos.data_ptr(), 0, Fd.data_ptr(),
                                 C.addressof(Eh), C.addressof(Wh))
    assert rc == 0
    assert np.array_equal(np.array(Eh[:]), E0)
    assert np.array_equal(np.array(Wh[:]).reshape(B, 6), W0)
    bad = x.copy()
    bad[off[3] + 1, 0] = np.nan
    pos2 = torch.tensor(np.c_[bad, c], dtype=torch.float64, device="cuda")
    rc = gpu_lib.mls6_batch_eval(bt.handle, pos2.data_ptr(), 0, Fd.data_ptr(),
                                 C.addressof(Eh), C.addressof(Wh))
    assert rc == gpu_lib.MLS6_ERR_NONFINITE
    # the batch stays usable
    rc = gpu_lib.mls6_batch_eval(bt.handle, pos.data_ptr(), 0, Fd.data_ptr(),
                                 C.addressof(Eh), C.addressof(Wh))
    assert rc == 0 and np.array_equal(np.array(Eh[:]), E0)


@pytest.mark.gpu
def test_batch_with_empty_replica(gpu_lib):
    """A replica without atoms gives E = W = 0 and leaves the others as
    their single plans."""
    boxes = [(9.0, 9.0, 9.0), (8.0, 8.0, 8.0), (10.0, 10.0, 12.0)]
    Ns = [500, 0, 800]
    xs, cs = [], []
    for r, (b, n) in enumerate(zip(boxes, Ns)):
        x, c = I.uniform_atoms(300 + r, n, b)
        xs.append(x if n else np.zeros((0, 3)))
        cs.append(c if n else np.zeros(0))
    x = np.concatenate(xs)
    c = np.concatenate(cs)
    bt = gpu_lib.Batch(boxes, Ns, 2.5, 1.0, 0)
    E, W, F, _ = _batch_eval(bt, x, c, "fp64")
    assert E[1] == 0.0 and np.all(W[1] == 0.0)
    off = bt.offsets
    info = bt.info()
    for r in (0, 2):
        w = I.Workload("r", Ns[r], boxes[r], None, (0.5, 1.5), 2.5, 1.0, 0, 0)
        sl = slice(off[r], off[r + 1])
        e1, w1, f1, _ = _single(gpu_lib, w, x[sl], c[sl], "fp64", info["pair_split"][r],
                                info["stencil_groups"][r])
        assert E[r] == e1 and np.array_equal(W[r], w1) and np.array_equal(F[sl], f1)


@pytest.mark.gpu
def test_persistent_batch_is_one_launch_equal_to_chains(gpu_lib, small_batch):
    """FP32 batches in persistent mode run one persistent kernel (work queue
    over stage, replica and block): the graph holds a single kernel, and
    every replica's energy, virial and forces equal those of the per-replica
    kernel chains (the default form) bit for bit (same kernel bodies, same
    shapes).  The autotuner tunes both forms and keeps the faster; the
    results stay those of single plans with the chosen shapes."""
    ws, x, c, off = small_batch
    bt = gpu_lib.Batch([w.box for w in ws], [w.N for w in ws], SMALL["a"], SMALL["h"], 0,
                       precision="fp32")
    assert gpu_lib.mls6_batch_mode(bt.handle) == 0
    gpu_lib.mls6_batch_set_mode(bt.handle, True)
    E, W, F, pos = _batch_eval(bt, x, c, "fp32")
    assert gpu_lib.mls6_batch_mode(bt.handle) == 1
    assert bt.info()["launches"] == 1
    gpu_lib.mls6_batch_set_mode(bt.handle, False)
    E2, W2, F2, _ = _batch_eval(bt, x, c, "fp32")
    assert gpu_lib.mls6_batch_mode(bt.handle) == 0
    assert bt.info()["launches"] > len(ws)
    assert np.array_equal(E, E2) and np.array_equal(W, W2) and np.array_equal(F, F2)
    t = bt.tune(pos, reps=2)
    assert t > 0 and gpu_lib.mls6_batch_mode(bt.handle) in (0, 1)
    E3, W3, F3, _ = _batch_eval(bt, x, c, "fp32")
    info = bt.info()
    for r, w in enumerate(ws):
        sl = slice(off[r], off[r + 1])
        e1, w1, f1, _ = _single(gpu_lib, w, x[sl], c[sl], "fp32", info["pair_split"][r],
                                info["stencil_groups"][r])
        assert E3[r] == e1 and np.array_equal(W3[r], w1) and np.array_equal(F3[sl], f1)


@pytest.mark.gpu
@pytest.mark.parametrize("item", [0, 7])
def test_persistent_batch_bounded_wait_runs_out(gpu_lib, small_batch, item):
    """The test hook withholds the completion count of one work item: the
    waits behind it run out after a short poll limit, every block leaves the
    kernel (nothing traps or faults), the call reports MLS6_ERR_TIMEOUT, and
    the batch evaluates normally once the hook is cleared."""
    import ctypes as C

    import torch

    ws, x, c, off = small_batch
    bt = gpu_lib.Batch([w.box for w in ws], [w.N for w in ws], SMALL["a"], SMALL["h"], 0,
                       precision="fp32")
    gpu_lib.mls6_batch_set_mode(bt.handle, True)
    E0, W0, F0, pos = _batch_eval(bt, x, c, "fp32")
    assert bt.info()["launches"] == 1
    B = len(ws)
    Eh = (C.c_double * B)()
    Fd = torch.empty((off[-1], 3), dtype=torch.float32, device="cuda")
    gpu_lib.mls6_batch_set_wait(bt.handle, 2000, item)
    rc = gpu_lib.mls6_batch_eval(bt.handle, pos.data_ptr(), 0, Fd.data_ptr(), C.addressof(Eh), 0)
    assert rc == gpu_lib.MLS6_ERR_TIMEOUT
    assert gpu_lib.mls6_batch_last_error(bt.handle) == gpu_lib.MLS6_ERR_TIMEOUT
    gpu_lib.mls6_batch_set_wait(bt.handle, 1 << 22, -1)
    rc = gpu_lib.mls6_batch_eval(bt.handle, pos.data_ptr(), 0, Fd.data_ptr(), C.addressof(Eh), 0)
    assert rc == 0
    assert np.array_equal(np.array(Eh[:]), E0)
    assert gpu_lib.mls6_batch_last_error(bt.handle) == 0
