"""GPU parity: the CUDA path (through the C-ABI) against the FP64 oracle on the
same seeded inputs.

Tolerances
  FP64 path (spec bar): |dE|/|E| <= 1e-12 and
      max_i |F_i - F_i^orc| / RMS(F^orc) <= 1e-11; the virial and per-atom
      energies are held to 1e-11 of their largest entry.
  FP32 path (pair kernel and grids in float, energy/virial accumulated in
      double): unit roundoff u = 2^-24 = 6.0e-8.  A force is a sum of ~100
      pair terms of size up to ~30 (6 c^2 r^-7 at r = 0.8) that cancel to
      O(1..10), plus a 64-node interpolation of grid potentials that are
      themselves ~10^3-term stencil sums; the accumulated rounding is
      bounded by ~ u * sqrt(terms) * max|term| ~ 6e-8 * 10 * 30 = 2e-5 of
      the RMS force, and the tests use 1e-4.  Per-atom energies carry
      u * sqrt(100) relative error and the total sums them in double, so
      |dE|/|E| <= 2e-6.
"""
import zlib

import numpy as np
import pytest

from paper_1308_4005_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL64 = dict(E=1e-12, F=1e-11, W=1e-11, eatom=1e-11)
TOL32 = dict(E=2e-6, F=1e-4, W=2e-5, eatom=2e-5)


def gpu_eval(mls6, box, a, h, levels, x, c, prec, packed=True, virial=True, atom_energy=True,
             shift=None):
    import torch

    dt = torch.float64 if prec == "fp64" else torch.float32
    N = len(c)
    plan = mls6.Plan(box, N, a, h, levels, precision=prec)
    xx = x if shift is None else x + shift
    if packed:
        pos = torch.tensor(np.c_[xx, c] if N else np.zeros((0, 4)), dtype=dt, device="cuda")
        cc = None
    else:
        pos = torch.tensor(xx if N else np.zeros((0, 3)), dtype=dt, device="cuda").contiguous()
        cc = torch.tensor(c, dtype=dt, device="cuda")
    r = plan.evaluate(pos, cc, virial=virial, atom_energy=atom_energy)
    torch.cuda.synchronize()
    assert mls6.mls6_last_error(plan.handle) == 0
    out = r["out"].cpu().numpy()
    res = dict(E=out[0], W=out[1:7], F=r["F"].cpu().double().numpy(), plan=plan)
    if atom_energy:
        res["eatom"] = r["eatom"].cpu().numpy()
    return res


def as_prec(x, c, prec):
    if prec == "fp32":
        return x.astype(np.float32).astype(np.float64), c.astype(np.float32).astype(np.float64)
    return x, c


def compare(g, o, tol, label=""):
    E_err = abs(g["E"] - o["E"]) / abs(o["E"])
    rms = np.sqrt(np.mean(np.sum(o["F"] ** 2, axis=1)))
    F_err = np.abs(g["F"] - o["F"]).max() / rms
    W_err = np.abs(g["W"] - o["W"]).max() / np.abs(o["W"]).max()
    msg = f"{label} dE={E_err:.3e} dF={F_err:.3e} dW={W_err:.3e}"
    assert E_err <= tol["E"], msg
    assert F_err <= tol["F"], msg
    assert W_err <= tol["W"], msg
    if "eatom" in g and "eatom" in o:
        ea_err = np.abs(g["eatom"] - o["eatom"]).max() / np.abs(o["eatom"]).max()
        assert ea_err <= tol["eatom"], f"{msg} deatom={ea_err:.3e}"
    return E_err, F_err, W_err


# ------------------------------------------------------------- FP64 parity

def test_cube1000_fp64_parity(gpu_lib, orc):
    """N=1000 cube, a=2.5, h=1 (-> 12^3, h=0.833), 3 levels, FP64."""
    w = I.workload("cube1000")
    x, c = I.generate(w)
    n = orc.grid_dims(w.box, w.h, w.levels)
    o = orc.evaluate(w.box, w.a, n, w.levels, x, c)
    g = gpu_eval(gpu_lib, w.box, w.a, w.h, w.levels, x, c, "fp64")
    compare(g, o, TOL64, "cube1000")
    assert g["eatom"].sum() == pytest.approx(g["E"], rel=1e-13)


def test_stage_grids_fp64(gpu_lib, orc):
    """Every grid of every level: xi^k, e^k, e^{k,tot}."""
    box, a, h, l = (8.0, 9.0, 10.0), 2.0, 0.5, 3
    x, c = I.uniform_atoms(17, 300, box)
    g = gpu_eval(gpu_lib, box, a, h, l, x, c, "fp64")
    n = orc.grid_dims(box, h, l)
    G = orc.grids(box, a, n, l, x, c)
    for k in range(1, l + 1):
        for which in range(3):
            ref = G[k - 1][which]
            got = gpu_lib.mls6_debug_grid(g["plan"].handle, k, which)
            assert got.shape == ref.shape
            assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), (k, which)


CASES = [
    # name, N, box, a, h, levels
    ("one_atom", 1, (6.0, 6.0, 6.0), 2.0, 0.75, 2),
    ("two_atoms", 2, (6.0, 7.0, 8.0), 2.0, 0.75, 2),
    ("ragged_aniso", 37, (5.0, 6.0, 9.0), 1.8, 0.6, 3),
    ("single_level", 300, (8.0, 8.0, 8.0), 2.0, 1.0, 1),
    ("box_below_2a", 60, (4.0, 4.5, 5.0), 2.5, 0.5, 2),
    ("tiny_top_grid", 200, (8.0, 8.0, 16.0), 1.5, 1.0, 4),
    ("slab_5_levels", 900, (9.6, 9.6, 38.4), 2.4, 0.6, 5),
    ("many_tiles", 3000, (16.0, 15.0, 14.0), 2.5, 0.7, 3),
]


@pytest.mark.parametrize("name,N,box,a,h,l", CASES, ids=[c[0] for c in CASES])
def test_small_cases_fp64(gpu_lib, orc, name, N, box, a, h, l):
    region = None
    if name.startswith("slab"):
        region = ((0, box[0]), (0, box[1]), (0.35 * box[2], 0.65 * box[2]))
    x, c = I.uniform_atoms(zlib.crc32(name.encode()) % 10000, N, box, region=region)
    n = orc.grid_dims(box, h, l)
    o = orc.evaluate(box, a, n, l, x, c)
    g = gpu_eval(gpu_lib, box, a, h, l, x, c, "fp64")
    compare(g, o, TOL64, name)


SHAPE_CASES = [c for c in CASES if c[0] in ("two_atoms", "ragged_aniso", "box_below_2a",
                                            "slab_5_levels", "many_tiles")]


# FP32 only where the energy is not a small difference of large terms (with
# two atoms the self term and the grid part cancel to ~1e-5 of FP32 rounding)
SHAPE_PARAMS = [c + ("fp64",) for c in SHAPE_CASES] + [
    c + ("fp32",) for c in SHAPE_CASES if c[1] >= 900]


@pytest.mark.parametrize("name,N,box,a,h,l,prec", SHAPE_PARAMS,
                         ids=[f"{c[0]}-{c[-1]}" for c in SHAPE_PARAMS])
def test_pair_kernel_shapes(gpu_lib, orc, name, N, box, a, h, l, prec):
    """Every pair-kernel shape (lanes per atom 1..8: one atom per lane
    group; 16, 32: warp form; 128, 256, 512: queue form with 2, 4, 8 atoms
    per warp; 1024: cluster form) against the oracle; the warp and queue
    forms are refused where the neighbour range is too wide for them, the
    cluster form also in FP64 and below 16 cells along x."""
    import torch

    region = None
    if name.startswith("slab"):
        region = ((0, box[0]), (0, box[1]), (0.35 * box[2], 0.65 * box[2]))
    x, c = I.uniform_atoms(zlib.crc32(name.encode()) % 10000, N, box, region=region)
    x, c = as_prec(x, c, prec)
    n = orc.grid_dims(box, h, l)
    o = orc.evaluate(box, a, n, l, x, c)
    dt = torch.float64 if prec == "fp64" else torch.float32
    plan = gpu_lib.Plan(box, N, a, h, l, precision=prec)
    pos = torch.tensor(np.c_[x, c], dtype=dt, device="cuda")
    tol = TOL64 if prec == "fp64" else TOL32
    ran = []
    for split in (1, 2, 4, 8, 16, 32, 128, 256, 512, 1024):
        try:
            gpu_lib.mls6_set_tuning(plan.handle, split, 0)
        except gpu_lib.MLS6Error:
            assert split > 8, split
            continue
        r = plan.evaluate(pos, virial=True, atom_energy=False)
        torch.cuda.synchronize()
        out = r["out"].cpu().numpy()
        g = dict(E=out[0], W=out[1:7], F=r["F"].cpu().double().numpy())
        compare(g, o, tol, f"{name} split={split}")
        r2 = plan.evaluate(pos, virial=True, atom_energy=False)
        torch.cuda.synchronize()
        assert torch.equal(r["F"], r2["F"]) and torch.equal(r["out"], r2["out"])
        ran.append(split)
    assert ran[:4] == [1, 2, 4, 8]
    if name in ("slab_5_levels", "many_tiles"):
        assert ran[4:] == [16, 32, 128, 256, 512]


def test_virial_strain_derivative_many_blocks(gpu_lib):
    """W_aa = -dE/d eps_aa (reading R8: the grids deform with the box) on a
    system large enough that the interpolation runs in several waves and its
    first blocks sum the virial records in slices (>= 608 blocks of 256
    atoms): the library's FP64 virial against central differences of its own
    energy under a diagonal strain (the grid counts stay fixed)."""
    import torch

    L = 57.0
    N = int(0.85 * L ** 3)
    assert (N + 255) // 256 >= 608
    box, a, h, l = (L, L, L), 2.5, 1.0, 4
    x, c = I.uniform_atoms(4242, N, box)

    def energy_virial(scale):
        b = tuple(L * s for s in scale)
        plan = gpu_lib.Plan(b, N, a, h, l, precision="fp64")
        pos = torch.tensor(np.c_[x * np.array(scale), c], dtype=torch.float64, device="cuda")
        r = plan.evaluate(pos, virial=True, atom_energy=False)
        torch.cuda.synchronize()
        out = r["out"].cpu().numpy().copy()
        plan.close()
        return out[0], out[1:7]

    _, W = energy_virial((1.0, 1.0, 1.0))
    d = 1e-5
    for k in range(3):
        sp = [1.0, 1.0, 1.0]
        sm = [1.0, 1.0, 1.0]
        sp[k] += d
        sm[k] -= d
        fd = -(energy_virial(sp)[0] - energy_virial(sm)[0]) / (2 * d)
        assert W[k] == pytest.approx(fd, rel=2e-5), (k, W[k], fd)


def test_no_atoms(gpu_lib):
    g = gpu_eval(gpu_lib, (8.0, 8.0, 8.0), 2.0, 1.0, 3, np.zeros((0, 3)), np.zeros(0), "fp64")
    assert g["E"] == 0.0
    assert np.all(g["W"] == 0.0)


def test_unwrapped_positions_and_separate_coefficients(gpu_lib, orc):
    box, a, h, l = (7.0, 8.0, 9.0), 2.0, 0.7, 3
    x, c = I.uniform_atoms(23, 200, box)
    n = orc.grid_dims(box, h, l)
    o = orc.evaluate(box, a, n, l, x, c)
    k = np.random.default_rng(5).integers(-3, 4, size=x.shape)
    g = gpu_eval(gpu_lib, box, a, h, l, x, c, "fp64", packed=False, shift=k * np.array(box))
    compare(g, o, dict(E=1e-12, F=1e-10, W=1e-11, eatom=1e-11), "unwrapped")


def test_repeatable_and_translation_by_coarsest_vector(gpu_lib):
    box, a, h, l = (8.0, 8.0, 8.0), 2.0, 0.5, 3
    x, c = I.uniform_atoms(29, 400, box)
    g1 = gpu_eval(gpu_lib, box, a, h, l, x, c, "fp64")
    g2 = gpu_eval(gpu_lib, box, a, h, l, x, c, "fp64")
    # every sum runs in a fixed order (cells sorted by input index,
    # fixed-point anterpolation, fixed-order reductions): bit for bit
    assert g2["E"] == g1["E"]
    assert np.array_equal(g2["F"], g1["F"]) and np.array_equal(g2["W"], g1["W"])
    assert np.array_equal(g2["eatom"], g1["eatom"])
    s = np.array(box) / 16 * 4 * np.array([1, 2, 0])
    g3 = gpu_eval(gpu_lib, box, a, h, l, x + s, c, "fp64")
    assert g3["E"] == pytest.approx(g1["E"], rel=1e-12)
    assert np.abs(g3["F"] - g1["F"]).max() <= 1e-11 * np.abs(g1["F"]).max()


def test_nonfinite_input_is_reported(gpu_lib):
    import torch

    box = (8.0, 8.0, 8.0)
    x, c = I.uniform_atoms(31, 50, box)
    x[7, 1] = np.nan
    plan = gpu_lib.Plan(box, 50, 2.0, 1.0, 2, precision="fp64")
    pos = torch.tensor(np.c_[x, c], dtype=torch.float64, device="cuda")
    F = torch.empty((50, 3), dtype=torch.float64, device="cuda")
    import ctypes as C

    E = C.c_double()
    rc = gpu_lib.mls6_eval(plan.handle, pos.data_ptr(), 0, F.data_ptr(), C.addressof(E), 0)
    assert rc == gpu_lib.MLS6_ERR_NONFINITE
    assert gpu_lib.mls6_last_error(plan.handle) == gpu_lib.MLS6_ERR_NONFINITE


# ------------------------------------------------ FP32 and full-size parity

def test_slab65536_fp32_parity(gpu_lib, orc):
    """N=65,536 liquid/vacuum slab (40x40x120, rho=0.8), a=3, h=1.25, 4 levels,
    FP32 with FP64 energy/virial: full comparison with the FP64 oracle."""
    w = I.workload("slab65536")
    x, c = I.generate(w)
    x, c = as_prec(x, c, "fp32")
    n = orc.grid_dims(w.box, w.h, w.levels)
    o = orc.evaluate(w.box, w.a, n, w.levels, x, c)
    g = gpu_eval(gpu_lib, w.box, w.a, w.h, w.levels, x, c, "fp32")
    compare(g, o, TOL32, "slab65536/fp32")


def test_slab65536_fp64_sampled(gpu_lib, orc):
    w = I.workload("slab65536")
    x, c = I.generate(w)
    idx = np.random.default_rng(3).choice(w.N, 400, replace=False)
    n = orc.grid_dims(w.box, w.h, w.levels)
    o = orc.evaluate_sample(w.box, w.a, n, w.levels, x, c, idx)
    g = gpu_eval(gpu_lib, w.box, w.a, w.h, w.levels, x, c, "fp64")
    # force scale from the oracle's sampled forces, not the GPU's own
    rms = np.sqrt(np.mean(np.sum(o["F"] ** 2, axis=1)))
    assert np.abs(g["F"][idx] - o["F"]).max() <= 1e-11 * rms
    assert np.abs(g["eatom"][idx] - o["eatom"]).max() <= 1e-11 * np.abs(o["eatom"]).max()
    assert g["eatom"].sum() == pytest.approx(g["E"], rel=1e-13)


@pytest.mark.slow
def test_cube1m_fp32_sampled(gpu_lib, orc):
    """N=1,048,576 cube at rho=0.85, a=3, h=1 (112^3), 5 levels, FP32: sampled
    atoms against the oracle (forces and per-atom energies), the total as the
    sum of per-atom energies (both formed from the same FP32 per-atom values;
    the total adds them in FP32 within warps, relative rounding of order
    2^-24 sqrt(32 / (N/32)) ~ 2e-9)."""
    w = I.workload("cube1m")
    x, c = I.generate(w)
    x, c = as_prec(x, c, "fp32")
    idx = np.random.default_rng(4).choice(w.N, 300, replace=False)
    n = orc.grid_dims(w.box, w.h, w.levels)
    o = orc.evaluate_sample(w.box, w.a, n, w.levels, x, c, idx)
    g = gpu_eval(gpu_lib, w.box, w.a, w.h, w.levels, x, c, "fp32")
    # force scale from the oracle's sampled forces, not the GPU's own
    rms = np.sqrt(np.mean(np.sum(o["F"] ** 2, axis=1)))
    assert np.abs(g["F"][idx] - o["F"]).max() <= TOL32["F"] * rms
    assert np.abs(g["eatom"][idx] - o["eatom"]).max() <= TOL32["eatom"] * np.abs(o["eatom"]).max()
    assert g["eatom"].sum() == pytest.approx(g["E"], rel=1e-8)


# ------------------------------------------------------ execution modes

def _fixed_buffers(N, prec):
    import torch

    dt = torch.float64 if prec == "fp64" else torch.float32
    return (torch.empty((N, 4), dtype=dt, device="cuda"),
            torch.empty((N, 3), dtype=dt, device="cuda"),
            torch.zeros(8, dtype=torch.float64, device="cuda"))


def test_graph_replay_matches_eager_and_tracks_inputs(gpu_lib):
    """The captured graph replays with the same buffers; new positions written
    into the same input buffer are picked up; eager launches agree."""
    import torch

    box, a, h, l = (9.0, 9.0, 12.0), 2.2, 0.75, 3
    x1, c = I.uniform_atoms(41, 500, box)
    x2, _ = I.uniform_atoms(42, 500, box)
    plan = gpu_lib.Plan(box, 500, a, h, l, precision="fp64")
    pos, F, out = _fixed_buffers(500, "fp64")
    res = {}
    for mode in ("graph", "eager"):
        gpu_lib.mls6_set_graph(plan.handle, mode == "graph")
        for tag, xx in (("x1", x1), ("x2", x2), ("x1b", x1)):
            pos.copy_(torch.tensor(np.c_[xx, c], dtype=torch.float64))
            rc = gpu_lib.mls6_eval(plan.handle, pos.data_ptr(), 0, F.data_ptr(), out.data_ptr(),
                                   out.data_ptr() + 8)
            assert rc == 0
            torch.cuda.synchronize()
            res[(mode, tag)] = (out[:7].cpu().numpy().copy(), F.cpu().numpy().copy())
    for tag in ("x1", "x2", "x1b"):
        (og, Fg), (oe, Fe) = res[("graph", tag)], res[("eager", tag)]
        assert np.allclose(og, oe, rtol=1e-14, atol=0)
        assert np.abs(Fg - Fe).max() <= 1e-13 * np.abs(Fe).max()
    assert not np.allclose(res[("graph", "x1")][0], res[("graph", "x2")][0])
    assert np.allclose(res[("graph", "x1")][0], res[("graph", "x1b")][0], rtol=1e-14, atol=0)


def test_caller_stream_ordering(gpu_lib):
    """Work on the caller's stream before and after mls6_eval is ordered
    with the library's internal streams."""
    import torch

    box, a, h, l = (9.0, 9.0, 9.0), 2.2, 0.75, 3
    x, c = I.uniform_atoms(43, 400, box)
    ref = gpu_eval(gpu_lib, box, a, h, l, x, c, "fp64", atom_energy=False)
    s = torch.cuda.Stream()
    plan = gpu_lib.Plan(box, 400, a, h, l, precision="fp64", stream=s.cuda_stream)
    pos, F, out = _fixed_buffers(400, "fp64")
    src = torch.tensor(np.c_[x, c], dtype=torch.float64).pin_memory()
    Fh = torch.empty((400, 3), dtype=torch.float64).pin_memory()
    with torch.cuda.stream(s):
        for _ in range(3):
            pos.zero_()
            F.fill_(7.0)
            pos.copy_(src, non_blocking=True)
            rc = gpu_lib.mls6_eval(plan.handle, pos.data_ptr(), 0, F.data_ptr(), out.data_ptr(),
                                   out.data_ptr() + 8)
            assert rc == 0
            Fh.copy_(F, non_blocking=True)
            s.synchronize()
            assert np.abs(Fh.numpy() - ref["F"]).max() <= 1e-13 * np.abs(ref["F"]).max()


CLUSTER_CASES = [
    # name, N, box, a, h, levels, continuity (>= 16 cells along x)
    ("cl_cube", 4001, (24.0, 14.0, 13.0), 2.5, 0.8, 3, 2),
    ("cl_slab_vacuum", 3000, (26.0, 12.0, 30.0), 3.0, 1.0, 3, 2),
    ("cl_thin_yz", 700, (30.0, 6.0, 5.5), 2.0, 0.6, 2, 2),
    ("cl_smoothing_c3", 2500, (22.0, 13.0, 12.0), 2.5, 0.8, 3, 3),
]


@pytest.mark.parametrize("name,N,box,a,h,l,cont", CLUSTER_CASES, ids=[c[0] for c in CLUSTER_CASES])
def test_pair_cluster_form(gpu_lib, orc, name, N, box, a, h, l, cont):
    """The FP32 cluster form (8 atoms per warp, segments of one cell row,
    branch-free candidates) against the oracle, with and without the
    virial, ragged atom counts, a slab with empty rows (segments split by
    row and by the 8-cell rule), boxes thinner than the neighbour range in
    y and z, and a C^3 smoothing function; repeatable bit for bit."""
    import torch

    region = None
    if "slab" in name:
        region = ((0, box[0]), (0, box[1]), (0.35 * box[2], 0.65 * box[2]))
    x, c = I.uniform_atoms(zlib.crc32(name.encode()) % 10000, N, box, region=region)
    x, c = as_prec(x, c, "fp32")
    n = orc.grid_dims(box, h, l)
    with orc.smoothing_order(cont):
        o = orc.evaluate(box, a, n, l, x, c)
    plan = gpu_lib.Plan(box, N, a, h, l, precision="fp32", continuity=cont)
    gpu_lib.mls6_set_tuning(plan.handle, 1024, 0)
    assert gpu_lib.mls6_get_tuning(plan.handle)[0] == 1024
    pos = torch.tensor(np.c_[x, c], dtype=torch.float32, device="cuda")
    for vir in (True, False):
        r = plan.evaluate(pos, virial=vir, atom_energy=False)
        torch.cuda.synchronize()
        out = r["out"].cpu().numpy()
        g = dict(E=out[0], W=out[1:7] if vir else o["W"], F=r["F"].cpu().double().numpy())
        compare(g, o, TOL32, f"{name} cluster virial={vir}")
        r2 = plan.evaluate(pos, virial=vir, atom_energy=False)
        torch.cuda.synchronize()
        assert torch.equal(r["F"], r2["F"]) and torch.equal(r["out"], r2["out"])


def test_pair_cluster_form_selection_and_refusals(gpu_lib):
    """The cluster form is selected by mls6_set_tuning only (the per-atom
    kernel stays the default); FP64 and boxes with < 16 cells along x
    refuse it."""
    c = I.workload("cube1m")
    for prec in ("fp32", "mixed"):
        p = gpu_lib.Plan(c.box, 40000, c.a, c.h, c.levels, precision=prec)
        assert gpu_lib.mls6_get_tuning(p.handle)[0] != 1024
        gpu_lib.mls6_set_tuning(p.handle, 1024, 0)
        assert gpu_lib.mls6_get_tuning(p.handle)[0] == 1024
    p64 = gpu_lib.Plan(c.box, 40000, c.a, c.h, c.levels, precision="fp64")
    with pytest.raises(gpu_lib.MLS6Error):
        gpu_lib.mls6_set_tuning(p64.handle, 1024, 0)
    narrow = gpu_lib.Plan((20.0, 20.0, 20.0), 5000, 3.0, 1.0, 2, precision="fp32")
    with pytest.raises(gpu_lib.MLS6Error):
        gpu_lib.mls6_set_tuning(narrow.handle, 1024, 0)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_positions_from_page_locked_host_memory(gpu_lib, prec):
    """Positions (and separate coefficients) in page-locked host memory are
    read by the binning kernel directly: the results equal those from device
    memory bit for bit, with and without the captured graph.  Host memory
    that is not page-locked is refused with MLS6_ERR_ARG before any kernel
    runs.  Forces and outputs stay in device memory."""
    import torch

    L = gpu_lib.load()
    box, a, h, l = (12.0, 11.0, 13.0), 2.5, 0.8, 3
    x, c = I.uniform_atoms(91, 1500, box)
    N = len(c)
    dt = torch.float64 if prec == "fp64" else torch.float32
    dev_xc = torch.tensor(np.c_[x, c], dtype=dt, device="cuda")
    host_xc = torch.tensor(np.c_[x, c], dtype=dt).pin_memory()
    host_x = torch.tensor(np.ascontiguousarray(x), dtype=dt).pin_memory()
    host_c = torch.tensor(np.ascontiguousarray(c), dtype=dt).pin_memory()
    plan = gpu_lib.Plan(box, N, a, h, l, precision=prec)

    def run(pos_ptr, c_ptr):
        F = torch.empty((N, 3), dtype=dt, device="cuda")
        out = torch.zeros(7, dtype=torch.float64, device="cuda")
        rc = L.mls6_eval(plan.handle, pos_ptr, c_ptr, F.data_ptr(), out.data_ptr(),
                         out.data_ptr() + 8)
        assert rc == 0, gpu_lib.status_string(rc)
        torch.cuda.synchronize()
        return F, out

    F0, o0 = run(dev_xc.data_ptr(), None)
    for graph in (1, 0):
        assert L.mls6_set_graph(plan.handle, graph) == 0
        F1, o1 = run(host_xc.data_ptr(), None)
        assert torch.equal(F1, F0) and torch.equal(o1, o0)
        F2, o2 = run(host_x.data_ptr(), host_c.data_ptr())
        assert torch.equal(F2, F0) and torch.equal(o2, o0)
    pageable = np.ascontiguousarray(np.c_[x, c], dtype=np.float64 if prec == "fp64" else np.float32)
    F = torch.empty((N, 3), dtype=dt, device="cuda")
    rc = L.mls6_eval(plan.handle, pageable.ctypes.data, None, F.data_ptr(), None, None)
    assert rc == gpu_lib.MLS6_ERR_ARG
