"""Host-side logic of the benchmark (no GPU): the exact sampled forces that
define eps_F, the pair count behind the pair kernel's algorithmic work, and
the equal-accuracy interpolation."""
import numpy as np
import pytest

import bench
from paper_1308_4005_gb300 import inputs as I


def test_exact_forces_match_brute_force(orc):
    """Direct image sums within R = 20 reproduce the oracle's brute-force
    periodic forces (windowed image sum with its continuum tail), for a
    small box (replicated images) and a box wider than 2R (minimum image)."""
    box = (9.0, 10.0, 11.0)
    x, c = I.uniform_atoms(3, 300, box)
    idx = np.arange(0, 300, 7)
    ref = orc.brute(box, x, c, r_img=8 * max(box))["F"]
    Fe = bench.exact_forces(x, c, box, idx)
    assert np.abs(Fe - ref[idx]).max() <= 1e-7 * np.abs(ref).max()
    big = (42.0, 41.0, 43.0)
    xb, cb = I.uniform_atoms(4, 400, big)
    ib = np.arange(0, 400, 5)
    refb = orc.brute(big, xb, cb, r_img=5 * max(big))["F"]
    Fb = bench.exact_forces(xb, cb, big, ib)
    assert np.abs(Fb - refb[ib]).max() <= 1e-6 * np.abs(refb).max()
    assert bench.eps_F(Fb, refb[ib]) <= 1e-7


def test_pair_count_is_ordered_pairs_inside_cutoff():
    from scipy.spatial import cKDTree

    box = (12.0, 13.0, 9.0)
    x, _ = I.uniform_atoms(5, 800, box)
    p = cKDTree(np.mod(x, box), boxsize=box).query_pairs(3.0, output_type="ndarray")
    assert bench.count_pairs(x, box, 3.0) == 2 * len(p)


def test_equal_accuracy_interpolation():
    pts = [{"eps_F": 4e-4, "value": 8.0}, {"eps_F": 1.6e-3, "value": 16.0},
           {"eps_F": 1e-4, "value": 4.0}]
    r = bench.at_target(pts, 1e-4)
    assert r["value"] == pytest.approx(4.0) and r["how"] == "interpolated"
    r = bench.at_target(pts, 2e-4)  # halfway in log between 1e-4 and 4e-4
    assert r["value"] == pytest.approx(4.0 * np.sqrt(2.0))
    assert bench.at_target(pts[:2], 1e-4)["how"] == "extrapolated"


def test_equal_accuracy_takes_the_fastest_spacing():
    """Each form's figure at the target error is taken on the grid spacing h
    whose cutoff sweep reaches it fastest; a bracketing (interpolated) h is
    preferred to an extrapolated one."""
    fine = [{"h": 1.0, "eps_F": 4e-4, "value": 8.0}, {"h": 1.0, "eps_F": 1e-4, "value": 4.0}]
    coarse = [{"h": 2.0, "eps_F": 4e-4, "value": 12.0}, {"h": 2.0, "eps_F": 1e-4, "value": 6.0}]
    r = bench.best_at_target(fine + coarse, 1e-4)
    assert r["h"] == 2.0 and r["value"] == pytest.approx(6.0) and r["how"] == "interpolated"
    # a faster but extrapolated h loses to an interpolated one
    far = [{"h": 3.0, "eps_F": 8e-4, "value": 50.0}, {"h": 3.0, "eps_F": 4e-4, "value": 40.0}]
    r = bench.best_at_target(fine + far, 1e-4)
    assert r["h"] == 1.0 and r["how"] == "interpolated"
    assert bench.best_at_target([], 1e-4)["value"] is None


def test_learned_configuration_workload():
    """slab4m: 4,194,304 atoms at density 0.8 in a centred slab of the
    160 x 160 x 240 box (thickness N / (0.8 * 160^2)), the coarse grid h = 2
    with the level count of the automatic rule."""
    from paper_1308_4005_gb300 import mls6

    w = I.workload("slab4m")
    assert w.N == 4194304 and w.box == (160.0, 160.0, 240.0)
    (x0, x1), (y0, y1), (z0, z1) = w.region
    t = z1 - z0
    assert (x1 - x0, y1 - y0) == (160.0, 160.0)
    assert w.N / (160.0 * 160.0 * t) == pytest.approx(0.8)
    assert z0 == pytest.approx(240.0 - z1)
    assert (w.a, w.h) == (3.0, 2.0)
    assert w.levels == mls6.mls6_auto_levels(w.box, w.h)
