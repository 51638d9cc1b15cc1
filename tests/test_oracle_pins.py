"""Pins of the FP64 CPU oracle against facts that do not come from the oracle.

Each test checks the oracle against something the paper or mathematics fixes:
closed-form values, identities of the kernel split, textbook special cases,
brute-force periodic sums, finite differences, symmetries and the error
behaviour of Sec. III.B/III.C.  A plausible slip in the oracle (dropped term,
wrong sign or index, transposed operator) breaks at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_1308_4005_gb300 import inputs as I

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))


# ---------------------------------------------------------------- closed forms

def test_gamma_golden_and_branches(orc):
    assert orc.gamma(0.0) == GOLD["gamma_at_0"]["value"]
    assert orc.gamma(1.0) == GOLD["gamma_at_1"]["value"]
    assert abs(orc.gamma(1.0 - 1e-15) - 1.0) < 1e-13
    for rho in (1.0, 1.5, 3.0, 10.0):
        assert orc.gamma(rho) == pytest.approx(rho ** -6, rel=1e-15)


def test_gamma_is_C2_not_C3_at_one(orc):
    """Eq. (gamma) is C^2 at rho = 1: value 1, slope -6, curvature 42 from
    both sides, third derivative discontinuous."""
    def d(f, x, k, s):
        # one-sided finite differences of order k with step s (s<0: left side)
        if k == 1:
            return (f(x + s) - f(x)) / s
        if k == 2:
            return (f(x + 2 * s) - 2 * f(x + s) + f(x)) / (s * s)
        return (f(x + 3 * s) - 3 * f(x + 2 * s) + 3 * f(x + s) - f(x)) / (s ** 3)

    g = orc.gamma
    assert orc.dgamma(1.0 - 1e-12) == pytest.approx(-6.0, rel=1e-9)
    assert orc.dgamma(1.0) == pytest.approx(-6.0, rel=1e-15)
    for s in (1e-4, -1e-4):
        assert d(g, 1.0, 1, s) == pytest.approx(-6.0, abs=0.03)
        assert d(g, 1.0, 2, s) == pytest.approx(42.0, rel=0.05)
    left, right = d(g, 1.0, 3, -1e-3), d(g, 1.0, 3, 1e-3)
    assert left == pytest.approx(2904.0, rel=0.1)      # d^3/drho^3 of the polynomial branch
    assert right == pytest.approx(-336.0, rel=0.1)     # d^3/drho^3 of rho^-6
    # derivative routine agrees with finite differences away from the joint
    for rho in (0.3, 0.8, 1.7):
        fd = (g(rho + 1e-6) - g(rho - 1e-6)) / 2e-6
        assert orc.dgamma(rho) == pytest.approx(fd, rel=1e-7, abs=1e-8)


@pytest.mark.parametrize("levels", [1, 2, 3, 4, 5])
def test_split_telescopes_to_r6(orc, levels):
    """Eq. (complete-splitting): sum_{k=0}^{l} g_k(r) = r^-6 pointwise."""
    a = 2.5
    rng = np.random.default_rng(7 + levels)
    for r in np.concatenate([rng.uniform(0.3, 50.0, 400), [a, 2 * a, 4 * a, 8 * a, 16 * a]]):
        s = sum(orc.gk(k, levels, a, r) for k in range(levels + 1))
        assert s == pytest.approx(r ** -6, rel=1e-13)


@pytest.mark.parametrize("levels", [1, 2, 3, 5])
def test_self_term_is_sum_of_grid_kernels_at_zero(orc, levels):
    """Eq. (self-interaction-energy): sum_{k>=1} g_k(0) = gamma(0)/a^6."""
    a = 1.7
    s = sum(orc.gk(k, levels, a, 0.0) for k in range(1, levels + 1))
    assert s == pytest.approx(15.0 / 8.0 / a ** 6, rel=1e-14)


def test_kernel_cutoffs_and_level_similarity(orc):
    """g_k vanishes beyond 2^k a for k < l (Sec. II.A.4), g_0 beyond a, and
    g_k(2^(k-1) r) = 2^(-6(k-1)) g_1(r) (Sec. II.A.4, same arguments on every
    grid)."""
    a, l = 3.0, 5
    for k in range(0, l):
        cut = a * 2 ** k
        assert orc.gk(k, l, a, cut) == 0.0
        assert orc.gk(k, l, a, cut * 1.01) == 0.0
        assert abs(orc.gk(k, l, a, cut * (1 - 1e-9))) < 1e-12 * abs(orc.gk(k, l, a, 0.5 * cut))
    for k in range(2, l):
        for r in (0.0, 0.7, 2.2, 4.9, 5.99):
            assert orc.gk(k, l, a, 2 ** (k - 1) * r) == pytest.approx(
                2.0 ** (-6 * (k - 1)) * orc.gk(1, l, a, r), rel=1e-13, abs=1e-300)
    assert orc.gk(l, l, a, 1e3) == pytest.approx(1e-18, rel=1e-12)  # g_l -> r^-6


def test_kernel_derivatives_match_finite_differences(orc):
    a, l = 2.0, 3
    for k in range(l + 1):
        for r in (0.45, 1.3, 2.6, 5.1, 9.0):
            f = lambda t: orc.gk(k, l, a, t)
            fd = (f(r + 1e-6) - f(r - 1e-6)) / 2e-6
            assert orc.dgk(k, l, a, r) == pytest.approx(fd, rel=1e-6, abs=1e-12)


def test_Phi_golden_half_integers(orc):
    g = GOLD["Phi_half_integers"]
    for t, v in zip(g["t"], g["value"]):
        assert orc.Phi(t) == v


def test_Phi_is_keys_cubic_convolution(orc):
    """Eq. (Phi-Hermite) equals Keys' cubic-convolution kernel with a = -1/2
    (textbook form (a+2)|x|^3-(a+3)|x|^2+1, a|x|^3-5a|x|^2+8a|x|-4a)."""
    A = -0.5
    for t in np.linspace(-2.5, 2.5, 1001):
        x = abs(t)
        if x <= 1:
            k = (A + 2) * x ** 3 - (A + 3) * x ** 2 + 1
        elif x < 2:
            k = A * x ** 3 - 5 * A * x ** 2 + 8 * A * x - 4 * A
        else:
            k = 0.0
        assert orc.Phi(t) == pytest.approx(k, abs=1e-14)


def test_Phi_reproduces_quadratics_not_cubics(orc):
    """Interpolation order p = 3 (Sec. III.B): sum_m Phi(t-m) m^j = t^j for
    j = 0, 1, 2 and not for j = 3."""
    for t in np.linspace(-0.99, 1.99, 37):
        ms = np.arange(-4, 6)
        w = np.array([orc.Phi(t - m) for m in ms])
        for j in range(3):
            assert np.dot(w, ms.astype(float) ** j) == pytest.approx(t ** j, abs=1e-14)
    t = 0.3
    w = np.array([orc.Phi(t - m) for m in np.arange(-4, 6)])
    assert abs(np.dot(w, np.arange(-4, 6) ** 3.0) - t ** 3) > 1e-3


def test_Phi_derivative_and_C1(orc):
    for t in np.linspace(-2.3, 2.3, 47):
        fd = (orc.Phi(t + 1e-7) - orc.Phi(t - 1e-7)) / 2e-7
        assert orc.dPhi(t) == pytest.approx(fd, abs=1e-7)
    for t0 in (-2.0, -1.0, 1.0, 2.0):  # C^1 at the joints
        assert orc.dPhi(t0 - 1e-12) == pytest.approx(orc.dPhi(t0 + 1e-12), abs=1e-9)


def test_grid_dims_golden(orc):
    for case in GOLD["grid_dims"]["cases"]:
        assert orc.grid_dims(case["L"], case["h"], case["levels"]) == tuple(case["n"])


# ------------------------------------------------------- exact periodic sums

def _sc_ewald(beta):
    """Independent Ewald evaluation of sum'_n |n|^-6 over the unit simple cubic
    lattice: real-space r^-6 Q(3, beta^2 r^2) + reciprocal Poisson sum of the
    smooth remainder - its value at r = 0 (beta^6/6)."""
    from scipy.special import erfc

    M = 6
    g = np.arange(-M, M + 1)
    n = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).astype(float)
    r2 = (n ** 2).sum(1)
    nz = r2 > 0
    x = beta ** 2 * r2[nz]
    real = np.sum(np.exp(-x) * (1 + x + 0.5 * x * x) / r2[nz] ** 3)
    k = 2 * np.pi * np.sqrt(r2)
    b = k / (2 * beta)
    Fk = (np.pi ** 1.5 * beta ** 3 / 3) * ((1 - 2 * b * b) * np.exp(-b * b)
                                           + 2 * np.sqrt(np.pi) * b ** 3 * erfc(b))
    return real + Fk.sum() - beta ** 6 / 6


def test_sc_lattice_sum_brute_vs_ewald(orc):
    """Simple-cubic sum'|n|^-6 = 8.40192...: the oracle's direct image sum with
    continuum tail against an Ewald summation written in this test."""
    e1, e2 = _sc_ewald(1.7), _sc_ewald(2.3)
    assert e1 == pytest.approx(e2, rel=1e-13)
    gold = GOLD["sc_lattice_sum_r6"]
    assert e1 == pytest.approx(gold["value"], rel=gold["rtol"])
    b = orc.brute(np.eye(3), np.zeros((1, 3)), np.ones(1), r_img=160.0)
    b80 = orc.brute(np.eye(3), np.zeros((1, 3)), np.ones(1), r_img=80.0)
    assert -2.0 * b["E"] == pytest.approx(e1, rel=1e-14)
    assert -2.0 * b80["E"] == pytest.approx(e1, rel=1e-14)
    assert np.abs(b["F"]).max() < 1e-12
    # virial of the isotropic lattice: W = 2E * I (tr W = 6E)
    assert b["W"][:3] == pytest.approx([2 * b["E"]] * 3, rel=1e-13)
    assert np.abs(b["W"][3:]).max() < 1e-12


def test_brute_force_converges_in_image_radius(orc):
    x, c = I.uniform_atoms(11, 30, (5.0, 6.0, 7.0))
    b1 = orc.brute((5.0, 6.0, 7.0), x, c, r_img=60.0)
    b2 = orc.brute((5.0, 6.0, 7.0), x, c, r_img=120.0)
    assert b1["E"] == pytest.approx(b2["E"], rel=1e-9)
    assert np.abs(b1["F"] - b2["F"]).max() < 1e-9 * np.abs(b2["F"]).max()
    assert b2["W"][:3].sum() == pytest.approx(6 * b2["E"], rel=1e-12)


# --------------------------------------------- MLS special case: exactness

@pytest.mark.parametrize("box,h,levels,a", [
    ((10.0, 10.0, 10.0), 10.0 / 12, 3, 2.5),
    ((8.0, 8.0, 12.0), 0.5, 3, 1.5),
    ((6.0, 6.0, 6.0), 0.75, 2, 2.0),
    ((9.0, 9.0, 9.0), 0.75, 1, 2.0),
])
def test_mls_exact_on_coarsest_lattice(orc, box, h, levels, a):
    """Atoms on nodes of the coarsest grid: anterpolation, restriction,
    prolongation and interpolation reduce to injection (Phi(integer) =
    delta), so by Eq. (complete-splitting) the MLS energy equals the exact
    periodic lattice energy (same image radius on both sides)."""
    n = orc.grid_dims(box, h, levels)
    top = [v // 2 ** (levels - 1) for v in n]
    x, c = I.lattice_atoms(5, box, top, min(0.6, 40.0 / np.prod(top)))
    R = 30.0 * max(box)  # window width >= 1.5 cell lengths: aliasing below 1e-15
    m = orc.evaluate(box, a, n, levels, x, c, r_img=R)
    b = orc.brute(box, x, c, r_img=R)
    assert m["E"] == pytest.approx(b["E"], rel=1e-12)
    # full lattice with equal coefficients: every atom is an inversion centre
    xf, _ = I.lattice_atoms(6, box, top, 1.1)
    cf = np.full(xf.shape[0], 0.9)
    mf = orc.evaluate(box, a, n, levels, xf, cf, r_img=R)
    assert np.abs(mf["F"]).max() < 1e-11 * abs(mf["E"])


# ------------------------------------------------ MLS against exact physics

def test_mls_converges_to_brute_force_with_paper_order(orc):
    """Sec. III.B: force error ~ h^n with n = 2 for C^2 gamma and p = 3.  At
    a/h = 8..12 the per-step order is already close to 2 (averaged over
    seeds); the energy error falls too (oscillating, Sec. III.C)."""
    box, a = (6.0, 6.0, 6.0), 3.0
    eF = {0.375: [], 0.25: []}
    eE = {0.75: [], 0.25: []}
    for seed in (200, 201):
        x, c = I.uniform_atoms(seed, 40, box)
        b = orc.brute(box, x, c, r_img=120.0)
        for h in (0.75, 0.375, 0.25):
            r = orc.evaluate(box, a, orc.grid_dims(box, h, 1), 1, x, c)
            if h in eF:
                eF[h].append(np.linalg.norm(r["F"] - b["F"]) / np.linalg.norm(b["F"]))
            if h in eE:
                eE[h].append(abs(r["E"] - b["E"]) / abs(b["E"]))
    slope = math.log(np.mean(eF[0.375]) / np.mean(eF[0.25])) / math.log(1.5)
    assert 1.5 <= slope <= 2.5, slope
    assert np.mean(eE[0.25]) < 0.25 * np.mean(eE[0.75])


def test_mls_error_falls_with_cutoff(orc):
    """Sec. III.C: at fixed h, a larger cutoff a gives smaller errors."""
    box = (9.6, 9.6, 9.6)
    x, c = I.uniform_atoms(300, 100, box)
    b = orc.brute(box, x, c, r_img=96.0)
    errs = []
    for a in (1.6, 2.4, 3.2):
        r = orc.evaluate(box, a, orc.grid_dims(box, 0.8, 2), 2, x, c)
        errs.append(np.linalg.norm(r["F"] - b["F"]) / np.linalg.norm(b["F"]))
    assert errs[0] > errs[1] > errs[2]
    assert errs[0] > 10 * errs[2]


def test_level_count_has_small_effect(orc):
    """Table II trend: with the finest grid fixed, using 2..4 levels changes
    the energy by much less than the MLS error itself."""
    box = (9.6, 9.6, 9.6)
    x, c = I.uniform_atoms(301, 100, box)
    b = orc.brute(box, x, c, r_img=96.0)
    n = orc.grid_dims(box, 0.6, 4)
    Es = [orc.evaluate(box, 2.4, n, l, x, c)["E"] for l in (2, 3, 4)]
    err = abs(Es[0] - b["E"])
    assert max(Es) - min(Es) < 0.1 * err


# ------------------------------------------------ derivatives of the energy

def _small_case():
    box = (5.0, 6.0, 5.5)
    x, c = I.uniform_atoms(42, 24, box)
    return box, x, c, 1.8, (8, 8, 8), 2


def test_forces_are_minus_energy_gradient(orc):
    box, x, c, a, n, l = _small_case()
    r = orc.evaluate(box, a, n, l, x, c, r_img=60.0)
    d = 1e-5
    for i in (0, 7, 19):
        for k in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, k] += d
            xm[i, k] -= d
            ep = orc.evaluate(box, a, n, l, xp, c, r_img=60.0)["E"]
            em = orc.evaluate(box, a, n, l, xm, c, r_img=60.0)["E"]
            assert r["F"][i, k] == pytest.approx(-(ep - em) / (2 * d), rel=1e-6, abs=1e-7)


def test_virial_is_strain_derivative(orc):
    """W_ab = -dE/d eps_ab with grids deforming with the cell (reading R8).
    The coarsest-level image sum is cut sharply at R; image points crossing
    |r| = R under the strain make jumps ~R^-6 (sum q)^2 that the difference
    quotient amplifies by 1/delta, so R is taken large here."""
    box, x, c, a, n, l = _small_case()
    H = np.diag(box)
    R = 300.0
    r = orc.evaluate(H, a, n, l, x, c, r_img=R)
    d = 1e-6
    comps = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    for idx, (p, q) in enumerate(comps):
        eps = np.zeros((3, 3))
        eps[p, q] += 0.5 * d
        eps[q, p] += 0.5 * d
        Ep = orc.evaluate((np.eye(3) + eps) @ H, a, n, l, x @ (np.eye(3) + eps).T, c, r_img=R)["E"]
        Em = orc.evaluate((np.eye(3) - eps) @ H, a, n, l, x @ (np.eye(3) - eps).T, c, r_img=R)["E"]
        fd = -(Ep - Em) / (2 * d)
        assert r["W"][idx] == pytest.approx(fd, rel=2e-6, abs=1e-6 * abs(r["W"][:3]).max())


def test_triclinic_cell_matches_orthorhombic_when_diagonal(orc):
    box, x, c, a, n, l = _small_case()
    r1 = orc.evaluate(box, a, n, l, x, c, r_img=60.0)
    r2 = orc.evaluate(np.diag(box), a, n, l, x, c, r_img=60.0)
    assert r1["E"] == r2["E"]


# ------------------------------------------------------------- invariances

def test_translation_by_coarsest_grid_vector(orc):
    box = (8.0, 8.0, 8.0)
    x, c = I.uniform_atoms(50, 60, box)
    n = orc.grid_dims(box, 0.5, 3)
    s = np.array(box) / np.array(n) * 4  # one coarsest-grid spacing
    r1 = orc.evaluate(box, 2.0, n, 3, x, c)
    r2 = orc.evaluate(box, 2.0, n, 3, x + s * np.array([1, 0, 2]), c)
    assert r2["E"] == pytest.approx(r1["E"], rel=1e-12)
    assert np.abs(r2["F"] - r1["F"]).max() < 1e-11 * np.abs(r1["F"]).max()
    # a generic shift changes E only at the discretisation-error level
    r3 = orc.evaluate(box, 2.0, n, 3, x + 0.37, c)
    assert r3["E"] == pytest.approx(r1["E"], rel=1e-3)
    assert r3["E"] != pytest.approx(r1["E"], rel=1e-12)


def test_scaling_laws(orc):
    """(x, L, a, h) -> s (x, L, a, h): E -> s^-6 E, F -> s^-7 F, W -> s^-6 W;
    c -> lam c: E -> lam^2 E."""
    box = np.array((7.0, 7.0, 8.0))
    x, c = I.uniform_atoms(51, 40, tuple(box))
    n = orc.grid_dims(box, 0.875, 2)
    r1 = orc.evaluate(box, 2.0, n, 2, x, c, r_img=70.0)
    s = 1.7
    r2 = orc.evaluate(box * s, 2.0 * s, n, 2, x * s, c, r_img=70.0 * s)
    assert r2["E"] == pytest.approx(r1["E"] * s ** -6, rel=1e-12)
    assert np.abs(r2["F"] - r1["F"] * s ** -7).max() < 1e-11 * np.abs(r1["F"]).max() * s ** -7
    assert r2["W"] == pytest.approx(r1["W"] * s ** -6, rel=1e-11, abs=1e-12)
    r3 = orc.evaluate(box, 2.0, n, 2, x, 1.3 * c, r_img=70.0)
    assert r3["E"] == pytest.approx(1.69 * r1["E"], rel=1e-13)


def test_atom_permutation(orc):
    box = (7.0, 7.0, 7.0)
    x, c = I.uniform_atoms(52, 40, box)
    n = orc.grid_dims(box, 0.875, 2)
    p = np.random.default_rng(3).permutation(40)
    r1 = orc.evaluate(box, 2.0, n, 2, x, c)
    r2 = orc.evaluate(box, 2.0, n, 2, x[p], c[p])
    assert r2["E"] == pytest.approx(r1["E"], rel=1e-13)
    assert np.abs(r2["F"] - r1["F"][p]).max() < 1e-12 * np.abs(r1["F"]).max()


def test_net_force_is_small(orc):
    """The local part conserves momentum exactly (pair antisymmetry); the grid
    part breaks continuous translation invariance, so only approximately."""
    box = (8.0, 8.0, 8.0)
    x, c = I.uniform_atoms(53, 80, box)
    n = orc.grid_dims(box, 0.5, 2)
    r = orc.evaluate(box, 2.4, n, 2, x, c)
    assert np.abs(r["F"].sum(0)).max() < 5e-3 * np.linalg.norm(r["F"], axis=1).sum()
    b = orc.brute(box, x, c, r_img=80.0)
    assert np.abs(b["F"].sum(0)).max() < 1e-10 * np.linalg.norm(b["F"], axis=1).sum()


# --------------------------------------------------- multilevel structure

def test_grid_adjointness_and_conservation(orc):
    """-1/2 q^1 . e^{1,tot} = sum_k -1/2 q^k . e^k (prolongation is the
    transpose of restriction) and sum q^k = sum c on every level."""
    box = (8.0, 8.0, 12.0)
    x, c = I.uniform_atoms(60, 70, box)
    n = orc.grid_dims(box, 0.5, 3)
    G = orc.grids(box, 2.0, n, 3, x, c)
    for q, e, et in G:
        assert q.sum() == pytest.approx(c.sum(), rel=1e-13)
    lhs = np.sum(G[0][0] * G[0][2])
    rhs = sum(np.sum(q * e) for q, e, _ in G)
    assert lhs == pytest.approx(rhs, rel=1e-13)
    r = orc.evaluate(box, 2.0, n, 3, x, c)
    le = r["level_energy"]
    assert le[2:5].sum() == pytest.approx(-0.5 * lhs, rel=1e-13)
    assert le[0] + le[1] + le[2:5].sum() == pytest.approx(r["E"], rel=1e-13)
    assert r["eatom"].sum() == pytest.approx(r["E"], rel=1e-13)


def _periodic_1d(n, fn):
    """Matrix with entries fn(i, j) summed over periodic images of j."""
    return fn


def test_dense_matrix_form_matches_loops(orc):
    """E_grid = -1/2 c^T P^T (K_1 + R^T K_2 R) P c with explicitly assembled
    periodic interpolation (P), restriction (R) and level (K) matrices."""
    box = np.array((4.0, 4.0, 6.0))
    a, l = 1.2, 2
    x, c = I.uniform_atoms(61, 9, tuple(box), dmin=0.6)
    n1 = np.array((4, 4, 8))
    n2 = n1 // 2
    h1 = box / n1

    def nodes(nv):
        g = np.stack(np.meshgrid(*[np.arange(v) for v in nv], indexing="ij"), -1)
        return g.transpose(2, 1, 0, 3).reshape(-1, 3)  # x-fastest order

    X1, X2 = nodes(n1), nodes(n2)

    def phi_per(t, nper):  # periodised Phi along one axis
        return sum(orc.Phi(t - p * nper) for p in range(-3, 4))

    P = np.array([[np.prod([phi_per(x[i, d] / h1[d] - X1[m, d], n1[d]) for d in range(3)])
                   for i in range(len(c))] for m in range(len(X1))])
    R = np.array([[np.prod([phi_per(X1[v, d] / 2.0 - X2[m, d], n2[d]) for d in range(3)])
                   for v in range(len(X1))] for m in range(len(X2))])
    K1 = np.zeros((len(X1), len(X1)))
    for u in range(len(X1)):
        for v in range(len(X1)):
            s = 0.0
            for img in np.stack(np.meshgrid(*[np.arange(-2, 3)] * 3, indexing="ij"), -1).reshape(-1, 3):
                r = np.linalg.norm((X1[u] - X1[v]) * h1 + img * box)
                s += orc.gk(1, l, a, r)
            K1[u, v] = s
    T, _ = orc.top_table(box, a, tuple(n2), l)
    K2 = np.zeros((len(X2), len(X2)))
    for u in range(len(X2)):
        for v in range(len(X2)):
            m = (X2[u] - X2[v]) % n2
            K2[u, v] = T[m[0] + n2[0] * (m[1] + n2[1] * m[2])]
    E_dense = -0.5 * c @ P.T @ (K1 + R.T @ K2 @ R) @ P @ c
    r = orc.evaluate(box, a, tuple(n1), l, x, c)
    assert r["level_energy"][2:4].sum() == pytest.approx(E_dense, rel=1e-12)
    assert np.allclose(P @ c, orc.grids(box, a, tuple(n1), l, x, c)[0][0].reshape(-1), rtol=0,
                       atol=1e-14)


def test_top_table_symmetry(orc):
    box = (8.0, 9.0, 10.0)
    nl = (3, 4, 5)
    T, V = orc.top_table(box, 1.0, nl, 3)
    Tg = T.reshape(nl[2], nl[1], nl[0])
    Tm = np.roll(Tg[::-1, ::-1, ::-1], 1, axis=(0, 1, 2))  # T(-m)
    assert np.allclose(Tg, Tm, rtol=1e-12, atol=0)


def test_oracle_is_thread_count_independent(orc):
    box = (8.0, 8.0, 8.0)
    x, c = I.uniform_atoms(70, 80, box)
    n = orc.grid_dims(box, 0.5, 3)
    orc.set_threads(1)
    r1 = orc.evaluate(box, 2.0, n, 3, x, c)
    orc.set_threads(4)
    r2 = orc.evaluate(box, 2.0, n, 3, x, c)
    orc.set_threads(0)
    assert r1["E"] == r2["E"]
    assert np.array_equal(r1["F"], r2["F"])
    assert np.array_equal(r1["W"], r2["W"])


# ------------------------------------------------ loop forms and sampled entry points

def _local_cases():
    tri = np.array([[9.0, 1.5, -0.7], [0.0, 8.5, 1.1], [0.0, 0.0, 10.0]])
    return [((8.0, 9.0, 10.0), 2.5, 300, 61),   # every axis holds >= 3 cells
            ((3.0, 9.0, 12.0), 2.5, 200, 62),   # x thinner than 2a: one cell, images -1..1
            ((2.0, 7.0, 8.0), 2.5, 60, 63),     # x thinner than a: images -2..2
            (tri, 2.2, 250, 64)]                # triclinic cell


@pytest.mark.parametrize("case", range(4))
def test_local_linked_cells_equal_all_pairs(orc, case):
    """The linked-cell local loop (Sec. III.D) visits exactly the (j, image)
    pairs of the plain all-atoms x all-images loop: e0, forces and virial
    records agree to rounding for every atom, including boxes thinner than
    the cutoff and a triclinic cell.  A missed or doubled pair changes a
    value by a whole pair term (>= 1e-4 of the largest here)."""
    box, a, N, seed = _local_cases()[case]
    H = np.diag(box) if np.ndim(box) == 1 else np.asarray(box)
    rng = np.random.default_rng(seed)
    x = rng.random((N, 3)) @ H.T + rng.normal(0.0, 3.0, (N, 3))  # some atoms outside the cell
    c = rng.uniform(0.7, 1.2, N)
    idx = np.arange(N)
    e1, F1, W1 = orc.local_forms(box, a, x, c, idx, "cells")
    e2, F2, W2 = orc.local_forms(box, a, x, c, idx, "allpairs")
    for u, v in ((e1, e2), (F1, F2), (W1, W2)):
        assert np.abs(u - v).max() <= 1e-13 * np.abs(v).max()
    assert np.abs(e2).max() > 0.0


def _sample_cases():
    return [((7.0, 8.0, 9.0), 2.0, 0.7, 3, 200, 71),
            ((6.0, 6.0, 15.0), 2.2, 0.75, 2, 150, 72),   # anisotropic box
            ((7.5, 7.5, 7.5), 2.0, 0.9, 1, 120, 73)]     # one level: no level stencils


@pytest.mark.parametrize("case", range(3))
def test_eval_sample_equals_eval(orc, case):
    """orc_eval_sample (the reference of the large sampled GPU tests) gives,
    at the listed atoms, the forces and per-atom energies of the full
    evaluation, its grid energy is the sum of the per-level energies
    -1/2 q^k . e^k of orc_eval, and orc_local's potentials reproduce the
    full evaluation's local energy -1/2 sum_i c_i e0_i."""
    box, a, h, l, N, seed = _sample_cases()[case]
    x, c = I.uniform_atoms(seed, N, box)
    n = orc.grid_dims(box, h, l)
    o = orc.evaluate(box, a, n, l, x, c)
    idx = np.random.default_rng(seed).permutation(N)[: N // 3]
    idx = np.r_[idx, idx[:5]]  # repeated indices are allowed
    s = orc.evaluate_sample(box, a, n, l, x, c, idx)
    assert np.abs(s["F"] - o["F"][idx]).max() <= 1e-14 * np.abs(o["F"]).max()
    assert np.abs(s["eatom"] - o["eatom"][idx]).max() <= 1e-14 * np.abs(o["eatom"]).max()
    le = o["level_energy"]
    assert s["grid_energy"] == pytest.approx(le[2:l + 2].sum(), rel=1e-14, abs=0)
    # total = local + self + grid levels
    assert le[0] + le[1] + le[2:l + 2].sum() == pytest.approx(o["E"], rel=1e-13)
    e0, Fl = orc.local(box, a, x, c, np.arange(N))
    assert -0.5 * np.sum(c * e0) == pytest.approx(le[0], rel=1e-13)
    # the local forces alone sum to zero (pair antisymmetry)
    assert np.abs(Fl.sum(axis=0)).max() <= 1e-12 * np.abs(Fl).max()


# ------------------------------------------------ smoothing functions of other continuity

@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_smoothing_continuity_order(orc, n):
    """gamma_n (Sec. II.A.3, compared for C^1..C^4 in Sec. III.B) meets rho^-6
    at rho = 1 with exactly n continuous derivatives: gamma_n - rho^-6
    vanishes like (1 - rho)^(n+1) from the left (log-log slope n+1, nonzero
    limit), equals rho^-6 on the right, and its derivative routine matches
    finite differences."""
    with orc.smoothing_order(n):
        ts = [0.005, 0.0025, 0.00125]
        d = [orc.gamma(1 - t) - (1 - t) ** -6 for t in ts]
        for k in range(2):
            slope = math.log(abs(d[k] / d[k + 1])) / math.log(2.0)
            assert slope == pytest.approx(n + 1, abs=0.08)
        assert abs(d[-1] / ts[-1] ** (n + 1)) > 1.0
        for rho in (1.0, 1.3, 2.0):
            assert orc.gamma(rho) == pytest.approx(rho ** -6, rel=1e-15)
        for rho in (0.2, 0.7, 0.95):
            fd = (orc.gamma(rho + 1e-6) - orc.gamma(rho - 1e-6)) / 2e-6
            assert orc.dgamma(rho) == pytest.approx(fd, rel=1e-7, abs=1e-8)


@pytest.mark.parametrize("n,gamma0", [(1, 3 / 2), (2, 15 / 8), (3, 35 / 16), (4, 315 / 128)])
def test_smoothing_self_term_and_telescoping(orc, n, gamma0):
    """gamma_n(0) is the order-n partial sum of the binomial series of
    (1 - x)^(-1/2) at x = 1, i.e. prod_{j=1..n} (2j+1)/(2j) (3/2, 15/8, 35/16,
    315/128); the split still telescopes to r^-6 and sum_{k>=1} g_k(0) =
    gamma_n(0)/a^6 for every n."""
    assert gamma0 == pytest.approx(math.prod((2 * j + 1) / (2 * j) for j in range(1, n + 1)))
    a, l = 2.5, 4
    with orc.smoothing_order(n):
        assert orc.gamma(0.0) == gamma0
        rng = np.random.default_rng(n)
        for r in rng.uniform(0.3, 40.0, 300):
            s = sum(orc.gk(k, l, a, r) for k in range(l + 1))
            assert s == pytest.approx(r ** -6, rel=1e-12)
        assert sum(orc.gk(k, l, a, 0.0) for k in range(1, l + 1)) == pytest.approx(
            gamma0 / a ** 6, rel=1e-14)
    assert orc.smoothing() == 2


@pytest.mark.parametrize("n", [1, 3, 4])
def test_smoothing_variants_exact_on_coarsest_lattice(orc, n):
    """Whatever gamma, atoms on a lattice commensurate with the coarsest grid
    make every transfer an injection, so the MLS energy equals the exact
    lattice sum (E/N = -1/2 c^2 S / s^6, S = 8.40192... for simple cubic)."""
    L, levels, h, a = 8.0, 3, 1.0, 2.0
    s = 4 * h
    m = int(L / s)
    x = np.array([[i, j, k] for i in range(m) for j in range(m) for k in range(m)], float) * s
    c = np.full(len(x), 1.1)
    nn = orc.grid_dims((L, L, L), h, levels)
    with orc.smoothing_order(n):
        o = orc.evaluate((L, L, L), a, nn, levels, x, c)
    S = 8.40192397482754
    assert o["E"] / len(x) == pytest.approx(-0.5 * 1.21 * S / s ** 6, rel=1e-10)
    assert np.abs(o["F"]).max() < 1e-12


def test_smoothing_variants_converge_with_cutoff(orc):
    """Every C^n MLS converges to the exact periodic forces as the cutoff
    grows at fixed a/h (Sec. III.B bounds ~ h^n / a^(n+7)).  (The paper's
    figure also shows C^1 converging more slowly than C^2 on its slab; on
    this small cube the two rates are within 5% and no ordering is
    asserted.)"""
    box = (9.0, 9.0, 9.0)
    x, c = I.uniform_atoms(808, 300, box)
    ex = orc.brute(box, x, c, r_img=10 * 9.0)["F"]
    errs = {}
    for n in (1, 2, 3, 4):
        with orc.smoothing_order(n):
            e = []
            for a in (1.5, 2.25):
                h = a / 3.0
                nn = orc.grid_dims(box, h, 2)
                F = orc.evaluate(box, a, nn, 2, x, c)["F"]
                e.append(np.linalg.norm(F - ex) / np.linalg.norm(ex))
            errs[n] = e
            assert e[1] < 0.2 * e[0]
