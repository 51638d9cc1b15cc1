"""Lorentz-Berthelot mixing for the oracle (TEST INFRASTRUCTURE ONLY, like
the rest of ``oracle/``).

Sec. II.D: with sigma_ij = (sigma_i + sigma_j)/2 and eps_ij = sqrt(eps_i eps_j)
the coefficient C_ij = 2 eps_ij sigma_ij^6 is expanded binomially as
    C_ij = sum_{k=0}^{6} xi_{i,k} xi_{j,6-k},
    xi_{i,k} = (1/8) sigma_i^k sqrt(binom(6,k) 2 eps_i)
(Eq. disp-pair-pot-multilevel-LorentzBerthelot; its index xi_{k-6} is read as
xi_{6-k}), so the energy is E = -1/2 sum_k xi_k^T G xi_{6-k}: seven
instances of the method.

Here each bilinear term comes from the oracle's single-coefficient
evaluation by polarization.  E(c) = -1/2 c^T G c (local part, grid part and
self term alike) is a quadratic form, so
    xi_a^T G xi_b = -[E(xi_a + xi_b) - E(xi_a) - E(xi_b)],
and the same identity holds for the forces, F(c) = -dE(c)/dx.  Eleven
single-coefficient evaluations give the LB energy and forces.
"""
from __future__ import annotations

import math

import numpy as np

from . import oracle as O


def xi(sigma, eps):
    """(7, N): xi_{i,k} for k = 0..6."""
    sigma = np.asarray(sigma, dtype=np.float64)
    eps = np.asarray(eps, dtype=np.float64)
    return np.stack([0.125 * sigma ** k * np.sqrt(math.comb(6, k) * 2.0 * eps)
                     for k in range(7)])


def c_lb(si, sj, ei, ej):
    """The Lorentz-Berthelot coefficient 2 sqrt(eps_i eps_j) ((si + sj)/2)^6."""
    return 2.0 * np.sqrt(ei * ej) * (0.5 * (si + sj)) ** 6


def _polarize(fn, X):
    """sum_k -1/2 xi_k^T G xi_{6-k} from a quadratic-form evaluator fn(c)
    returning (E, F); the terms k and 6-k are equal, so four mixed
    evaluations suffice."""
    single = [fn(X[k]) for k in range(7)]
    E = 0.0
    F = np.zeros_like(single[0][1])
    for k in range(4):
        m = 6 - k
        if k == m:
            Ek, Fk = single[k]
        else:
            Ej, Fj = fn(X[k] + X[m])
            # -1/2 xi_k G xi_m = 1/2 [E(xi_k + xi_m) - E(xi_k) - E(xi_m)],
            # and the (m, k) term is the same: count it twice
            Ek = Ej - single[k][0] - single[m][0]
            Fk = Fj - single[k][1] - single[m][1]
        E += Ek
        F += Fk
    return E, F


def evaluate_lb(box, a, n, levels, x, sigma, eps, r_img=0.0):
    """MLS energy and forces under Lorentz-Berthelot mixing (FP64)."""
    X = xi(sigma, eps)

    def fn(c):
        r = O.evaluate(box, a, n, levels, x, c, r_img)
        return r["E"], r["F"]

    E, F = _polarize(fn, X)
    return dict(E=E, F=F)


def brute_lb(box, x, sigma, eps, r_img):
    """Exact periodic Lorentz-Berthelot sum by polarization of the brute
    force."""
    X = xi(sigma, eps)

    def fn(c):
        r = O.brute(box, x, c, r_img)
        return r["E"], r["F"]

    E, F = _polarize(fn, X)
    return dict(E=E, F=F)
