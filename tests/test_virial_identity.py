"""The virial identity the pair kernel uses, checked by brute force on the
host (no GPU, no library): over all ordered pairs (i, j, n) inside the
cutoff, with t = c_i c_j G(r) d and d = x_j - x_i + n L,

    1/2 sum t (x) d  =  -sum_i c_i F0_i (x) x_i  +  1/2 sum_{n != 0} t (x) d,

F0_i = sum_{j, n = 0} c_j G(r) d the zero-image part of atom i's force sum
and x_i the wrapped position.  A zero-image pair is met from both of its
atoms with opposite d, which is what makes the identity exact; the
symmetric parts of the two sides agree to rounding."""
import itertools

import numpy as np
import pytest


def _pairs(x, box, a):
    """Every ordered (i, j, n) with 0 < |x_j - x_i + n L| < a."""
    L = np.asarray(box)
    reach = [int(np.ceil(a / l)) for l in L]
    out = []
    for n in itertools.product(*(range(-r, r + 1) for r in reach)):
        shift = np.asarray(n) * L
        d = x[None, :, :] - x[:, None, :] + shift
        r2 = (d * d).sum(-1)
        ii, jj = np.nonzero((r2 > 0) & (r2 < a * a))
        for i, j in zip(ii, jj):
            out.append((i, j, n, d[i, j]))
    return out


@pytest.mark.parametrize("box,a,N,seed", [((6.0, 7.0, 8.0), 2.5, 60, 1),
                                          ((4.0, 4.5, 5.0), 2.6, 40, 2)])
def test_pair_virial_identity(box, a, N, seed):
    rng = np.random.default_rng(seed)
    x = rng.random((N, 3)) * np.asarray(box)
    c = rng.uniform(0.7, 1.2, N)

    def G(r2):  # any radial pair function: here g'(r)/r of r^-6
        return -6.0 * r2 ** -4

    W = np.zeros((3, 3))
    Wsh = np.zeros((3, 3))
    F0 = np.zeros((N, 3))
    for i, j, n, d in _pairs(x, box, a):
        g = G(float(d @ d))
        t = c[i] * c[j] * g * d
        W += 0.5 * np.outer(t, d)
        if any(n):
            Wsh += 0.5 * np.outer(t, d)
        else:
            F0[i] += c[j] * g * d
    W_id = -np.einsum("i,ia,ib->ab", c, F0, x) + Wsh
    sym = 0.5 * (W_id + W_id.T)
    assert np.allclose(sym, W, rtol=1e-12, atol=1e-12 * np.abs(W).max())
    # the zero-image terms alone do not vanish: the identity is not trivial
    assert np.abs(np.einsum("i,ia,ib->ab", c, F0, x)).max() > 1e-3 * np.abs(W).max()
