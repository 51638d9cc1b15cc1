"""FP64 reference of the learned force correction (TEST INFRASTRUCTURE ONLY,
like the rest of ``oracle/``; it shares no code with the GPU library).

The correction is not part of the paper: a small network reads, for each atom,
the finest-grid potential of a coarse multilevel-summation evaluation around
the atom and predicts the force residual to a finer evaluation.  This module
states the two pieces the GPU kernels compute, in plain numpy:

features(E1, h, x)
    E1: the level-1 total potential e^{1,tot} (shape (nz, ny, nx), as
    ``oracle.grids`` returns it), h: the level-1 spacing per axis, x: wrapped
    positions.  For the 27 offsets d in {-1, 0, 1}^3 (x fastest) the potential
    e and its gradient at x_i + h*d, interpolated with the basis of the
    method (Eq. interpolation: products of Phi over the 4x4x4 nodes around
    the point, Phi from the oracle library), then sin and cos of 2 pi times
    the fractional grid coordinate of x_i per axis; zero padding to 128.

MLP
    128 -> 64 -> 64 -> 64 -> 8 (outputs 0..2 used), tanh after the hidden
    layers; parameters in one flat vector: W1 (128 x 64, row k = input k),
    b1, W2 (64 x 64), b2, W3, b3, W4 (64 x 8), b4.  loss = (1/N) sum_i
    sum_{c<3} (y_ic - t_ic)^2 with its analytic gradient.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O

NF = 128
SIZES = [(128, 64), (64, 64), (64, 64), (64, 8)]


def n_params() -> int:
    return sum(k * n + n for k, n in SIZES)


def unpack(p):
    out, off = [], 0
    for k, n in SIZES:
        W = p[off:off + k * n].reshape(k, n)
        off += k * n
        b = p[off:off + n]
        off += n
        out.append((W, b))
    return out


def _phi_weights(t):
    """Weights and derivatives of the four nodes b-1, b, b+1, b+2 around a
    point with fractional offset t in [0, 1) from node b."""
    off = np.array([1.0 + t, t, 1.0 - t, 2.0 - t])
    w = np.array([O.Phi(v) for v in off])
    # d/du Phi(u - m) at the four nodes: Phi'(u - m) with u - m = off * sign
    s = np.array([1.0, 1.0, -1.0, -1.0])
    dw = np.array([O.dPhi(s[j] * off[j]) for j in range(4)])
    return w, dw


def features(E1, h, x):
    """N x 128 FP64 features (see module docstring)."""
    nz, ny, nx = E1.shape
    n = (nx, ny, nz)
    h = np.asarray(h, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    N = x.shape[0]
    F = np.zeros((N, NF))
    for i in range(N):
        u = x[i] / h
        base = np.floor(u).astype(int)
        t = u - base
        W = [_phi_weights(t[d]) for d in range(3)]
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    idx = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)
                    b = base + np.array([dx, dy, dz])
                    e = gx = gy = gz = 0.0
                    for c in range(4):
                        iz = (b[2] - 1 + c) % n[2]
                        for bb in range(4):
                            iy = (b[1] - 1 + bb) % n[1]
                            for a in range(4):
                                ix = (b[0] - 1 + a) % n[0]
                                v = E1[iz, iy, ix]
                                wx, dwx = W[0][0][a], W[0][1][a]
                                wy, dwy = W[1][0][bb], W[1][1][bb]
                                wz, dwz = W[2][0][c], W[2][1][c]
                                e += wx * wy * wz * v
                                gx += dwx * wy * wz * v
                                gy += wx * dwy * wz * v
                                gz += wx * wy * dwz * v
                    F[i, 4 * idx:4 * idx + 4] = (e, gx / h[0], gy / h[1], gz / h[2])
        for d in range(3):
            F[i, 108 + 2 * d] = np.sin(2.0 * np.pi * t[d])
            F[i, 109 + 2 * d] = np.cos(2.0 * np.pi * t[d])
    return F


def forward(p, X):
    """Output (N x 8) and the hidden activations."""
    L = unpack(p)
    H = [X]
    a = X
    for j, (W, b) in enumerate(L):
        z = a @ W + b
        a = np.tanh(z) if j < 3 else z
        H.append(a)
    return a, H


def loss_grad(p, X, T):
    """loss and its gradient with respect to the flat parameter vector."""
    N = X.shape[0]
    Y, H = forward(p, X)
    R = Y[:, :3] - T
    loss = float(np.sum(R * R) / N)
    dY = np.zeros_like(Y)
    dY[:, :3] = 2.0 * R / N
    L = unpack(p)
    grads = [None] * 4
    d = dY
    for j in (3, 2, 1, 0):
        W, _ = L[j]
        A = H[j]
        grads[j] = (A.T @ d, d.sum(axis=0))
        if j > 0:
            d = (d @ W.T) * (1.0 - H[j] ** 2)
    g = np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in grads])
    return loss, g
