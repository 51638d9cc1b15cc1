"""Training data, normalisation, training loop and accuracy measurement of the
learned force correction (``mls6_mlp_*`` in ``include/mls6.h``).

Everything numeric runs in the library's kernels; this module only drives
them.  Data comes from the method itself: for seeded synthetic slabs, a
coarse evaluation (finest spacing ``h_coarse``) gives the features, and the
target is the force residual to a finer evaluation (``h_fine``), divided by
c_i (the correction is applied as c_i * s * y_i).  Accuracy is measured as
eps_F = ||F - F_ref|| / ||F_ref|| over all components, with F_ref a
converged evaluation (larger cutoff, finer grid).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import inputs as I
from . import mls6


@dataclasses.dataclass
class Setup:
    a: float = 3.0
    h_coarse: float = 2.0
    h_fine: float = 1.0
    a_ref: float = 4.5
    h_ref: float = 0.75
    precision: str = "fp32"


def slab_system(N: int, seed: int, rho: float = 0.8, c6=(0.5, 1.5)):
    """A liquid slab with the proportions of the 4,194,304-atom slab
    (box 160 x 160 x 240 scaled to N atoms, density rho inside, slab
    thickness N / (rho Lx Ly), centred)."""
    s = (N / 4194304.0) ** (1.0 / 3.0)
    Lx, Lz = 160.0 * s, 240.0 * s
    t = N / (rho * Lx * Lx)
    z0 = 0.5 * (Lz - t)
    w = I.Workload(f"slab{N}_s{seed}", N, (Lx, Lx, Lz), ((0.0, Lx), (0.0, Lx), (z0, z0 + t)),
                   tuple(c6), 3.0, 1.0, 0, seed)
    x, c = I.generate(w)
    return w.box, x, c


def _forces(box, x, c, a, h, precision, levels=0):
    import torch

    dt = torch.float64 if precision == "fp64" else torch.float32
    plan = mls6.Plan(box, len(c), a, h, levels, precision=precision)
    pos = torch.tensor(np.c_[x, c], dtype=dt, device="cuda")
    r = plan.evaluate(pos, virial=False)
    return plan, pos, r["F"]


def make_data(box, x, c, st: Setup, model: "mls6.MLP"):
    """(X f32 features with the model's current normalisation, T targets
    (N x 3), coarse forces, the coarse plan and its positions)."""
    import torch

    plan_c, pos_c, Fc = _forces(box, x, c, st.a, st.h_coarse, st.precision)
    X = model.features(plan_c, fmt="f32")
    _, _, Ff = _forces(box, x, c, st.a, st.h_fine, st.precision)
    cc = torch.tensor(c, dtype=torch.float32, device="cuda")[:, None]
    T = ((Ff.float() - Fc.float()) / cc).contiguous()
    torch.cuda.synchronize()
    return X, T, Fc, plan_c, pos_c


def fit_norm(X, T):
    """Per-feature shift/scale (mean, 1/std with a floor) and the output
    scale (RMS of the targets)."""
    Xd = X.double()
    mu = Xd.mean(0)
    sd = Xd.std(0)
    scale = torch_where_small(sd)
    out_scale = float(T.double().pow(2).mean().sqrt())
    return mu.float().cpu().numpy(), scale.float().cpu().numpy(), max(out_scale, 1e-30)


def torch_where_small(sd):
    import torch

    return torch.where(sd > 1e-12 * sd.max().clamp(min=1e-300), 1.0 / sd,
                       torch.zeros_like(sd))


def train(model: "mls6.MLP", Xs, Ts, steps: int = 2000, batch: int = 16384, lr: float = 2e-3,
          seed: int = 0, log=None):
    """Adam on minibatches drawn from the concatenated (X, T) (bf16 features,
    targets already divided by the output scale); cosine learning-rate
    decay.  Returns the loss history."""
    import torch

    X = torch.cat(Xs).to(torch.bfloat16).contiguous()
    T = torch.cat(Ts).float().contiguous()
    n = X.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    hist = []
    for s in range(steps):
        idx = torch.randint(0, n, (min(batch, n),), generator=g).cuda()
        lr_s = lr * 0.5 * (1.0 + math.cos(math.pi * s / steps))
        loss = model.train_step(X[idx].contiguous(), T[idx].contiguous(), max(lr_s, lr * 1e-3))
        hist.append(loss)
        if log and (s % max(1, steps // 10) == 0 or s == steps - 1):
            log(f"step {s} loss {loss:.4e}")
    return hist


def eps_F(F, Fref):
    Fd = F.double() if hasattr(F, "double") else F
    Rd = Fref.double() if hasattr(Fref, "double") else Fref
    return float(((Fd - Rd).pow(2).sum() / Rd.pow(2).sum()).sqrt())


def build_model(st: Setup, train_systems, steps=2000, batch=16384, lr=2e-3, seed=1, log=None):
    """Train a correction on the given (box, x, c) systems.  Returns the
    model (normalisation set) and the loss history."""
    import torch

    model = mls6.MLP(seed)
    raw = [make_data(b, x, c, st, model) for (b, x, c) in train_systems]
    X0 = torch.cat([r[0] for r in raw])
    T0 = torch.cat([r[1] for r in raw])
    shift, scale, out_scale = fit_norm(X0, T0)
    model.set_norm(shift, scale, out_scale)
    Xs, Ts = [], []
    for (b, x, c) in train_systems:
        X, T, _, _, _ = make_data(b, x, c, st, model)
        Xs.append(X)
        Ts.append(T / out_scale)
    hist = train(model, Xs, Ts, steps=steps, batch=batch, lr=lr, seed=seed, log=log)
    return model, hist


def accuracy(model: "mls6.MLP", st: Setup, box, x, c):
    """eps_F of the coarse, coarse + correction and fine evaluations against
    the reference, on one system."""
    import torch

    plan_c, pos_c, Fc = _forces(box, x, c, st.a, st.h_coarse, st.precision)
    torch.cuda.synchronize()
    Fl = Fc.clone()
    torch.cuda.synchronize()
    model.apply(plan_c, Fl)
    _, _, Ff = _forces(box, x, c, st.a, st.h_fine, st.precision)
    _, _, Fr = _forces(box, x, c, st.a_ref, st.h_ref, st.precision)
    torch.cuda.synchronize()
    return dict(coarse=eps_F(Fc, Fr), learned=eps_F(Fl, Fr), fine=eps_F(Ff, Fr))
