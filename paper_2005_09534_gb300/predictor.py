"""Driver of the learned spectral predictor (argument marshalling and batching).

The network's forward, backward and Adam kernels, the labels (Lanczos bounds
and the KPM eigenvalue count, polfed_spectral_labels) and the feature/target
conventions all live in libpolfed.so; this module only loops over
realizations, stacks arrays and feeds batches.

Labels are invariant under the symmetries of the periodic chain of Eq. (1):
cyclic shifts and reflection of the fields, and the global spin flip
(h -> -h maps the S^z = 0 sector onto itself).  ``symmetric_copies`` uses them
to multiply the training set by 4L.
"""
from __future__ import annotations

import time

import numpy as np

from . import MLP, Model, mlp_features, mlp_targets, spectral_labels


def symmetric_copies(h: np.ndarray, periodic: bool = True):
    """Field vectors with the same spectrum as h (4L for a ring, 4 for an open chain)."""
    h = np.asarray(h, dtype=np.float64)
    out = []
    shifts = range(h.size) if periodic else [0]
    for s in shifts:
        r = np.roll(h, s)
        for v in (r, r[::-1]):
            out.append(v)
            out.append(-v)
    return out


def labels_for(ctx, models, eps=0.5, n_mom=256, R=16):
    """[n, 3] array of (E_min, E_max, rho_eps) from the method's own machinery."""
    return np.array([spectral_labels(ctx, m, eps, n_mom, R) for m in models])


def dataset(models, Ws, labels, augment=True):
    """Feature rows x = (h, W) and target rows y = (E_min/L, E_max/L, log rho_eps)."""
    X, Y = [], []
    for m, W, lab in zip(models, Ws, labels):
        y = mlp_targets(m.L, lab)
        hs = symmetric_copies(m.h, m.periodic) if augment else [m.h]
        for h in hs:
            X.append(mlp_features(Model(m.L, m.J1, m.J2, m.Delta, h, m.periodic), W))
            Y.append(y)
    return np.stack(X).astype(np.float32), np.stack(Y).astype(np.float32)


def fit(net: MLP, X: np.ndarray, Y: np.ndarray, steps=3000, lr=1e-3, batch=256, seed=0, device="cuda:0"):
    """Standardize with the training set's mean/std and run `steps` Adam steps on
    random batches, the learning rate decaying by a cosine from lr to lr/20;
    returns (final full-set loss, seconds)."""
    import torch
    xm, xs = X.mean(axis=0), X.std(axis=0) + 1e-6
    ym, ys = Y.mean(axis=0), Y.std(axis=0) + 1e-6
    net.set_scaling(xm, xs, ym, ys)
    dX = torch.from_numpy(X).to(device)
    dY = torch.from_numpy(Y).to(device)
    n = X.shape[0]
    b = min(batch, n)
    rng = np.random.default_rng(seed)
    xb = torch.empty((b, X.shape[1]), dtype=torch.float32, device=device)
    yb = torch.empty((b, Y.shape[1]), dtype=torch.float32, device=device)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(steps):
        idx = torch.from_numpy(rng.integers(0, n, b)).to(device)
        torch.index_select(dX, 0, idx, out=xb)
        torch.index_select(dY, 0, idx, out=yb)
        torch.cuda.synchronize()
        lr_k = lr * (0.05 + 0.95 * 0.5 * (1.0 + np.cos(np.pi * k / steps)))
        net.train_step(xb, yb, b, float(lr_k))
    loss = net.grad(dX, dY, n)
    return loss, time.perf_counter() - t0
