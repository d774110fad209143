"""Plain FP64 CPU oracle of the learned spectral predictor.

TEST INFRASTRUCTURE ONLY (see the package docstring): nothing in the GPU
library imports or calls this module.

The paper has no learned component; this is the network the GPU library
trains (two tanh hidden layers, linear output), written out with numpy:
  * ``forward``       -- x' = (x - x_mean) / x_std, a1 = tanh(W1 x' + b1),
                         a2 = tanh(W2 a1 + b2), y = W3 a2 + b3.
  * ``loss_and_grad`` -- L = 0.5 / B sum_b |y_b - (t_b - y_mean) / y_std|^2 and
                         its gradient by the chain rule (tanh' = 1 - tanh^2).
  * ``adam_step``     -- Kingma & Ba, ICLR 2015, Algorithm 1 (bias-corrected).
Parameter layout: W1 [H x d_in] row-major, b1 [H], W2 [H x H], b2 [H],
W3 [d_out x H], b3 [d_out], concatenated.
"""
from __future__ import annotations

from typing import Dict, Optional, Tuple

import numpy as np


def n_params(d_in: int, H: int, d_out: int) -> int:
    return H * d_in + H + H * H + H + d_out * H + d_out


def unpack(p: np.ndarray, d_in: int, H: int, d_out: int) -> Dict[str, np.ndarray]:
    p = np.asarray(p, dtype=np.float64)
    sizes = [("W1", (H, d_in)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (d_out, H)), ("b3", (d_out,))]
    out, k = {}, 0
    for name, shp in sizes:
        n = int(np.prod(shp))
        out[name] = p[k:k + n].reshape(shp)
        k += n
    assert k == p.size
    return out


def pack(d: Dict[str, np.ndarray]) -> np.ndarray:
    return np.concatenate([d[k].ravel() for k in ("W1", "b1", "W2", "b2", "W3", "b3")])


def identity_scaling(d_in: int, d_out: int):
    return np.zeros(d_in), np.ones(d_in), np.zeros(d_out), np.ones(d_out)


def forward(p, x, d_in, H, d_out, scaling=None) -> Tuple[np.ndarray, dict]:
    """Standardized outputs y [B x d_out] and the activations."""
    xm, xs, ym, ys = scaling if scaling is not None else identity_scaling(d_in, d_out)
    w = unpack(p, d_in, H, d_out)
    xp = (np.asarray(x, dtype=np.float64) - xm) / xs
    a1 = np.tanh(xp @ w["W1"].T + w["b1"])
    a2 = np.tanh(a1 @ w["W2"].T + w["b2"])
    y = a2 @ w["W3"].T + w["b3"]
    return y, {"xp": xp, "a1": a1, "a2": a2, "w": w}


def predict(p, x, d_in, H, d_out, scaling=None) -> np.ndarray:
    """Outputs in target units: y * y_std + y_mean."""
    xm, xs, ym, ys = scaling if scaling is not None else identity_scaling(d_in, d_out)
    y, _ = forward(p, x, d_in, H, d_out, scaling)
    return y * ys + ym


def loss_and_grad(p, x, t, d_in, H, d_out, scaling=None) -> Tuple[float, np.ndarray]:
    xm, xs, ym, ys = scaling if scaling is not None else identity_scaling(d_in, d_out)
    y, c = forward(p, x, d_in, H, d_out, scaling)
    B = y.shape[0]
    r = y - (np.asarray(t, dtype=np.float64) - ym) / ys
    loss = 0.5 * float(np.sum(r * r)) / B
    w = c["w"]
    dy = r / B                                   # dL/dy
    g = {"W3": dy.T @ c["a2"], "b3": dy.sum(axis=0)}
    dz2 = (dy @ w["W3"]) * (1.0 - c["a2"] ** 2)  # through tanh of layer 2
    g["W2"] = dz2.T @ c["a1"]
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ w["W2"]) * (1.0 - c["a1"] ** 2)
    g["W1"] = dz1.T @ c["xp"]
    g["b1"] = dz1.sum(axis=0)
    return loss, pack(g)


def adam_step(p, grad, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update at step t (1-based); returns (p, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def glorot_params(d_in: int, H: int, d_out: int, rng: np.random.Generator) -> np.ndarray:
    """Uniform +-sqrt(6 / (fan_in + fan_out)) weights, zero biases (the GPU's init
    uses its own stream; tests pass parameters explicitly)."""
    d = {"W1": rng.uniform(-1, 1, (H, d_in)) * np.sqrt(6.0 / (d_in + H)), "b1": np.zeros(H),
         "W2": rng.uniform(-1, 1, (H, H)) * np.sqrt(6.0 / (2 * H)), "b2": np.zeros(H),
         "W3": rng.uniform(-1, 1, (d_out, H)) * np.sqrt(6.0 / (H + d_out)), "b3": np.zeros(d_out)}
    return pack(d)
