"""CPU oracle of the surrogate MLP used to screen PSO candidates.

TEST INFRASTRUCTURE ONLY (imported by tests, never by the product package).

Network: 5 -> W -> W -> W -> 1 with ReLU on the hidden layers.  Weights and
layer inputs are rounded to bfloat16 (round to nearest even) before every
matrix product, exactly where the GPU rounds them; the products and sums are
carried in float64 here (the GPU accumulates in float32).  Loss:
L = (1 / 2N) sum_n (y_n - t_n)^2 over the samples with a finite target.
The backward pass is the plain chain rule of that forward pass (the bf16
rounding is treated as the identity, as in mixed-precision training).
"""
from __future__ import annotations

import numpy as np

WIDTH = 256
N_IN = 5


def bf16(a: np.ndarray) -> np.ndarray:
    """Round float values to bfloat16 (nearest, ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    out = u.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if np.any(nan):
        out = np.where(nan, np.nan, out)
    return out


def param_shapes(width: int = WIDTH):
    return [("W1", (width, N_IN)), ("b1", (width,)), ("W2", (width, width)), ("b2", (width,)),
            ("W3", (width, width)), ("b3", (width,)), ("W4", (1, width)), ("b4", (1,))]


def unflatten(theta: np.ndarray, width: int = WIDTH) -> dict:
    out, o = {}, 0
    for name, shp in param_shapes(width):
        n = int(np.prod(shp))
        out[name] = np.asarray(theta[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


def flatten(p: dict, width: int = WIDTH) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in param_shapes(width)])


def forward(theta: np.ndarray, X: np.ndarray, width: int = WIDTH, keep: bool = False):
    p = unflatten(theta, width)
    a = bf16(X)
    acts = [a]
    for l in (1, 2, 3):
        z = a @ bf16(p[f"W{l}"]).T + p[f"b{l}"]
        a = bf16(np.maximum(z, 0.0))
        acts.append(a)
    y = (a @ bf16(p["W4"]).T)[:, 0] + p["b4"][0]
    return (y, acts) if keep else y


def loss_and_grad(theta: np.ndarray, X: np.ndarray, t: np.ndarray, width: int = WIDTH):
    p = unflatten(theta, width)
    y, acts = forward(theta, X, width, keep=True)
    ok = np.isfinite(t)
    n = max(int(ok.sum()), 1)
    r = np.where(ok, y - np.where(ok, t, 0.0), 0.0)
    L = 0.5 * np.sum(r * r) / n
    dy = r / n
    g = {"W4": dy[None, :] @ acts[3], "b4": np.array([dy.sum()])}
    d = dy[:, None] * bf16(p["W4"])                      # dL/da3
    for l in (3, 2, 1):
        dz = d * (acts[l] > 0)
        g[f"W{l}"] = dz.T @ acts[l - 1]
        g[f"b{l}"] = dz.sum(axis=0)
        d = dz @ bf16(p[f"W{l}"])
    return L, flatten(g, width)


def adam(theta, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (bias-corrected), step counted from 1."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
