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


def loss_and_grad(theta: np.ndarray, X: np.ndarray, t: np.ndarray, width: int = WIDTH,
                  bf16_deltas: bool = False):
    """Loss and its gradient by the chain rule.  bf16_deltas = True rounds each
    layer's back-propagated delta dL/dz (after the ReLU mask) to bfloat16, the
    storage precision of the deltas in a mixed-precision backward pass whose
    next products take bf16 operands; the plain chain rule otherwise."""
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
        if bf16_deltas:
            dz = bf16(dz)
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





def grad_tolerance(theta: np.ndarray, X: np.ndarray, t: np.ndarray, width: int = WIDTH,
                   c: float = 4.0, amb: float = 1e-4):
    """Elementwise tolerance for comparing a reduced-precision gradient with
    loss_and_grad(..., bf16_deltas=True), per parameter:

        c 2^-8 sum_n |term_n|  +  sum over ambiguous terms |term_n|

    where term_n is the parameter's per-sample product in the chain rule
    (delta times layer input; delta alone for a bias).  An evaluation that
    rounds at the same points but accumulates in fp32 differs from the oracle
    only where a value lands on the other side of a bf16 rounding boundary,
    i.e. by one bf16 unit (2^-8 relative at most) in a few stored values, so
    each gradient moves by a small multiple of 2^-8 of its absolute terms.
    The exception is a ReLU unit whose pre-activation z lies so close to zero
    (|z| <= amb times the sum of its absolute terms, far above fp32's
    accumulation error) that its mask may differ: its whole term may then
    differ, and goes into the tolerance in full, together with everything it
    feeds in the layers below."""
    p = unflatten(theta, width)
    Wb = {l: bf16(p[f"W{l}"]) for l in (1, 2, 3, 4)}
    acts, ambig = [bf16(X)], []
    for l in (1, 2, 3):
        a = acts[-1]
        z = a @ Wb[l].T + p[f"b{l}"]
        zabs = np.abs(a) @ np.abs(Wb[l]).T + np.abs(p[f"b{l}"])
        ambig.append(np.abs(z) <= amb * zabs)
        acts.append(bf16(np.maximum(z, 0.0)))
    y = (acts[3] @ Wb[4].T)[:, 0] + p["b4"][0]
    ok = np.isfinite(t)
    n = max(int(ok.sum()), 1)
    r = np.where(ok, y - np.where(ok, t, 0.0), 0.0)
    dy = r / n
    u = c * 2.0 ** -8
    tol = {"W4": u * (np.abs(dy)[None, :] @ np.abs(acts[3])), "b4": np.array([u * np.abs(dy).sum()])}
    d = dy[:, None] * Wb[4]
    extra = np.zeros_like(d)        # |delta| a mask flip at this or a higher layer may change
    for l in (3, 2, 1):
        on = acts[l] > 0
        dz = bf16(d * on)
        flip = ambig[l - 1]
        ex = extra * (on | flip) + flip * np.abs(d)
        tol[f"W{l}"] = u * (np.abs(dz).T @ np.abs(acts[l - 1])) + ex.T @ np.abs(acts[l - 1])
        tol[f"b{l}"] = u * np.abs(dz).sum(axis=0) + ex.sum(axis=0)
        if l > 1:
            d = dz @ Wb[l]
            extra = ex @ np.abs(Wb[l])
    return flatten(tol, width)


def grad_abs_terms(theta: np.ndarray, X: np.ndarray, t: np.ndarray, width: int = WIDTH):
    """For every parameter, the sum of the absolute values of the terms its
    gradient sums over the samples (the same chain rule as loss_and_grad with
    bf16_deltas = True, each product taken in absolute value): the scale
    against which rounding differences of a reduced-precision evaluation are
    measured elementwise."""
    p = unflatten(theta, width)
    y, acts = forward(theta, X, width, keep=True)
    ok = np.isfinite(t)
    n = max(int(ok.sum()), 1)
    r = np.where(ok, y - np.where(ok, t, 0.0), 0.0)
    dy = np.abs(r / n)
    g = {"W4": dy[None, :] @ np.abs(acts[3]), "b4": np.array([dy.sum()])}
    d = (r / n)[:, None] * bf16(p["W4"])
    for l in (3, 2, 1):
        dz = bf16(d * (acts[l] > 0))
        g[f"W{l}"] = np.abs(dz).T @ np.abs(acts[l - 1])
        g[f"b{l}"] = np.abs(dz).sum(axis=0)
        d = dz @ bf16(p[f"W{l}"])
    return flatten(g, width)
