"""Pins of the surrogate network's elementwise gradient tolerance (CPU).

An independent float32 re-implementation of the backward pass, rounding to
bf16 at the same points as a bf16 network does (weights, layer outputs,
deltas) and accumulating in float32, must lie inside the tolerance of
mlp_oracle.grad_tolerance element by element; planted mistakes of the kind
the comparison must catch (a sign error in a few hundred weights, two
swapped rows, a transposed block) must not.  The bf16 storage of the deltas
moves the gradient by far less than the tolerance of the norm check it
replaces.
"""
import numpy as np
import pytest

import mlp_checks as K
from oracle import mlp_oracle as M


def bf16_32(a):
    return M.bf16(a).astype(np.float32)


def emulate_grad(theta, X, t, W):
    p = M.unflatten(theta, W)
    Wb = {l: bf16_32(p[f"W{l}"]) for l in (1, 2, 3, 4)}
    b = {l: p[f"b{l}"].astype(np.float32) for l in (1, 2, 3, 4)}
    a = [bf16_32(X)]
    for l in (1, 2, 3):
        a.append(bf16_32(np.maximum(a[-1] @ Wb[l].T + b[l], 0)))
    y = (a[3] @ Wb[4].T)[:, 0] + b[4][0]
    ok = np.isfinite(t)
    n = np.float32(max(ok.sum(), 1))
    r = np.where(ok, y - np.where(ok, t, 0).astype(np.float32), 0).astype(np.float32)
    dy = (r / n).astype(np.float32)
    g = {"W4": dy[None, :] @ a[3], "b4": np.array([dy.sum()])}
    dz = bf16_32(dy[:, None] * Wb[4] * (a[3] > 0))
    for l in (3, 2, 1):
        g[f"W{l}"] = dz.T @ a[l - 1]
        g[f"b{l}"] = dz.sum(axis=0)
        if l > 1:
            dz = bf16_32((dz @ Wb[l]) * (a[l - 1] > 0))
    return M.flatten({k: np.asarray(v, np.float64) for k, v in g.items()}, W)


def case(W, N, seed):
    rng = np.random.default_rng(seed)
    parts = []
    for name, shp in M.param_shapes(W):
        fan = shp[1] if len(shp) == 2 else 1
        parts.append(rng.uniform(-1, 1, size=int(np.prod(shp))) * np.sqrt(6.0 / fan))
    th = np.concatenate(parts).astype(np.float32).astype(np.float64)
    X = rng.random((N, 5)).astype(np.float32).astype(np.float64)
    t = (np.sin(4 * X[:, 0]) + X[:, 1] - X[:, 2] * X[:, 4]).astype(np.float32).astype(np.float64)
    t[::13] = np.nan
    return th, X, t


@pytest.mark.parametrize("W,N,seed", [(256, 1000, 1), (256, 77, 333), (128, 300, 3), (64, 77, 4)])
def test_float32_emulation_lies_inside_the_tolerance(W, N, seed):
    th, X, t = case(W, N, seed)
    K.assert_elementwise(emulate_grad(th, X, t, W), th, X, t, W)


def test_planted_gradient_mistakes_are_caught():
    W, N = 256, 1000
    th, X, t = case(W, N, 1)
    g = emulate_grad(th, X, t, W)
    rng = np.random.default_rng(9)
    o2 = W * 5 + W
    o3 = o2 + W * W + W
    mistakes = []
    bad = g.copy()
    bad[o2 + rng.choice(W * W, 300, replace=False)] *= -1.0            # sign of 300 weights
    mistakes.append(("W2", bad))
    bad = g.copy()
    blk = bad[o3:o3 + W * W].reshape(W, W)
    blk[[3, 7]] = blk[[7, 3]]                                           # two rows swapped
    mistakes.append(("W3", bad))
    bad = g.copy()
    bad[o3:o3 + W * W] = g[o3:o3 + W * W].reshape(W, W).T.ravel()       # transposed
    mistakes.append(("W3", bad))
    bad = g.copy()
    bad[o2 + W * W:o2 + W * W + W] = g[W * 5:W * 5 + W]                 # b2 from the wrong layer
    mistakes.append(("b2", bad))
    for name, bad in mistakes:
        outside, worst, _ = K.compare(bad, th, X, t, W)[name]
        assert outside > K.MAX_OUTSIDE, name


def test_bf16_deltas_stay_close_to_the_plain_chain_rule():
    W, N = 256, 1000
    th, X, t = case(W, N, 1)
    _, g0 = M.loss_and_grad(th, X, t, W)
    _, g1 = M.loss_and_grad(th, X, t, W, bf16_deltas=True)
    o = 0
    for name, shp in M.param_shapes(W):
        n = int(np.prod(shp))
        assert np.linalg.norm(g1[o:o + n] - g0[o:o + n]) <= 2e-3 * np.linalg.norm(g0[o:o + n]) + 1e-300, name
        o += n
