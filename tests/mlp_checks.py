"""Elementwise gradient comparison of the surrogate network (shared by the
CPU pins of the tolerance and the GPU tests).

The reference is the oracle's chain rule with the back-propagated deltas
stored in bf16 (mlp_oracle.loss_and_grad(..., bf16_deltas=True)), the same
rounding points as a bf16 backward pass; the tolerance is
mlp_oracle.grad_tolerance (C x 2^-8 times each gradient's absolute terms,
plus the full terms of ReLU units on the edge of their mask).  An evaluation
that differs only by fp32 accumulation order stays inside it except where a
bf16 rounding flip cascades through one sample (about one element in 10^5
in the CPU emulation), so the rule allows a fraction MAX_OUTSIDE of the
elements outside the tolerance, and none beyond MAX_RATIO times it.  A sign
error or a swapped index in a few hundred live weights of a 256 x 256 layer
puts about 10^-3 of the block outside.
"""
import numpy as np

from oracle import mlp_oracle as M

C_TOL = 8.0
MAX_OUTSIDE = 2e-4
MAX_RATIO = 32.0
MIN_PROTECTED = 0.70    # live elements on which a sign error would exceed the tolerance


def compare(g, theta, X, t, width):
    """Per parameter block: (fraction outside the tolerance, max |g - g_o| /
    tolerance, fraction of live elements protected against a sign error)."""
    _, go = M.loss_and_grad(theta, X, t, width, bf16_deltas=True)
    tol = M.grad_tolerance(theta, X, t, width, c=C_TOL)
    G = M.grad_abs_terms(theta, X, t, width)
    out = {}
    o = 0
    for name, shp in M.param_shapes(width):
        n = int(np.prod(shp))
        sl = slice(o, o + n)
        o += n
        r = np.abs(g[sl] - go[sl]) / np.maximum(tol[sl], 1e-300)
        r[(tol[sl] == 0) & (g[sl] == go[sl])] = 0.0
        live = G[sl] > 0
        prot = float(np.mean((2.0 * np.abs(go[sl]) > tol[sl])[live])) if live.any() else 1.0
        out[name] = (float(np.mean(r > 1.0)), float(r.max()), prot)
    return out


def assert_elementwise(g, theta, X, t, width):
    res = compare(g, theta, X, t, width)
    for name, (outside, worst, prot) in res.items():
        assert outside <= MAX_OUTSIDE, (name, outside, worst)
        assert worst <= MAX_RATIO, (name, worst)
        assert prot >= MIN_PROTECTED, (name, prot)
    return res
