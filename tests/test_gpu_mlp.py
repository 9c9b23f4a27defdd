"""Surrogate MLP on the tensor cores against the CPU oracle (same bf16
rounding points, fp64 sums): forward pass, loss, gradients, Adam training.

Gradients are compared element by element with the oracle's chain rule at
the GPU's rounding points (bf16 deltas), within the tolerance of
tests/mlp_checks.py (a multiple of the bf16 unit of each gradient's absolute
terms), and by norm with the plain chain rule."""
import numpy as np
import pytest

import mlp_checks as K
from oracle import mlp_oracle as M

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fst():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_10797_gb300 import fstat
    fstat.load()
    return fstat


def rand_theta(W, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    parts = []
    for name, shp in M.param_shapes(W):
        fan = shp[1] if len(shp) == 2 else 1
        parts.append(rng.uniform(-1, 1, size=int(np.prod(shp))) * scale * np.sqrt(6.0 / fan))
    return np.concatenate(parts)


@pytest.mark.parametrize("W,N", [(256, 1000), (64, 77)])
def test_forward_and_gradients_match_oracle(fst, W, N):
    theta = rand_theta(W, 1)
    theta32 = theta.astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(2)
    X = rng.random((N, 5)).astype(np.float32)
    t = (np.sin(4 * X[:, 0]) + X[:, 1] - X[:, 2] * X[:, 4]).astype(np.float32)
    t[::13] = np.nan
    net = fst.MLP(W, max_batch=2048, seed=0)
    net.set_params(torch.from_numpy(theta32.astype(np.float32)).cuda())
    y = net.forward(torch.from_numpy(X).cuda()).cpu().numpy().astype(np.float64)
    yo = M.forward(theta32, X.astype(np.float64), W)
    scale = np.max(np.abs(yo))
    assert np.max(np.abs(y - yo)) <= 1e-2 * scale
    assert np.median(np.abs(y - yo)) <= 1e-4 * scale
    L, g = net.loss_grad(torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda())
    Lo, go = M.loss_and_grad(theta32, X.astype(np.float64), t.astype(np.float64), W)
    assert float(L) == pytest.approx(Lo, rel=1e-3)
    g = g.cpu().numpy().astype(np.float64)
    K.assert_elementwise(g, theta32, X.astype(np.float64), t.astype(np.float64), W)
    o = 0
    for name, shp in M.param_shapes(W):
        n = int(np.prod(shp))
        gi, goi = g[o:o + n], go[o:o + n]
        assert np.linalg.norm(gi - goi) <= 1e-2 * np.linalg.norm(goi) + 1e-12, name
        o += n
    net.close()


def test_training_fits_smooth_target_and_is_deterministic(fst):
    rng = np.random.default_rng(3)
    X = torch.from_numpy(rng.random((4096, 5)).astype(np.float32)).cuda()
    Xc = X.cpu().numpy()
    t = torch.from_numpy((10.0 + 3.0 * (np.sin(3 * Xc[:, 0]) + Xc[:, 1] ** 2 - Xc[:, 2] * Xc[:, 3]))
                         .astype(np.float32)).cuda()
    runs = []
    for _ in range(2):
        net = fst.MLP(256, max_batch=4096, seed=11)
        losses = net.train(X, t, steps=300, lr=2e-3).cpu().numpy()
        y = net.forward(X)
        runs.append((losses, y.cpu().numpy(), net.params().cpu().numpy()))
        net.close()
    losses, y, th = runs[0]
    assert losses[-1] < 0.02 * losses[0]
    # predictions come back in the units of the targets
    rel = np.sqrt(np.mean((y - t.cpu().numpy()) ** 2)) / np.std(t.cpu().numpy())
    assert rel < 0.15
    assert np.array_equal(runs[0][2], runs[1][2]) and np.array_equal(runs[0][1], runs[1][1])


@pytest.mark.parametrize("W,N", [(256, 1000), (256, 77), (128, 300)])
def test_tcgen05_path_matches_oracle_and_mma_sync(fst, W, N):
    """The tcgen05 GEMMs (TMEM accumulators) give the oracle's forward pass,
    loss and gradients to the same bf16 tolerance as the mma.sync GEMMs, and
    agree with them closely (fp32 sums in another order)."""
    theta = rand_theta(W, 4)
    theta32 = theta.astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(5)
    X = rng.random((N, 5)).astype(np.float32)
    t = (np.cos(3 * X[:, 0]) - X[:, 3] + X[:, 1] * X[:, 2]).astype(np.float32)
    t[::11] = np.nan
    out = {}
    for tc in (0, 1, 2):      # mma.sync; tcgen05 throughout; tcgen05 forward + mma.sync backward
        net = fst.MLP(W, max_batch=2048, seed=0)
        net.set_tensor_path(tc)
        net.set_params(torch.from_numpy(theta32.astype(np.float32)).cuda())
        y = net.forward(torch.from_numpy(X).cuda()).cpu().numpy().astype(np.float64)
        L, g = net.loss_grad(torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda())
        assert net.tensor_status()
        out[tc] = (y, float(L), g.cpu().numpy().astype(np.float64))
        net.close()
    yo = M.forward(theta32, X.astype(np.float64), W)
    Lo, go = M.loss_and_grad(theta32, X.astype(np.float64), t.astype(np.float64), W)
    scale = np.max(np.abs(yo))
    y, L, g = out[1]
    assert np.max(np.abs(y - yo)) <= 1e-2 * scale
    assert np.median(np.abs(y - yo)) <= 1e-4 * scale
    assert L == pytest.approx(Lo, rel=1e-3)
    for tc in (0, 1, 2):
        K.assert_elementwise(out[tc][2], theta32, X.astype(np.float64), t.astype(np.float64), W)
    o = 0
    for name, shp in M.param_shapes(W):
        n = int(np.prod(shp))
        assert np.linalg.norm(g[o:o + n] - go[o:o + n]) <= 1e-2 * np.linalg.norm(go[o:o + n]) + 1e-12, name
        o += n
    y0, L0, g0 = out[0]
    assert np.array_equal(out[2][0], y)      # the two tcgen05 paths share the forward layers
    assert np.max(np.abs(y - y0)) <= 1e-2 * scale
    assert np.linalg.norm(g - g0) <= 1e-2 * np.linalg.norm(g0)


def test_tcgen05_training_is_deterministic_and_fits(fst):
    rng = np.random.default_rng(7)
    X = torch.from_numpy(rng.random((4096, 5)).astype(np.float32)).cuda()
    Xc = X.cpu().numpy()
    t = torch.from_numpy((5.0 + 2.0 * (np.sin(3 * Xc[:, 0]) + Xc[:, 1] ** 2 - Xc[:, 2] * Xc[:, 3]))
                         .astype(np.float32)).cuda()
    runs = []
    for _ in range(2):
        net = fst.MLP(256, max_batch=4096, seed=13)
        net.set_tensor_path(True)
        losses = net.train(X, t, steps=200, lr=2e-3).cpu().numpy()
        assert net.tensor_status()
        runs.append((losses, net.params().cpu().numpy()))
        net.close()
    assert runs[0][0][-1] < 0.05 * runs[0][0][0]
    assert np.array_equal(runs[0][1], runs[1][1])


def test_first_adam_step_moves_each_weight_by_lr(fst):
    """Adam's bias-corrected first step is -lr g / (|g| + eps) (Kingma and
    Ba): every weight whose gradient is clearly non-zero moves by lr against
    the sign of its gradient, and no weight moves by more than lr. Targets
    are pre-standardised, so the training call's own standardisation leaves
    the gradient of fs_mlp_loss_grad unchanged."""
    rng = np.random.default_rng(8)
    Xc = rng.random((512, 5)).astype(np.float32)
    t = np.sin(3 * Xc[:, 0]) + Xc[:, 1]
    t = ((t - t.mean()) / t.std()).astype(np.float32)
    X = torch.from_numpy(Xc).cuda()
    tt = torch.from_numpy(t).cuda()
    net = fst.MLP(64, max_batch=512, seed=4)
    th0 = net.params().cpu().numpy()
    _, g = net.loss_grad(X, tt)
    g = g.cpu().numpy()
    lr = 1e-3
    net.train(X, tt, 1, lr)
    step = (net.params().cpu().numpy() - th0) / lr
    clear = np.abs(g) > 1e-4 * np.abs(g).max()
    assert clear.mean() > 0.25
    assert np.all(np.abs(step) <= 1.0 + 1e-3)
    assert np.allclose(step[clear], -np.sign(g[clear]), atol=1e-2)
    net.close()
