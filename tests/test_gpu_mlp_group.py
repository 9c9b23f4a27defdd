"""A batch of G surrogate networks (one fs_mlp, every kernel over all G)
against G networks created and run one by one: same seeds (seed + g), same
summation order, so every result must be identical bit for bit."""
import numpy as np
import pytest

from paper_2407_10797_gb300 import synth as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

G, W, CAP = 3, 64, 512


@pytest.fixture(scope="module")
def fs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_10797_gb300 import fstat
    fstat.load()
    return fstat


def data(n, seed, nan_every=0):
    g = torch.Generator().manual_seed(seed)
    X = torch.rand(G, n, 5, generator=g)
    t = (X[..., 0] * 3 - X[..., 1] ** 2 + 0.5 * torch.sin(6 * X[..., 2])) * 40 + 100
    if nan_every:
        t[:, ::nan_every] = float("nan")
    return X.cuda(), t.cuda()


@pytest.mark.parametrize("tc5", [0, 1, 2])
def test_batch_equals_separate_networks(fs, tc5):
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        batch = fs.MLP(W, max_batch=CAP, seed=7, stream=s, groups=G)
        single = [fs.MLP(W, max_batch=CAP, seed=7 + g, stream=s) for g in range(G)]
        for net in [batch] + single:
            net.set_tensor_path(tc5)
    assert batch.groups == G and batch.params().shape == (G, batch.P)
    for g in range(G):
        assert torch.equal(batch.params()[g], single[g].params())
    # forward over more rows than max_batch (chunked), before any training
    X, _ = data(CAP + 333, 1)
    with torch.cuda.stream(s):
        yb = batch.forward(X)
        ys = [single[g].forward(X[g]) for g in range(G)]
    s.synchronize()
    assert yb.shape == (G, CAP + 333)
    for g in range(G):
        assert torch.equal(yb[g], ys[g])
    # loss and gradient with ignored (NaN) targets
    X, t = data(CAP - 17, 2, nan_every=5)
    with torch.cuda.stream(s):
        Lb, gb = batch.loss_grad(X, t)
        ref = [single[g].loss_grad(X[g], t[g]) for g in range(G)]
    s.synchronize()
    for g in range(G):
        assert torch.equal(Lb[g:g + 1], ref[g][0])
        assert torch.equal(gb[g * batch.P:(g + 1) * batch.P], ref[g][1])
    # Adam training (standardised targets), then predictions in target units
    with torch.cuda.stream(s):
        lb = batch.train(X, t, 4, 2e-3)
        ls = [single[g].train(X[g], t[g], 4, 2e-3) for g in range(G)]
        Xq, _ = data(200, 3)
        yb = batch.forward(Xq)
        ys = [single[g].forward(Xq[g]) for g in range(G)]
    s.synchronize()
    assert lb.shape == (4, G)
    for g in range(G):
        assert torch.equal(lb[:, g], ls[g])
        assert torch.equal(batch.params()[g], single[g].params())
        assert torch.equal(yb[g], ys[g])
    assert not torch.equal(batch.params()[0], batch.params()[1])
    assert batch.tensor_status() and all(n.tensor_status() for n in single)


def test_batch_rejects_bad_shapes(fs):
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        batch = fs.MLP(W, max_batch=CAP, seed=1, stream=s, groups=G)
        with pytest.raises(ValueError):
            batch.forward(torch.rand(10, 5, device="cuda"))
        with pytest.raises(fs.FstatError):
            fs.MLP(W, max_batch=CAP, seed=1, stream=s, groups=0)
        with pytest.raises(fs.FstatError):
            batch.train(*data(CAP + 1, 4), 1, 1e-3)   # training rows must fit max_batch


@pytest.fixture(scope="module")
def swarm_env(fs):
    g = S.tiny_grid(n=20000, f_min=0.02)
    psd = S.lisa_like_psd(g.freqs())
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan = fs.Plan.from_grid(g, mode=fs.FS_MIXED, stream=s)
        plan.set_data(torch.from_numpy(S.gaussian_noise(g, psd, 5)).cuda(), torch.from_numpy(psd).cuda())
    box = np.zeros((6, 5, 2))
    box[:, 0] = (20.0, 40.0)
    box[:, 1] = (0.0, g.T_obs)
    box[:, 2] = (-1.0, 1.0)
    box[:, 3] = (0.0, 2 * np.pi)
    box[:, 4] = (0.0, 0.1)
    return plan, s, box


def run_search(fs, plan, s, box, nets, rings, graphs):
    """Five captured iterations (evaluate + record, screened step) with one
    captured training round after the third."""
    with torch.cuda.stream(s):
        sw = fs.Swarm(plan, 6, 30, box)
        sw.init(17)
        g1 = sw.graph_build_ex(1 | 2, 4, 9, ring=rings)
        g2 = sw.graph_build_ex(8, 4, 9, mlp=nets, n_cand=8)
        gt = fs.mlp_train_graph(nets, rings, 3, 2e-3) if graphs else None
        for it in range(5):
            g1.run(1)
            if it == 2:
                if graphs:
                    gt.run(1)
                else:
                    for net, r in zip(nets, rings):
                        net.train(r.x, r.f, 3, 2e-3)
            g2.run(1)
    torch.cuda.synchronize()
    for gr in (g1, g2, gt):
        if gr is not None:
            gr.close()
    return sw.x.clone(), sw.pbest_f.clone()


def test_batch_in_screened_search(fs, swarm_env):
    """Three boxes' networks as one batch (rings from SampleRing.batch, one
    training graph) move the swarm exactly as three separate networks do."""
    plan, s, box = swarm_env
    with torch.cuda.stream(s):
        batch = fs.MLP(W, max_batch=CAP, seed=40, stream=s, groups=3)
        single = [fs.MLP(W, max_batch=CAP, seed=40 + g, stream=s) for g in range(3)]
        rings_b = fs.SampleRing.batch(3, 256)
        rings_s = [fs.SampleRing(256) for _ in range(3)]
    xb, fb = run_search(fs, plan, s, box, [batch], rings_b, graphs=True)
    xs, fsep = run_search(fs, plan, s, box, single, rings_s, graphs=False)
    assert torch.equal(xb, xs) and torch.equal(fb, fsep)
    for g in range(3):
        assert torch.equal(rings_b[g].x, rings_s[g].x)
        assert torch.equal(batch.params()[g], single[g].params())
    # two batches of networks side by side cover the boxes in order
    with torch.cuda.stream(s):
        b1 = fs.MLP(W, max_batch=CAP, seed=40, stream=s, groups=1)
        b2 = fs.MLP(W, max_batch=CAP, seed=41, stream=s, groups=2)
        rings_2 = [fs.SampleRing(256)] + fs.SampleRing.batch(2, 256)
    x2, f2 = run_search(fs, plan, s, box, [b1, b2], rings_2, graphs=True)
    assert torch.equal(x2, xs) and torch.equal(f2, fsep)
    # rings of a batch that are not slices of one buffer are refused
    with pytest.raises(fs.FstatError):
        fs.mlp_train_graph([batch], rings_s, 1, 1e-3)
