"""Surrogate plumbing of the search: per-box networks in the screened PSO step
and per-box sample rings, eager and captured.

The screened step gives network g the candidates of the g-th equal group of
runs, so a run's move depends only on its own group's network; the recorder
sends each group's (position, fitness) pairs to its own ring.
"""
import numpy as np
import pytest

from paper_2407_10797_gb300 import synth as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_10797_gb300 import fstat
    fstat.load()
    g = S.tiny_grid(n=20000, f_min=0.02)
    psd = S.lisa_like_psd(g.freqs())
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan = fstat.Plan.from_grid(g, mode=fstat.FS_MIXED, stream=s)
        plan.set_data(torch.from_numpy(S.gaussian_noise(g, psd, 3)).cuda(), torch.from_numpy(psd).cuda())
    box = np.zeros((4, 5, 2))
    box[:, 0] = (20.0, 40.0)
    box[:, 1] = (0.0, g.T_obs)
    box[:, 2] = (-1.0, 1.0)
    box[:, 3] = (0.0, 2 * np.pi)
    box[:, 4] = (0.0, 0.1)
    return fstat, plan, s, box


def nets(fstat, s, seeds):
    out = []
    for sd in seeds:
        out.append(fstat.MLP(64, max_batch=4096, seed=sd, stream=s))
    return out


def swarm_after_step(fstat, plan, s, box, mlps):
    with torch.cuda.stream(s):
        sw = fstat.Swarm(plan, 4, 40, box)
        sw.init(11)
        sw.evaluate(4)
        sw.step_screened(mlps, 16, 5, -1)
        sw.evaluate(4)
        sw.step_screened(mlps, 16, 5, -1)
    torch.cuda.synchronize()
    return sw.x.clone(), sw.v.clone()


def test_one_network_per_group_of_runs(env):
    fstat, plan, s, box = env
    A, B = nets(fstat, s, (1, 2))
    A2 = nets(fstat, s, (1,))[0]              # same seed: same weights as A
    B2 = nets(fstat, s, (2,))[0]
    xa, va = swarm_after_step(fstat, plan, s, box, [A])
    xaa, vaa = swarm_after_step(fstat, plan, s, box, [A, A2])
    assert torch.equal(xa, xaa) and torch.equal(va, vaa)
    xab, vab = swarm_after_step(fstat, plan, s, box, [A, B])
    xbb, vbb = swarm_after_step(fstat, plan, s, box, [B, B2])
    # runs 0-1 follow network A, runs 2-3 network B
    assert torch.equal(xab[:2], xa[:2]) and torch.equal(vab[:2], va[:2])
    assert torch.equal(xab[2:], xbb[2:]) and torch.equal(vab[2:], vbb[2:])
    assert not torch.equal(xa[2:], xbb[2:])
    with pytest.raises(fstat.FstatError):
        swarm_after_step(fstat, plan, s, box, [A, B, A2])   # 4 runs are not 3 equal groups


def test_rings_take_their_groups_samples(env):
    fstat, plan, s, box = env
    with torch.cuda.stream(s):
        sw = fstat.Swarm(plan, 4, 40, box)
        sw.init(3)
        sw.evaluate(4)
        rings = [fstat.SampleRing(100), fstat.SampleRing(100)]
        sw.record(rings)
        sw.record(rings)                       # 2 x 80 samples into 100 slots: wraps around
    torch.cuda.synchronize()
    x = sw.x.reshape(2, 80, 5).float()
    f = sw.fit.reshape(2, 80)
    for gidx, r in enumerate(rings):
        assert int(r.count.item()) == 160
        for slot in range(100):
            # append 1: sample i -> slot i; append 2: sample i -> slot (80 + i) mod 100
            i = slot + 20 if slot < 60 else (slot if slot < 80 else slot - 80)
            assert torch.equal(r.x[slot], x[gidx, i])
            fv = float(f[gidx, i])
            if np.isfinite(fv):
                assert float(r.f[slot]) == np.float32(fv)
            else:
                assert np.isnan(float(r.f[slot]))


def test_captured_screened_iteration_matches_eager(env):
    fstat, plan, s, box = env
    out = []
    for captured in (True, False):
        A, B = nets(fstat, s, (4, 5))
        with torch.cuda.stream(s):
            sw = fstat.Swarm(plan, 4, 40, box)
            sw.init(21)
            rings = [fstat.SampleRing(256), fstat.SampleRing(256)]
            if captured:
                g1 = sw.graph_build_ex(1 | 2, 4, 9, ring=rings)
                g2 = sw.graph_build_ex(8, 4, 9, mlp=[A, B], n_cand=8)
            for it in range(5):
                if captured:
                    g1.run(1)
                else:
                    sw.evaluate(4)
                    sw.record(rings)
                if it == 2:
                    for net, r in zip((A, B), rings):
                        net.train(r.x[:240], r.f[:240], 5, 1e-3)
                if captured:
                    g2.run(1)
                else:
                    sw.step_screened([A, B], 8, 9, -1)
        torch.cuda.synchronize()
        out.append((sw.x.clone(), sw.pbest_f.clone(), [r.x.clone() for r in rings]))
        if captured:
            g1.close()
            g2.close()
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
    for a, b in zip(out[0][2], out[1][2]):
        assert torch.equal(a, b)


def test_training_graph_matches_eager(env):
    """A captured training round (every network on its whole ring, empty
    slots ignored) replayed twice equals the same eager calls: the Adam step
    count and bias corrections live on the device."""
    fstat, plan, s, box = env
    with torch.cuda.stream(s):
        sw = fstat.Swarm(plan, 4, 40, box)
        sw.init(8)
        sw.evaluate(4)
        rings = [fstat.SampleRing(512), fstat.SampleRing(512)]
        for _ in range(3):
            sw.record(rings)                   # 240 of 512 slots written per ring
    torch.cuda.synchronize()
    eager = nets(fstat, s, (31, 32))
    captured = nets(fstat, s, (31, 32))
    with torch.cuda.stream(s):
        for _ in range(2):
            for net, r in zip(eager, rings):
                net.train(r.x, r.f, 3, 2e-3)
        g = fstat.mlp_train_graph(captured, rings, 3, 2e-3)
        g.run(2)
    torch.cuda.synchronize()
    for a, b in zip(eager, captured):
        assert torch.equal(a.params(), b.params())
    assert not torch.equal(eager[0].params(), nets(fstat, s, (31,))[0].params())   # training moved the weights
    g.close()


def test_many_rings_in_batches_of_launches(env):
    """40 rings (one launch covers 32): every ring holds its own runs'
    samples after two appends that wrap its 7 slots."""
    fstat, plan, s, _ = env
    box = np.zeros((40, 5, 2))
    box[:, 0] = (20.0, 40.0)
    box[:, 1] = (0.0, 1e7)
    box[:, 2] = (-1.0, 1.0)
    box[:, 3] = (0.0, 2 * np.pi)
    box[:, 4] = (0.0, 0.1)
    with torch.cuda.stream(s):
        sw = fstat.Swarm(plan, 40, 4, box)
        sw.init(5)
        sw.evaluate(4)
        rings = fstat.SampleRing.batch(40, 7)
        sw.record(rings)
        sw.record(rings)                       # 2 x 4 samples into 7 slots
    torch.cuda.synchronize()
    x = sw.x.reshape(40, 4, 5).float()
    f = sw.fit.reshape(40, 4)
    for g, r in enumerate(rings):
        assert int(r.count.item()) == 8
        for slot in range(7):
            # append 1 wrote samples 0-3 to slots 0-3, append 2 samples 0-3 to slots 4, 5, 6, 0
            i = 3 if slot == 0 else (slot if slot < 4 else slot - 4)
            assert torch.equal(r.x[slot], x[g, i])
            fv = float(f[g, i])
            assert (np.isnan(float(r.f[slot])) if not np.isfinite(fv) else float(r.f[slot]) == np.float32(fv))
