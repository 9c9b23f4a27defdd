"""Device PSO step (Sec. III.A) against the CPU oracle, bit for bit, and the
captured PSO iteration against eager launches."""

import numpy as np
import pytest

from oracle import oracle as O
from paper_2407_10797_gb300 import synth as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fst():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_10797_gb300 import fstat
    fstat.load()
    return fstat


@pytest.fixture(scope="module")
def plan(fst):
    g = S.tiny_grid(n=6000, f_min=0.02, stride=4)
    psd = S.lisa_like_psd(g.freqs())
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        p = fst.Plan.from_grid(g, mode=fst.FS_MIXED, stream=s)
        p.set_data(torch.from_numpy(S.gaussian_noise(g, psd, 3)).cuda(), torch.from_numpy(psd).cuda())
    torch.cuda.synchronize()
    p.grid = g
    p.psd = psd
    yield p
    p.close()


def unit_box(R):
    return np.tile(np.array([[10.0, 50.0], [0.0, 1e8], [-1.0, 1.0], [0.0, 2 * np.pi], [0.0, 0.1]]), (R, 1, 1))


def test_init_matches_oracle(fst, plan):
    R, Np = 3, 40
    sw = fst.Swarm(plan, R, Np, unit_box(R))
    sw.init(seed=12345)
    torch.cuda.synchronize()
    xo, vo = O.pso_init(R, Np, 5, 12345)
    assert np.array_equal(sw.x.cpu().numpy(), xo)
    assert np.array_equal(sw.v.cpu().numpy(), vo)
    assert np.all(np.isneginf(sw.pbest_f.cpu().numpy()))


def dmu_box(R):
    """The unit box with delta_mu in the paper's [0, 0.9] as a sixth coordinate."""
    b = unit_box(R)
    return np.concatenate([b, np.tile(np.array([[0.0, 0.9]]), (R, 1, 1))], axis=1)


@pytest.mark.parametrize("dims", [5, 6])
def test_steps_bit_exact_with_oracle(fst, plan, dims):
    """Random fitness arrays with NaN, -inf and ties; several iterations; the
    5-D space and the 6-D one with delta_mu free."""
    R, Np, seed, n_iter = 4, 40, 99, 7
    sw = fst.Swarm(plan, R, Np, unit_box(R) if dims == 5 else dmu_box(R), dims=dims)
    sw.init(seed)
    torch.cuda.synchronize()
    x = sw.x.cpu().numpy().copy()
    v = sw.v.cpu().numpy().copy()
    pbx = sw.pbest_x.cpu().numpy().copy()
    pbf = sw.pbest_f.cpu().numpy().copy()
    rng = np.random.default_rng(0)
    lb_dev = torch.zeros(R, Np, dtype=torch.int32, device="cuda")
    for it in range(n_iter):
        fit = np.round(rng.normal(size=(R, Np)), 1)          # many ties
        fit[rng.random((R, Np)) < 0.1] = -np.inf
        fit[rng.random((R, Np)) < 0.05] = np.nan
        sw.fit.copy_(torch.from_numpy(fit))
        sw.step(seed, it, w0=0.9, w1=0.4, n_iter=n_iter, c1=2.0, c2=2.0, vmax=0.5, lbest=lb_dev)
        w = 0.9 - (0.9 - 0.4) * (it / (n_iter - 1))
        lb = O.pso_step(x, v, pbx, pbf, fit, seed, it, w, 2.0, 2.0, 0.5)
        torch.cuda.synchronize()
        assert np.array_equal(lb_dev.cpu().numpy(), lb)
        assert np.array_equal(sw.pbest_f.cpu().numpy(), pbf)
        assert np.array_equal(sw.pbest_x.cpu().numpy(), pbx)
        assert np.array_equal(sw.v.cpu().numpy(), v)
        assert np.array_equal(sw.x.cpu().numpy(), x)


def test_device_iteration_counter_and_graph_replay(fst, plan):
    R, Np, seed = 2, 40, 5
    box = unit_box(R)
    g = plan.grid
    box[:, 1] = [0.3 * g.T_obs, 1.5 * g.T_obs]

    def fresh():
        sw = fst.Swarm(plan, R, Np, box)
        with torch.cuda.stream(plan.stream):
            sw.init(seed)
        return sw

    eager, graphed = fresh(), fresh()
    with torch.cuda.stream(plan.stream):
        for it in range(5):
            eager.evaluate(16)
            eager.step(seed, -1, n_iter=5)
        graphed.graph_build(16, seed, n_iter=5)
        graphed.graph_run(5)
    torch.cuda.synchronize()
    assert int(graphed.iter.item()) == 5 and int(eager.iter.item()) == 5
    for name in ("x", "v", "pbest_x", "pbest_f", "fit"):
        assert torch.equal(getattr(eager, name), getattr(graphed, name)), name


def test_evaluate_is_F_hat_and_let_them_fly(fst, plan):
    R, Np = 2, 40
    g = plan.grid
    box = unit_box(R)
    box[:, 1] = [0.3 * g.T_obs, 1.5 * g.T_obs]
    sw = fst.Swarm(plan, R, Np, box)
    with torch.cuda.stream(plan.stream):
        sw.init(7)
        sw.x[0, :5] += 2.0   # outside the unit box
        sw.evaluate(8)
    torch.cuda.synchronize()
    fit = sw.fit.cpu().numpy()
    assert np.all(np.isneginf(fit[0, :5]))
    # the inside particles: F_sum / N_p of the mapped parameters
    x = sw.x.cpu().numpy()
    y = box[:, None, :, 0] + x * (box[:, None, :, 1] - box[:, None, :, 0])
    P = np.stack([y[..., 0], y[..., 1], np.arcsin(np.clip(y[..., 2], -1, 1)), y[..., 3], y[..., 4],
                  np.ones_like(y[..., 0])], axis=-1).reshape(-1, 6)
    with torch.cuda.stream(plan.stream):
        F, _ = plan.fstat(torch.from_numpy(P).cuda(), 8)
    torch.cuda.synchronize()
    Fh = F.cpu().numpy().reshape(R, Np) / 8
    inside = ~np.isneginf(fit)
    # the host mapping rounds t_c differently from the device FMA by an ulp,
    # which moves F by ~1e-9; a wrong mapping would move it by O(1)
    assert np.allclose(fit[inside], Fh[inside], rtol=1e-6, atol=0)


def test_graph_reads_its_own_edges_after_other_calls(fst, plan):
    """A captured iteration with global edges A still uses A when it is
    replayed after an evaluation with edges B (and after another graph with
    edges B) on the same plan: each evaluation converts its own edge
    frequencies on the stream, so no captured graph depends on what an
    earlier call left in the plan."""
    R, Np, seed = 2, 40, 21
    g = plan.grid
    box = unit_box(R)
    box[:, 1] = [0.3 * g.T_obs, 1.5 * g.T_obs]
    eA = torch.tensor(g.edge_freqs([0, 1500, 3000, 4500, 6000]), dtype=torch.float64, device="cuda")
    eB = torch.tensor(g.edge_freqs([100, 200, 5900]), dtype=torch.float64, device="cuda")

    def fresh():
        sw = fst.Swarm(plan, R, Np, box)
        with torch.cuda.stream(plan.stream):
            sw.init(seed)
        return sw

    eager, graphed, other = fresh(), fresh(), fresh()
    with torch.cuda.stream(plan.stream):
        graphed.graph_build(4, seed, edges=eA, n_iter=6)
        other.graph_build(2, seed, edges=eB, n_iter=6)
        for it in range(3):
            eager.evaluate(4, edges=eA)
            eager.step(seed, -1, n_iter=6)
            graphed.graph_run(1)
            other.graph_run(1)
            other.evaluate(2, edges=eB)       # overwrites the plan's segment starts with B
    torch.cuda.synchronize()
    for name in ("x", "v", "pbest_x", "pbest_f", "fit"):
        assert torch.equal(getattr(eager, name), getattr(graphed, name)), name
    assert plan.check() == 0


def test_six_dimensional_swarm_maps_delta_mu_to_the_mass_ratio(fst, plan):
    """With delta_mu free, a particle's fitness is F-hat at the mass ratio
    q = (1 + delta_mu)/(1 - delta_mu) of its sixth coordinate (Sec. II.A's
    dimensionless mass difference), and the init draws the oracle's 6-D
    positions."""
    R, Np = 2, 40
    g = plan.grid
    box = dmu_box(R)
    box[:, 1] = [0.3 * g.T_obs, 1.5 * g.T_obs]
    sw = fst.Swarm(plan, R, Np, box, dims=6)
    with torch.cuda.stream(plan.stream):
        sw.init(11)
        sw.evaluate(4)
    torch.cuda.synchronize()
    xo, vo = O.pso_init(R, Np, 6, 11)
    assert np.array_equal(sw.x.cpu().numpy(), xo) and np.array_equal(sw.v.cpu().numpy(), vo)
    x = sw.x.cpu().numpy()
    y = box[:, None, :, 0] + x * (box[:, None, :, 1] - box[:, None, :, 0])
    dmu = y[..., 5]
    P = np.stack([y[..., 0], y[..., 1], np.arcsin(np.clip(y[..., 2], -1, 1)), y[..., 3], y[..., 4],
                  (1.0 + dmu) / (1.0 - dmu)], axis=-1).reshape(-1, 6)
    with torch.cuda.stream(plan.stream):
        F, _ = plan.fstat(torch.from_numpy(P).cuda(), 4)
    torch.cuda.synchronize()
    fit = sw.fit.cpu().numpy()
    Fh = F.cpu().numpy().reshape(R, Np) / 4
    inside = ~np.isneginf(fit)
    assert inside.sum() > 40 and np.any(np.abs(dmu - 0.45) > 0.3)
    assert np.allclose(fit[inside], Fh[inside], rtol=1e-6, atol=0)
    # the screened step needs the networks' 5 inputs
    with pytest.raises(fst.FstatError) as ei:
        net = fst.MLP(64, max_batch=512, seed=0, stream=plan.stream)
        sw.step_screened(net, 4, 11, 0)
    assert ei.value.status == fst.FS_EUNSUPPORTED


def test_rings_hold_the_swarms_dimensions(fst, plan):
    """A ring declares its floats per sample; a 6-D swarm appends only to a
    6-float ring (a 5-float one would overflow and is refused), and the
    samples are the positions as floats."""
    R, Np = 2, 40
    sw = fst.Swarm(plan, R, Np, dmu_box(R), dims=6)
    with torch.cuda.stream(plan.stream):
        sw.init(3)
        sw.evaluate(4)
        with pytest.raises(fst.FstatError) as ei:
            sw.record(fst.SampleRing(256))
        assert ei.value.status == fst.FS_EINVAL
        ring = fst.SampleRing(256, dims=6)
        sw.record(ring)
    torch.cuda.synchronize()
    assert int(ring.count.item()) == R * Np
    assert torch.equal(ring.x[:R * Np], sw.x.reshape(-1, 6).float())
