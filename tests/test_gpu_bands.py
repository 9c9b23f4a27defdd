"""Band edges of the particles (Sec. II: the template's band runs from its
frequency at t = 0 to its frequency at t = T_obs, in bins: first bin with
t(f_k) >= 0, last with t(f_k) <= T_obs) from the setup kernel, bit-exact
against the oracle's root find, on random draws and on the cases where the
band reaches an end of the grid or is empty."""
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


def gpu_bands(fst, g, P):
    plan = fst.Plan.from_grid(g, mode=fst.FS_FP64)
    psd = S.lisa_like_psd(g.freqs())
    plan.set_data(torch.zeros(g.n, dtype=torch.complex128).cuda(), torch.from_numpy(psd).cuda())
    b = plan.bands(torch.from_numpy(np.ascontiguousarray(P)).cuda()).cpu().numpy()
    plan.close()
    return b


def special(g, n_each=8, seed=3):
    """Coalescence long before, inside and long after the observation, prior
    corners in M_c and e0."""
    rng = np.random.default_rng(seed)
    rows = []
    for Mc in (10.0, 50.0):
        for e0 in (0.0, 0.1):
            for tc in (-1e7, -10.0, 0.0, 0.5 * g.T_obs, g.T_obs, g.T_obs + 10.0, 2 * g.T_obs, 40 * g.T_obs):
                rows.append([Mc, tc, np.arcsin(rng.uniform(-1, 1)), rng.uniform(0, 2 * np.pi), e0, 1.0])
    return np.array(rows)


def test_bands_match_oracle_paper_grid(fst):
    w = S.paper_workload()
    g = w.grid
    P = np.vstack([S.draw_params(w.prior, 3000, 21), special(g)])
    m = O.OracleModel.from_grid(g)
    ref = np.array([O.band(p, m) for p in P])
    got = gpu_bands(fst, g, P)
    bad = np.flatnonzero(np.any(got != ref, axis=1))
    assert bad.size == 0, (bad[:5], got[bad[:5]], ref[bad[:5]])
    assert np.any(ref[:, 0] == 0) and np.any(ref[:, 1] == g.n - 1) and np.any(ref[:, 0] > ref[:, 1])


@pytest.mark.parametrize("n", [20, 4096])
def test_bands_match_oracle_small_grids(fst, n):
    g = S.tiny_grid(n=n, f_min=0.02, stride=64)
    rng = np.random.default_rng(n)
    P = np.column_stack([rng.uniform(10, 50, 400), rng.uniform(-0.2, 1.5, 400) * g.T_obs,
                         np.arcsin(rng.uniform(-1, 1, 400)), rng.uniform(0, 2 * np.pi, 400),
                         rng.uniform(0, 0.1, 400), np.ones(400)])
    P = np.vstack([P, special(g)])
    m = O.OracleModel.from_grid(g)
    ref = np.array([O.band(p, m) for p in P])
    got = gpu_bands(fst, g, P)
    assert np.array_equal(got, ref)
