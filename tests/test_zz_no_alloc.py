"""fs_fstat_batch_noalloc: the F-statistic for callers that cannot allocate
device memory (its workspace is the library's fixed device array).

Two calls in a row, on different grids and segment layouts, must each match
fs_fstat_batch (the plan-based entry point) to the FP64 parity bar, so a call
never depends on what the previous call left in the shared workspace.  Sampled
particles are also checked against the CPU oracle, a call without F_part
(per-segment sums in the shared array) and a call at all three limits at once
against the plan entry point.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2407_10797_gb300 import synth as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-9


@pytest.fixture(scope="module")
def fst():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_10797_gb300 import fstat
    fstat.load()
    return fstat


def _case(grid, B, seed, Np, global_edges):
    psd = S.lisa_like_psd(grid.freqs())
    d = S.gaussian_noise(grid, psd, seed)
    P = S.draw_params(S.Prior(tc_lo=0.0, tc_hi=1.2 * grid.T_obs), B, seed)
    m = P[:, 0] * S.MSUN_S
    f_ref = grid.f_min + 0.5 * grid.n * grid.df
    P[:, 1] += 5.0 / 256.0 * m * (np.pi * m * f_ref) ** (-8.0 / 3.0) * (not global_edges)
    edges = grid.edge_freqs(np.linspace(0, grid.n, Np + 1).astype(np.int64)) if global_edges else None
    return (torch.from_numpy(d).cuda(), torch.from_numpy(psd).cuda(), torch.from_numpy(P).cuda(), edges)


def _with_plan(fst, grid, d, psd, P, Np, edges):
    plan = fst.Plan.from_grid(grid)
    plan.set_data(d, psd)
    F, Fp = plan.fstat(P, Np, edges=edges)
    torch.cuda.synchronize()
    out = F.cpu().numpy(), Fp.cpu().numpy()
    plan.close()
    return out


def _close(a, b, Np):
    assert np.array_equal(np.isnan(a), np.isnan(b))
    ok = ~np.isnan(b)
    return np.max(np.abs(a[ok] - b[ok]) / np.maximum(np.abs(b[ok]), 2.0 * Np), initial=0.0) <= TOL64


def test_noalloc_matches_plan_entry_point_on_two_calls(fst):
    n = 1 << 15
    df = 0.01 / n
    g1 = S.Grid(f_min=0.015, df=df, n=n, T_obs=1.0 / df)           # the 2^15-bin workload, global edges
    g2 = S.tiny_grid(n=20000, f_min=0.02, stride=8)                  # a 2.5 yr slice, per-particle segments
    calls = [(g1, 1024, 0, 8, True), (g2, 333, 4, 64, False)]
    results = []
    for g, B, seed, Np, glob in calls:
        d, psd, P, edges = _case(g, B, seed, Np, glob)
        Fp = torch.empty(B, Np, dtype=torch.float64, device="cuda")
        F, _ = fst.fstat_batch_noalloc(g, d, psd, P, Np, edges=edges, F_part=Fp)
        torch.cuda.synchronize()
        results.append((F.cpu().numpy(), Fp.cpu().numpy(), g, d, psd, P, Np, edges))
    for F, Fp, g, d, psd, P, Np, edges in results:
        Fr, Fpr = _with_plan(fst, g, d, psd, P, Np, edges)
        assert _close(F, Fr, Np)
        assert _close(Fp.ravel(), Fpr.ravel(), 1)
        # a few particles against the oracle, which shares nothing with either entry point
        idx = np.arange(0, P.shape[0], max(1, P.shape[0] // 6))[:6]
        Pn = P.cpu().numpy()[idx]
        Fo, _ = O.fstat_batch(Pn, O.OracleModel.from_grid(g), d.cpu().numpy(),
                              psd.cpu().numpy(), Np, edges_hz=edges)
        assert _close(F[idx], Fo, Np)


def test_noalloc_without_F_part_and_at_every_limit_at_once(fst):
    """n_bins = 32768, B = 1024 and N_p = 64 in one call (the largest layout
    the fixed array holds), with F_part = NULL so that the per-segment values
    go to the array's own region; then a small call, to see that the second
    does not depend on the first."""
    n = 1 << 15
    df = 0.01 / n
    g = S.Grid(f_min=0.015, df=df, n=n, T_obs=1.0 / df)
    g2 = S.tiny_grid(n=5000, f_min=0.02, stride=8)
    for grid, B, Np, glob, seed in ((g, 1024, 64, True, 6), (g2, 50, 3, False, 7)):
        d, psd, P, edges = _case(grid, B, seed, Np, glob)
        F, Fp = fst.fstat_batch_noalloc(grid, d, psd, P, Np, edges=edges)
        assert Fp is None
        F = F.cpu().numpy()
        Fr, _ = _with_plan(fst, grid, d, psd, P, Np, edges)
        assert _close(F, Fr, Np)


def test_noalloc_rejects_sizes_beyond_its_limits(fst):
    g = S.tiny_grid(n=32769, f_min=0.02, stride=8)
    d = torch.zeros(g.n, dtype=torch.complex128, device="cuda")
    psd = torch.ones(g.n, dtype=torch.float64, device="cuda")
    P = torch.zeros(4, 6, dtype=torch.float64, device="cuda")
    with pytest.raises(fst.FstatError) as ei:
        fst.fstat_batch_noalloc(g, d, psd, P, 8)
    assert ei.value.status == fst.FS_EINVAL and "limit" in str(ei.value)
    g = S.tiny_grid(n=1000, f_min=0.02, stride=8)
    d = torch.zeros(g.n, dtype=torch.complex128, device="cuda")
    psd = torch.ones(g.n, dtype=torch.float64, device="cuda")
    with pytest.raises(fst.FstatError):
        fst.fstat_batch_noalloc(g, d, psd, P, 65)
    with pytest.raises(fst.FstatError):
        fst.fstat_batch_noalloc(g, d, psd, torch.zeros(1025, 6, dtype=torch.float64, device="cuda"), 8)
