"""fs_fstat_batch_noalloc: the F-statistic for callers that cannot allocate
device memory (its workspace is the library's fixed device array).

Two calls in a row, on different grids and segment layouts, must each match
fs_fstat_batch (the plan-based entry point) to the FP64 parity bar, so a call
never depends on what the previous call left in the shared workspace.  This
file is collected last on purpose.
"""
import numpy as np
import pytest

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
    edges = np.linspace(0, grid.n, Np + 1).astype(np.int64) if global_edges else None
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
