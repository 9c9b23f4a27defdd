"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bar (FP64 mode): |F_gpu - F_oracle| / max(|F_oracle|, 2 N_p) <= 1e-9 for the
sum, and the same with max(|F_p|, 2) per segment.  The normalisation by the
noise-only mean E[F_sum] = 2 N_p keeps the bar meaningful where F is small.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2407_10797_gb300 import synth as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-9


def tc_for(Mc, f, t):
    m = Mc * S.MSUN_S
    return t + 5.0 / 256.0 * m * (np.pi * m * f) ** (-8.0 / 3.0)


@pytest.fixture(scope="module")
def fst():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_10797_gb300 import fstat
    fstat.load()
    return fstat


def make_data(grid, seed, inj=None, snr=12.0):
    """Noise + (optionally) an oracle-made injection limited to its band."""
    psd = S.lisa_like_psd(grid.freqs())
    d = S.gaussian_noise(grid, psd, seed)
    if inj is not None:
        m = O.OracleModel.from_grid(grid)
        a = O.extrinsic_to_a(1.0, S.INJ_PSI, S.INJ_IOTA, S.INJ_PHIC)
        k0, k1 = O.band(inj, m)
        h = O.inject(inj, m, a, k0, k1 + 1)
        d = d + h * (snr / math.sqrt(O.inner(h, h, psd, grid.df)))
    return d, psd


def run_gpu(fst, grid, d, psd, P, Np, edges=None, mode=0, edges_hz=None):
    """F and F_part on the GPU; global segments as start bins (edges) or frequencies (edges_hz)."""
    plan = fst.Plan.from_grid(grid, mode=mode)
    plan.set_data(torch.from_numpy(d).cuda(), torch.from_numpy(psd).cuda())
    if edges is not None:
        edges_hz = grid.edge_freqs(edges)
    F, Fp = plan.fstat(torch.from_numpy(np.ascontiguousarray(P)).cuda(), Np, edges=edges_hz)
    torch.cuda.synchronize()
    out = F.cpu().numpy(), Fp.cpu().numpy()
    plan.close()
    return out


def assert_parity(Fg, Fpg, Fo, Fpo, Np, tol):
    both_nan = np.isnan(Fg) & np.isnan(Fo)
    ok = ~both_nan
    err = np.abs(Fg[ok] - Fo[ok]) / np.maximum(np.abs(Fo[ok]), 2.0 * Np)
    assert np.all(np.isnan(Fg) == np.isnan(Fo))
    assert err.max(initial=0.0) <= tol, f"max rel err {err.max():.3e}"
    if Fpg is not None:
        errp = np.abs(Fpg[ok] - Fpo[ok]) / np.maximum(np.abs(Fpo[ok]), 2.0)
        assert errp.max(initial=0.0) <= tol, f"max per-segment rel err {errp.max():.3e}"
    return err.max(initial=0.0)


def in_band_params(grid, B, seed, f_ref, spread=(0.1, 0.9)):
    P = S.draw_params(S.Prior(tc_lo=spread[0] * grid.T_obs, tc_hi=spread[1] * grid.T_obs), B, seed)
    P[:, 1] = tc_for(P[:, 0], f_ref, P[:, 1])
    return P


# ---------------------------------------------------------------- small cases
@pytest.mark.parametrize("Np", [1, 3, 16, 256])
def test_fp64_per_particle_segments_small(fst, Np):
    """5000 bins (two full tiles and a ragged third) of the 2.5 yr grid;
    37 particles (a partial particle group) with bands that start and end
    at different bins; injection + noise."""
    g = S.tiny_grid(n=5000, f_min=0.02, stride=16)
    P = in_band_params(g, 37, 5, 0.02 + 2500 * g.df, spread=(-0.3, 1.3))
    inj = in_band_params(g, 1, 6, 0.02 + 2500 * g.df, spread=(0.5, 0.5))[0]
    d, psd = make_data(g, 3, inj=inj)
    Fg, Fpg = run_gpu(fst, g, d, psd, P, Np)
    Fo, Fpo = O.fstat_batch(P, O.OracleModel.from_grid(g), d, psd, Np)
    assert np.any(Fo > 0) and np.any(Fo == 0)   # some particles have no band at all
    assert_parity(Fg, Fpg, Fo, Fpo, Np, TOL64)


@pytest.mark.parametrize("edges", [
    [0, 1024, 2048, 3072, 4096, 5120, 6144, 7168, 8192],
    [0, 3, 3, 100, 2047, 2049, 5000, 8191],                 # empty and tiny segments
    [17, 8000],
])
def test_fp64_global_edges_small(fst, edges):
    n = 8192
    df = 0.01 / (1 << 15)
    g = S.Grid(f_min=0.015, df=df, n=n, T_obs=1.0 / df)
    P = S.draw_params(S.Prior(tc_lo=0.0, tc_hi=g.T_obs), 41, 8)
    d, psd = make_data(g, 1)
    Np = len(edges) - 1
    e = np.array(edges, dtype=np.int64)
    Fg, Fpg = run_gpu(fst, g, d, psd, P, Np, edges=e)
    Fo, Fpo = O.fstat_batch(P, O.OracleModel.from_grid(g), d, psd, Np, edges=e)
    assert_parity(Fg, Fpg, Fo, Fpo, Np, TOL64)


def test_fp64_edge_frequencies_on_bins_and_outside_the_grid(fst):
    """Edges given as frequencies that sit exactly on bin frequencies (the
    bin belongs to the segment that starts there; the last edge is closed),
    below the first bin and above the last one: the device's conversion to
    bins matches the oracle's membership rule (e_p <= f_k < e_{p+1})."""
    n = 8192
    df = 0.01 / (1 << 15)
    g = S.Grid(f_min=0.015, df=df, n=n, T_obs=1.0 / df)
    P = S.draw_params(S.Prior(tc_lo=0.0, tc_hi=g.T_obs), 29, 12)
    d, psd = make_data(g, 3)
    f = g.freqs()
    m = O.OracleModel.from_grid(g)
    cases = [
        np.array([f[0], f[100], f[100], f[4095], f[8191]]),
        np.array([g.f_min - 10 * df, f[3] + 0.3 * df, f[7000], g.f_min + (n + 5) * df]),
        np.array([f[2000], f[2000] + 0.49 * df, f[2001], f[2004]]),
    ]
    for e in cases:
        Np = len(e) - 1
        starts = O.edge_starts(m, e, Np)
        Fg, Fpg = run_gpu(fst, g, d, psd, P, Np, edges_hz=e)
        Fo, Fpo = O.fstat_batch(P, m, d, psd, Np, edges=starts)
        assert_parity(Fg, Fpg, Fo, Fpo, Np, TOL64)


def test_fp64_noise_free_injection_recovers_half_snr2(fst):
    g = S.tiny_grid(n=4096, f_min=0.02, stride=4)
    p = np.array([28.0, tc_for(28.0, 0.02 + 2048 * g.df, 0.5 * g.T_obs), 0.4, 2.0, 0.04, 1.0])
    m = O.OracleModel.from_grid(g)
    psd = S.lisa_like_psd(g.freqs())
    a = O.extrinsic_to_a(1.0, S.INJ_PSI, S.INJ_IOTA, S.INJ_PHIC)
    k0, k1 = O.band(p, m)
    h = O.inject(p, m, a, k0, k1 + 1)
    h *= 10.0 / math.sqrt(O.inner(h, h, psd, g.df))
    for Np in (1, 7):
        Fg, _ = run_gpu(fst, g, h, psd, p[None], Np)
        assert Fg[0] == pytest.approx(50.0, rel=1e-9)


def test_edge_cases(fst):
    g = S.tiny_grid(n=3000, f_min=0.02, stride=8)
    d, psd = make_data(g, 2)
    P = in_band_params(g, 6, 2, 0.02 + 1500 * g.df)
    P[1, 0] = np.nan                       # non-finite -> NaN
    P[2, 1] = -1e9                         # merged before the data: empty band -> 0
    P[3, 4] = 0.0                          # circular
    P[4, 0] = -5.0                         # unphysical -> NaN
    Fg, Fpg = run_gpu(fst, g, d, psd, P, 8)
    Fo, Fpo = O.fstat_batch(P, O.OracleModel.from_grid(g), d, psd, 8)
    assert np.isnan(Fg[1]) and np.isnan(Fg[4]) and Fg[2] == 0.0
    assert_parity(Fg, Fpg, Fo, Fpo, 8, TOL64)
    # B = 0 launches nothing and succeeds
    plan = fst.Plan.from_grid(g)
    plan.set_data(torch.from_numpy(d).cuda(), torch.from_numpy(psd).cuda())
    F, Fp = plan.fstat(torch.zeros(0, 6, dtype=torch.float64, device="cuda"), 4)
    assert F.numel() == 0
    # invalid sizes are rejected before any launch
    for bad in (dict(Np=0), dict(Np=5000)):
        with pytest.raises(fst.FstatError) as ei:
            plan.fstat(torch.from_numpy(P).cuda(), bad["Np"])
        assert ei.value.status == fst.FS_EINVAL
    # edge frequencies live on the device: decreasing or non-finite ones give
    # NaN for every particle, and fs_plan_check reports them afterwards
    assert plan.check() == 0
    f = g.freqs()
    for bad in ([f[5], f[3], f[9]], [f[5], np.nan, f[9]]):
        F, Fp = plan.fstat(torch.from_numpy(P).cuda(), 2, edges=bad)
        assert torch.isnan(F).all() and torch.isnan(Fp).all()
        with pytest.raises(fst.FstatError) as ei:
            plan.check()
        assert ei.value.status == fst.FS_EINVAL
        assert plan.check() == 0          # the flag is cleared by the check
    # a valid call after an invalid one is not affected
    F, _ = plan.fstat(torch.from_numpy(P).cuda(), 2, edges=[f[0], f[1000], f[2999]])
    Fo, _ = O.fstat_batch(P, O.OracleModel.from_grid(g), d, psd, 2, edges_hz=[f[0], f[1000], f[2999]])
    assert_parity(F.cpu().numpy(), None, Fo, None, 2, TOL64)
    plan.close()
    with pytest.raises(fst.FstatError):
        fst.Plan(0, 0.01, 1e-6, 1e7)


def test_runs_are_bitwise_deterministic(fst):
    g = S.tiny_grid(n=6000, f_min=0.02, stride=4)
    d, psd = make_data(g, 5)
    P = torch.from_numpy(in_band_params(g, 64, 1, 0.02 + 3000 * g.df, spread=(-0.2, 1.2))).cuda()
    plan = fst.Plan.from_grid(g)
    plan.set_data(torch.from_numpy(d).cuda(), torch.from_numpy(psd).cuda())
    a = [plan.fstat(P, 16)[0].clone() for _ in range(3)]
    torch.cuda.synchronize()
    assert torch.equal(a[0], a[1]) and torch.equal(a[0], a[2])
    plan.close()


def test_add_signal_matches_oracle_template(fst):
    g = S.tiny_grid(n=4000, f_min=0.02, stride=4)
    psd = S.lisa_like_psd(g.freqs())
    p = np.array([33.0, tc_for(33.0, 0.02 + 2000 * g.df, 0.6 * g.T_obs), -0.3, 5.0, 0.07, 1.0])
    a = np.array([0.3, -1.2, 0.8, 0.45])
    m = O.OracleModel.from_grid(g)
    k0, k1 = O.band(p, m)
    ho = O.inject(p, m, a, k0, k1 + 1)
    plan = fst.Plan.from_grid(g)
    plan.set_data(torch.zeros(g.n, dtype=torch.complex128, device="cuda"), torch.from_numpy(psd).cuda())
    hg = torch.zeros(g.n, dtype=torch.complex128, device="cuda")
    plan.add_signal(p, a, hg)
    hg = hg.cpu().numpy()
    plan.close()
    scale = np.abs(ho).max()
    assert np.max(np.abs(hg - ho)) <= 1e-9 * scale
    assert np.all(hg[:k0] == 0) and np.all(hg[k1 + 1:] == 0)


# ---------------------------------------------------------------- full-size cases
def test_small_workload_full_size_sampled(fst):
    """2^15 bins, B = 1024, N_p = 8 global edges (the timed small workload):
    every particle finite and >= 0, 24 sampled particles against the oracle."""
    w = S.small_workload()
    g = w.grid
    P = S.draw_params(w.prior, w.B, w.seed)
    d, psd = make_data(g, w.seed)
    edges = np.arange(9, dtype=np.int64) * (g.n // 8)
    Fg, Fpg = run_gpu(fst, g, d, psd, P, 8, edges=edges)
    assert np.all(np.isfinite(Fg)) and np.all(Fg >= 0)
    idx = np.r_[0:8, 511:519, 1016:1024]
    Fo, Fpo = O.fstat_batch(P[idx], O.OracleModel.from_grid(g), d, psd, 8, edges=edges)
    assert_parity(Fg[idx], Fpg[idx], Fo, Fpo, 8, TOL64)


@pytest.mark.slow
def test_paper_workload_full_size_sampled(fst):
    """3,155,760 bins (2.5 yr, 10-50 mHz), B = 320, N_p in {256, 64, 16, 1}:
    sampled in-band particles against the oracle."""
    w = S.paper_workload()
    g = w.grid
    P = S.draw_params(w.prior, w.B, w.seed)
    d, psd = make_data(g, w.seed)
    m = O.OracleModel.from_grid(g)
    bands = np.array([O.band(p, m) for p in P])
    nb = np.maximum(bands[:, 1] - bands[:, 0] + 1, 0)
    order = np.argsort(nb)
    idx = np.unique(np.r_[order[-2:], order[len(order) // 2], np.flatnonzero(nb == 0)[:1]])
    for Np in w.Np_list:
        Fg, Fpg = run_gpu(fst, g, d, psd, P, Np)
        assert np.all(np.isfinite(Fg)) and np.all(Fg >= 0)
        Fo, Fpo = O.fstat_batch(P[idx], m, d, psd, Np)
        assert_parity(Fg[idx], Fpg[idx], Fo, Fpo, Np, TOL64)


def test_set_data_with_a_frequency_grid(fst):
    """fs_plan_set_data's f_grid: the plan's own uniform grid (computed here
    in another order, so a few ulp apart) is accepted and gives the same F;
    a grid with one bin moved by a millionth of a bin is refused with
    FS_EUNSUPPORTED and loads nothing."""
    g = S.tiny_grid(n=5000, f_min=0.02, stride=4)
    d, psd = make_data(g, 7)
    P = in_band_params(g, 16, 3, 0.02 + 2500 * g.df)
    plan = fst.Plan.from_grid(g)
    dt, pt = torch.from_numpy(d).cuda(), torch.from_numpy(psd).cuda()
    plan.set_data(dt, pt)
    F0 = plan.fstat(torch.from_numpy(P).cuda(), 4)[0].clone()
    f = torch.from_numpy(g.f_min + g.df * np.arange(g.n, dtype=np.float64)).cuda()
    plan.set_data(dt, pt, f_grid=f)
    F1 = plan.fstat(torch.from_numpy(P).cuda(), 4)[0]
    assert torch.equal(F0, F1)
    bad = f.clone()
    bad[1234] += 1e-6 * g.df
    with pytest.raises(fst.FstatError) as ei:
        plan.set_data(2.0 * dt, pt, f_grid=bad)
    assert ei.value.status == fst.FS_EUNSUPPORTED
    assert torch.equal(plan.fstat(torch.from_numpy(P).cuda(), 4)[0], F0)   # the earlier data stay loaded
    plan.close()
