"""Mixed-precision mode (FS_MIXED): FP64 anchors with exact fixed-point phase
steps, FP32 response and products.

Bar: |F_mixed - F_ref| / max(|F_ref|, 2 N_p) <= 1e-4, the reference being
the CPU oracle on small cases and the FP64 mode (itself within 1e-9 of the
oracle) on the full paper-scale workload.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2407_10797_gb300 import synth as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-4


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


def rel_err(F, Fref, Np):
    ok = ~np.isnan(Fref)
    assert np.array_equal(np.isnan(F), np.isnan(Fref))
    return np.max(np.abs(F[ok] - Fref[ok]) / np.maximum(np.abs(Fref[ok]), 2.0 * Np), initial=0.0)


def gpu_F(fst, g, d, psd, P, Np, mode, edges=None, parts=False):
    plan = fst.Plan.from_grid(g, mode=mode)
    plan.set_data(torch.as_tensor(d).cuda(), torch.as_tensor(psd).cuda())
    F, Fp = plan.fstat(torch.as_tensor(np.ascontiguousarray(P)).cuda(), Np,
                       edges=None if edges is None else g.edge_freqs(edges))
    torch.cuda.synchronize()
    out = (F.cpu().numpy(), Fp.cpu().numpy())
    plan.close()
    return out if parts else out[0]


def data_with_injection(g, seed, inj, snr=12.0):
    psd = S.lisa_like_psd(g.freqs())
    d = S.gaussian_noise(g, psd, seed)
    m = O.OracleModel.from_grid(g)
    a = O.extrinsic_to_a(1.0, S.INJ_PSI, S.INJ_IOTA, S.INJ_PHIC)
    k0, k1 = O.band(inj, m)
    h = O.inject(inj, m, a, k0, k1 + 1)
    return d + h * (snr / math.sqrt(O.inner(h, h, psd, g.df))), psd


@pytest.mark.parametrize("Np", [1, 16, 256])
def test_mixed_matches_oracle_small(fst, Np):
    """40000 bins of the 2.5 yr grid (ragged tiles and spans), 45 particles
    with bands that start, end or lie inside the data, injection + noise."""
    g = S.tiny_grid(n=40000, f_min=0.02)
    fr = 0.02 + 20000 * g.df
    P = S.draw_params(S.Prior(tc_lo=-0.2 * g.T_obs, tc_hi=1.2 * g.T_obs), 45, 7)
    P[:, 1] = tc_for(P[:, 0], fr, P[:, 1] * 0.01)
    inj = P[3].copy()
    inj[1] = tc_for(inj[0], fr, 0.5 * g.T_obs)
    d, psd = data_with_injection(g, 2, inj)
    P[3] = inj
    Fm, Fpm = gpu_F(fst, g, d, psd, P, Np, fst.FS_MIXED, parts=True)
    Fo, Fpo = O.fstat_batch(P, O.OracleModel.from_grid(g), d, psd, Np)
    assert np.sum(Fo > 0) >= 10
    assert rel_err(Fm, Fo, Np) <= TOL_MIXED
    assert Fm[3] > 40.0   # the injection is recovered


def test_mixed_global_edges_small(fst):
    g = S.tiny_grid(n=70000, f_min=0.012)
    P = S.draw_params(S.Prior(tc_lo=0.0, tc_hi=g.T_obs), 24, 3)
    P[:, 1] = tc_for(P[:, 0], 0.012 + 35000 * g.df, P[:, 1] * 0.002)
    psd = S.lisa_like_psd(g.freqs())
    d = S.gaussian_noise(g, psd, 4)
    edges = np.array([0, 5000, 5001, 33000, 40000, 69999], dtype=np.int64)
    Np = len(edges) - 1
    Fm = gpu_F(fst, g, d, psd, P, Np, fst.FS_MIXED, edges=edges)
    Fo, _ = O.fstat_batch(P, O.OracleModel.from_grid(g), d, psd, Np, edges=edges)
    assert rel_err(Fm, Fo, Np) <= TOL_MIXED


def test_mixed_falls_back_to_fp64_on_aliased_grid(fst):
    """The 2^15-bin small workload has ~2000 rad of phase per bin, where no
    1024-bin Taylor anchor is valid: every tile takes the bin-by-bin FP64 path."""
    w = S.small_workload()
    g = w.grid
    P = S.draw_params(w.prior, 64, 5)
    psd = S.lisa_like_psd(g.freqs())
    d = S.gaussian_noise(g, psd, 5)
    edges = np.arange(9, dtype=np.int64) * (g.n // 8)
    Fm = gpu_F(fst, g, d, psd, P, 8, fst.FS_MIXED, edges=edges)
    Fo, _ = O.fstat_batch(P, O.OracleModel.from_grid(g), d, psd, 8, edges=edges)
    assert rel_err(Fm, Fo, 8) <= TOL_MIXED


def test_mixed_matches_fp64_paper_workload(fst):
    """Full 3,155,760-bin paper workload, B = 320, every N_p of the schedule."""
    w = S.paper_workload()
    g = w.grid
    P = S.draw_params(w.prior, w.B, w.seed)
    psd = S.lisa_like_psd(g.freqs())
    d = torch.from_numpy(S.gaussian_noise(g, psd, w.seed)).cuda()
    psd_t = torch.from_numpy(psd).cuda()
    Pt = torch.from_numpy(P).cuda()
    errs = {}
    for mode in (fst.FS_FP64, fst.FS_MIXED):
        plan = fst.Plan.from_grid(g, mode=mode)
        plan.set_data(d, psd_t)
        errs[mode] = {Np: plan.fstat(Pt, Np, want_parts=False)[0].cpu().numpy() for Np in w.Np_list}
        plan.close()
    for Np in w.Np_list:
        e = rel_err(errs[fst.FS_MIXED][Np], errs[fst.FS_FP64][Np], Np)
        assert e <= TOL_MIXED, (Np, e)


@pytest.mark.slow
def test_mixed_noise_only_chi_square_1e5_particles(fst):
    """Noise-only paper-scale data: 2F of particles whose every segment has
    >= 64 bins follows chi^2 with 4 N_p degrees of freedom (10^5 particles)."""
    from scipy import stats
    w = S.paper_workload()
    g = w.grid
    psd = S.lisa_like_psd(g.freqs())
    d = torch.from_numpy(S.gaussian_noise(g, psd, 1)).cuda()
    P = S.draw_params(w.prior, 100000, 11)
    plan = fst.Plan.from_grid(g, mode=fst.FS_MIXED)
    plan.set_data(d, torch.from_numpy(psd).cuda())
    Pt = torch.from_numpy(P).cuda()
    bands = plan.bands(Pt).cpu().numpy()
    nb = bands[:, 1] - bands[:, 0] + 1
    for Np in (1, 16):
        keep = nb >= 64 * Np
        F = plan.fstat(Pt, Np, want_parts=False)[0].cpu().numpy()[keep]
        assert keep.sum() > 20000
        ks = stats.kstest(2.0 * F, stats.chi2(4 * Np).cdf)
        assert ks.pvalue > 1e-4, (Np, ks)
    plan.close()


def test_mixed_is_deterministic(fst):
    g = S.tiny_grid(n=50000, f_min=0.03)
    psd = S.lisa_like_psd(g.freqs())
    d = torch.from_numpy(S.gaussian_noise(g, psd, 9)).cuda()
    P = S.draw_params(S.Prior(tc_lo=0.0, tc_hi=g.T_obs), 77, 9)
    P[:, 1] = tc_for(P[:, 0], 0.03 + 25000 * g.df, P[:, 1] * 0.01)
    plan = fst.Plan.from_grid(g, mode=fst.FS_MIXED)
    plan.set_data(d, torch.from_numpy(psd).cuda())
    Pt = torch.from_numpy(P).cuda()
    runs = [plan.fstat(Pt, 64)[0].clone() for _ in range(3)]
    torch.cuda.synchronize()
    assert torch.equal(runs[0], runs[1]) and torch.equal(runs[0], runs[2])
    plan.close()
