"""Spacecraft orbits to second order in eccentricity (Sec. IV; fs_plan_set_orbit)
on the GPU against the CPU oracle.

The oracle forms the arms from its written-out orbit series and the
detectors by vector geometry (the three vertex Michelsons for A and E); the
library evaluates the same orbits with its own angle-addition form, the
normalised arms' projections and, with the response series, their analytic
derivatives.  Bar 1e-9 on |dF| / max(|F|, 2 N_p), as for the rigid form.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2407_10797_gb300 import synth as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-9
E_LISA = 2.5e9 / (2.0 * math.sqrt(3.0) * 1.495978707e11)


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


@pytest.fixture(scope="module")
def case():
    """8000 bins of the 2.5-yr grid at 20 mHz, LISA-like noise plus an injection
    made with the eccentric orbits at SNR 15, 30 particles in and around the data."""
    g = S.tiny_grid(n=8000, f_min=0.02)
    psd = S.lisa_like_psd(g.freqs())
    fr = 0.02 + 4000 * g.df
    P = S.draw_params(S.Prior(tc_lo=-0.3 * g.T_obs, tc_hi=1.3 * g.T_obs), 30, 77)
    P[:, 1] = tc_for(P[:, 0], fr, P[:, 1])
    inj = np.array([27.0, tc_for(27.0, fr, 0.4 * g.T_obs), -0.5, 0.9, 0.06, 1.0])
    P[7] = inj
    m = O.OracleModel.from_grid(g, ecc=E_LISA)
    a = O.extrinsic_to_a(1.0, S.INJ_PSI, S.INJ_IOTA, S.INJ_PHIC)
    k0, k1 = O.band(inj, m)
    h = O.inject(inj, m, a, k0, k1 + 1)
    d = S.gaussian_noise(g, psd, 21) + h * (15.0 / math.sqrt(O.inner(h, h, psd, g.df)))
    return g, psd, d, P


def gpu_F(fst, g, d, psd, P, Np, ecc, N=-1, K=0, edges=None, tdi=None, variant=None):
    kw = {} if tdi is None else {"tdi": tdi}
    plan = fst.Plan.from_grid(g, mode=fst.FS_FP64, **kw)
    plan.set_data(torch.as_tensor(d).cuda(), torch.as_tensor(psd).cuda())
    plan.set_orbit(ecc)
    assert plan.get_orbit() == ecc
    plan.set_response(N, K)
    if variant is not None:
        plan.set_variant(variant)
    F, Fp = plan.fstat(torch.as_tensor(np.ascontiguousarray(P)).cuda(), Np,
                       edges=None if edges is None else g.edge_freqs(edges))
    out = F.cpu().numpy(), Fp.cpu().numpy()
    assert plan.check() == 0
    plan.close()
    return out


@pytest.mark.parametrize("N,K", [(-1, 0), (2, 1)])
@pytest.mark.parametrize("Np", [1, 16])
def test_orbit_matches_oracle(fst, case, N, K, Np):
    g, psd, d, P = case
    Fg, Fpg = gpu_F(fst, g, d, psd, P, Np, E_LISA, N, K)
    m = O.OracleModel.from_grid(g, ecc=E_LISA, mb_order=N, mb_kmax=K)
    Fo, Fpo = O.fstat_batch(P, m, d, psd, Np)
    assert np.any(Fo > 50.0) and np.any(Fo == 0.0)
    assert rel_err(Fg, Fo, Np) <= TOL64
    ok = ~np.isnan(Fpo)
    assert np.max(np.abs(Fpg[ok] - Fpo[ok]) / np.maximum(np.abs(Fpo[ok]), 2.0)) <= TOL64


def test_orbit_two_channels_global_edges(fst, case):
    g, _, _, P = case
    psd = S.tdi_psds(g.freqs(), S.TDI_AE)
    for N, K in ((-1, 0), (1, 1)):
        ms = [O.OracleModel.from_grid(g, channel=c, ecc=E_LISA, mb_order=N, mb_kmax=K) for c in (1, 2)]
        inj = P[7]
        a = O.extrinsic_to_a(1.0, S.INJ_PSI, S.INJ_IOTA, S.INJ_PHIC)
        k0, k1 = O.band(inj, ms[0])
        h = np.stack([O.inject(inj, m, a, k0, k1 + 1) for m in ms])
        hh = sum(O.inner(h[c], h[c], psd[c], g.df) for c in range(2))
        d = np.stack([S.gaussian_noise(g, psd[c], 9, channel=c) for c in range(2)]) + h * (14.0 / math.sqrt(hh))
        edges = np.array([0, 1000, 1000, 2048, 5000, 8000], dtype=np.int64)
        Np = len(edges) - 1
        Fg, _ = gpu_F(fst, g, d, psd, P, Np, E_LISA, N, K, edges=edges, tdi=fst.FS_TDI_AE)
        Fo, _ = O.fstat_batch_channels(P, ms, d, psd, Np, edges=edges)
        assert rel_err(Fg, Fo, Np) <= TOL64, (N, K)


def test_orbit_variants_agree_and_injection(fst, case):
    g, psd, d, P = case
    ref, _ = gpu_F(fst, g, d, psd, P, 4, E_LISA, variant=0)
    for v in (1, 2, 4):
        F, _ = gpu_F(fst, g, d, psd, P, 4, E_LISA, variant=v)
        assert rel_err(F, ref, 4) <= 1e-12, v
    inj = P[7]
    m = O.OracleModel.from_grid(g, ecc=E_LISA)
    a = np.array([0.4, -0.9, 1.1, 0.2])
    k0, k1 = O.band(inj, m)
    ho = O.inject(inj, m, a, k0, k1 + 1)
    plan = fst.Plan.from_grid(g, mode=fst.FS_FP64)
    plan.set_data(torch.zeros(g.n, dtype=torch.complex128).cuda(), torch.as_tensor(psd).cuda())
    plan.set_orbit(E_LISA)
    hg = torch.zeros(g.n, dtype=torch.complex128).cuda()
    plan.add_signal(inj, a, hg)
    hg = hg.cpu().numpy()
    plan.close()
    assert np.max(np.abs(hg - ho)) <= 1e-9 * np.max(np.abs(ho))


def test_orbit_changes_F_and_needs_fp64(fst, case):
    g, psd, d, P = case
    F0, _ = gpu_F(fst, g, d, psd, P, 1, 0.0)
    Fe, _ = gpu_F(fst, g, d, psd, P, 1, E_LISA)
    assert abs(Fe[7] - F0[7]) > 3e-7 * abs(F0[7])   # the injection was made with the eccentric orbits
    plan = fst.Plan.from_grid(g, mode=fst.FS_MIXED)
    with pytest.raises(fst.FstatError) as ei:
        plan.set_orbit(E_LISA)
    assert ei.value.status == fst.FS_EUNSUPPORTED
    plan.set_orbit(0.0)
    plan.close()
