"""Several TDI channels (Sec. II.A, Eq. eq2): the A and E channels of the
long-wavelength response, summed in every segment's N and M, on the GPU
against the oracle (which builds A and E from the three vertex Michelsons
by vector geometry; the library turns the X Michelson in the constellation
plane and scales it).

Bars: 1e-9 (FP64 mode) and 1e-4 (mixed mode) on |dF| / max(|F|, 2 N_p).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2407_10797_gb300 import synth as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def models(g):
    return [O.OracleModel.from_grid(g, channel=1), O.OracleModel.from_grid(g, channel=2)]


@pytest.fixture(scope="module")
def case():
    """40000 bins of the 2.5-yr grid, A and E noise, an injection at SNR 12
    summed over both channels, 45 particles with bands in and around the data."""
    g = S.tiny_grid(n=40000, f_min=0.02)
    fr = 0.02 + 20000 * g.df
    P = S.draw_params(S.Prior(tc_lo=-0.2 * g.T_obs, tc_hi=1.2 * g.T_obs), 45, 17)
    P[:, 1] = tc_for(P[:, 0], fr, P[:, 1] * 0.01)
    inj = P[3].copy()
    inj[1] = tc_for(inj[0], fr, 0.5 * g.T_obs)
    P[3] = inj
    psd = S.tdi_psds(g.freqs(), S.TDI_AE)
    ms = models(g)
    a = O.extrinsic_to_a(1.0, S.INJ_PSI, S.INJ_IOTA, S.INJ_PHIC)
    k0, k1 = O.band(inj, ms[0])
    h = np.stack([O.inject(inj, m, a, k0, k1 + 1) for m in ms])
    hh = sum(O.inner(h[c], h[c], psd[c], g.df) for c in range(2))
    d = np.stack([S.gaussian_noise(g, psd[c], 6, channel=c) for c in range(2)]) + h * (12.0 / math.sqrt(hh))
    return g, d, psd, P, ms


def gpu_F(fst, g, d, psd, P, Np, mode, edges=None, variant=None):
    plan = fst.Plan.from_grid(g, mode=mode, tdi=fst.FS_TDI_AE)
    assert plan.nch == 2
    plan.set_data(torch.as_tensor(d).cuda(), torch.as_tensor(psd).cuda())
    if variant is not None:
        plan.set_variant(variant)
    F, Fp = plan.fstat(torch.as_tensor(np.ascontiguousarray(P)).cuda(), Np,
                       edges=None if edges is None else g.edge_freqs(edges))
    out = F.cpu().numpy(), Fp.cpu().numpy()
    assert plan.check() == 0
    plan.close()
    return out


@pytest.mark.parametrize("Np", [1, 7, 64])
def test_two_channel_fp64_matches_oracle(fst, case, Np):
    g, d, psd, P, ms = case
    Fo, Fpo = O.fstat_batch_channels(P, ms, d, psd, Np)
    assert np.sum(Fo > 0) >= 10 and Fo[3] > 40.0
    for v in (0, 4):
        Fg, Fpg = gpu_F(fst, g, d, psd, P, Np, fst.FS_FP64, variant=v)
        assert rel_err(Fg, Fo, Np) <= 1e-9, v
        ok = ~np.isnan(Fpo)
        assert np.max(np.abs(Fpg[ok] - Fpo[ok]) / np.maximum(np.abs(Fpo[ok]), 2.0)) <= 1e-9, v


def test_two_channel_global_edges(fst, case):
    g, d, psd, P, ms = case
    edges = np.array([0, 5000, 5001, 23000, 39999], dtype=np.int64)
    Np = len(edges) - 1
    Fo, _ = O.fstat_batch_channels(P, ms, d, psd, Np, edges=edges)
    Fg, _ = gpu_F(fst, g, d, psd, P, Np, fst.FS_FP64, edges=edges)
    assert rel_err(Fg, Fo, Np) <= 1e-9
    Fm, _ = gpu_F(fst, g, d, psd, P, Np, fst.FS_MIXED, edges=edges)
    assert rel_err(Fm, Fo, Np) <= 1e-4


@pytest.mark.parametrize("Np", [1, 16])
def test_two_channel_mixed_matches_oracle_and_variants_agree(fst, case, Np):
    g, d, psd, P, ms = case
    Fo, _ = O.fstat_batch_channels(P, ms, d, psd, Np)
    outs = [gpu_F(fst, g, d, psd, P, Np, fst.FS_MIXED, variant=v)[0] for v in range(5)]
    for F in outs[1:]:
        assert np.array_equal(F, outs[0])
    assert rel_err(outs[0], Fo, Np) <= 1e-4


def test_two_channel_noise_free_F_is_half_snr_squared_and_add_signal(fst):
    """Noise-free injection built by fs_add_signal in both channels: the data
    match the oracle's per-channel signal, and F at the truth is SNR^2 / 2
    for any segmentation."""
    g = S.tiny_grid(n=4096, f_min=0.02, stride=4)
    p = np.array([28.0, tc_for(28.0, 0.02 + 2048 * g.df, 0.5 * g.T_obs), 0.4, 2.0, 0.04, 1.0])
    psd = S.tdi_psds(g.freqs(), S.TDI_AE)
    ms = models(g)
    a = O.extrinsic_to_a(1.0, S.INJ_PSI, S.INJ_IOTA, S.INJ_PHIC)
    k0, k1 = O.band(p, ms[0])
    h = np.stack([O.inject(p, m, a, k0, k1 + 1) for m in ms])
    hh = sum(O.inner(h[c], h[c], psd[c], g.df) for c in range(2))
    scale = 10.0 / math.sqrt(hh)
    plan = fst.Plan.from_grid(g, mode=fst.FS_FP64, tdi=fst.FS_TDI_AE)
    dgpu = torch.zeros(2, g.n, dtype=torch.complex128, device="cuda")
    plan.set_data(dgpu, torch.from_numpy(psd).cuda())
    plan.add_signal(p, a * scale, dgpu)
    torch.cuda.synchronize()
    hg = dgpu.cpu().numpy()
    assert np.max(np.abs(hg - h * scale)) <= 1e-9 * np.max(np.abs(h * scale))
    plan.set_data(dgpu, torch.from_numpy(psd).cuda())
    for Np in (1, 5):
        F, _ = plan.fstat(torch.from_numpy(p[None]).cuda(), Np)
        assert float(F[0]) == pytest.approx(50.0, rel=1e-9)
    plan.close()
