"""The response series of Sec. IV, Eq. (freDres), on the GPU (fs_plan_set_response)
against the CPU oracle.

The oracle evaluates the series from its definition: the kernel G at the
stencil points t_f + j T_f from the vector-geometry antenna pattern at the
retarded time, G' by central differences, the filter weights by solving
their moment conditions, the 4x4 system of each segment by Cholesky.  The
library evaluates it with analytic derivatives of its harmonic antenna
expansion, closed-form weights and the Hermitian 2x2 solve.  Bars as for the
paper's form: 1e-9 on |dF| / max(|F|, 2 N_p) (per segment max(|F_p|, 2)),
amplitudes to 1e-9 of |a|.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2407_10797_gb300 import synth as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-9
ORDERS = [(0, 0), (0, 1), (1, 1), (2, 0), (2, 1)]


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
    """6000 bins of the 2.5-yr grid at 20 mHz (three 2048-bin tiles, the last
    ragged), LISA-like noise plus an injection made with the order-2, k <= 1
    series at SNR 15, 26 particles with bands in, across and outside the data."""
    g = S.tiny_grid(n=6000, f_min=0.02)
    psd = S.lisa_like_psd(g.freqs())
    fr = 0.02 + 3000 * g.df
    P = S.draw_params(S.Prior(tc_lo=-0.3 * g.T_obs, tc_hi=1.3 * g.T_obs), 26, 41)
    P[:, 1] = tc_for(P[:, 0], fr, P[:, 1])
    inj = np.array([31.0, tc_for(31.0, fr, 0.55 * g.T_obs), 0.6, 2.2, 0.04, 1.0])
    P[5] = inj
    m = O.OracleModel.from_grid(g, mb_order=2, mb_kmax=1)
    a = O.extrinsic_to_a(1.0, S.INJ_PSI, S.INJ_IOTA, S.INJ_PHIC)
    k0, k1 = O.band(inj, m)
    h = O.inject(inj, m, a, k0, k1 + 1)
    d = S.gaussian_noise(g, psd, 12) + h * (15.0 / math.sqrt(O.inner(h, h, psd, g.df)))
    return g, psd, d, P


def gpu_F(fst, g, d, psd, P, Np, N, K, edges=None, tdi=None, variant=None):
    kw = {} if tdi is None else {"tdi": tdi}
    plan = fst.Plan.from_grid(g, mode=fst.FS_FP64, **kw)
    plan.set_data(torch.as_tensor(d).cuda(), torch.as_tensor(psd).cuda())
    plan.set_response(N, K)
    assert plan.get_response() == (N, K)
    if variant is not None:
        plan.set_variant(variant)
    F, Fp = plan.fstat(torch.as_tensor(np.ascontiguousarray(P)).cuda(), Np,
                       edges=None if edges is None else g.edge_freqs(edges))
    out = F.cpu().numpy(), Fp.cpu().numpy()
    assert plan.check() == 0
    plan.close()
    return out


@pytest.mark.parametrize("N,K", ORDERS)
@pytest.mark.parametrize("Np", [1, 16])
def test_series_matches_oracle_per_particle_segments(fst, case, N, K, Np):
    g, psd, d, P = case
    Fg, Fpg = gpu_F(fst, g, d, psd, P, Np, N, K)
    m = O.OracleModel.from_grid(g, mb_order=N, mb_kmax=K)
    Fo, Fpo = O.fstat_batch(P, m, d, psd, Np)
    assert np.any(Fo > 50.0) and np.any(Fo == 0.0)
    assert rel_err(Fg, Fo, Np) <= TOL64
    ok = ~np.isnan(Fpo)
    assert np.max(np.abs(Fpg[ok] - Fpo[ok]) / np.maximum(np.abs(Fpo[ok]), 2.0)) <= TOL64


def test_series_launch_variants_agree(fst, case):
    # the direct tiles of 1024 and 4096 bins, and the anchored variant numbers (which the
    # series runs with the default tile)
    g, psd, d, P = case
    ref, _ = gpu_F(fst, g, d, psd, P, 8, 2, 1, variant=0)
    for v in (1, 2, 3, 4):
        F, _ = gpu_F(fst, g, d, psd, P, 8, 2, 1, variant=v)
        assert rel_err(F, ref, 8) <= 1e-12, v


def test_series_global_edges_two_channels(fst, case):
    g, _, _, P = case
    psd = S.tdi_psds(g.freqs(), S.TDI_AE)
    ms = [O.OracleModel.from_grid(g, channel=c, mb_order=2, mb_kmax=1) for c in (1, 2)]
    inj = P[5]
    a = O.extrinsic_to_a(1.0, S.INJ_PSI, S.INJ_IOTA, S.INJ_PHIC)
    k0, k1 = O.band(inj, ms[0])
    h = np.stack([O.inject(inj, m, a, k0, k1 + 1) for m in ms])
    hh = sum(O.inner(h[c], h[c], psd[c], g.df) for c in range(2))
    d = np.stack([S.gaussian_noise(g, psd[c], 7, channel=c) for c in range(2)]) + h * (13.0 / math.sqrt(hh))
    edges = np.array([0, 700, 701, 2048, 3000, 4097, 6000], dtype=np.int64)   # an empty segment, a tile edge
    Np = len(edges) - 1
    Fg, _ = gpu_F(fst, g, d, psd, P, Np, 2, 1, edges=edges, tdi=fst.FS_TDI_AE)
    Fo, _ = O.fstat_batch_channels(P, ms, d, psd, Np, edges=edges)
    assert rel_err(Fg, Fo, Np) <= TOL64


def test_series_noise_free_injection_recovers_amplitudes(fst, case):
    """Noise-free data made by the oracle's series: at the injected parameters
    F = SNR^2 / 2 in every segment tiling (Eq. coherent_F_stat) and the
    amplitudes M^-1 N of each segment are the injected ones (Eq. aandMN3)."""
    g, psd, _, P = case
    inj = P[5:6].copy()
    m = O.OracleModel.from_grid(g, mb_order=2, mb_kmax=1)
    a = O.extrinsic_to_a(1.0, S.INJ_PSI, S.INJ_IOTA, S.INJ_PHIC)
    k0, k1 = O.band(inj[0], m)
    h = O.inject(inj[0], m, a, k0, k1 + 1)
    s = 20.0 / math.sqrt(O.inner(h, h, psd, g.df))
    d = h * s
    plan = fst.Plan.from_grid(g, mode=fst.FS_FP64)
    plan.set_data(torch.as_tensor(d).cuda(), torch.as_tensor(psd).cuda())
    plan.set_response(2, 1)
    for Np in (1, 4):
        F, amp, _ = plan.amplitudes(torch.as_tensor(inj).cuda(), Np)
        F, amp = F.cpu().numpy(), amp.cpu().numpy()
        assert abs(F[0] - 200.0) <= 1e-9 * 200.0
        assert np.max(np.abs(amp[0] - a * s)) <= 1e-8 * np.max(np.abs(a * s))
    plan.close()


def test_series_amplitudes_match_oracle_solve(fst, case):
    g, psd, d, P = case
    Np = 3
    plan = fst.Plan.from_grid(g, mode=fst.FS_FP64)
    plan.set_data(torch.as_tensor(d).cuda(), torch.as_tensor(psd).cuda())
    plan.set_response(2, 1)
    F, amp, _ = plan.amplitudes(torch.as_tensor(np.ascontiguousarray(P)).cuda(), Np)
    amp = amp.cpu().numpy()
    plan.close()
    m = O.OracleModel.from_grid(g, mb_order=2, mb_kmax=1)
    checked = 0
    for b in range(len(P)):
        N, M, nb = O.segment_sums(P[b], m, d, psd, Np)
        for p in range(Np):
            if nb[p] < 4 or M[p, 0, 0] * M[p, 1, 1] - M[p, 0, 1] ** 2 <= 1e-12 * M[p, 0, 0] * M[p, 1, 1]:
                continue
            ao = np.linalg.solve(M[p], N[p])
            assert np.max(np.abs(amp[b, p] - ao)) <= 1e-9 * max(np.max(np.abs(ao)), 1e-300), (b, p)
            checked += 1
    assert checked >= 20


def test_series_signal_synthesis_matches_oracle(fst, case):
    g, psd, _, P = case
    inj = P[5]
    m = O.OracleModel.from_grid(g, mb_order=1, mb_kmax=1)
    a = np.array([0.3, -1.2, 0.7, 0.25])
    k0, k1 = O.band(inj, m)
    ho = O.inject(inj, m, a, k0, k1 + 1)
    plan = fst.Plan.from_grid(g, mode=fst.FS_FP64)
    plan.set_data(torch.zeros(g.n, dtype=torch.complex128).cuda(), torch.as_tensor(psd).cuda())
    plan.set_response(1, 1)
    data = torch.zeros(g.n, dtype=torch.complex128).cuda()
    plan.add_signal(inj, a, data)
    hg = data.cpu().numpy()
    plan.close()
    assert np.max(np.abs(hg - ho)) <= 1e-9 * np.max(np.abs(ho))
    assert np.all(hg[:k0] == 0) and np.all(hg[k1 + 1:] == 0)


def test_series_differs_from_the_paper_form_and_needs_fp64(fst, case):
    g, psd, d, P = case
    Fpaper, _ = gpu_F(fst, g, d, psd, P, 1, -1, 0)
    Fser, _ = gpu_F(fst, g, d, psd, P, 1, 2, 1)
    # at the injection (made with the series) the two templates give F 2e-5 apart on this slice
    assert abs(Fser[5] - Fpaper[5]) > 2e-6 * abs(Fpaper[5])
    plan = fst.Plan.from_grid(g, mode=fst.FS_MIXED)
    with pytest.raises(fst.FstatError) as ei:
        plan.set_response(2, 1)
    assert ei.value.status == fst.FS_EUNSUPPORTED
    plan.set_response(-1, 0)   # the paper's form is always accepted
    plan.close()
