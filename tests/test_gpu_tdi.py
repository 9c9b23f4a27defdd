"""The finite-arm TDI response (Sec. IV; fs_plan_set_arm) on the GPU against the
CPU oracle.

The oracle writes each link as the difference of its two retarded phase
factors over 2 (1 - k.n) and combines the vertex Michelsons; the library uses
the equivalent sinc form per arm and its own position code.  Bar 1e-9 on
|dF| / max(|F|, 2 N_p); amplitudes to 1e-9 of |a|.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2407_10797_gb300 import synth as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-9
L_ARM = 2.5e9 / 299792458.0
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
    """7000 bins of the 2.5-yr grid at 30 mHz (pi f L = 0.8), LISA-like noise plus
    an injection made with the finite-arm response at SNR 15, 28 particles."""
    g = S.tiny_grid(n=7000, f_min=0.03)
    psd = S.lisa_like_psd(g.freqs())
    fr = 0.03 + 3500 * g.df
    P = S.draw_params(S.Prior(Mc_lo=20.0, Mc_hi=50.0, tc_lo=-0.3 * g.T_obs, tc_hi=1.3 * g.T_obs), 28, 91)
    P[:, 1] = tc_for(P[:, 0], fr, P[:, 1])
    inj = np.array([36.0, tc_for(36.0, fr, 0.5 * g.T_obs), 0.2, 3.3, 0.03, 1.0])
    P[4] = inj
    m = O.OracleModel.from_grid(g, arm_s=L_ARM)
    a = O.extrinsic_to_a(1.0, S.INJ_PSI, S.INJ_IOTA, S.INJ_PHIC)
    k0, k1 = O.band(inj, m)
    h = O.inject(inj, m, a, k0, k1 + 1)
    d = S.gaussian_noise(g, psd, 33) + h * (15.0 / math.sqrt(O.inner(h, h, psd, g.df)))
    return g, psd, d, P


def gpu_F(fst, g, d, psd, P, Np, arm, ecc=0.0, edges=None, tdi=None, variant=None):
    kw = {} if tdi is None else {"tdi": tdi}
    plan = fst.Plan.from_grid(g, mode=fst.FS_FP64, **kw)
    plan.set_data(torch.as_tensor(d).cuda(), torch.as_tensor(psd).cuda())
    plan.set_arm(arm)
    assert plan.get_arm() == arm
    plan.set_orbit(ecc)
    if variant is not None:
        plan.set_variant(variant)
    F, Fp = plan.fstat(torch.as_tensor(np.ascontiguousarray(P)).cuda(), Np,
                       edges=None if edges is None else g.edge_freqs(edges))
    out = F.cpu().numpy(), Fp.cpu().numpy()
    assert plan.check() == 0
    plan.close()
    return out


@pytest.mark.parametrize("ecc", [0.0, E_LISA])
@pytest.mark.parametrize("Np", [1, 16])
def test_finite_arm_matches_oracle(fst, case, ecc, Np):
    g, psd, d, P = case
    Fg, Fpg = gpu_F(fst, g, d, psd, P, Np, L_ARM, ecc)
    m = O.OracleModel.from_grid(g, arm_s=L_ARM, ecc=ecc)
    Fo, Fpo = O.fstat_batch(P, m, d, psd, Np)
    assert np.any(Fo > 50.0) and np.any(Fo == 0.0)
    assert rel_err(Fg, Fo, Np) <= TOL64
    ok = ~np.isnan(Fpo)
    assert np.max(np.abs(Fpg[ok] - Fpo[ok]) / np.maximum(np.abs(Fpo[ok]), 2.0)) <= TOL64


def test_finite_arm_two_channels_global_edges_and_variants(fst, case):
    g, _, _, P = case
    psd = S.tdi_psds(g.freqs(), S.TDI_AE)
    ms = [O.OracleModel.from_grid(g, channel=c, arm_s=L_ARM) for c in (1, 2)]
    inj = P[4]
    a = O.extrinsic_to_a(1.0, S.INJ_PSI, S.INJ_IOTA, S.INJ_PHIC)
    k0, k1 = O.band(inj, ms[0])
    h = np.stack([O.inject(inj, m, a, k0, k1 + 1) for m in ms])
    hh = sum(O.inner(h[c], h[c], psd[c], g.df) for c in range(2))
    d = np.stack([S.gaussian_noise(g, psd[c], 35, channel=c) for c in range(2)]) + h * (14.0 / math.sqrt(hh))
    edges = np.array([0, 1500, 1500, 4096, 7000], dtype=np.int64)
    Np = len(edges) - 1
    Fg, _ = gpu_F(fst, g, d, psd, P, Np, L_ARM, edges=edges, tdi=fst.FS_TDI_AE)
    Fo, _ = O.fstat_batch_channels(P, ms, d, psd, Np, edges=edges)
    assert rel_err(Fg, Fo, Np) <= TOL64
    for v in (1, 2, 4):
        Fv, _ = gpu_F(fst, g, d, psd, P, Np, L_ARM, edges=edges, tdi=fst.FS_TDI_AE, variant=v)
        assert rel_err(Fv, Fg, Np) <= 1e-12, v


def test_finite_arm_amplitudes_and_injection(fst, case):
    g, psd, d, P = case
    Np = 2
    plan = fst.Plan.from_grid(g, mode=fst.FS_FP64)
    plan.set_data(torch.as_tensor(d).cuda(), torch.as_tensor(psd).cuda())
    plan.set_arm(L_ARM)
    _, amp, _ = plan.amplitudes(torch.as_tensor(np.ascontiguousarray(P)).cuda(), Np)
    amp = amp.cpu().numpy()
    m = O.OracleModel.from_grid(g, arm_s=L_ARM)
    checked = 0
    for b in range(len(P)):
        N, M, nb = O.segment_sums(P[b], m, d, psd, Np)
        for p in range(Np):
            if nb[p] < 4 or M[p, 0, 0] * M[p, 1, 1] - M[p, 0, 1] ** 2 <= 1e-12 * M[p, 0, 0] * M[p, 1, 1]:
                continue
            ao = np.linalg.solve(M[p], N[p])
            assert np.max(np.abs(amp[b, p] - ao)) <= 1e-9 * np.max(np.abs(ao)), (b, p)
            checked += 1
    assert checked >= 20
    inj = P[4]
    a = np.array([0.2, 1.1, -0.6, 0.4])
    k0, k1 = O.band(inj, m)
    ho = O.inject(inj, m, a, k0, k1 + 1)
    hg = torch.zeros(g.n, dtype=torch.complex128).cuda()
    plan.add_signal(inj, a, hg)
    hg = hg.cpu().numpy()
    plan.close()
    assert np.max(np.abs(hg - ho)) <= 1e-9 * np.max(np.abs(ho))


def test_finite_arm_changes_F_and_its_limits(fst, case):
    g, psd, d, P = case
    F0, _ = gpu_F(fst, g, d, psd, P, 1, 0.0)
    F1, _ = gpu_F(fst, g, d, psd, P, 1, L_ARM)
    # over this 89 uHz slice the arm transfer is nearly a common complex factor, which the
    # amplitudes absorb: F at the injection moves by 1e-5 (it is made with finite arms)
    assert abs(F1[4] - F0[4]) > 3e-6 * abs(F1[4])
    plan = fst.Plan.from_grid(g, mode=fst.FS_FP64)
    plan.set_arm(L_ARM)
    with pytest.raises(fst.FstatError) as ei:
        plan.set_response(2, 1)
    assert ei.value.status == fst.FS_EUNSUPPORTED
    plan.set_arm(0.0)
    plan.set_response(2, 1)
    with pytest.raises(fst.FstatError) as ei:
        plan.set_arm(L_ARM)
    assert ei.value.status == fst.FS_EUNSUPPORTED
    plan.close()
    plan = fst.Plan.from_grid(g, mode=fst.FS_MIXED)
    with pytest.raises(fst.FstatError) as ei:
        plan.set_arm(L_ARM)
    assert ei.value.status == fst.FS_EUNSUPPORTED
    plan.close()
