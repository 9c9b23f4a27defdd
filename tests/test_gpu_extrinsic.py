"""Maximum-likelihood amplitudes (Eq. aandMN3) and extrinsic parameters
(App. B, Eqs. B2-B3) on the GPU, against the CPU oracle.

The oracle side solves the full 4x4 system M a = N of each segment
(np.linalg.solve on the oracle's long-double sums) and maps a to
(D_L, iota, psi, phi_c) with its own App. B routine.  Bars: a to 1e-9 of
|a| in FP64 mode (the sums behind it match to that level), the extrinsic
parameters to 1e-8, and in noise-free data the injected amplitudes come back.
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


@pytest.fixture(scope="module")
def case():
    g = S.tiny_grid(n=60000, f_min=0.02)
    psd = S.lisa_like_psd(g.freqs())
    m = O.OracleModel.from_grid(g)
    inj = np.array([25.0, tc_for(25.0, 0.02 + 30000 * g.df, 0.45 * g.T_obs), -0.7, 4.0, 0.03, 1.0])
    a_inj = O.extrinsic_to_a(1.0, S.INJ_PSI, S.INJ_IOTA, S.INJ_PHIC)
    k0, k1 = O.band(inj, m)
    h = O.inject(inj, m, a_inj, k0, k1 + 1)
    s = 20.0 / math.sqrt(O.inner(h, h, psd, g.df))
    return g, psd, m, inj, h * s, a_inj * s


def gpu_amplitudes(fst, g, d, psd, P, Np, mode=0):
    plan = fst.Plan.from_grid(g, mode=mode)
    plan.set_data(torch.from_numpy(d).cuda(), torch.from_numpy(psd).cuda())
    F, a, ext = plan.amplitudes(torch.from_numpy(np.ascontiguousarray(P)).cuda(), Np)
    torch.cuda.synchronize()
    out = F.cpu().numpy(), a.cpu().numpy(), ext.cpu().numpy()
    plan.close()
    return out


def angle_diff(x, y, period):
    d = (x - y) % period
    return min(d, period - d)


def test_noise_free_injection_amplitudes_and_extrinsics(fst, case):
    g, psd, m, inj, h, a_inj = case
    F, a, ext = gpu_amplitudes(fst, g, h, psd, inj[None], 1)
    assert np.allclose(a[0, 0], a_inj, rtol=0, atol=1e-9 * np.linalg.norm(a_inj))
    DL, iota, psi, phic = O.a_to_extrinsic(a_inj)
    assert ext[0, 0, 0] == pytest.approx(DL, rel=1e-8)
    assert ext[0, 0, 1] == pytest.approx(iota, abs=1e-8)
    assert ext[0, 0, 1] == pytest.approx(S.INJ_IOTA, abs=1e-8)
    # (psi, phi_c) are defined modulo the symmetry (psi + pi/2, phi_c + pi)
    assert angle_diff(2 * ext[0, 0, 2], 2 * psi, 2 * np.pi) < 1e-8
    assert angle_diff(ext[0, 0, 3], phic, np.pi) < 1e-8
    # and they map back to the injected amplitudes through Eq. B1
    back = O.extrinsic_to_a(ext[0, 0, 0], ext[0, 0, 2], ext[0, 0, 1], ext[0, 0, 3])
    assert np.allclose(back, a_inj, rtol=0, atol=1e-8 * np.linalg.norm(a_inj))
    assert F[0] == pytest.approx(200.0, rel=1e-9)   # F = SNR^2 / 2


@pytest.mark.parametrize("Np", [1, 4])
def test_amplitudes_match_oracle_solve_in_noise(fst, case, Np):
    g, psd, m, inj, h, a_inj = case
    d = S.gaussian_noise(g, psd, 31) + h
    P = S.draw_params(S.Prior(tc_lo=0.2 * g.T_obs, tc_hi=0.8 * g.T_obs), 12, 32)
    P[:, 1] = tc_for(P[:, 0], 0.02 + 30000 * g.df, P[:, 1])
    P[0] = inj
    F, a, ext = gpu_amplitudes(fst, g, d, psd, P, Np)
    checked = 0
    for b in range(len(P)):
        N, M, nb = O.segment_sums(P[b], m, d, psd, Np)
        for s in range(Np):
            if nb[s] < 64:
                continue
            a_ref = np.linalg.solve(M[s], N[s])
            scale = np.linalg.norm(a_ref)
            assert np.max(np.abs(a[b, s] - a_ref)) <= 1e-9 * scale, (b, s)
            ref = O.a_to_extrinsic(a[b, s])
            assert ext[b, s, 0] == pytest.approx(ref[0], rel=1e-9)
            assert ext[b, s, 1] == pytest.approx(ref[1], abs=1e-9)
            assert angle_diff(2 * ext[b, s, 2], 2 * ref[2], 2 * np.pi) < 1e-9
            assert angle_diff(ext[b, s, 3], ref[3], np.pi) < 1e-9
            checked += 1
    assert checked >= 3 * Np


def test_degenerate_and_invalid_particles(fst, case):
    g, psd, m, inj, h, a_inj = case
    P = np.stack([inj, inj, inj])
    P[1, 1] = -10.0 * g.T_obs          # no in-band bin: every segment degenerate
    P[2, 0] = float("nan")             # invalid parameters
    F, a, ext = gpu_amplitudes(fst, g, h, psd, P, 2)
    assert np.all(a[1] == 0.0) and np.all(np.isnan(ext[1])) and F[1] == 0.0
    assert np.all(np.isnan(a[2])) and np.all(np.isnan(ext[2])) and np.isnan(F[2])
    assert np.all(np.isfinite(a[0])) and np.all(np.isfinite(ext[0]))


def test_mixed_mode_amplitudes_close_to_fp64(fst, case):
    g, psd, m, inj, h, a_inj = case
    d = S.gaussian_noise(g, psd, 33) + h
    _, a64, _ = gpu_amplitudes(fst, g, d, psd, inj[None], 1, mode=0)
    _, am, _ = gpu_amplitudes(fst, g, d, psd, inj[None], 1, mode=1)
    assert np.max(np.abs(am - a64)) <= 1e-4 * np.linalg.norm(a64)
