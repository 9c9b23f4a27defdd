"""Pins of the semi-coherent statistic (Sec. II, Eq. 9-12) carried through the
CUDA path:

- in Gaussian noise 2 F_sum follows a chi-square law with 4 N_p degrees of
  freedom (four amplitudes maximised per segment), in FP64 mode on 10^5
  particles of the 2.5-yr grid;
- on noise-free data a brute-force (M_c, t_c) scan peaks at the injected
  parameters, and the oracle, the FP64 mode and the mixed mode pick the same
  grid cell (Fig. 1's peak, its width growing with N_p).
"""
import math

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


def tc_for(Mc, f, t):
    """Coalescence time of a Newtonian chirp at frequency f at time t."""
    m = Mc * S.MSUN_S
    return t + 5.0 / 256.0 * m * (np.pi * m * f) ** (-8.0 / 3.0)


@pytest.mark.slow
def test_fp64_noise_only_chi_square_1e5_particles(fst):
    """2F of particles whose every segment holds >= 64 bins is chi^2_{4 N_p}
    (Kolmogorov-Smirnov against the chi-square CDF; mean 4 N_p)."""
    from scipy import stats
    w = S.paper_workload()
    g = w.grid
    psd = S.lisa_like_psd(g.freqs())
    plan = fst.Plan.from_grid(g, mode=fst.FS_FP64)
    plan.set_data(torch.from_numpy(S.gaussian_noise(g, psd, 2)).cuda(), torch.from_numpy(psd).cuda())
    Pt = torch.from_numpy(S.draw_params(w.prior, 100000, 12)).cuda()
    bands = plan.bands(Pt).cpu().numpy()
    nb = bands[:, 1] - bands[:, 0] + 1
    for Np in (1, 16):
        keep = nb >= 64 * Np
        assert keep.sum() > 20000
        F = plan.fstat(Pt, Np, want_parts=False)[0].cpu().numpy()[keep]
        ks = stats.kstest(2.0 * F, stats.chi2(4 * Np).cdf)
        assert ks.pvalue > 1e-4, (Np, ks)
        # the sample mean of 2F within 5 standard errors of 4 N_p
        assert abs(np.mean(2.0 * F) - 4 * Np) < 5.0 * math.sqrt(8.0 * Np / keep.sum())
    plan.close()


def test_brute_force_grid_argmax_identical_in_oracle_and_both_modes(fst):
    """Noise-free data with one injection (SNR 20): a 21 x 21 (M_c, t_c) grid
    centred on the truth, its spans scaled with the peak width (x1 for
    N_p = 1, x16 for N_p = 16), peaks at the centre cell in the oracle and
    the FP64 mode; the FP64 values agree with the oracle to 1e-9 and the
    mixed ones to 1e-4 (|dF| / max(|F|, 2 N_p)). The mixed mode picks the
    same cell where the oracle's top two cells differ by more than its
    tolerance (N_p = 1); along the M_c-t_c ridge of N_p = 16 the top cells
    differ by ~1e-6 and any cell within the tolerance of the maximum is a
    correct answer."""
    g = S.tiny_grid(n=2048, f_min=0.02, stride=64)
    psd = S.lisa_like_psd(g.freqs())
    m = O.OracleModel.from_grid(g)
    Mc0 = 30.0
    p = np.array([Mc0, tc_for(Mc0, 0.02, 0.9 * g.T_obs), 0.4, 2.1, 0.01, 1.0])
    a = O.extrinsic_to_a(1.0, S.INJ_PSI, S.INJ_IOTA, S.INJ_PHIC)
    k0, k1 = O.band(p, m)
    h = O.inject(p, m, a, k0, k1 + 1)
    d = h * (20.0 / math.sqrt(O.inner(h, h, psd, g.df)))
    n = 21
    centre = (n // 2) * n + n // 2
    plans = {}
    for mode in (fst.FS_FP64, fst.FS_MIXED):
        plans[mode] = fst.Plan.from_grid(g, mode=mode)
        plans[mode].set_data(torch.from_numpy(d).cuda(), torch.from_numpy(psd).cuda())
    for Np, span in ((1, 1.0), (16, 16.0)):
        P = np.repeat(p[None], n * n, axis=0)
        P[:, 0] = np.repeat(Mc0 * (1.0 + span * np.linspace(-4e-5, 4e-5, n)), n)
        P[:, 1] = np.tile(p[1] + span * np.linspace(-200.0, 200.0, n), n)
        Fo, _ = O.fstat_batch(P, m, d, psd, Np)
        assert int(np.argmax(Fo)) == centre
        top2 = np.sort(Fo)[-2:]
        gap = (top2[1] - top2[0]) / max(top2[1], 2.0 * Np)
        Pt = torch.from_numpy(np.ascontiguousarray(P)).cuda()
        for mode, tol in ((fst.FS_FP64, 1e-9), (fst.FS_MIXED, 1e-4)):
            F = plans[mode].fstat(Pt, Np, want_parts=False)[0].cpu().numpy()
            err = np.max(np.abs(F - Fo) / np.maximum(np.abs(Fo), 2.0 * Np))
            assert err <= tol, (Np, mode, err)
            k = int(np.argmax(F))
            if gap > 2.0 * tol:
                assert k == centre, (Np, mode, gap)
            else:
                assert (Fo[centre] - Fo[k]) / max(Fo[centre], 2.0 * Np) <= 2.0 * tol, (Np, mode)
    for pl in plans.values():
        pl.close()
