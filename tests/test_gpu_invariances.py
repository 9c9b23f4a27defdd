"""Invariances of the F-statistic (what the mathematics fixes, independent of
any implementation) on the CUDA path, in both precision modes:

- (d, S) -> (c d, c^2 S) leaves every F_p unchanged (the noise-weighted inner
  product is invariant; c a power of two changes no rounding);
- data outside a particle's band does not contribute: changing it leaves F
  unchanged (per-particle segments);
- a constant phase on the data, d -> d e^{i phi}, leaves F unchanged (it is
  absorbed by the amplitudes a_i), up to rounding;
- F_sum(N_p = 1) equals F computed with one global segment over the band.
"""
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
    g = S.tiny_grid(n=70000, f_min=0.02)
    fr = 0.02 + 35000 * g.df
    P = S.draw_params(S.Prior(tc_lo=0.1 * g.T_obs, tc_hi=0.9 * g.T_obs), 40, 17)
    P[:, 1] = tc_for(P[:, 0], fr, P[:, 1])
    psd = S.lisa_like_psd(g.freqs())
    m = O.OracleModel.from_grid(g)
    a = O.extrinsic_to_a(1.0, S.INJ_PSI, S.INJ_IOTA, S.INJ_PHIC)
    k0, k1 = O.band(P[0], m)
    h = O.inject(P[0], m, a, k0, k1 + 1)
    d = S.gaussian_noise(g, psd, 18) + h * (20.0 / np.sqrt(O.inner(h, h, psd, g.df)))
    return g, d, psd, P


def run(fst, g, d, psd, P, Np, mode, edges=None):
    plan = fst.Plan.from_grid(g, mode=mode)
    plan.set_data(torch.from_numpy(np.ascontiguousarray(d)).cuda(), torch.from_numpy(np.ascontiguousarray(psd)).cuda())
    Pt = torch.from_numpy(P).cuda()
    F, Fp = plan.fstat(Pt, Np, edges=None if edges is None else g.edge_freqs(edges))
    out = F.cpu().numpy(), Fp.cpu().numpy(), plan.bands(Pt).cpu().numpy()
    plan.close()
    return out


@pytest.mark.parametrize("mode", [0, 1])
def test_scale_invariance(fst, case, mode):
    g, d, psd, P = case
    F, Fp, _ = run(fst, g, d, psd, P, 16, mode)
    F2, Fp2, _ = run(fst, g, d * 8.0, psd * 64.0, P, 16, mode)
    assert np.array_equal(F, F2) and np.array_equal(Fp, Fp2)


@pytest.mark.parametrize("mode", [0, 1])
def test_data_outside_the_band_is_ignored(fst, case, mode):
    g, d, psd, P = case
    F, Fp, bands = run(fst, g, d, psd, P, 8, mode)
    lo, hi = bands[0]
    assert hi > lo
    d2 = d.copy()
    d2[:lo] = 1e3 * (1 + 1j)
    d2[hi + 1:] = -7e2j
    F2, Fp2, _ = run(fst, g, d2, psd, P[:1], 8, mode)
    assert np.array_equal(F2, F[:1]) and np.array_equal(Fp2, Fp[:1])


@pytest.mark.parametrize("mode,tol", [(0, 1e-11), (1, 1e-5)])
def test_constant_phase_is_absorbed(fst, case, mode, tol):
    g, d, psd, P = case
    F, _, _ = run(fst, g, d, psd, P, 4, mode)
    F2, _, _ = run(fst, g, d * np.exp(1j * 1.234), psd, P, 4, mode)
    assert np.max(np.abs(F2 - F) / np.maximum(np.abs(F), 8.0)) <= tol
    assert F[0] > 100.0   # the injection


def test_one_segment_equals_one_global_segment_over_the_band(fst, case):
    g, d, psd, P = case
    F, _, bands = run(fst, g, d, psd, P, 1, 0)
    for b in range(5):
        lo, hi = bands[b]
        if hi <= lo:
            continue
        Fg, _, _ = run(fst, g, d, psd, P[b:b + 1], 1, 0, edges=np.array([lo, hi + 1], dtype=np.int64))
        assert Fg[0] == pytest.approx(F[b], rel=1e-12, abs=1e-12)
