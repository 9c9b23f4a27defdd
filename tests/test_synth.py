"""The seeded input generators (paper_2407_10797_gb300/synth.py) give the
inputs the design states: noise with Re, Im of n_k i.i.d. N(0, S_k T/4)
(independent per channel and seed, reproducible bit for bit), particles
from the stated prior (sin(lat) and the longitude uniform, e0 and M_c in
range, q = 1), the paper grid of 2.5 yr at 1/T over [10, 50) mHz, and a
positive, smooth PSD."""
import numpy as np
import pytest

from paper_2407_10797_gb300 import synth as S

scipy_stats = pytest.importorskip("scipy.stats")


def test_noise_is_complex_gaussian_with_variance_S_T_over_4():
    g = S.tiny_grid(n=1 << 16, f_min=0.01)
    psd = S.lisa_like_psd(g.freqs())
    n = S.gaussian_noise(g, psd, 5)
    z = n / np.sqrt(psd * g.T_obs / 4.0)
    for x in (z.real, z.imag):
        assert abs(np.mean(x)) < 5.0 / np.sqrt(x.size)
        assert abs(np.var(x) - 1.0) < 5.0 * np.sqrt(2.0 / x.size)
        assert scipy_stats.kstest(x, "norm").pvalue > 1e-3
    assert abs(np.corrcoef(z.real, z.imag)[0, 1]) < 5.0 / np.sqrt(z.size)
    # E|n_k|^2 = S_k T / 2
    assert abs(np.mean(np.abs(z) ** 2) - 2.0) < 5.0 * 2.0 / np.sqrt(z.size)


def test_noise_is_reproducible_and_independent_across_seeds_and_channels():
    g = S.tiny_grid(n=1 << 14)
    psd = np.ones(g.n)
    a = S.gaussian_noise(g, psd, 7)
    assert np.array_equal(a, S.gaussian_noise(g, psd, 7))
    for other in (S.gaussian_noise(g, psd, 8), S.gaussian_noise(g, psd, 7, channel=1)):
        r = np.corrcoef(np.concatenate([a.real, a.imag]), np.concatenate([other.real, other.imag]))[0, 1]
        assert abs(r) < 5.0 / np.sqrt(2 * g.n)


def test_uniforms_lie_in_the_unit_interval_and_are_uniform():
    u = S.uniforms(3, S.STREAM_PARTICLES, 100001)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert scipy_stats.kstest(u, "uniform").pvalue > 1e-3
    # an offset in blocks continues the same sequence
    assert np.array_equal(S.uniforms(3, S.STREAM_PARTICLES, 10, offset=7), u[14:24])


def test_particles_follow_the_prior():
    pr = S.Prior(Mc_lo=12.0, Mc_hi=40.0, tc_lo=-1e6, tc_hi=3e7, e0_hi=0.08)
    P = S.draw_params(pr, 20000, 2)
    assert P.shape == (20000, 6)
    assert P[:, 0].min() >= 12.0 and P[:, 0].max() < 40.0
    assert P[:, 1].min() >= -1e6 and P[:, 1].max() < 3e7
    assert P[:, 4].min() >= 0.0 and P[:, 4].max() < 0.08
    assert np.all(P[:, 5] == 1.0)
    # uniform on the sphere: sin(lat) ~ U[-1, 1]; lon ~ U[0, 2 pi)
    assert scipy_stats.kstest((np.sin(P[:, 2]) + 1.0) / 2.0, "uniform").pvalue > 1e-3
    assert scipy_stats.kstest(P[:, 3] / (2.0 * np.pi), "uniform").pvalue > 1e-3
    assert scipy_stats.kstest((P[:, 0] - 12.0) / 28.0, "uniform").pvalue > 1e-3
    # particles o .. o + B - 1 of one long draw, for every offset
    for o in range(6):
        assert np.array_equal(S.draw_params(pr, 3, 2, offset=o), P[o:o + 3])


def test_paper_grid_and_psd():
    w = S.paper_workload()
    g = w.grid
    assert g.n == 3155760 and g.df == 1.0 / g.T_obs and g.T_obs == 2.5 * S.YEAR_S
    f = g.freqs()
    assert f[0] == 0.01 and f[-1] < 0.05 and f[-1] + g.df >= 0.05 - 1e-12
    psd = S.lisa_like_psd(f[::997])
    assert np.all(np.isfinite(psd)) and np.all(psd > 0.0)
    # smooth: neighbouring samples of the thinned grid differ by well under 1%
    assert np.max(np.abs(np.diff(np.log(psd)))) < 1e-2
    assert w.B == 320 and tuple(w.Np_list) == (256, 64, 16, 1)
