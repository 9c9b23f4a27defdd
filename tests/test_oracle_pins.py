"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
known-answer vectors, closed forms, exact invariants of the F-statistic,
textbook special cases and brute force on tiny inputs.  None of these needs a
GPU.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_2407_10797_gb300 import synth as S

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def tc_for(Mc, f, t):
    """Coalescence time that puts the Newtonian stationary-phase time of
    frequency f at t (test helper: chooses in-band particles)."""
    m = Mc * S.MSUN_S
    return t + 5.0 / 256.0 * m * (np.pi * m * f) ** (-8.0 / 3.0)


@pytest.fixture(scope="module")
def tiny():
    g = S.tiny_grid(n=4096, f_min=0.02)
    psd = S.lisa_like_psd(g.freqs())
    return g, psd, O.OracleModel.from_grid(g)


def _inject(p, m, psd, df, snr):
    """Signal of particle p, present only at the bins swept during [0, T]."""
    a = O.extrinsic_to_a(1.0, S.INJ_PSI, S.INJ_IOTA, S.INJ_PHIC)
    k0, k1 = O.band(p, m)
    h = O.inject(p, m, a, k0, k1 + 1)
    s = snr / math.sqrt(O.inner(h, h, psd, df))
    return h * s, a * s


# ---------------------------------------------------------------- Philox
def _kat():
    rows = []
    for line in open(os.path.join(GOLD, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        rows.append((w[:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers_oracle():
    for ctr, key, out in _kat():
        assert list(O.philox(ctr, key)) == out


def test_philox_known_answers_input_generator():
    for ctr, key, out in _kat():
        got = S.philox4x32_10(np.array(ctr, np.uint32), np.array(key, np.uint32))
        assert list(got) == out


# ---------------------------------------------------------------- p1: (h|h)
def test_inner_product_matches_analytic_integral():
    """Test-mode response (F+ = 1, Fx = 0, no Doppler), flat PSD S0:
    <A1, A1> = 4 df sum f_k^-7/3 / S0 is the midpoint rule of
    4/S0 int f^-7/3 df = (3/S0)(fa^-4/3 - fb^-4/3) over [f_lo - df/2, f_hi + df/2]."""
    g = S.tiny_grid(n=20000, f_min=0.01, stride=200)
    m = O.OracleModel.from_grid(g, response=1)
    S0 = 3.7e-40
    psd = np.full(g.n, S0)
    p = np.array([20.0, 0.0, 0.1, 0.2, 0.0, 1.0])
    edges = np.array([0, 7000, 20000], dtype=np.int64)
    N, M, nb = O.segment_sums(p, m, np.zeros(g.n, complex), psd, 2, edges)
    for s in range(2):
        k0, k1 = edges[s], edges[s + 1]
        fa = g.f_min + (k0 - 0.5) * g.df
        fb = g.f_min + (k1 - 0.5) * g.df
        exact = 3.0 / S0 * (fa ** (-4 / 3) - fb ** (-4 / 3))
        # midpoint-rule error bound: (b-a) h^2 max|f''| / 24, f'' = (7/3)(10/3) x^(-13/3)
        bound = 4.0 / S0 * (fb - fa) * g.df ** 2 * (70.0 / 9.0) * fa ** (-13 / 3) / 24.0
        assert abs(M[s, 0, 0] - exact) <= bound
        assert abs(M[s, 0, 0] - exact) <= 1e-4 * exact
        # A3 = -i A1 has the same norm and is orthogonal to A1
        assert M[s, 2, 2] == pytest.approx(M[s, 0, 0], rel=1e-14)
        assert M[s, 0, 2] == 0.0
        assert nb[s] == k1 - k0


# ---------------------------------------------------------------- p2/p3
@pytest.mark.parametrize("Np", [1, 3, 8, 16])
def test_F_equals_half_snr_squared_at_truth(tiny, Np):
    g, psd, m = tiny
    p = np.array([30.0, tc_for(30.0, 0.02, 0.5 * g.T_obs), 0.3, 1.0, 0.05, 1.0])
    d, a = _inject(p, m, psd, g.df, 12.0)
    F, Fp = O.fstat_batch(p[None], m, d, psd, Np)
    assert F[0] == pytest.approx(72.0, rel=1e-12)
    # per segment: F_p = (h|h)_p / 2
    N, M, nb = O.segment_sums(p, m, d, psd, Np)
    for s in range(Np):
        hh = a @ M[s] @ a
        assert Fp[0, s] == pytest.approx(0.5 * hh, rel=1e-10)


def test_amplitudes_recovered_and_appendix_b_round_trip(tiny):
    g, psd, m = tiny
    p = np.array([25.0, tc_for(25.0, 0.02, 0.4 * g.T_obs), -0.7, 4.0, 0.02, 1.0])
    d, a = _inject(p, m, psd, g.df, 10.0)
    N, M, nb = O.segment_sums(p, m, d, psd, 1)
    a_hat = np.linalg.solve(M[0], N[0])          # Eq. (aandMN3)
    assert np.allclose(a_hat, a, rtol=1e-9, atol=0)
    # Appendix B: a -> (D_L, iota, psi, phi_c) -> a
    DL, iota, psi, phic = O.a_to_extrinsic(a_hat)
    a_back = O.extrinsic_to_a(DL, psi, iota, phic)
    assert np.allclose(a_back, a_hat, rtol=1e-10, atol=0)
    # the injected extrinsics (Table I) are recovered modulo the (psi, phi_c) -> (psi + pi/2, phi_c + pi) symmetry
    assert iota == pytest.approx(S.INJ_IOTA, abs=1e-8)
    two_psi = (2 * psi - 2 * S.INJ_PSI) % (2 * np.pi)
    assert min(two_psi, 2 * np.pi - two_psi) == pytest.approx(0.0, abs=1e-8) or \
        abs(two_psi - np.pi) < 1e-8


# ---------------------------------------------------------------- p4: chi^2
@pytest.mark.parametrize("Np", [1, 4])
def test_noise_only_2F_is_chi_square_4Np(Np):
    from scipy import stats
    g = S.tiny_grid(n=1024, f_min=0.02)
    psd = S.lisa_like_psd(g.freqs())
    m = O.OracleModel.from_grid(g)
    noise = S.gaussian_noise(g, psd, 11)
    P = S.draw_params(S.Prior(tc_lo=0.2 * g.T_obs, tc_hi=0.8 * g.T_obs), 600, 3)
    P[:, 1] = tc_for(P[:, 0], 0.02, P[:, 1])
    F, Fp = O.fstat_batch(P, m, noise, psd, Np)
    assert np.all(F > 0)
    ks = stats.kstest(2.0 * F, stats.chi2(4 * Np).cdf)
    assert ks.pvalue > 1e-3
    assert np.mean(2 * F) == pytest.approx(4 * Np, rel=5 * np.sqrt(8 * Np / 600) / (4 * Np))


# ---------------------------------------------------------------- p5: invariances
def test_invariances(tiny):
    g, psd, m = tiny
    noise = S.gaussian_noise(g, psd, 2)
    P = S.draw_params(S.Prior(tc_lo=0.3 * g.T_obs, tc_hi=0.7 * g.T_obs), 6, 9)
    P[:, 1] = tc_for(P[:, 0], 0.02, P[:, 1])
    d = noise + _inject(P[0], m, psd, g.df, 8.0)[0]
    F0, _ = O.fstat_batch(P, m, d, psd, 4)
    # constant phase of the data (phi_c, pi/4 are absorbed by the amplitudes)
    F1, _ = O.fstat_batch(P, m, d * np.exp(0.731j), psd, 4)
    assert np.allclose(F1, F0, rtol=1e-11)
    # (d, S) -> (c d, c^2 S)
    F2, _ = O.fstat_batch(P, m, 3.0e5 * d, 9.0e10 * psd, 4)
    assert np.allclose(F2, F0, rtol=1e-11)


def test_bins_outside_band_do_not_contribute():
    """Per-particle segments: data outside [f_lo, f_hi] is ignored."""
    g = S.tiny_grid(n=3000, f_min=0.03, stride=300)
    psd = S.lisa_like_psd(g.freqs())
    m = O.OracleModel.from_grid(g)
    p = np.array([10.0, tc_for(10.0, 0.03, -0.05 * g.T_obs), 0.2, 2.0, 0.03, 1.0])
    k0, k1 = O.band(p, m)
    assert 0 < k0 <= k1 < g.n - 1
    noise = S.gaussian_noise(g, psd, 4)
    F0, _ = O.fstat_batch(p[None], m, noise, psd, 8)
    d2 = noise.copy()
    d2[:k0] *= -7.0
    d2[k1 + 1:] = 1e3 * d2[k1 + 1:] + 1.0
    F1, _ = O.fstat_batch(p[None], m, d2, psd, 8)
    assert F1[0] == F0[0]


# ---------------------------------------------------------------- p6: t(f)
def test_time_is_derivative_of_phase(tiny):
    g, psd, m = tiny
    for Mc, e0 in [(12.0, 0.0), (30.0, 0.08), (48.0, 0.03)]:
        p = np.array([Mc, tc_for(Mc, 0.02, 0.5 * g.T_obs), 0.3, 1.0, e0, 1.0])
        for f in (0.0200, 0.02003):
            h = 1e-7
            dphi = (O.phase_orb_cycles(p, m, f + h) - O.phase_orb_cycles(p, m, f - h)) / (2 * h)
            t = O.time_of_freq(p, m, f)
            assert dphi == pytest.approx(t, abs=0.05)


def test_newtonian_time_and_band_edges():
    """pn_order 0 and e0 = 0: t(f) = t_c - (5/256) Mc (pi Mc f)^(-8/3), and the
    band edges are the bins around f(t) = (1/pi) (5/(256 (t_c - t)))^(3/8) Mc^(-5/8)."""
    g = S.Grid(f_min=0.01, df=1e-5, n=4000, T_obs=2.5 * S.YEAR_S)
    m = O.OracleModel.from_grid(g, pn_order=0)
    for Mc, tcf in [(15.0, 0.9), (30.0, 0.6), (45.0, 1.3)]:
        p = np.array([Mc, tcf * g.T_obs, 0.1, 0.5, 0.0, 1.0])
        mc = Mc * S.MSUN_S
        for f in (0.012, 0.03, 0.045):
            t = O.time_of_freq(p, m, f)
            assert t - p[1] == pytest.approx(-5.0 / 256.0 * mc * (np.pi * mc * f) ** (-8 / 3), rel=1e-12)

        def f_of_t(t):
            if t >= p[1]:
                return np.inf
            return (5.0 / (256.0 * (p[1] - t))) ** 0.375 * mc ** (-0.625) / np.pi

        klo, khi = O.band(p, m)
        flo, fhi = f_of_t(0.0), f_of_t(g.T_obs)
        exp_lo = max(0, math.ceil((flo - g.f_min) / g.df))
        exp_hi = g.n - 1 if not np.isfinite(fhi) else min(g.n - 1, math.floor((fhi - g.f_min) / g.df))
        assert klo == exp_lo and khi == exp_hi


def test_pn_coefficients_from_energy_balance():
    """t(f) of the oracle equals the stationary-phase time obtained from the
    textbook 2PN binding energy and flux (non-spinning, circular):
    E = -(mu v^2/2)[1 - (3/4 + eta/12) v^2 - (27/8 - 19 eta/8 + eta^2/24) v^4],
    F = (32/5) eta^2 v^10 [1 - (1247/336 + 35 eta/12) v^2 + 4 pi v^3
        - (44711/9072 - 9271 eta/504 - 65 eta^2/18) v^4],
    dt/dv = -(dE/dv)/F expanded to O(v^4) and integrated term by term."""
    import sympy as sp
    v, eta = sp.symbols("v eta", positive=True)
    e2 = -(sp.Rational(3, 4) + eta / 12)
    e4 = -(sp.Rational(27, 8) - sp.Rational(19, 8) * eta + eta ** 2 / 24)
    f2 = -(sp.Rational(1247, 336) + sp.Rational(35, 12) * eta)
    f3 = 4 * sp.pi
    f4 = -(sp.Rational(44711, 9072) - sp.Rational(9271, 504) * eta - sp.Rational(65, 18) * eta ** 2)
    num = 1 + 2 * e2 * v ** 2 + 3 * e4 * v ** 4     # -(dE/dv)/(mu v)
    den = 1 + f2 * v ** 2 + f3 * v ** 3 + f4 * v ** 4
    R = sp.series(num / den, v, 0, 5).removeO()
    # t(v) = t_c - (5 M /(32 eta)) sum_k r_k v^(k-8)/(8-k)
    tv = sum(-sp.Rational(5, 32) / eta * R.coeff(v, k) * v ** (k - 8) / (8 - k) for k in range(5))
    tfun = sp.lambdify((v, eta), tv, "math")
    g = S.tiny_grid(n=10, f_min=0.01)
    m = O.OracleModel.from_grid(g)
    for Mc, q in [(10.0, 1.0), (37.0, 1.0), (20.0, 3.0)]:
        p = np.array([Mc, 1.0e7, 0.0, 0.0, 0.0, q])
        et = q / (1 + q) ** 2
        M = Mc * S.MSUN_S * et ** (-0.6)
        for f in (0.01, 0.02, 0.05):
            vv = (np.pi * M * f) ** (1 / 3)
            expect = tfun(vv, et) * M
            got = O.time_of_freq(p, m, f) - p[1]
            assert got == pytest.approx(expect, rel=1e-12)


# ---------------------------------------------------------------- p7: antenna
def test_antenna_sky_polarisation_average():
    """<F+^2 + Fx^2> over the sky = 2 * 3/20 for a 60-degree Michelson
    (the psi-average of F+^2 is (F+^2 + Fx^2)/2 and <F+^2> = (2/5) D:D =
    (2/5)(1/2) sin^2(60 deg)).  F+^2 + Fx^2 is a degree-4 polynomial in the
    direction, so a Gauss-Legendre x uniform-longitude rule is exact."""
    g = S.tiny_grid(n=10)
    m = O.OracleModel.from_grid(g)
    xs, ws = np.polynomial.legendre.leggauss(6)
    nl = 12
    for t in (0.0, 0.37 * S.YEAR_S, 1.71 * S.YEAR_S):
        acc = 0.0
        for x, w in zip(xs, ws):
            for j in range(nl):
                p = np.array([20.0, 0.0, math.asin(x), 2 * np.pi * j / nl, 0.0, 1.0])
                fp, fx = O.antenna(p, m, t)
                acc += w * (fp * fp + fx * fx) / nl
        assert acc / 2.0 == pytest.approx(2 * 3.0 / 20.0, rel=1e-12)


def test_doppler_vanishes_at_ecliptic_poles_and_peaks_in_plane():
    g = S.tiny_grid(n=10)
    m = O.OracleModel.from_grid(g)
    for t in (0.0, 1.0e7, 5.5e7):
        for lat in (np.pi / 2, -np.pi / 2):
            assert abs(O.doppler_delay([20, 0, lat, 1.0, 0, 1], m, t)) < 1e-12 * S.AU_S
    # in the ecliptic plane, facing the guiding centre: d = R
    assert O.doppler_delay([20, 0, 0.0, 0.0, 0, 1], m, 0.0) == pytest.approx(S.AU_S, rel=1e-15)


def test_orbit_and_cartwheel_repeat_after_one_year():
    """A 1 AU circular orbit takes one year (Kepler's third law) and the rigid
    constellation turns once per orbit: the Doppler delay and the detector
    tensor repeat after a year, and the delay changes sign after half a year
    (the guiding centre on the far side of the Sun)."""
    m = O.OracleModel.from_grid(S.tiny_grid(n=10))
    rng = np.random.default_rng(4)
    for _ in range(20):
        p = [20.0, 0.0, math.asin(rng.uniform(-0.9, 0.9)), rng.uniform(0, 2 * np.pi), 0.0, 1.0]
        t = rng.uniform(0, 2 * S.YEAR_S)
        d = O.doppler_delay(p, m, t)
        assert O.doppler_delay(p, m, t + S.YEAR_S) == pytest.approx(d, abs=1e-9 * S.AU_S)
        assert O.doppler_delay(p, m, t + 0.5 * S.YEAR_S) == pytest.approx(-d, abs=1e-9 * S.AU_S)
        assert np.allclose(O.detector_tensor(m, t + S.YEAR_S), O.detector_tensor(m, t), atol=1e-12)


def test_detector_is_a_60_degree_michelson_in_a_plane_inclined_60_degrees():
    """The constellation is an equilateral triangle whose plane is inclined by
    60 degrees to the ecliptic. The tensor (a a - b b)/2 of two unit arms 60
    degrees apart is traceless with eigenvalues -sin(60)/2, 0, +sin(60)/2; its
    null vector is the normal of the plane, at 60 degrees from the ecliptic
    pole."""
    m = O.OracleModel.from_grid(S.tiny_grid(n=10))
    for t in np.linspace(0.0, S.YEAR_S, 9):
        D = O.detector_tensor(m, t)
        assert np.allclose(D, D.T, atol=1e-15) and abs(np.trace(D)) < 1e-14
        w, V = np.linalg.eigh(D)
        assert np.allclose(w, [-math.sqrt(3) / 4, 0.0, math.sqrt(3) / 4], atol=1e-13)
        assert abs(V[2, 1]) == pytest.approx(0.5, abs=1e-12)


def test_antenna_is_the_transverse_traceless_projection_along_the_source():
    """F+^2 + Fx^2 = 2 |D^TT|^2 with D^TT = P D P - (1/2) P tr(P D),
    P = I - n n and n = (cos b cos l, cos b sin l, sin b) the source direction
    of the Doppler delay: the basis-free form of the polarisation sum, which
    holds only for polarisation tensors transverse to that same direction."""
    m = O.OracleModel.from_grid(S.tiny_grid(n=10))
    rng = np.random.default_rng(5)
    for _ in range(50):
        b, l, t = math.asin(rng.uniform(-1, 1)), rng.uniform(0, 2 * np.pi), rng.uniform(0, S.YEAR_S)
        fp, fx = O.antenna([20.0, 0.0, b, l, 0.0, 1.0], m, t)
        n = np.array([math.cos(b) * math.cos(l), math.cos(b) * math.sin(l), math.sin(b)])
        P = np.eye(3) - np.outer(n, n)
        D = O.detector_tensor(m, t)
        Dtt = P @ D @ P - 0.5 * P * np.trace(P @ D)
        assert fp * fp + fx * fx == pytest.approx(2.0 * np.sum(Dtt * Dtt), rel=1e-10, abs=1e-14)


def test_doppler_phase_is_the_arrival_time_shift():
    """A wave from direction n reaches a detector at r a time n.r/c before the
    solar-system barycentre: h_det(t) = h_ssb(t + tau(t)), tau = n.r/c (the
    Doppler delay), so the frequency f is observed at the detector time t with
    f = F_ssb(t + tau(t)) (1 + tau'(t)), F_ssb the inverse of the barycentric
    t(f). The template's group delay dPhi/df at f must be that time. The
    template keeps the response to first order in the orbital motion (Sec.
    IV, N = 0, d evaluated at t_f), so the two agree to a few per cent of the
    shift."""
    m0 = O.OracleModel.from_grid(S.tiny_grid(n=10, f_min=0.01))
    Mc, f_star = 30.0, 0.02
    alpha_star = 2 * np.pi * 0.3
    for lon in (alpha_star - np.pi / 2, alpha_star + np.pi / 2, 2.0):
        p = np.array([Mc, tc_for(Mc, f_star, 0.3 * S.YEAR_S), 0.0, lon, 0.0, 1.0])

        def f_ssb(s):   # inverse of the barycentric t(f), by bisection
            lo, hi = 1e-3, 0.2
            for _ in range(200):
                mid = 0.5 * (lo + hi)
                lo, hi = (mid, hi) if O.time_of_freq(p, m0, mid) < s else (lo, mid)
            return 0.5 * (lo + hi)

        def observed(t):
            tau = O.doppler_delay(p, m0, t)
            rate = (O.doppler_delay(p, m0, t + 10.0) - O.doppler_delay(p, m0, t - 10.0)) / 20.0
            return f_ssb(t + tau) * (1.0 + rate)

        lo, hi = 0.2 * S.YEAR_S, 0.4 * S.YEAR_S
        for _ in range(80):
            mid = 0.5 * (lo + hi)
            lo, hi = (mid, hi) if observed(mid) < f_star else (lo, mid)
        t_det = 0.5 * (lo + hi)
        shift = t_det - O.time_of_freq(p, m0, f_star)
        df = 1e-10
        m = O.OracleModel.from_grid(S.Grid(f_min=f_star - 5 * df, df=df, n=11, T_obs=2.5 * S.YEAR_S))
        ph = np.unwrap(2 * np.pi * np.array([O.phase_frac(p, m, k) for k in range(11)])) / (2 * np.pi)
        group_delay = (ph[6] - ph[4]) / (2 * df)
        assert abs(shift) > 1000.0
        assert abs(group_delay - t_det) <= 0.02 * abs(shift) + 1.0, (lon, shift, group_delay - t_det)


def test_band_edges_by_brute_force():
    """On a 2.5-yr grid (bins ~20 s of chirp time apart) the band is the first
    bin with t(f_k) >= 0 and the last with t(f_k) <= T_obs, found by scanning
    every bin."""
    g = S.tiny_grid(n=3000, f_min=0.02)
    m = O.OracleModel.from_grid(g)
    f_mid = g.f_min + 1500 * g.df
    for Mc, t_mid in [(30.0, 0.0), (12.0, 0.0), (45.0, g.T_obs), (25.0, g.T_obs)]:
        p = np.array([Mc, 0.0, 0.3, 1.1, 0.02, 1.0])
        p[1] = t_mid - O.time_of_freq(p, m, f_mid)   # the edge crossing at bin 1500
        t = np.array([O.time_of_freq(p, m, g.f_min + k * g.df) for k in range(g.n)])
        ok_lo, ok_hi = np.flatnonzero(t >= 0.0), np.flatnonzero(t <= g.T_obs)
        klo, khi = O.band(p, m)
        assert klo == (ok_lo[0] if ok_lo.size else g.n)
        assert khi == (ok_hi[-1] if ok_hi.size else -1)
        assert 0 < klo < g.n - 1 or 0 < khi < g.n - 1   # an edge inside the grid


# ---------------------------------------------------------------- p8: eccentricity
def test_eccentric_correction_scales_as_e0_squared():
    g = S.tiny_grid(n=10)
    m = O.OracleModel.from_grid(g)
    base = np.array([25.0, 1.0e8, 0.0, 0.0, 0.0, 1.0])
    for f in (0.01, 0.02, 0.04):
        ph0 = O.phase_orb_cycles(base, m, f)
        d1 = O.phase_orb_cycles(base + [0, 0, 0, 0, 0.03, 0], m, f) - ph0
        d2 = O.phase_orb_cycles(base + [0, 0, 0, 0, 0.06, 0], m, f) - ph0
        assert d2 / d1 == pytest.approx(4.0, rel=1e-7)
        # and matches -(2355/1462) e0^2 (3/128)(pi Mc f)^-5/3 (f0/f)^(19/9) / (2 pi)
        mc = 25.0 * S.MSUN_S
        expect = -(2355 / 1462) * 0.03 ** 2 * 3 / 128 * (np.pi * mc * f) ** (-5 / 3) \
            * (0.01 / f) ** (19 / 9) / (2 * np.pi)
        assert d1 == pytest.approx(expect, rel=1e-7)


# ---------------------------------------------------------------- segments
def test_segment_membership_exact():
    """Bin k lies in segment p iff e_p <= f_k < e_{p+1} (last one closed), with
    e_p = f_lo + p (f_hi - f_lo)/Np, checked in exact rational arithmetic."""
    g = S.Grid(f_min=0.01, df=1.0 / 1024.0 / 1024.0 / 32.0, n=3001, T_obs=2.5 * S.YEAR_S)
    m = O.OracleModel.from_grid(g)
    for Mc, tcf, Np in [(20.0, 0.9, 7), (33.0, 0.95, 256), (45.0, 0.8, 64), (11.0, 1.05, 3)]:
        p = np.array([Mc, tcf * g.T_obs, 0.1, 0.5, 0.02, 1.0])
        p[1] = tc_for(Mc, 0.01 + 1500 * g.df, tcf * g.T_obs * 0.5)
        klo, khi = O.band(p, m)
        _, _, nb = O.segment_sums(p, m, np.zeros(g.n, complex), np.ones(g.n), Np)
        fmin, df = Fraction(g.f_min), Fraction(g.df)
        fk = lambda k: fmin + k * df
        cnt = np.zeros(Np, dtype=np.int64)
        if klo <= khi:
            flo, fhi = fk(klo), fk(khi)
            for k in range(klo, khi + 1):
                e = [flo + Fraction(j) * (fhi - flo) / Np for j in range(Np + 1)]
                for s in range(Np):
                    if e[s] <= fk(k) < e[s + 1] or (s == Np - 1 and fk(k) == e[Np]):
                        cnt[s] += 1
                        break
        assert list(nb) == list(cnt)


def test_global_edge_frequencies_follow_the_membership_rule():
    """Global edges given as frequencies: the oracle's segment start bins give
    each bin the segment p with e_p <= f_k < e_{p+1} (the last one closed at
    e_{N_p}, bins outside [e_0, e_{N_p}] in none), checked bin by bin with the
    grid's own frequencies: edges on bins, between bins, repeated, and outside
    the grid; decreasing or non-finite edges are refused."""
    g = S.Grid(f_min=0.02, df=1.0e-7, n=500, T_obs=1.0e7)
    m = O.OracleModel.from_grid(g)
    f = g.freqs()
    cases = [
        [f[0], f[100], f[100], f[250], f[499]],
        [f[0] - 3e-7, f[7] + 0.4e-7, f[300], f[499] + 1e-3],
        [f[10], f[10] + 0.5e-7, f[11], f[11]],
        list(g.edge_freqs([0, 17, 17, 300, 500])),
    ]
    for e in cases:
        Np = len(e) - 1
        starts = O.edge_starts(m, e, Np)
        seg = np.full(g.n, -1)
        for k in range(g.n):
            for p in range(Np):
                if e[p] <= f[k] < e[p + 1] or (p == Np - 1 and f[k] == e[Np]):
                    seg[k] = p
                    break
        for p in range(Np):
            assert np.array_equal(np.nonzero(seg == p)[0], np.arange(starts[p], starts[p + 1])), (e, p)
        assert np.all(seg[:starts[0]] == -1) and np.all(seg[starts[Np]:] == -1)
    assert list(O.edge_starts(m, cases[3], 4)) == [0, 17, 17, 300, 500]
    for bad in ([f[5], f[3], f[9]], [f[5], np.nan, f[9]], [f[5], f[6], np.inf]):
        with pytest.raises(ValueError):
            O.edge_starts(m, bad, 2)


def test_degenerate_segments_give_zero():
    N = np.array([1.0, 2.0, 3.0, 4.0])
    M = np.eye(4)
    assert O.segment_F(N, M, 3) == 0.0
    assert O.segment_F(N, M, 4) == pytest.approx(15.0)
    Ms = np.diag([1.0, 1.0, 1.0, 1.0])
    Ms[0, 1] = Ms[1, 0] = 1.0 - 1e-14          # M11 M22 - M12^2 below 1e-12 M11 M22
    assert O.segment_F(N, Ms, 100) == 0.0


def test_nonfinite_parameters_give_nan(tiny):
    g, psd, m = tiny
    P = np.array([[np.nan, 1e8, 0, 0, 0, 1], [20.0, 1e8, 0, 0, 0, 1]])
    F, Fp = O.fstat_batch(P, m, np.zeros(g.n, complex), psd, 2)
    assert np.isnan(F[0]) and np.all(np.isnan(Fp[0]))


# ---------------------------------------------------------------- p9: brute force
def test_brute_force_scan_peaks_at_truth_and_broadens_with_Np():
    """Noise-free 1-D M_c scan: the argmax is the injected M_c for every Np and
    the half-maximum width grows with Np (Fig. 1, left panel)."""
    g = S.tiny_grid(n=2048, f_min=0.02, stride=64)
    psd = S.lisa_like_psd(g.freqs())
    m = O.OracleModel.from_grid(g)
    Mc0 = 30.0
    p = np.array([Mc0, tc_for(Mc0, 0.02, 0.9 * g.T_obs), 0.4, 2.1, 0.01, 1.0])
    d, _ = _inject(p, m, psd, g.df, 20.0)
    grid = Mc0 * (1.0 + np.linspace(-4e-5, 4e-5, 81))
    P = np.repeat(p[None], len(grid), axis=0)
    P[:, 0] = grid
    widths = []
    for Np in (1, 16):
        F, _ = O.fstat_batch(P, m, d, psd, Np)
        assert np.argmax(F) == 40
        widths.append(np.sum(F > 0.5 * F.max()))
    assert widths[1] > widths[0]


# ---------------------------------------------------------------- PSO
def test_pso_converges_on_sphere_function():
    R, Np, D = 2, 40, 5
    x, v = O.pso_init(R, Np, D, seed=7)
    assert np.all((x >= 0) & (x < 1)) and np.all(x + v >= 0) and np.all(x + v <= 1)
    pbx = x.copy()
    pbf = np.full((R, Np), -np.inf)
    target = np.array([0.3, 0.7, 0.5, 0.2, 0.9])
    iters = 300
    for it in range(iters):
        inside = np.all((x >= 0) & (x <= 1), axis=2)
        fit = np.where(inside, -np.sum((x - target) ** 2, axis=2), -np.inf)
        w = 0.9 - 0.5 * it / (iters - 1)
        O.pso_step(x, v, pbx, pbf, fit, seed=7, iteration=it, w=w)
    best = pbx[np.arange(R), np.argmax(pbf, axis=1)]
    assert np.all(np.abs(best - target) < 1e-3)


def test_pso_step_rules():
    """pbest only on strictly greater fitness, lbest on the ring with ties to
    the lowest index, symmetric velocity clamp."""
    R, Np, D = 1, 6, 2
    x = np.arange(R * Np * D, dtype=float).reshape(R, Np, D) / 20
    v = np.zeros_like(x)
    pbx = x.copy() + 0.5
    pbf = np.array([[1.0, 2.0, 2.0, 0.5, 3.0, 3.0]])
    fit = np.array([[1.0, 5.0, -np.inf, np.nan, 3.0, 1.0]])
    pbx0 = pbx.copy()
    lb = O.pso_step(x, v, pbx, pbf, fit, seed=1, iteration=3, w=0.5, vmax=0.05)
    assert list(pbf[0]) == [1.0, 5.0, 2.0, 0.5, 3.0, 3.0]
    assert np.array_equal(pbx[0, 0], pbx0[0, 0]) and np.array_equal(pbx[0, 1], x[0, 1] - v[0, 1])
    # ring neighbourhoods {5,0,1} {0,1,2} {1,2,3} {2,3,4} {3,4,5} {4,5,0}
    assert list(lb[0]) == [1, 1, 1, 4, 4, 4]
    assert np.all(np.abs(v) <= 0.05)


def test_pso_velocity_clamp_is_symmetric():
    """Attractions of either sign beyond v_max are clamped to -v_max and +v_max
    (reading c10)."""
    R, Np, D = 1, 40, 5
    x = np.full((R, Np, D), 0.5)
    v = np.zeros_like(x)
    pbx = np.where(np.arange(Np)[None, :, None] % 2 == 0, 0.0, 1.0) * np.ones_like(x)
    pbf = np.zeros((R, Np))   # equal fitness: lbest = lowest ring index, an even particle for most
    O.pso_step(x, v, pbx, pbf, np.full((R, Np), -np.inf), seed=3, iteration=0, w=0.0, vmax=0.05)
    assert v.min() == -0.05 and v.max() == 0.05


@pytest.mark.parametrize("which", ["cognitive", "social"])
def test_pso_terms_pull_toward_their_own_attractor(which):
    """With w = 0 and only one acceleration constant the step is c r (a - x)
    with r in [0, 1): a = the particle's personal best for c1, its ring's best
    for c2. Personal and ring bests are placed on opposite sides of x, so
    every coordinate's ratio v / (a - x) must lie in [0, c)."""
    R, Np, D = 2, 8, 5
    rng = np.random.default_rng(6)
    x = rng.uniform(0.4, 0.6, (R, Np, D))
    v = np.zeros_like(x)
    pbx = np.zeros_like(x)
    pbx[:, 0] = 1.0                        # particle 0: personal best above every x
    pbf = np.full((R, Np), -1.0)
    pbf[:, 0] = 5.0                        # ... and the best of its ring
    pbx[:, 1:] = 0.0                       # the others' personal bests below x
    c1, c2 = (1.7, 0.0) if which == "cognitive" else (0.0, 1.7)
    lb = O.pso_step(x, v, pbx, pbf, np.full((R, Np), -np.inf), seed=9, iteration=2, w=0.0,
                    c1=c1, c2=c2, vmax=10.0)
    x0 = x - v                             # the step moved x by v
    for r in range(R):
        for i in (1, 7):                   # ring best is particle 0, personal best below
            a = pbx[r, i] if which == "cognitive" else pbx[r, lb[r, i]]
            ratio = v[r, i] / (a - x0[r, i])
            assert lb[r, i] == 0
            assert np.all(ratio >= 0.0) and np.all(ratio < (c1 if which == "cognitive" else c2))


def test_pso_random_numbers_are_uniform_on_the_unit_interval():
    """With w = 0, c1 = 1, c2 = 0 and the personal best one unit above x, the
    velocity is r1 itself: 10^4 draws must follow U[0, 1) (Kolmogorov-Smirnov)."""
    from scipy import stats
    R, Np, D = 10, 40, 5
    draws = []
    for it in range(5):
        x = np.zeros((R, Np, D))
        v = np.zeros_like(x)
        pbx = np.ones_like(x)
        pbf = np.zeros((R, Np))
        O.pso_step(x, v, pbx, pbf, np.full((R, Np), -np.inf), seed=11, iteration=it, w=0.0, c1=1.0, c2=0.0,
                   vmax=10.0)
        draws.append(v.ravel())
    u = np.concatenate(draws)
    assert np.all((u >= 0) & (u < 1))
    assert stats.kstest(u, "uniform").pvalue > 1e-3


def test_constants_agree_with_input_module():
    src = open(os.path.join(os.path.dirname(O.__file__), "fstat_oracle.c")).read()

    def grab(name):
        for line in src.splitlines():
            if line.startswith(f"#define {name} "):
                return float(line.split()[2])
        raise KeyError(name)

    assert grab("OR_MSUN_S") == S.MSUN_S
    assert grab("OR_YEAR_S") == S.YEAR_S
    assert grab("OR_AU_S") == S.AU_S


# ---------------------------------------------------------------- p11: MLP oracle
def test_mlp_oracle_bf16_rounding_known_values():
    from oracle import mlp_oracle as M
    # exact bf16 values stay, halfway cases round to even, 1 + 2^-9 rounds down
    vals = np.array([1.0, -2.5, 1.0 + 2 ** -8, 1.0 + 2 ** -9, 1.0 + 3 * 2 ** -9, 65504.0])
    got = M.bf16(vals)
    assert got[0] == 1.0 and got[1] == -2.5
    assert got[2] == 1.0            # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to even -> 1
    assert got[3] == 1.0
    assert got[4] == 1.0 + 2 ** -7  # above halfway
    assert got[5] == 65536.0


def test_mlp_oracle_gradient_matches_finite_differences():
    """Central differences of the loss in float64 without the bf16 rounding of
    the weights (rounding removed so the loss is smooth) match the analytic
    gradient of the same network."""
    from oracle import mlp_oracle as M
    rng = np.random.default_rng(1)
    W = 16
    shapes = M.param_shapes(W)
    theta = np.concatenate([rng.normal(scale=0.5, size=int(np.prod(s))) for _, s in shapes])
    X = rng.random((20, 5))
    t = rng.normal(size=20)
    t[3] = np.nan                   # ignored sample
    orig = M.bf16
    try:
        M.bf16 = lambda a: np.asarray(a, dtype=np.float64)
        L0, g = M.loss_and_grad(theta, X, t, W)
        idx = rng.choice(len(theta), 40, replace=False)
        for i in idx:
            h = 1e-6
            tp = theta.copy()
            tp[i] += h
            tm = theta.copy()
            tm[i] -= h
            fd = (M.loss_and_grad(tp, X, t, W)[0] - M.loss_and_grad(tm, X, t, W)[0]) / (2 * h)
            assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-9)
    finally:
        M.bf16 = orig


def test_mlp_oracle_loss_of_a_constant_network():
    """All weights zero: the network outputs b4 everywhere, so the loss is half
    the mean squared difference to the finite targets (NaN targets are not
    counted) and the only non-zero gradient is dL/db4 = mean(b4 - t)."""
    from oracle import mlp_oracle as M
    W = 8
    theta = np.zeros(sum(int(np.prod(s)) for _, s in M.param_shapes(W)))
    theta[-1] = 0.75
    X = np.random.default_rng(3).random((6, 5))
    t = np.array([1.0, np.nan, -0.5, 2.0, np.nan, 0.25])
    L, g = M.loss_and_grad(theta, X, t, W)
    ok = np.isfinite(t)
    assert L == pytest.approx(0.5 * np.mean((0.75 - t[ok]) ** 2), rel=1e-15)
    assert g[-1] == pytest.approx(np.mean(0.75 - t[ok]), rel=1e-15)
    assert np.all(g[:-1] == 0.0)


def test_mlp_oracle_adam_steps_have_closed_forms():
    """Adam with bias correction (Kingma and Ba): under a constant gradient
    every step is -lr sign(g) (to eps); after g then -g the second step is
    +lr (1 - beta1)/(1 + beta1) sign(g), since the corrected second moment is
    g^2 and the corrected first moment -(1 - beta1)/(1 + beta1) g."""
    from oracle import mlp_oracle as M
    g = np.array([3.0, -0.02, 1e3])
    lr = 1e-3
    th, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
    for step in range(1, 6):
        th_new, m, v = M.adam(th, g, m, v, step, lr)
        assert np.allclose(th_new - th, -lr * np.sign(g), rtol=1e-6, atol=0)
        th = th_new
    th, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
    th1, m, v = M.adam(th, g, m, v, 1, lr)
    th2, m, v = M.adam(th1, -g, m, v, 2, lr)
    assert np.allclose(th2 - th1, lr * 0.1 / 1.9 * np.sign(g), rtol=1e-6, atol=0)


def test_mlp_oracle_adam_fits_a_smooth_function():
    from oracle import mlp_oracle as M
    rng = np.random.default_rng(2)
    W = 32
    theta = np.concatenate([rng.uniform(-1, 1, size=int(np.prod(s))) * np.sqrt(6.0 / (s[1] if len(s) == 2 else 1))
                            * (len(s) == 2) for _, s in M.param_shapes(W)])
    X = rng.random((256, 5))
    t = np.sin(3 * X[:, 0]) + X[:, 1] ** 2 - X[:, 2] * X[:, 3]
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    L_first = M.loss_and_grad(theta, X, t, W)[0]
    for s in range(1, 301):
        L, g = M.loss_and_grad(theta, X, t, W)
        theta, m, v = M.adam(theta, g, m, v, s, 3e-3)
    assert L < 0.05 * L_first


# ---------------------------------------------------------------- TDI channels (Sec. II.A, Eq. eq2)
def test_tdi_T_vanishes_and_A_E_are_orthogonal_michelsons_turned_in_the_plane():
    """Long-wavelength TDI: X + Y + Z = 0, so T vanishes; A and E are
    orthogonal, each of norm sqrt(3/2) times a Michelson's, and equal to the
    X Michelson with the constellation turned in its plane by 75 and 30
    degrees (three tensors 120 degrees apart in the plane of traceless
    in-plane tensors, where a turn by r moves a tensor by 2r), times
    sqrt(3/2)."""
    g = S.tiny_grid(n=10)
    ms = [O.OracleModel.from_grid(g, channel=c) for c in range(4)]
    for t in (0.0, 0.37 * S.YEAR_S, 1.71 * S.YEAR_S):
        DX, DA, DE, DT = (O.detector_tensor(m, t) for m in ms)
        assert np.abs(DT).max() < 1e-15
        assert abs(np.sum(DA * DE)) < 1e-15
        assert np.sum(DA * DA) == pytest.approx(1.5 * np.sum(DX * DX), rel=1e-13)
        assert np.sum(DE * DE) == pytest.approx(1.5 * np.sum(DX * DX), rel=1e-13)
        for D, deg in ((DA, 75.0), (DE, 30.0)):
            turned = O.detector_tensor(O.OracleModel.from_grid(g, channel=0, orient=np.deg2rad(deg)), t)
            assert np.allclose(D, np.sqrt(1.5) * turned, rtol=0, atol=1e-15)


def test_tdi_A_E_sky_averages():
    """<F_A^2> = <F_E^2> = 3/2 x 3/20 (sky and polarisation average) and
    <F_A F_E> = 0: A and E see the sky with equal sensitivity and their
    responses are uncorrelated (Gauss-Legendre x uniform longitude, exact
    for these degree-4 polynomials in the direction)."""
    g = S.tiny_grid(n=10)
    mA = O.OracleModel.from_grid(g, channel=1)
    mE = O.OracleModel.from_grid(g, channel=2)
    xs, ws = np.polynomial.legendre.leggauss(6)
    nl = 12
    for t in (0.0, 0.9 * S.YEAR_S):
        aa = ee = ae = 0.0
        for x, w in zip(xs, ws):
            for j in range(nl):
                p = np.array([20.0, 0.0, math.asin(x), 2 * np.pi * j / nl, 0.0, 1.0])
                pa, xa = O.antenna(p, mA, t)
                pe, xe = O.antenna(p, mE, t)
                aa += w * (pa * pa + xa * xa) / nl
                ee += w * (pe * pe + xe * xe) / nl
                ae += w * (pa * pe + xa * xe) / nl
        assert aa / 2.0 == pytest.approx(2 * 1.5 * 3.0 / 20.0, rel=1e-12)
        assert ee / 2.0 == pytest.approx(2 * 1.5 * 3.0 / 20.0, rel=1e-12)
        assert abs(ae) < 1e-13


def _two_channel_case(g, p, snr, seed=None):
    psd = S.tdi_psds(g.freqs(), S.TDI_AE)
    ms = [O.OracleModel.from_grid(g, channel=1), O.OracleModel.from_grid(g, channel=2)]
    a = O.extrinsic_to_a(1.0, S.INJ_PSI, S.INJ_IOTA, S.INJ_PHIC)
    k0, k1 = O.band(p, ms[0])
    h = np.stack([O.inject(p, m, a, k0, k1 + 1) for m in ms])
    hh = sum(O.inner(h[c], h[c], psd[c], g.df) for c in range(2))
    h *= snr / math.sqrt(hh)
    d = h.copy()
    if seed is not None:
        d += np.stack([S.gaussian_noise(g, psd[c], seed, channel=c) for c in range(2)])
    return d, psd, ms, h


@pytest.mark.parametrize("Np", [1, 5])
def test_two_channel_F_is_half_the_summed_snr_squared(Np):
    """Noise-free A and E data: F_sum at the truth = (sum over channels of
    (h_c|h_c)) / 2 = SNR^2 / 2 -- the amplitudes are common to the channels."""
    g = S.tiny_grid(n=4096, f_min=0.02, stride=4)
    p = np.array([30.0, tc_for(30.0, 0.02 + 2048 * g.df, 0.5 * g.T_obs), 0.3, 1.0, 0.05, 1.0])
    d, psd, ms, h = _two_channel_case(g, p, 12.0)
    F, _ = O.fstat_batch_channels(p[None], ms, d, psd, Np)
    assert F[0] == pytest.approx(72.0, rel=1e-11)


def test_two_channel_F_reduces_to_one_channel():
    """With the second channel's data zero and its noise PSD 10^30 times
    larger, its inner products vanish and F equals the one-channel F."""
    g = S.tiny_grid(n=4096, f_min=0.02, stride=4)
    p = np.array([26.0, tc_for(26.0, 0.02 + 2048 * g.df, 0.4 * g.T_obs), -0.4, 2.0, 0.03, 1.0])
    d, psd, ms, h = _two_channel_case(g, p, 10.0, seed=3)
    P = np.stack([p, p + np.array([0.2, 30.0, 0.01, 0.0, 0.0, 0.0])])
    d2 = d.copy()
    d2[1] = 0.0
    psd2 = psd.copy()
    psd2[1] *= 1e30
    F2, Fp2 = O.fstat_batch_channels(P, ms, d2, psd2, 3)
    F1, Fp1 = O.fstat_batch(P, ms[0], d2[0], psd2[0], 3)
    assert np.allclose(F2, F1, rtol=1e-10, atol=1e-12)
    assert np.allclose(Fp2, Fp1, rtol=1e-10, atol=1e-12)


def test_two_channel_noise_only_2F_is_chi_square_4Np():
    """Gaussian noise in A and E: 2 F_sum ~ chi^2 with 4 N_p degrees of
    freedom (the four amplitudes per segment are common to the channels)."""
    from scipy import stats
    g = S.tiny_grid(n=3000, f_min=0.02)          # bins of width 1/T, as the noise model assumes
    psd = S.tdi_psds(g.freqs(), S.TDI_AE)
    ms = [O.OracleModel.from_grid(g, channel=1), O.OracleModel.from_grid(g, channel=2)]
    Np = 2
    P = S.draw_params(S.Prior(tc_lo=0.2 * g.T_obs, tc_hi=0.8 * g.T_obs), 40, 5)
    P[:, 1] = tc_for(P[:, 0], 0.02 + 1500 * g.df, P[:, 1])
    vals = []
    for seed in range(40):
        d = np.stack([S.gaussian_noise(g, psd[c], 100 + seed, channel=c) for c in range(2)])
        F, _ = O.fstat_batch_channels(P[seed % 40:seed % 40 + 5], ms, d, psd, Np)
        vals.extend(2.0 * F)
    vals = np.array(vals)
    assert abs(np.mean(vals) - 4 * Np) < 0.6
    assert stats.kstest(vals, stats.chi2(4 * Np).cdf).pvalue > 1e-3
