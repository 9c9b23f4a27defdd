"""Pins of the oracle's Eq. (freDres) response series (Sec. IV) against the
definition it approximates.

The series stands for the Fourier transform of the single-arm response
x(t) = F(t) h(t + d(t)).  The brute-force pin builds that time series
directly: h(t) is the exact inverse discrete Fourier transform of a tapered
frequency-domain chirp h(f) = f^-7/6 exp(-2 pi i Phi_orb(f)), evaluated at the
delayed times t + d(t) by the band-limited (direct) Fourier sum, multiplied by
the antenna pattern, and transformed back by an FFT.  The oracle's basis
waveform A1 = T+ h0 (A2 = Tx h0) must reproduce that spectrum, and each term
of the series must bring it closer: the paper's form misses the
second-order Doppler phase (about pi f^2 ddot^2 / fdot, 1e-2 rad here), the
filter of order N removes it to O(eps^(2N+2)) with eps = 2 pi f ddot T_f, and
the k = 1 term the amplitude slope T_A1 G'.  Planting any one mistake in
the oracle's series (no retarded time, no 1/(1 + ddot), no (1 - ddot) in the
phase, the sign of T_A1, T_f^2 = |dt/df|, the conjugate filter weights) lifts
the order-2 error from 5e-7 to at least 8e-5.
"""
import numpy as np
import pytest

from oracle import oracle as O

T_WIN = 2.0 ** 20          # s: period of the discrete transforms
M_T = 8192                 # time samples (128 s apart, heterodyned band +-3.9 mHz)
F_LO, F_HI = 0.0515, 0.0550
TAPER = 0.12               # raised-cosine taper on each side (fraction of the band)
O_MSUN = 4.925490947e-6    # s


def _setup(lat, lon, Mc=50.0):
    df = 1.0 / T_WIN
    kmin, kmax = int(F_LO / df), int(F_HI / df)
    f_min = kmin * df
    n = kmax - kmin
    p = np.array([Mc, 0.0, lat, lon, 0.0, 1.0])
    m0 = O.OracleModel(f_min, df, n, T_WIN)
    p[1] = 0.5 * T_WIN - O.time_of_freq(p, m0, 0.5 * (F_LO + F_HI))   # chirp centred in the window
    return p, m0


def _brute_force_spectrum(p, m0):
    """Spectra of F+(t) h(t + d(t)) and Fx(t) h(t + d(t)) at the grid bins."""
    n, df, f_min = m0.n, m0.df, m0.f_min
    fk = f_min + df * np.arange(n)
    ph = np.array([O.phase_orb_cycles(p, m0, f) for f in fk])
    x = (fk - F_LO) / (F_HI - F_LO)
    w = np.ones(n)
    lo, hi = x < TAPER, x > 1.0 - TAPER
    w[lo] = 0.5 - 0.5 * np.cos(np.pi * x[lo] / TAPER)
    w[hi] = 0.5 - 0.5 * np.cos(np.pi * (1.0 - x[hi]) / TAPER)
    ht = w * fk ** (-7.0 / 6.0) * np.exp(-2j * np.pi * (ph - np.round(ph)))
    dt = T_WIN / M_T
    tj = dt * np.arange(M_T)
    d = np.array([O.doppler_delay(p, m0, t) for t in tj])
    F = np.array([O.antenna(p, m0, t) for t in tj])
    tp = tj + d
    h = np.zeros(M_T, complex)
    kk = np.arange(n)
    for c0 in range(0, M_T, 256):
        sl = slice(c0, c0 + 256)
        arg = np.outer(tp[sl] / T_WIN, kk)
        arg -= np.round(arg)
        h[sl] = (np.exp(2j * np.pi * arg) @ ht) * df * np.exp(2j * np.pi * ((f_min * tp[sl]) % 1.0))
    het = np.exp(-2j * np.pi * ((f_min * tj) % 1.0))
    X = [np.fft.fft(F[:, c] * h * het)[:n] * dt for c in range(2)]
    flat = np.nonzero((x > TAPER + 0.08) & (x < 1.0 - TAPER - 0.08))[0]
    return X, flat


def _err(p, m0, X, flat, N, K):
    m = O.OracleModel(m0.f_min, m0.df, m0.n, m0.T_obs, mb_order=N, mb_kmax=K)
    A = O.basis(p, m, int(flat[0]), int(flat[-1]) + 1)
    out = []
    for c in range(2):
        a = A[c][flat - flat[0]]
        out.append(np.max(np.abs(X[c][flat] - a)) / np.max(np.abs(a)))
    return max(out)


@pytest.mark.parametrize("lat,lon", [(0.35, 1.1), (-0.8, 4.0)])
def test_series_converges_to_the_fourier_transform_of_the_delayed_response(lat, lon):
    p, m0 = _setup(lat, lon)
    X, flat = _brute_force_spectrum(p, m0)
    assert len(flat) > 2000
    e = {nk: _err(p, m0, X, flat, *nk) for nk in [(-1, 0), (0, 0), (1, 1), (2, 0), (2, 1)]}
    assert e[(-1, 0)] > 5e-3            # the paper's form: second-order Doppler phase missing
    assert e[(0, 0)] > 2e-3             # the full kernel G without the filter: still missing it
    assert e[(1, 1)] < 3e-4             # filter of order 1
    assert e[(2, 1)] < 3e-6             # order 2 with the k = 1 term
    assert e[(2, 0)] > 20.0 * e[(2, 1)]  # the k = 1 term (T_A1 G') matters at this level


def test_filter_weights_reproduce_the_kernel_moments():
    # the even moments of exp(i pi fdot s^2) are <s^2m> = (2m - 1)!! (i T_f^2 / pi)^m: check
    # them by quadrature along the rotated contour s = e^{i pi/4} u (a real Gaussian), then
    # the weights against them
    u = np.linspace(-12.0, 12.0, 200001)
    g = np.exp(-np.pi * u ** 2)   # fdot = 1, T_f^2 = 1/2 (unit-free check)
    Tf2 = 0.5
    for N in range(3):
        a = O.mb_weights(N)
        for mm in range(N + 1):
            mom = np.trapezoid((np.exp(1j * np.pi / 4) * u) ** (2 * mm) * g, u) / np.trapezoid(g, u)
            filt = sum(a[j] * (j * j * Tf2) ** mm if j else (a[0] if mm == 0 else 0.0) for j in range(N + 1))
            assert abs(filt - mom) < 1e-9 * max(1.0, abs(mom))
    assert O.mb_weights(0)[0] == 1.0


def test_doppler_rates_are_the_derivatives_of_the_delay():
    p = np.array([30.0, 1e7, 0.4, 2.0, 0.05, 1.0])
    m = O.OracleModel(0.01, 1e-8, 100, 7.9e7)
    for t in (0.0, 3.3e6, 2.1e7):
        h = 2.0e4
        d = [O.doppler_delay(p, m, t + k * h) for k in (-2, -1, 0, 1, 2)]
        dd_fd = (-d[4] + 8 * d[3] - 8 * d[1] + d[0]) / (12 * h)
        d2_fd = (-d[4] + 16 * d[3] - 30 * d[2] + 16 * d[1] - d[0]) / (12 * h * h)
        dd, d2 = O.doppler_rates(p, m, t)
        assert abs(dd - dd_fd) < 1e-10
        assert abs(d2 - d2_fd) < 1e-14


def test_tf_width_newtonian_closed_form():
    # t(f) = t_c - (5/256) Mc (pi Mc f)^(-8/3) at Newtonian order with e0 = 0, so
    # T_f^2 = |dt/df| / 2 = (1/2) (8/3) (5/256) Mc (pi Mc f)^(-8/3) / f
    p = np.array([25.0, 1e7, 0.1, 0.2, 0.0, 1.0])
    m = O.OracleModel(0.01, 1e-8, 100, 7.9e7, pn_order=0, mb_order=0)
    Mc = 25.0 * O_MSUN
    for f in (0.012, 0.03, 0.047):
        Tf = O.mb_response(p, m, f)[3]
        want = np.sqrt(0.5 * (8.0 / 3.0) * (5.0 / 256.0) * Mc * (np.pi * Mc * f) ** (-8.0 / 3.0) / f)
        assert abs(Tf / want - 1.0) < 1e-10


def test_series_without_response_is_the_bare_chirp():
    # test mode (F+ = 1, Fx = 0, no Doppler): G = 1 for all tau, so every order gives T = 1
    p = np.array([30.0, 3e6, 0.4, 2.0, 0.05, 1.0])
    for N in range(3):
        for K in (0, 1):
            m = O.OracleModel(0.02, 1e-7, 4096, 7.9e7, response=1, mb_order=N, mb_kmax=K)
            Tp, Tx, D0, _ = O.mb_response(p, m, 0.0201)
            assert abs(Tp - 1.0) < 1e-12 and Tx == 0.0 and D0 == 0.0

