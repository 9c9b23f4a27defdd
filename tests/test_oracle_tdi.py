"""Pins of the oracle's finite-arm TDI response (Sec. IV: a TDI combination is
a sum of time-delayed single-arm responses).

The brute-force pin simulates the first-generation Michelson X in the time
domain from its definition: every link s -> r carries
y_sr(t) = n.H(t - L - k.x_s).n - n.H(t - k.x_r).n over 2 (1 - k.n), the wave
H = h e_A with h(t) the exact inverse DFT of a tapered chirp, evaluated at
each retarded time by the band-limited Fourier sum; the Michelson is
y_12(t - L) + y_21(t) - y_13(t - L) - y_31(t); its FFT divided by -4 pi i f L
must equal the oracle's A1 = T+ h0 (A2 = Tx h0).  At 52 mHz (pi f L = 1.4) the
long-wavelength form misses it at order one.  On the orbits to second order
in eccentricity the three vertex Michelsons, each arm delayed by its own
length, combine into X, A, E and T, which the oracle's channels must match.
The Doppler delay is switched off on both sides so that the arm transfer is
tested alone.
"""
import numpy as np

from oracle import oracle as O

T_WIN = 2.0 ** 20
M_T = 8192
F_LO, F_HI = 0.0515, 0.0550
TAPER = 0.12
L_ARM = 2.5e9 / 299792458.0     # s


def _setup():
    df = 1.0 / T_WIN
    kmin, kmax = int(F_LO / df), int(F_HI / df)
    f_min = kmin * df
    n = kmax - kmin
    p = np.array([50.0, 0.0, 0.35, 1.1, 0.0, 1.0])
    m0 = O.OracleModel(f_min, df, n, T_WIN, no_doppler=1)
    p[1] = 0.5 * T_WIN - O.time_of_freq(p, m0, 0.5 * (F_LO + F_HI))
    return p, m0


def _michelson_spectra(p, m0, vertices=(0,), ecc=0.0):
    """Spectra of the vertex Michelsons R_v (v in `vertices`) simulated in the time
    domain, per polarisation, divided by -4 pi i f L; the spacecraft on the orbits
    of eccentricity `ecc` (0: rigid), every arm delay its own length."""
    n, df, f_min = m0.n, m0.df, m0.f_min
    fk = f_min + df * np.arange(n)
    ph = np.array([O.phase_orb_cycles(p, m0, f) for f in fk])
    x = (fk - F_LO) / (F_HI - F_LO)
    w = np.ones(n)
    lo, hi = x < TAPER, x > 1.0 - TAPER
    w[lo] = 0.5 - 0.5 * np.cos(np.pi * x[lo] / TAPER)
    w[hi] = 0.5 - 0.5 * np.cos(np.pi * (1.0 - x[hi]) / TAPER)
    ht = w * fk ** (-7.0 / 6.0) * np.exp(-2j * np.pi * (ph - np.round(ph)))
    kk = np.arange(n)

    def h_at(tt):
        out = np.zeros(tt.size, complex)
        for c0 in range(0, tt.size, 512):
            sl = slice(c0, c0 + 512)
            arg = np.outer(tt[sl] / T_WIN, kk)
            arg -= np.round(arg)
            out[sl] = (np.exp(2j * np.pi * arg) @ ht) * df * np.exp(2j * np.pi * ((f_min * tt[sl]) % 1.0))
        return out

    dt = T_WIN / M_T
    tj = dt * np.arange(M_T)
    sb, cb, sl_, cl = np.sin(p[2]), np.cos(p[2]), np.sin(p[3]), np.cos(p[3])
    pv, qv = np.array([sb * cl, sb * sl_, -cb]), np.array([-sl_, cl, 0.0])
    k = -np.array([cb * cl, cb * sl_, sb])
    ep, ex = np.outer(pv, pv) - np.outer(qv, qv), np.outer(pv, qv) + np.outer(qv, pv)
    # spacecraft offsets (seconds) at every sample time
    mo = O.OracleModel(m0.f_min, m0.df, m0.n, m0.T_obs, ecc=ecc)
    pos = np.zeros((M_T, 3, 3))
    for j, t in enumerate(tj):
        a = 2.0 * np.pi * t / 31557600.0
        for i in range(3):
            pos[j, i] = O.sc_offset(mo, i, a) * L_ARM / (2.0 * np.sqrt(3.0))

    def link(s, r, delayed):
        """y_sr per polarisation (constellation at the sample time), received at t,
        or one arm length L_sr(t) earlier when `delayed`."""
        d = pos[:, r] - pos[:, s]
        Ls = np.linalg.norm(d, axis=1)
        t_rx = tj - Ls if delayed else tj
        nv = d / Ls[:, None]
        kn = nv @ k
        h_emit = h_at(t_rx - Ls - pos[:, s] @ k)
        h_recv = h_at(t_rx - pos[:, r] @ k)
        out = []
        for e in (ep, ex):
            q = np.einsum("ti,ij,tj->t", nv, e, nv)
            out.append(q * (h_emit - h_recv) / (2.0 * (1.0 - kn)))
        return out

    het = np.exp(-2j * np.pi * ((f_min * tj) % 1.0))
    spectra = {}
    for v in vertices:
        a_, b_ = (v + 1) % 3, (v + 2) % 3
        yva, yav = link(v, a_, True), link(a_, v, False)
        yvb, ybv = link(v, b_, True), link(b_, v, False)
        out = []
        for A in range(2):
            R = yva[A] + yav[A] - yvb[A] - ybv[A]
            Rf = np.fft.fft(R * het)[:n] * dt
            out.append(Rf / (-4j * np.pi * fk * L_ARM))
        spectra[v] = out
    flat = np.nonzero((x > TAPER + 0.08) & (x < 1.0 - TAPER - 0.08))[0]
    return spectra, flat


def _max_rel(X, A, flat):
    e = 0.0
    for c in range(2):
        a = A[c][flat - flat[0]]
        e = max(e, np.max(np.abs(X[c][flat] - a)) / np.max(np.abs(a)))
    return e


def test_finite_arm_response_is_the_fourier_transform_of_the_delayed_links():
    p, m0 = _setup()
    R, flat = _michelson_spectra(p, m0)
    errs = {}
    for name, arm in (("finite", L_ARM), ("long-wavelength", 0.0)):
        m = O.OracleModel(m0.f_min, m0.df, m0.n, m0.T_obs, no_doppler=1, arm_s=arm)
        A = O.basis(p, m, int(flat[0]), int(flat[-1]) + 1)
        errs[name] = _max_rel(R[0], A, flat)
    assert errs["finite"] < 3e-5           # 7.5e-6 measured: the constellation frozen at t_f
    assert errs["long-wavelength"] > 0.1


def test_finite_arm_channels_on_eccentric_orbits_are_the_delayed_links():
    """All three vertex Michelsons on the orbits to second order in LISA's
    eccentricity (unequal, breathing arms, each delay its own length), combined
    into X, A = (Z - X)/sqrt2, E = (X - 2Y + Z)/sqrt6 and T = (X + Y + Z)/sqrt3:
    the oracle's channels with the same orbit match them (measured 7.4e-6, 2.6e-5,
    1.0e-5, 4.2e-5 of each channel's scale: the constellation frozen at t_f),
    while the rigid orbit's channels miss by 4e-3 to 4e-2.  T, zero in the
    long-wavelength limit, is as large as X at pi f L = 1.4."""
    p, m0 = _setup()
    ecc = 2.5e9 / (2.0 * np.sqrt(3.0) * 1.495978707e11)
    R, flat = _michelson_spectra(p, m0, vertices=(0, 1, 2), ecc=ecc)
    X, Y, Z = R[0], R[1], R[2]
    chans = {0: X,
             1: [(Z[c] - X[c]) / np.sqrt(2.0) for c in range(2)],
             2: [(X[c] - 2.0 * Y[c] + Z[c]) / np.sqrt(6.0) for c in range(2)],
             3: [(X[c] + Y[c] + Z[c]) / np.sqrt(3.0) for c in range(2)]}
    scale = {}
    for ch, sim in chans.items():
        m = O.OracleModel(m0.f_min, m0.df, m0.n, m0.T_obs, no_doppler=1, arm_s=L_ARM, ecc=ecc, channel=ch)
        A = O.basis(p, m, int(flat[0]), int(flat[-1]) + 1)
        assert _max_rel(sim, A, flat) < (3e-5 if ch == 0 else 1e-4), ch
        scale[ch] = max(np.max(np.abs(A[c])) for c in range(2))
        # the rigid orbit's channel misses it: the e^2 terms matter at this bar
        mr = O.OracleModel(m0.f_min, m0.df, m0.n, m0.T_obs, no_doppler=1, arm_s=L_ARM, channel=ch)
        assert _max_rel(sim, O.basis(p, mr, int(flat[0]), int(flat[-1]) + 1), flat) > 2e-3, ch
    assert scale[3] > 0.5 * scale[0]


def _long_wavelength(p, m, t):
    """Limit f L -> 0 of the Michelsons, arm lengths kept: D_v = (L_a a a - L_b b b) / (2 L),
    combined into the model's channel, projected on e+ and ex."""
    a_ = 2.0 * np.pi * t / 31557600.0
    x = np.array([O.sc_offset(m, i, a_) for i in range(3)]) * L_ARM / (2.0 * np.sqrt(3.0))
    D = []
    for v in range(3):
        u = x[(v + 1) % 3] - x[v]
        w = x[(v + 2) % 3] - x[v]
        D.append((np.outer(u, u) / np.linalg.norm(u) - np.outer(w, w) / np.linalg.norm(w)) / (2.0 * L_ARM))
    D = {0: D[0], 1: (D[2] - D[0]) / np.sqrt(2.0), 2: (D[0] - 2.0 * D[1] + D[2]) / np.sqrt(6.0)}[m.channel]
    sb, cb, sl, cl = np.sin(p[2]), np.cos(p[2]), np.sin(p[3]), np.cos(p[3])
    pv, qv = np.array([sb * cl, sb * sl, -cb]), np.array([-sl, cl, 0.0])
    return np.sum(D * (np.outer(pv, pv) - np.outer(qv, qv))), np.sum(D * (np.outer(pv, qv) + np.outer(qv, pv)))


def test_finite_arm_response_tends_to_the_long_wavelength_patterns():
    p = np.array([30.0, 1e7, -0.4, 5.0, 0.05, 1.0])
    for channel in (0, 1, 2):
        for ecc in (0.0, 0.0048):
            m = O.OracleModel(0.01, 1e-8, 10, 7.9e7, channel=channel, ecc=ecc, arm_s=L_ARM)
            m0 = O.OracleModel(0.01, 1e-8, 10, 7.9e7, channel=channel, ecc=ecc)
            for t in (0.0, 1.1e7, 2.5e7):
                Tp, Tx = O.tdi_response(p, m, 1e-9, t)
                Fp, Fx = _long_wavelength(p, m, t)
                assert abs(Tp - Fp) < 1e-7 and abs(Tx - Fx) < 1e-7
                if ecc == 0.0:   # equal arms: the unit-vector pattern of the long-wavelength response
                    Gp, Gx = O.antenna(p, m0, t)
                    assert abs(Fp - Gp) < 1e-12 and abs(Fx - Gx) < 1e-12
                # the first correction is a phase of order 2 pi f times the vertex offset
                Tp3, _ = O.tdi_response(p, m, 1e-4, t)
                assert 1e-6 < abs(Tp3 - Fp) < 1e-2
