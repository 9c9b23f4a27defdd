"""Pins of the oracle's spacecraft orbits to second order in eccentricity
(Sec. IV; the orbit the paper uses is accurate to that order).

The oracle writes the orbits out as a series in e.  These tests solve
Kepler's equation numerically for the same three ellipses (semi-major axis
R, eccentricity e, inclination sqrt(3) e, perihelia 120 degrees apart in
mean anomaly) and check that the series is their expansion: its error
shrinks as e^3 (in units of R), while the first-order (rigid) form misses
by e^2; and the second-order arm lengths breathe as the exact ones do.
"""
import numpy as np

from oracle import oracle as O


def kepler_offsets(e, alpha, orient=0.0):
    """Exact positions of the three spacecraft minus the guiding centre
    (cos alpha, sin alpha, 0), in units of e R: [3, 3]."""
    iota = np.sqrt(3.0) * e
    out = np.zeros((3, 3))
    for n in range(3):
        beta = 2.0 * np.pi * n / 3.0 + orient
        M = alpha - beta
        E = M
        for _ in range(50):   # Newton on E - e sin E = M
            E -= (E - e * np.sin(E) - M) / (1.0 - e * np.cos(E))
        X, Y = np.cos(E) - e, np.sqrt(1.0 - e * e) * np.sin(E)
        xp, z = X * np.cos(iota), -X * np.sin(iota)
        pos = np.array([xp * np.cos(beta) - Y * np.sin(beta), xp * np.sin(beta) + Y * np.cos(beta), z])
        out[n] = (pos - np.array([np.cos(alpha), np.sin(alpha), 0.0])) / e
    return out


def model(ecc, orient=0.0):
    return O.OracleModel(0.01, 1e-8, 10, 7.9e7, orient=orient, ecc=ecc)


ALPHAS = np.linspace(0.0, 2.0 * np.pi, 97)[:-1]


def max_offset_error(e, ecc_model, orient=0.0):
    m = model(ecc_model, orient)
    return max(np.max(np.abs(np.array([O.sc_offset(m, n, a) for n in range(3)]) - kepler_offsets(e, a, orient)))
               for a in ALPHAS)


def test_second_order_series_is_the_expansion_of_the_kepler_orbits():
    for orient in (0.0, 0.7):
        e1, e2 = 0.01, 0.02
        err1, err2 = max_offset_error(e1, e1, orient), max_offset_error(e2, e2, orient)
        # error in units of e R is O(e^2) (positions O(e^3) R: 3.67 e^3 R at most), quadrupling
        # when e doubles
        assert err1 < 4.0 * e1 ** 2 and err2 < 4.0 * e2 ** 2
        assert 3.9 < err2 / err1 < 4.1
        # the first-order (rigid) form misses the e^2 R terms: O(e) in units of e R (3.46 e)
        assert max_offset_error(e1, 0.0, orient) > 3.0 * e1


def test_lisa_eccentricity_error_and_breathing_arms():
    e = 2.5e9 / (2.0 * np.sqrt(3.0) * 1.495978707e11)   # arm length 2.5 Gm at 1 AU
    assert max_offset_error(e, e) < 4.0 * e ** 2
    m = model(e)
    lens_model, lens_exact = [], []
    for a in ALPHAS:
        r = np.array([O.sc_offset(m, n, a) for n in range(3)])
        x = kepler_offsets(e, a)
        for i, j in ((0, 1), (1, 2), (2, 0)):
            lens_model.append(np.linalg.norm(r[i] - r[j]))
            lens_exact.append(np.linalg.norm(x[i] - x[j]))
    lens_model, lens_exact = np.array(lens_model), np.array(lens_exact)
    # first order: all arms 2 sqrt(3) e R; the second order makes them breathe by O(e)
    assert abs(lens_model.mean() / (2.0 * np.sqrt(3.0)) - 1.0) < 5.0 * e
    swing = (lens_model.max() - lens_model.min()) / lens_model.mean()
    assert 0.5 * e < swing < 10.0 * e
    assert np.max(np.abs(lens_model - lens_exact)) < 10.0 * e ** 2
    r0 = np.array([O.sc_offset(model(0.0), n, 0.4) for n in range(3)])
    assert np.allclose([np.linalg.norm(r0[i] - r0[j]) for i, j in ((0, 1), (1, 2), (2, 0))], 2.0 * np.sqrt(3.0),
                       rtol=0, atol=1e-14)


def test_detector_tends_to_the_rigid_one_and_moves_by_order_e():
    e = 0.0048
    p = np.array([30.0, 1e7, 0.4, 2.0, 0.05, 1.0])
    dmax = 0.0
    for t in np.linspace(0.0, 3.15e7, 23):
        D0 = O.detector_tensor(model(0.0), t)
        Dtiny = O.detector_tensor(model(1e-12), t)
        assert np.max(np.abs(Dtiny - D0)) < 1e-11
        De = O.detector_tensor(model(e), t)
        assert abs(np.trace(De)) < 1e-14 and np.allclose(De, De.T, atol=0)
        dmax = max(dmax, np.max(np.abs(De - D0)))
        Fp0, Fx0 = O.antenna(p, model(0.0), t)
        Fpe, Fxe = O.antenna(p, model(e), t)
        assert abs(Fpe - Fp0) < 10.0 * e and abs(Fxe - Fx0) < 10.0 * e
    assert 0.1 * e < dmax < 10.0 * e
