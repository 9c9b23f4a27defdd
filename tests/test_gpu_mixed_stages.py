"""Mixed-precision mode, stage by stage, on the 2.5-yr paper grid.

Every stage of the FS_MIXED body is compared, bin by bin, with an FP64
evaluation of the same quantity:

  orb     fixed-point cubic phase polynomial (orbital phase minus the
          anchor's Doppler phase)        vs the oracle's long-double phase
  dalpha  orbital-phase offset from the anchor, quadratic in the bin offset
                                         vs 2 pi (t(f_k) - t(f_a)) / yr, oracle t(f)
  dop     Doppler polynomial (FP32)      vs f_k d(t_k) - f_a d(t_a), oracle delay
  ph      phase fed to sincos            vs the oracle's total phase mod 1
  G1, G2  antenna polynomials (FP32, FP64 constant terms)
                                         vs the oracle's vector-geometry F+, Fx
                                            rotated by the segment's (c, s)
  sincos  SFU __sincosf                  vs FP64 cos, sin of the same FP32 phase
  tables  FP32 dw, W                     vs FP64 4 df d f^-7/6 / S, 4 df f^-7/3 / S
  terms   FP32 products                  vs FP64 products of the same FP32 inputs
  sums    compensated FP32 sums (F_p of the production kernel)
                                         vs FP64 sums of the kernel's own terms
  F       the production F_p             vs the FP64 mode and the oracle

fs_mixed_probe returns the values the production per-bin code feeds into the
sums (Sec. II.B segment inner product).  Each stage's bound is the one the
design states for it (validity limits of the anchor expansions, unit
roundoff u = 2^-24 of the FP32 steps, the SFU's absolute error); the
measured maxima are printed (run with -s) for the precision table.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2407_10797_gb300 import synth as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
N_SAMPLE = 6000          # bins per probed particle compared with the oracle bin by bin
NP_LIST = (256, 64, 16, 1)


def wrap(x):
    return x - np.rint(x)


@pytest.fixture(scope="module")
def fst():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_10797_gb300 import fstat
    fstat.load()
    return fstat


@pytest.fixture(scope="module")
def setup(fst):
    """Paper grid, noise + an injection at SNR 12.5; three probed particles
    with long bands (the injection among them) inside a 320-particle batch."""
    w = S.paper_workload()
    g = w.grid
    P = S.draw_params(w.prior, w.B, w.seed)
    m = O.OracleModel.from_grid(g)
    psd = S.lisa_like_psd(g.freqs())
    plan = fst.Plan.from_grid(g, mode=fst.FS_MIXED)
    d = S.gaussian_noise(g, psd, 3)
    plan.set_data(torch.from_numpy(d).cuda(), torch.from_numpy(psd).cuda())
    bands = plan.bands(torch.from_numpy(P).cuda()).cpu().numpy()
    nb = bands[:, 1] - bands[:, 0] + 1
    order = np.argsort(-nb)
    probe = [int(i) for i in order[[0, 5, 20]]]
    inj = probe[0]
    a = O.extrinsic_to_a(1.0, S.INJ_PSI, S.INJ_IOTA, S.INJ_PHIC)
    k0, k1 = bands[inj]
    h = O.inject(P[inj], m, a, int(k0), int(k1) + 1)
    d = d + h * (12.5 / math.sqrt(O.inner(h, h, psd, g.df)))
    plan.set_data(torch.from_numpy(d).cuda(), torch.from_numpy(psd).cuda())
    yield dict(g=g, P=P, m=m, d=d, psd=psd, plan=plan, bands=bands, probe=probe)
    plan.close()


def probe_records(fst, st, b, Np):
    plan, P, bands = st["plan"], st["P"], st["bands"]
    k0, k1 = int(bands[b, 0]), int(bands[b, 1]) + 1
    rec = plan.mixed_probe(torch.from_numpy(P).cuda(), Np, b, k0, k1 - k0).cpu().numpy().astype(np.float64)
    F = fst.Plan.PROBE_FIELDS
    return k0, {name: rec[:, i] for i, name in enumerate(F)}


def segment_F_from_terms(r, Np):
    """F_p from FP64 sums of the kernel's per-bin terms (the solve of the
    reduction kernel: 2x2 Gram matrix in the rotated basis, c9 rule)."""
    seg = r["seg"].astype(np.int64)
    ok = r["mode"] > 0
    Fp = np.zeros(Np)
    for p in range(Np):
        sel = ok & (seg == p)
        nb = int(sel.sum())
        if nb < 4:
            continue
        S7 = [np.sum(r[f"t{c}"][sel]) for c in range(7)]
        X1r, X1i, X2r, X2i, K11, K12, K22 = S7
        det = K11 * K22 - K12 * K12
        c = r["rot_c"][sel][0] + r["rot_c_lo"][sel][0]
        s = r["rot_s"][sel][0] + r["rot_s_lo"][sel][0]
        Pp = c * c * K11 - 2 * c * s * K12 + s * s * K22
        Rr = s * s * K11 + 2 * c * s * K12 + c * c * K22
        if det > 1e-12 * Pp * Rr:
            Fp[p] = 0.5 * (K22 * (X1r ** 2 + X1i ** 2) - 2 * K12 * (X1r * X2r + X1i * X2i)
                           + K11 * (X2r ** 2 + X2i ** 2)) / det
    return Fp


def test_mixed_stage_errors_against_fp64(fst, setup):
    st = setup
    g, P, m = st["g"], st["P"], st["m"]
    f = g.freqs()
    yr = S.YEAR_S
    om = 2.0 * np.pi / yr
    rows = {}
    low_share = []
    rng = np.random.default_rng(1)

    def note(name, val):
        rows[name] = max(rows.get(name, 0.0), float(val))

    # per-bin template stages: N_p independent (use N_p = 16 for the rotation)
    for b in st["probe"]:
        k0, r = probe_records(fst, st, b, 16)
        poly = np.nonzero(np.isin(r["mode"], (1, 3)))[0]
        assert poly.size > 0.9 * r["mode"].size      # the paper grid runs the FP32 body
        low_share.append(float(np.mean(r["mode"][poly] == 3)))   # low-degree tier (mode 3)
        idx = rng.choice(poly, size=min(N_SAMPLE, poly.size), replace=False)
        p = P[b]
        for i in idx:
            k = k0 + int(i)
            ka = int(r["k_anchor"][i])
            fk, fa = f[k], f[ka]
            tk, ta = O.time_of_freq(p, m, fk), O.time_of_freq(p, m, fa)
            dk, da = O.doppler_delay(p, m, tk), O.doppler_delay(p, m, ta)
            ph = O.phase_frac(p, m, k)                  # orb(f_k) - f_k d_k, mod 1
            orb = wrap(ph + fk * dk - fa * da)           # orb(f_k) - f_a d_a, mod 1
            note("orb_cycles", abs(wrap(r["orb"][i] - orb)))
            note("dalpha_rad", abs(r["dalpha"][i] - om * (tk - ta)))
            note("dop_cycles", abs(r["dop"][i] - (fk * dk - fa * da)))
            note("ph_cycles", abs(wrap(r["ph"][i] - ph)))
            Fp, Fx = O.antenna(p, m, tk)
            c = r["rot_c"][i] + r["rot_c_lo"][i]
            s = r["rot_s"][i] + r["rot_s_lo"][i]
            scale = math.hypot(Fp, Fx)
            note("G_rel", max(abs(r["G1"][i] - (c * Fp + s * Fx)), abs(r["G2"][i] - (c * Fx - s * Fp))) / scale)
        # SFU sincos against FP64 of the same FP32 phase
        ph32 = r["ph"][poly]
        note("sincos_abs", np.max(np.abs(r["cos"][poly] - np.cos(2 * np.pi * ph32))))
        note("sincos_abs", np.max(np.abs(r["sin"][poly] - np.sin(2 * np.pi * ph32))))
        # FP32 tables against the FP64 tables (scaled by one power of two)
        kk = k0 + poly
        dw = 4.0 * g.df * st["d"][kk] * f[kk] ** (-7.0 / 6.0) / st["psd"][kk]
        W = 4.0 * g.df * f[kk] ** (-7.0 / 3.0) / st["psd"][kk]
        sW = np.exp2(np.rint(np.log2(np.median(r["tw_W"][poly] / W))))
        sd = math.sqrt(sW)
        note("table_rel", np.max(np.abs(r["tw_W"][poly] - W * sW) / (W * sW)))
        note("table_rel", np.max(np.abs(r["tw_re"][poly] - dw.real * sd) / np.abs(dw * sd)))
        note("table_rel", np.max(np.abs(r["tw_im"][poly] - dw.imag * sd) / np.abs(dw * sd)))
        # FP32 products against FP64 products of the same FP32 inputs
        x, y, Wt = r["tw_re"][poly], r["tw_im"][poly], r["tw_W"][poly]
        cs, sn, G1, G2 = r["cos"][poly], r["sin"][poly], r["G1"][poly], r["G2"][poly]
        zr, zi = x * cs - y * sn, x * sn + y * cs
        zabs = np.abs(x * cs) + np.abs(y * sn) + np.abs(x * sn) + np.abs(y * cs)
        ref = [G1 * zr, G1 * zi, G2 * zr, G2 * zi, Wt * G1 * G1, Wt * G1 * G2, Wt * G2 * G2]
        mag = [np.abs(G1) * zabs, np.abs(G1) * zabs, np.abs(G2) * zabs, np.abs(G2) * zabs,
               Wt * G1 * G1, Wt * np.abs(G1 * G2), Wt * G2 * G2]
        for c in range(7):
            tiny = mag[c] > 0
            note("term_rel", np.max(np.abs(r[f"t{c}"][poly][tiny] - ref[c][tiny]) / mag[c][tiny]))

    # sums: production F_p (compensated FP32 sums) against F_p from FP64 sums of
    # the same per-bin terms, and both against the FP64 mode and the oracle
    Pt = torch.from_numpy(P).cuda()
    fp64 = fst.Plan.from_grid(g, mode=fst.FS_FP64)
    fp64.set_data(torch.from_numpy(st["d"]).cuda(), torch.from_numpy(st["psd"]).cuda())
    sel = np.array(st["probe"])
    Fo_all = {}
    for Np in NP_LIST:
        _, Fpm = st["plan"].fstat(Pt, Np)
        _, Fpd = fp64.fstat(Pt, Np)
        Fpm, Fpd = Fpm.cpu().numpy(), Fpd.cpu().numpy()
        _, Fpo = O.fstat_batch(P[sel], m, st["d"], st["psd"], Np)
        Fo_all[Np] = Fpo
        for j, b in enumerate(st["probe"]):
            _, r = probe_records(fst, st, b, Np)
            Fterm = segment_F_from_terms(r, Np)
            den = np.maximum(np.abs(Fpd[b]), 2.0)
            note(f"sums_F_rel_Np{Np}", np.max(np.abs(Fpm[b] - Fterm) / den))
            note(f"F_vs_fp64_Np{Np}", np.max(np.abs(Fpm[b] - Fpd[b]) / den))
            note(f"F_vs_oracle_Np{Np}", np.max(np.abs(Fpm[b] - Fpo[j]) / np.maximum(np.abs(Fpo[j]), 2.0)))
            note(f"fp64_vs_oracle_Np{Np}", np.max(np.abs(Fpd[b] - Fpo[j]) / np.maximum(np.abs(Fpo[j]), 2.0)))
    fp64.close()

    print("\nshare of polynomial bins in the low-degree tier per probed particle:", low_share)
    print("\nFS_MIXED stage errors (max over probed bins / segments):")
    for k in sorted(rows):
        print(f"  {k:28s} {rows[k]:.3e}")

    # the paper grid's tiles are mostly short in d(alpha): the low-degree tier carries many of them
    assert min(low_share) > 0.25
    # bounds the design states for each stage
    assert rows["orb_cycles"] <= 2e-6        # quartic remainder <= 1e-6 cycle, 2^-32 steps, FP32 rendering
    assert rows["dalpha_rad"] <= 2e-6        # cubic t(f) remainder <= 1e-6 rad, FP32
    assert rows["dop_cycles"] <= 3e-5        # <= max f AD (25 cycles/rad) x d(alpha) bound + FP32 polynomial
    assert rows["ph_cycles"] <= 3.5e-5
    assert rows["G_rel"] <= 5e-6             # antenna harmonics <= 4: |dF/dalpha| <= 4 |F| x d(alpha) bound
    assert rows["sincos_abs"] <= 6e-7        # SFU 2^-21.4 plus the FP32 product 2 pi ph
    assert rows["table_rel"] <= 0.51 * 2 * U32   # one rounding to FP32
    assert rows["term_rel"] <= 4 * U32       # <= 3 FP32 roundings per term
    for Np in NP_LIST:
        assert rows[f"F_vs_oracle_Np{Np}"] <= 1e-4       # the mixed-mode bar
        assert rows[f"fp64_vs_oracle_Np{Np}"] <= 1e-9    # the FP64 bar
        assert rows[f"sums_F_rel_Np{Np}"] <= 1e-5
