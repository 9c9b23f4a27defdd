"""Launch variants of the fused kernel and the autotuner that picks among them.

FS_MIXED: the grid and persistent forms (2 or 3 CTAs per SM) compute the same
per-(span, particle) partial sums in the same order, so F must be bitwise
equal across the four.  FS_FP64: the tile length changes how partial sums are
grouped, so the three agree to rounding and each stays within 1e-9 of the
oracle; the anchored FP64 variants (3, 4: per-tile expansions with bounded
truncation) agree with the direct ones to 1e-10 and with the oracle to 1e-9.
The autotuner records a valid choice per (N_p, edge kind) and the plan then
uses it.
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


def rel_err(F, Fref, Np):
    ok = ~np.isnan(Fref)
    assert np.array_equal(np.isnan(F), np.isnan(Fref))
    return np.max(np.abs(F[ok] - Fref[ok]) / np.maximum(np.abs(Fref[ok]), 2.0 * Np), initial=0.0)


@pytest.fixture(scope="module")
def small_case():
    """100000 bins of the 2.5 yr grid (4 spans of 32768 bins, the last one
    ragged), 53 particles (not a multiple of the 8 warps of a CTA) whose
    bands start, end or lie inside the data; noise only."""
    g = S.tiny_grid(n=100000, f_min=0.02)
    fr = 0.02 + 50000 * g.df
    P = S.draw_params(S.Prior(tc_lo=-0.2 * g.T_obs, tc_hi=1.2 * g.T_obs), 53, 21)
    P[:, 1] = tc_for(P[:, 0], fr, P[:, 1] * 0.01)
    psd = S.lisa_like_psd(g.freqs())
    d = S.gaussian_noise(g, psd, 22)
    return g, d, psd, P


@pytest.mark.parametrize("Np", [1, 16, 256])
def test_mixed_variants_bitwise_equal(fst, small_case, Np):
    g, d, psd, P = small_case
    plan = fst.Plan.from_grid(g, mode=fst.FS_MIXED)
    plan.set_data(torch.from_numpy(d).cuda(), torch.from_numpy(psd).cuda())
    Pt = torch.from_numpy(P).cuda()
    outs = []
    assert plan.n_variants == 5
    for v in range(plan.n_variants):
        plan.set_variant(v)
        F, Fp = plan.fstat(Pt, Np)
        outs.append((F.clone(), Fp.clone()))
    torch.cuda.synchronize()
    assert plan.check() == 0          # no bounded wait of the staged form ran out
    for F, Fp in outs[1:]:
        assert torch.equal(F, outs[0][0]) and torch.equal(Fp, outs[0][1])
    Fo, _ = O.fstat_batch(P, O.OracleModel.from_grid(g), d, psd, Np)
    assert np.sum(Fo > 0) >= 10
    assert rel_err(outs[0][0].cpu().numpy(), Fo, Np) <= 1e-4
    plan.close()


@pytest.mark.parametrize("variant", [2, 4])
def test_mixed_persistent_repeats_and_empty_batches(fst, small_case, variant):
    """The persistent form resets its device-side item counter on every
    launch, and the staged form's barriers start afresh in every CTA:
    repeated calls, a batch with no in-band particle and a single particle
    (a CTA with one busy warp and seven idle ones) all come out right."""
    g, d, psd, P = small_case
    plan = fst.Plan.from_grid(g, mode=fst.FS_MIXED)
    plan.set_data(torch.from_numpy(d).cuda(), torch.from_numpy(psd).cuda())
    plan.set_variant(variant)
    Pt = torch.from_numpy(P).cuda()
    F0 = plan.fstat(Pt, 16)[0].clone()
    far = P.copy()
    far[:, 1] = -10.0 * g.T_obs           # merged long before the data: no in-band bin
    Fz = plan.fstat(torch.from_numpy(far).cuda(), 16)[0].cpu().numpy()
    assert np.all(Fz == 0.0)
    F1 = plan.fstat(Pt, 16)[0]
    assert torch.equal(F0, F1)
    one = plan.fstat(Pt[5:6].contiguous(), 16)[0]
    assert torch.equal(one, F0[5:6])
    assert plan.check() == 0
    plan.close()


@pytest.mark.parametrize("Np", [1, 16, 256])
def test_fp64_variants_match_oracle(fst, small_case, Np):
    g, d, psd, P = small_case
    plan = fst.Plan.from_grid(g, mode=fst.FS_FP64)
    plan.set_data(torch.from_numpy(d).cuda(), torch.from_numpy(psd).cuda())
    Pt = torch.from_numpy(P).cuda()
    Fo, Fpo = O.fstat_batch(P, O.OracleModel.from_grid(g), d, psd, Np)
    assert plan.n_variants == 5
    outs = []
    for v in range(plan.n_variants):
        plan.set_variant(v)
        F, Fp = plan.fstat(Pt, Np)
        outs.append((F.cpu().numpy(), Fp.cpu().numpy()))
    for v, (F, Fp) in enumerate(outs):
        assert rel_err(F, Fo, Np) <= 1e-9, v
        ok = ~np.isnan(Fpo)
        assert np.max(np.abs(Fp[ok] - Fpo[ok]) / np.maximum(np.abs(Fpo[ok]), 2.0), initial=0.0) <= 1e-9, v
        assert rel_err(F, outs[0][0], Np) <= (1e-12 if v < 3 else 1e-10), v
    # the two anchored forms compute the same sums in the same order
    assert np.array_equal(outs[3][0], outs[4][0]) and np.array_equal(outs[3][1], outs[4][1])
    plan.close()


def test_fp64_anchored_global_edges_and_injection(fst):
    """Global edges (a segment of one bin, a segment ending inside a tile) and
    an injected signal with its band inside the data."""
    g = S.tiny_grid(n=70000, f_min=0.012)
    fr = 0.012 + 35000 * g.df
    P = S.draw_params(S.Prior(tc_lo=0.0, tc_hi=g.T_obs), 24, 3)
    P[:, 1] = tc_for(P[:, 0], fr, P[:, 1] * 0.002)
    inj = P[0].copy()
    inj[1] = tc_for(inj[0], fr, 0.5 * g.T_obs)
    P[0] = inj
    psd = S.lisa_like_psd(g.freqs())
    m = O.OracleModel.from_grid(g)
    a = O.extrinsic_to_a(1.0, S.INJ_PSI, S.INJ_IOTA, S.INJ_PHIC)
    k0, k1 = O.band(inj, m)
    h = O.inject(inj, m, a, k0, k1 + 1)
    d = S.gaussian_noise(g, psd, 4) + h * (15.0 / np.sqrt(O.inner(h, h, psd, g.df)))
    plan = fst.Plan.from_grid(g, mode=fst.FS_FP64)
    plan.set_data(torch.from_numpy(d).cuda(), torch.from_numpy(psd).cuda())
    Pt = torch.from_numpy(P).cuda()
    for edges in (np.array([0, 5000, 5001, 33000, 40000, 69999], dtype=np.int64), None):
        Np = 5
        Fo, _ = O.fstat_batch(P, m, d, psd, Np, edges=edges)
        for v in (3, 4):
            plan.set_variant(v)
            F = plan.fstat(Pt, Np, edges=None if edges is None else g.edge_freqs(edges))[0].cpu().numpy()
            assert rel_err(F, Fo, Np) <= 1e-9, (v, edges is None)
        assert Fo[0] > 50.0
    plan.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_autotuner_records_choice(fst, small_case, mode):
    g, d, psd, P = small_case
    plan = fst.Plan.from_grid(g, mode=mode)
    plan.set_data(torch.from_numpy(d).cuda(), torch.from_numpy(psd).cuda())
    Pt = torch.from_numpy(P).cuda()
    default = 3 if mode == fst.FS_MIXED else 4
    assert plan.get_variant(16) == default
    v, ms = plan.autotune(Pt, 16, reps=2)
    assert 0 <= v < plan.n_variants and len(ms) == plan.n_variants
    assert all(m > 0 for m in ms) and ms[v] == min(ms)
    assert plan.get_variant(16) == v and plan.get_variant(64) == default
    assert plan.get_variant(16, global_edges=True) == default
    plan.set_variant_for(64, plan.n_variants - 1)
    assert plan.get_variant(64) == plan.n_variants - 1
    plan.set_variant(1)
    assert plan.get_variant(16) == 1
    plan.set_variant(-1)
    assert plan.get_variant(16) == v
    with pytest.raises(fst.FstatError):
        plan.set_variant(plan.n_variants)
    # the tuned plan still computes the same F as variant 0 (mixed: bitwise)
    F = plan.fstat(Pt, 16)[0].cpu().numpy()
    plan.set_variant(0)
    F0 = plan.fstat(Pt, 16)[0].cpu().numpy()
    if mode == fst.FS_MIXED:
        assert np.array_equal(F, F0)
    else:
        assert rel_err(F, F0, 16) <= 1e-10
    plan.close()


def test_fp64_anchored_paper_workload(fst):
    """Full 3,155,760-bin paper grid, B = 320, every N_p of the schedule: the
    anchored forms against the direct form (itself pinned to the oracle on
    sampled particles), and the widest-band particle against the oracle."""
    w = S.paper_workload()
    g = w.grid
    P = S.draw_params(w.prior, w.B, w.seed)
    psd = S.lisa_like_psd(g.freqs())
    d = S.gaussian_noise(g, psd, w.seed)
    plan = fst.Plan.from_grid(g, mode=fst.FS_FP64)
    plan.set_data(torch.from_numpy(d).cuda(), torch.from_numpy(psd).cuda())
    Pt = torch.from_numpy(P).cuda()
    bands = plan.bands(Pt).cpu().numpy()
    wide = int(np.argmax(bands[:, 1] - bands[:, 0]))
    m = O.OracleModel.from_grid(g)
    for Np in w.Np_list:
        out = {}
        for v in (0, 3, 4):
            plan.set_variant(v)
            out[v] = plan.fstat(Pt, Np)[0].cpu().numpy()
        assert np.array_equal(out[3], out[4])
        assert rel_err(out[3], out[0], Np) <= 1e-10, Np
        if Np == 16:
            Fo, _ = O.fstat_batch(P[wide:wide + 1], m, d, psd, Np)
            assert rel_err(out[4][wide:wide + 1], Fo, Np) <= 1e-9
            # the tiers that evaluate the phase remainder in FP32 (census modes 6, 7 and 8, antenna degree
            # 6, 5 and 4) carry most bins here, so the 1e-10 agreement above covers them
            plan.set_variant(4)
            c = plan.census(Pt, Np)
            assert c[6] + c[7] + c[8] > 0.5 * sum(c), c
    plan.close()


def test_swarm_autotune_leaves_swarm_unchanged(fst, small_case):
    g, d, psd, P = small_case
    plan = fst.Plan.from_grid(g, mode=fst.FS_MIXED)
    plan.set_data(torch.from_numpy(d).cuda(), torch.from_numpy(psd).cuda())
    box = np.zeros((2, 5, 2))
    box[:, 0] = (10.0, 50.0)
    box[:, 1] = (0.0, g.T_obs)
    box[:, 2] = (-1.0, 1.0)
    box[:, 3] = (0.0, 2.0 * np.pi)
    box[:, 4] = (0.0, 0.1)
    sw = fst.Swarm(plan, 2, 40, box)
    sw.init(5)
    before = [t.clone() for t in (sw.x, sw.v, sw.pbest_x, sw.pbest_f, sw.fit)]
    v, ms = sw.autotune(64, reps=1)
    assert 0 <= v < plan.n_variants and plan.get_variant(64) == v
    after = (sw.x, sw.v, sw.pbest_x, sw.pbest_f, sw.fit)
    for a, b in zip(before, after):
        assert torch.equal(a, b)
    plan.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_census_counts_every_in_band_bin(fst, small_case, mode):
    """fs_plan_census: the anchored kernels' per-mode counts add up to the
    in-band particle*bins of the batch (the mixed mode uses modes 1, 2 and 3
    only); the direct FP64 form has no anchors.  On the 2^15-bin aliased
    workload with 8 global segments every mixed tile is bin by bin."""
    g, d, psd, P = small_case
    plan = fst.Plan.from_grid(g, mode=mode)
    plan.set_data(torch.from_numpy(d).cuda(), torch.from_numpy(psd).cuda())
    Pt = torch.from_numpy(P).cuda()
    b = plan.bands(Pt).cpu().numpy()
    inband = int(np.maximum(b[:, 1] - b[:, 0] + 1, 0).sum())
    for Np in (1, 256):
        c = plan.census(Pt, Np)
        assert c[0] == 0 and sum(c) == inband, (Np, c)
        if mode == fst.FS_MIXED:
            assert c[4] == 0 and c[5] == 0 and c[6] == 0 and c[7] == 0 and c[8] == 0
    if mode == fst.FS_FP64:
        plan.set_variant(0)
        assert plan.census(Pt, 16) == [0] * 9
    plan.close()
    w = S.small_workload()
    g = w.grid
    Ps = S.draw_params(w.prior, 64, 5)
    psd = S.lisa_like_psd(g.freqs())
    plan = fst.Plan.from_grid(g, mode=fst.FS_MIXED)
    plan.set_data(torch.from_numpy(S.gaussian_noise(g, psd, 5)).cuda(), torch.from_numpy(psd).cuda())
    c = plan.census(torch.from_numpy(Ps).cuda(), 8, edges=g.edge_freqs(np.arange(9, dtype=np.int64) * (g.n // 8)))
    assert c[1] == 0 and c[3] == 0 and c[2] > 0
    plan.close()
