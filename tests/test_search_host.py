"""Host logic of the hierarchical search (Sec. III.B's stages), on the CPU:
sub-range and follow-up boxes, the coordinate maps, and checkpoint resume,
with the GPU part of a stage replaced by a deterministic stand-in."""
import math
import types

import numpy as np
import pytest

from paper_2407_10797_gb300 import search
from paper_2407_10797_gb300 import synth as S

PRIOR = S.Prior(Mc_lo=10.0, Mc_hi=50.0, tc_lo=0.0, tc_hi=0.5 * S.YEAR_S, e0_hi=0.1)


class StandIn(search.HierarchicalSearch):
    """PSO runs replaced by a fixed function of the stage, box and index."""
    calls = 0

    def _run_boxes(self, i, boxes, k0, k1):
        type(self).calls += 1
        win, wf = [], []
        for k in range(k0, k1):
            u = 0.1 + 0.8 * (((3 * k + i) % 7) / 6.0)
            p = search.to_physical(np.full(5, u), boxes[k], self.q)
            win.append([float(x) for x in p])
            wf.append(float(-abs(p[0] - 27.0) + 0.001 * k))
        return win, wf, 0


def make(seed=1, stages=None, ckpt=None):
    plan = types.SimpleNamespace(mode=1, stream=None)
    return StandIn(plan, PRIOR, stages or search.default_stages(10), n_boxes=6, runs_per_box=2, n_part=4,
                   seed=seed, autotune=False, checkpoint_dir=ckpt)


def test_box_around_stays_in_prior_keeps_width_and_centre():
    pb = search.prior_box(PRIOR)
    rng = np.random.default_rng(0)
    widths = (2.0, 0.01 * S.YEAR_S, 0.4, 0.4, 0.006)
    for _ in range(500):
        c = pb[:, 0] + rng.uniform(-0.1, 1.1, 5) * (pb[:, 1] - pb[:, 0])
        b = search.box_around(c, widths, pb)
        for j, w in enumerate(widths):
            if j == 3:   # periodic longitude: centred, never clipped
                assert b[j, 0] == pytest.approx(c[j] - w / 2) and b[j, 1] == pytest.approx(c[j] + w / 2)
                continue
            assert pb[j, 0] <= b[j, 0] < b[j, 1] <= pb[j, 1]
            assert b[j, 1] - b[j, 0] == pytest.approx(min(w, pb[j, 1] - pb[j, 0]), rel=1e-12)
            if pb[j, 0] + w / 2 <= c[j] <= pb[j, 1] - w / 2:
                assert 0.5 * (b[j, 0] + b[j, 1]) == pytest.approx(c[j], rel=1e-12, abs=1e-12)
    b = search.box_around(pb.mean(axis=1), (None, None, None, None, None), pb)
    assert np.array_equal(b, pb)


def test_coordinate_maps_round_trip():
    pb = search.prior_box(PRIOR)
    rng = np.random.default_rng(1)
    for _ in range(200):
        x = rng.uniform(0, 1, 5)
        p = search.to_physical(x, pb, 1.0)
        assert p[5] == 1.0 and -math.pi / 2 <= p[2] <= math.pi / 2
        y = search.to_normal_coords(p[:5])
        assert np.allclose(y, pb[:, 0] + x * (pb[:, 1] - pb[:, 0]), rtol=1e-12, atol=1e-12)


def test_stage_one_splits_tc_into_contiguous_sub_ranges():
    s1, s1b, s2 = make(seed=1), make(seed=1), make(seed=2)
    b1, b1b, b2 = s1.stage_boxes(0), s1b.stage_boxes(0), s2.stage_boxes(0)
    assert np.array_equal(b1, b1b) and not np.array_equal(b1, b2)
    pb = search.prior_box(PRIOR)
    for b in (b1, b2):
        assert b.shape == (6, 5, 2)
        assert b[0, 1, 0] == pb[1, 0] and b[-1, 1, 1] == pytest.approx(pb[1, 1], rel=1e-15)
        assert np.all(b[1:, 1, 0] == b[:-1, 1, 1]) and np.all(b[:, 1, 1] > b[:, 1, 0])
        others = np.delete(b, 1, axis=1)
        assert np.all(others == np.delete(pb, 1, axis=0)[None])


def test_follow_up_boxes_centre_on_winners_and_mirror_the_best():
    s = make()
    res = s.run(extrinsic=False)
    assert len(res["stages"]) == 4 and StandIn.calls > 0
    pb = search.prior_box(PRIOR)
    # stage 2: one box per stage-1 winner, 0.6 Msun x 0.01 yr, other coordinates the prior's
    prev = s.results[0]
    b = s.stage_boxes(1)
    for k, w in enumerate(prev.winners):
        c = search.to_normal_coords(np.array(w))
        assert b[k, 0, 1] - b[k, 0, 0] == pytest.approx(0.6)
        assert b[k, 1, 1] - b[k, 1, 0] == pytest.approx(0.01 * S.YEAR_S)
        assert np.array_equal(b[k, 2:], pb[2:]) or np.allclose(b[k, 2:], pb[2:])
        assert b[k, 0, 0] <= c[0] <= b[k, 0, 1]
    # last stage: boxes alternate between the best winner and its theta -> pi - theta mirror
    prev = s.results[2]
    best = search.to_normal_coords(np.array(prev.winners[int(np.argmax(prev.winner_f))]))
    b = s.stage_boxes(3)
    for k in range(6):
        mid = 0.5 * (b[k, 2, 0] + b[k, 2, 1])
        want = best[2] if k % 2 == 0 else -best[2]
        if abs(want) + 0.1 <= 1.0:   # not shifted by the prior edge
            assert mid == pytest.approx(want, abs=1e-12)


def test_checkpoints_resume_and_reject_another_search(tmp_path):
    StandIn.calls = 0
    first = make(ckpt=str(tmp_path)).run(extrinsic=False)
    n = StandIn.calls
    assert n == 4
    again = make(ckpt=str(tmp_path)).run(extrinsic=False)   # every stage from its checkpoint
    assert StandIn.calls == n and again == first
    with pytest.raises(ValueError):
        make(seed=9, ckpt=str(tmp_path)).run(extrinsic=False)
    with pytest.raises(ValueError):
        make(stages=search.default_stages(11), ckpt=str(tmp_path)).run(extrinsic=False)


def test_delta_mu_free_search_coordinates_and_boxes():
    """delta_mu as a sixth search coordinate: prior box [0, 0.9] (Table I),
    q = (1 + delta_mu)/(1 - delta_mu) and back, and every stage keeps
    delta_mu's full range (Sec. III.B stage 3) while narrowing the others."""
    pb = search.prior_box(PRIOR, 0.9)
    assert pb.shape == (6, 2) and list(pb[5]) == [0.0, 0.9]
    rng = np.random.default_rng(3)
    for _ in range(100):
        x = rng.uniform(0, 1, 6)
        p = search.to_physical(x, pb)
        dmu = 0.9 * x[5]
        assert p[5] == pytest.approx((1 + dmu) / (1 - dmu), rel=1e-14)
        eta = p[5] / (1 + p[5]) ** 2
        assert eta == pytest.approx((1 - dmu * dmu) / 4, rel=1e-13)
        y = search.to_normal_coords(p, 6)
        assert np.allclose(y, pb[:, 0] + x * (pb[:, 1] - pb[:, 0]), rtol=1e-12, atol=1e-12)
    widths = (0.3, 0.004 * S.YEAR_S, 0.4, 0.4, 0.006)
    c = search.to_normal_coords(search.to_physical(np.full(6, 0.5), pb), 6)
    b = search.box_around(c, widths, pb)
    assert b.shape == (6, 2) and list(b[5]) == [0.0, 0.9]
    assert b[0, 1] - b[0, 0] == pytest.approx(0.3)


def test_paper_budget_layout_per_stage():
    """The paper's own layout (Sec. III.B): 24 t_c intervals x 24 runs x 128
    particles, then 24 boxes x 8 runs around the 24 stage-1 winners, then the
    best winner and its mirror x 48 runs; iterations 8000/8000/15000 x scale."""
    st = search.paper_budget_stages(1.0)
    assert [s.Np for s in st] == [16, 16, 1]
    assert [s.n_iter for s in st] == [8000, 8000, 15000]
    assert [s.n_iter for s in search.paper_budget_stages(0.25)] == [2000, 2000, 3750]
    s = make(stages=st)
    assert [s.stage_layout(i) for i in range(3)] == [(24, 24, 128), (24, 8, 128), (2, 48, 128)]
    # a stage without its own counts takes the search's
    assert make().stage_layout(0) == (6, 2, 4)
    res = s.run(extrinsic=False)
    assert [len(r["winners"]) for r in res["stages"]] == [24, 24, 2]
    b0 = s.stage_boxes(0)
    assert b0.shape[0] == 24 and np.all(b0[1:, 1, 0] == b0[:-1, 1, 1])
    b1 = s.stage_boxes(1)
    for k, w in enumerate(s.results[0].winners):
        c = search.to_normal_coords(np.array(w))
        assert b1[k, 0, 0] <= c[0] <= b1[k, 0, 1] and b1[k, 1, 0] <= c[1] <= b1[k, 1, 1]
    assert s.stage_boxes(2).shape[0] == 2
    for world in (1, 2, 5):
        seen = []
        for rank in range(world):
            s.comm = types.SimpleNamespace(rank=rank, world=world)
            k0, k1 = s.local_boxes(2)
            seen.extend(range(k0, k1))
        assert seen == [0, 1]
    s.comm = None
