"""Hierarchical search controller (Sec. III.B): stages of PSO runs over
search boxes, each stage narrowing the boxes around the previous winners.

All runs of a stage -- n_boxes boxes x runs_per_box runs x n_part particles,
each run with its own box -- are one swarm on the device, so one PSO iteration
is one batched F-statistic launch; the iteration (map, F-statistic, fitness,
update) is captured once as a CUDA graph and replayed n_iter times.  The host
only builds boxes and picks best-of-runs winners between stages.

Stage layout (the paper's three stages, Sec. III.B, generalised to the
four-stage N_p = 256 -> 64 -> 16 -> 1 schedule with a fixed number of boxes
per stage):
  stage 1: the t_c prior split into n_boxes contiguous intervals of uneven
           (Dirichlet) widths, every other parameter over its full prior;
  stage 2: boxes centred on the stage-1 winners, narrowed in t_c and M_c;
  stage 3: boxes centred on the stage-2 winners, narrowed in every parameter;
  stage 4: boxes centred on the best stage-3 winner and on its mirror image
           in ecliptic latitude (theta -> pi - theta, Sec. III.B stage 3),
           fully coherent (N_p = 1).
Best-of-runs and ties: the run with the largest fitness, lowest index first.
"""
from __future__ import annotations

import json
import math
import os
import time
from dataclasses import asdict, dataclass, field

import numpy as np

from . import fstat
from . import synth as S

YEAR = S.YEAR_S


@dataclass
class StageSpec:
    Np: int
    n_iter: int
    rule: str                      # "split_tc" | "around" | "around_best_mirror"
    widths: tuple = ()             # full widths (M_c [Msun], t_c [s], sin(lat), lon [rad], e0); None = prior
    w0: float = 0.9
    w1: float = 0.4
    boxes: int | None = None       # boxes, runs per box and particles per run of this stage
    runs: int | None = None        # (None: the search's n_boxes, runs_per_box, n_part)
    particles: int | None = None


def default_stages(n_iter: int = 2000) -> list[StageSpec]:
    """Widths follow the paper's stage 2 (0.01 yr, 0.6 Msun) and stage 3
    (0.004 yr, 0.3 Msun, 0.4 rad, 0.4 rad, 0.006) boxes; stage 4 halves stage 3."""
    return [
        StageSpec(256, n_iter, "split_tc"),
        StageSpec(64, n_iter, "around", (0.6, 0.01 * YEAR, None, None, None)),
        StageSpec(16, n_iter, "around", (0.3, 0.004 * YEAR, 0.4, 0.4, 0.006)),
        StageSpec(1, n_iter, "around_best_mirror", (0.15, 0.002 * YEAR, 0.2, 0.2, 0.003)),
    ]


def paper_stages(n_iter: int = 2000) -> list[StageSpec]:
    """The paper's three stages (Sec. III.B): N_seg = 16 over t_c sub-ranges;
    N_seg = 16 in boxes of 0.01 yr x 0.6 Msun around the stage-1 winners;
    N_seg = 1 in a box of 0.004 yr, 0.3 Msun, 0.4 rad, 0.4 rad, 0.006 around
    the best winner and its theta -> pi - theta mirror."""
    return [
        StageSpec(16, n_iter, "split_tc"),
        StageSpec(16, n_iter, "around", (0.6, 0.01 * YEAR, None, None, None)),
        StageSpec(1, n_iter, "around_best_mirror", (0.3, 0.004 * YEAR, 0.4, 0.4, 0.006)),
    ]


def paper_budget_stages(scale: float = 1.0) -> list[StageSpec]:
    """The paper's three stages with its own layout and budget (Sec. III.B):
    stage 1, N_seg = 16, the t_c range in 24 intervals x 24 PSO runs of 128
    particles, 8000 iterations; stage 2, N_seg = 16, 24 boxes (0.01 yr x 0.6
    Msun) around the stage-1 winners x 8 runs, 8000 iterations; stage 3,
    N_seg = 1, the best winner's box (0.004 yr, 0.3 Msun, 0.4 rad, 0.4 rad,
    0.006) and its theta -> pi - theta mirror x 48 runs, 15000 iterations.
    scale multiplies every iteration count."""
    it = lambda n: max(2, int(round(n * scale)))
    return [
        StageSpec(16, it(8000), "split_tc", boxes=24, runs=24, particles=128),
        StageSpec(16, it(8000), "around", (0.6, 0.01 * YEAR, None, None, None), boxes=24, runs=8, particles=128),
        StageSpec(1, it(15000), "around_best_mirror", (0.3, 0.004 * YEAR, 0.4, 0.4, 0.006), boxes=2, runs=48,
                  particles=128),
    ]


def prior_box(prior: S.Prior, dmu_hi: float = 0.0) -> np.ndarray:
    """Search box of the prior in search coordinates (M_c, t_c, sin(lat), lon,
    e0), with a sixth row [0, dmu_hi] for delta_mu when dmu_hi > 0."""
    rows = [[prior.Mc_lo, prior.Mc_hi], [prior.tc_lo, prior.tc_hi], [-1.0, 1.0], [0.0, 2.0 * np.pi],
            [0.0, prior.e0_hi]]
    if dmu_hi > 0.0:
        rows.append([0.0, dmu_hi])
    return np.array(rows)


def q_of_dmu(dmu: float) -> float:
    """Mass ratio m1/m2 of the dimensionless mass difference (m1 - m2)/M."""
    return (1.0 + dmu) / (1.0 - dmu)


def to_physical(xn: np.ndarray, box: np.ndarray, q: float = 1.0) -> np.ndarray:
    """Normalised position [D] in box [D, 2] -> (M_c, t_c, lat, lon, e0, q);
    with D = 6 the sixth coordinate is delta_mu and fixes q."""
    y = box[:, 0] + xn * (box[:, 1] - box[:, 0])
    qq = q_of_dmu(y[5]) if len(y) == 6 else q
    return np.array([y[0], y[1], math.asin(max(-1.0, min(1.0, y[2]))), y[3], y[4], qq])


def to_normal_coords(p: np.ndarray, dims: int = 5) -> np.ndarray:
    """(M_c, t_c, lat, lon, e0, q) -> the search coordinates (M_c, t_c,
    sin(lat), lon, e0), with delta_mu = (q - 1)/(q + 1) sixth when dims = 6."""
    c = [p[0], p[1], math.sin(p[2]), p[3], p[4]]
    if dims == 6:
        c.append((p[5] - 1.0) / (p[5] + 1.0))
    return np.array(c)


def box_around(center: np.ndarray, widths, prior: np.ndarray) -> np.ndarray:
    """Box of the given full widths centred on `center` (search coordinates),
    shifted to stay inside the prior; None keeps the prior range."""
    b = prior.copy()
    for j, wj in enumerate(widths):
        if wj is None or j >= len(b):
            continue
        lo, hi = center[j] - 0.5 * wj, center[j] + 0.5 * wj
        if j == 3:   # longitude is periodic: no clipping
            b[j] = [lo, hi]
            continue
        if lo < prior[j, 0]:
            lo, hi = prior[j, 0], min(prior[j, 1], prior[j, 0] + wj)
        if hi > prior[j, 1]:
            lo, hi = max(prior[j, 0], prior[j, 1] - wj), prior[j, 1]
        b[j] = [lo, hi]
    return b


@dataclass
class SurrogateSpec:
    """Surrogate screening of PSO moves (not in the paper): every exact
    evaluation adds its (position, F-hat) pairs to its box's ring of `buffer`
    samples (the latest ones: about six iterations of a box's 8 x 40
    particles at the default), each box's MLP is retrained every
    `train_every` iterations for `train_steps` full-ring Adam steps, and after
    `warm` iterations each particle takes the best of `n_cand` candidate moves
    as ranked by its box's network.  The number of exact F-statistic
    evaluations is unchanged."""
    n_cand: int = 16
    warm: int = 20
    train_every: int = 10
    train_steps: int = 20
    lr: float = 1e-3
    buffer: int = 2048
    width: int = 256


@dataclass
class StageResult:
    stage: int
    Np: int
    boxes: list
    winners: list          # physical parameters of the best run of every box
    winner_f: list         # their fitness (F-hat)
    seconds: float
    variant: int = -1      # launch variant of the fused kernel this stage used


class Comm:
    """The search's only exchange between processes: gathering every
    process's box winners at the end of a stage (torch.distributed, any
    backend; objects of a few KB)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self._dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def allgather(self, obj) -> list:
        out = [None] * self.world
        self._dist.all_gather_object(out, obj, group=self.group)
        return out


class HierarchicalSearch:
    def __init__(self, plan: "fstat.Plan", prior: S.Prior, stages: list[StageSpec] | None = None,
                 n_boxes: int = 16, runs_per_box: int = 8, n_part: int = 40, seed: int = 0, q: float = 1.0,
                 checkpoint_dir: str | None = None, c1: float = 2.0, c2: float = 2.0, vmax: float = 0.5,
                 bounds: np.ndarray | None = None, surrogate: SurrogateSpec | None = None,
                 autotune: bool | None = None, use_graphs: bool = True, record_history: bool = False,
                 comm: "Comm | None" = None, dmu_hi: float = 0.0, progress_every: int = 0,
                 on_progress=None):
        """bounds: optional [D, 2] search bounds overriding the prior's (a zero
        width pins a coordinate).  dmu_hi > 0: search delta_mu in [0, dmu_hi]
        as a sixth coordinate (the paper's [0, 0.9], Table I), its full range
        kept in every stage as the paper does (Sec. III.B, stage 3); q is then
        each particle's own.  The surrogate needs 5 coordinates.
        progress_every > 0: every that many iterations of a stage, append
        (stage, iteration, best F-hat, its physical parameters) over all of
        this process's runs to `progress` (a small device-to-host read; the
        captured iterations replay in chunks of that length).  autotune: time the fused kernel's launch
        variants on each stage's first swarm and use the fastest; None = only
        for FS_MIXED plans, whose variants give bitwise-equal F (FP64 variants
        differ by rounding, which can steer a PSO run differently).  use_graphs:
        replay captured iterations (eager launches otherwise; same results).
        record_history: keep the best fitness after every iteration of a
        surrogate-screened stage in `history`.  comm: split every stage's boxes
        over processes (Comm), one GPU each; None = this process runs all."""
        self.plan = plan
        self.prior = prior
        self.dmu_hi = float(dmu_hi)
        self.dims = 6 if self.dmu_hi > 0.0 else 5
        if self.dims == 6 and surrogate is not None:
            raise ValueError("the surrogate networks take 5 coordinates: no surrogate with delta_mu free")
        self.bounds = None if bounds is None else np.asarray(bounds, dtype=np.float64)
        self.stages = stages if stages is not None else default_stages()
        self.n_boxes, self.runs_per_box, self.n_part = n_boxes, runs_per_box, n_part
        self.seed, self.q = seed, q
        self.ckpt = checkpoint_dir
        self.c1, self.c2, self.vmax = c1, c2, vmax
        self.results: list[StageResult] = []
        self.surrogate = surrogate
        self.mlp = None
        self.mlps: list = []
        self.history: dict[int, list] = {}   # best fitness after each iteration (surrogate runs)
        self.autotune = (plan.mode == fstat.FS_MIXED) if autotune is None else bool(autotune)
        self.use_graphs = use_graphs
        self.record_history = record_history
        self.comm = comm
        self.progress_every = int(progress_every)
        self.progress: list = []
        self.on_progress = on_progress   # optional callable, given each progress entry as it is made

    # ---------------------------------------------------------------- boxes
    def stage_layout(self, i: int) -> tuple[int, int, int]:
        """(boxes, runs per box, particles per run) of stage i."""
        spec = self.stages[i]
        return (spec.boxes or self.n_boxes, spec.runs or self.runs_per_box, spec.particles or self.n_part)

    def stage_boxes(self, i: int) -> np.ndarray:
        spec = self.stages[i]
        n_boxes = self.stage_layout(i)[0]
        pb = prior_box(self.prior, self.dmu_hi) if self.bounds is None else self.bounds.copy()
        if spec.rule == "split_tc":
            u = S.uniforms(self.seed, 0x53504C54, n_boxes)                # "SPLT"
            w = -np.log1p(-u)                                              # Dirichlet(1) via exponentials
            edges = pb[1, 0] + (pb[1, 1] - pb[1, 0]) * np.concatenate([[0.0], np.cumsum(w) / np.sum(w)])
            boxes = np.repeat(pb[None], n_boxes, axis=0)
            boxes[:, 1, 0] = edges[:-1]
            boxes[:, 1, 1] = edges[1:]
            return boxes
        prev = self.results[i - 1]
        if spec.rule == "around":
            # box k around winner k of the previous stage (cyclically if this stage has more boxes)
            centers = [to_normal_coords(np.array(prev.winners[k % len(prev.winners)]), self.dims)
                       for k in range(n_boxes)]
        elif spec.rule == "around_best_mirror":
            best = np.array(prev.winners[int(np.argmax(prev.winner_f))])
            c = to_normal_coords(best, self.dims)
            m = c.copy()
            m[2] = -m[2]                                                   # theta -> pi - theta
            centers = [c if k % 2 == 0 else m for k in range(n_boxes)]
        else:
            raise ValueError(spec.rule)
        return np.stack([box_around(c, spec.widths, pb) for c in centers])

    # ---------------------------------------------------------------- one stage
    def local_boxes(self, i: int = 0) -> tuple[int, int]:
        """The contiguous block [k0, k1) of stage i's boxes this process
        searches (all of them without a communicator)."""
        n_boxes = self.stage_layout(i)[0] if self.stages else self.n_boxes
        if self.comm is None:
            return 0, n_boxes
        r, w = self.comm.rank, self.comm.world
        return n_boxes * r // w, n_boxes * (r + 1) // w

    def run_stage(self, i: int) -> StageResult:
        """One stage: every process runs the PSO runs of its block of boxes on
        its GPU; the best of each box's runs (a few hundred bytes per box) is
        then exchanged, so every process holds the stage's full result and
        derives the next stage's boxes from it.  The Philox counters use
        global run indices, so the result does not depend on the number of
        processes."""
        spec = self.stages[i]
        boxes = self.stage_boxes(i)
        k0, k1 = self.local_boxes(i)
        t0 = time.perf_counter()
        local = self._run_boxes(i, boxes, k0, k1) if k1 > k0 else ([], [], -1)
        seconds = time.perf_counter() - t0
        winners, wf, variant = local
        if self.comm is not None:
            parts = self.comm.allgather((k0, winners, wf, seconds, variant))
            parts.sort(key=lambda t: t[0])
            winners = [w for part in parts for w in part[1]]
            wf = [f for part in parts for f in part[2]]
            seconds = max(part[3] for part in parts)
            variant = parts[0][4]
        res = StageResult(i, spec.Np, boxes.tolist(), winners, wf, seconds, int(variant))
        if self.comm is None or self.comm.rank == 0:
            self._save(res)
        return res

    def _run_boxes(self, i: int, boxes: np.ndarray, k0: int, k1: int):
        """PSO runs of boxes [k0, k1) of stage i on this process's GPU: the
        best position (physical parameters) and fitness of each box, and the
        launch variant used."""
        import torch
        spec = self.stages[i]
        _, runs_per_box, n_part = self.stage_layout(i)
        nb = k1 - k0
        R = nb * runs_per_box
        run_boxes = np.repeat(boxes[k0:k1], runs_per_box, axis=0)
        stage_seed = (self.seed << 8) + i
        with torch.cuda.stream(self.plan.stream):
            sw = fstat.Swarm(self.plan, R, n_part, run_boxes, self.q, run0=k0 * runs_per_box, dims=self.dims)
            sw.init(stage_seed)
            variant = sw.autotune(spec.Np, reps=2)[0] if self.autotune else self.plan.get_variant(spec.Np)
            if self.surrogate is None:
                sw.graph_build(spec.Np, stage_seed, n_iter=spec.n_iter, w0=spec.w0, w1=spec.w1, c1=self.c1,
                               c2=self.c2, vmax=self.vmax)
                done = 0
                chunk = self.progress_every if self.progress_every > 0 else spec.n_iter - 1
                while done < spec.n_iter - 1:      # the graph does evaluate + step
                    k = min(chunk, spec.n_iter - 1 - done)
                    sw.graph_run(k)
                    done += k
                    if self.progress_every > 0:
                        self._note_progress(i, done, sw, run_boxes)
                sw.graph_free()
            else:
                self._run_screened(sw, spec, stage_seed, i, k0, nb, run_boxes)
            sw.evaluate(spec.Np)               # fitness of the final positions
            sw.step(stage_seed, -1, w0=spec.w0, w1=spec.w1, n_iter=spec.n_iter)   # folds them into pbest
            best_f, best_i = sw.best()
            bf = best_f.cpu().numpy()
            bi = best_i.cpu().numpy()
            pbx = sw.pbest_x.cpu().numpy()
        winners, wf = [], []
        for k in range(nb):
            runs = np.arange(k * runs_per_box, (k + 1) * runs_per_box)
            r = runs[int(np.argmax(bf[runs]))]
            winners.append(to_physical(pbx[r, bi[r]], run_boxes[r], self.q).tolist())
            wf.append(float(bf[r]))
        return winners, wf, int(variant)

    def _note_progress(self, stage: int, it: int, sw, run_boxes):
        """Best personal best over the swarm's runs after `it` iterations."""
        best_f, best_i = sw.best()
        bf = best_f.cpu().numpy()
        bi = best_i.cpu().numpy()
        r = int(np.argmax(bf))
        x = sw.pbest_x[r, int(bi[r])].cpu().numpy()
        self.progress.append((stage, it, float(bf[r]), to_physical(x, run_boxes[r], self.q).tolist()))
        if self.on_progress is not None:
            self.on_progress(self.progress[-1])

    def _run_screened(self, sw, spec: StageSpec, stage_seed: int, stage: int, k0: int = 0, nb: int | None = None,
                      run_boxes=None):
        """n_iter - 1 iterations of evaluate + record + (screened) step with one
        network and one sample ring per search box: positions are normalised
        to each run's box, so the runs of a box share a landscape and the
        boxes do not.  The boxes' networks form one batch (every kernel of a
        forward or training pass covers all of them) and their rings are
        slices of one buffer.  Every train_every iterations after the warm-up
        each network trains on its box's ring.  With graphs (default) an
        iteration is two captured launches, (evaluate + record) and the step,
        with the captured training round in between when due; the eager form
        makes the same calls."""
        import torch
        sp = self.surrogate
        nb = self.stage_layout(stage)[0] if nb is None else nb
        dev = sw.x.device
        # network k of the batch belongs to box k0 + k and is seeded by that global index
        self.mlp = fstat.MLP(sp.width, max_batch=max(sp.buffer, 4096), seed=self.seed * 1000 + 97 * stage + k0,
                             stream=self.plan.stream, groups=nb)
        self.mlps = [self.mlp]
        rings = fstat.SampleRing.batch(nb, sp.buffer, device=dev)
        step_kw = dict(w0=spec.w0, w1=spec.w1, n_iter=spec.n_iter, c1=self.c1, c2=self.c2, vmax=self.vmax)
        graphs = None
        if self.use_graphs:
            graphs = (sw.graph_build_ex(1 | 2, spec.Np, stage_seed, ring=rings, **step_kw),
                      sw.graph_build_ex(4, spec.Np, stage_seed, **step_kw),
                      sw.graph_build_ex(8, spec.Np, stage_seed, mlp=self.mlps, n_cand=sp.n_cand, **step_kw),
                      fstat.mlp_train_graph(self.mlps, rings, sp.train_steps, sp.lr))
        hist = []
        for it in range(spec.n_iter - 1):
            if graphs:
                graphs[0].run(1)
            else:
                sw.evaluate(spec.Np)
                sw.record(rings)
            screened = it >= sp.warm
            if screened and (it - sp.warm) % sp.train_every == 0:
                # the whole ring: slots not yet written hold NaN targets, which the loss ignores
                if graphs:
                    graphs[3].run(1)
                else:
                    self.mlp.train(torch.stack([r.x for r in rings]), torch.stack([r.f for r in rings]),
                                   sp.train_steps, sp.lr)
            if graphs:
                graphs[2 if screened else 1].run(1)
            elif screened:
                sw.step_screened(self.mlps, sp.n_cand, stage_seed, -1, **step_kw)
            else:
                sw.step(stage_seed, -1, **step_kw)
            if self.record_history:
                hist.append(sw.pbest_f.max())
            if self.progress_every > 0 and run_boxes is not None and (it + 1) % self.progress_every == 0:
                self._note_progress(stage, it + 1, sw, run_boxes)
        if graphs:
            for gr in graphs:
                gr.close()
        self.history[stage] = [float(h) for h in torch.stack(hist).cpu().numpy()] if hist else []

    # ---------------------------------------------------------------- checkpoints
    def _path(self, i):
        return None if not self.ckpt else os.path.join(self.ckpt, f"stage{i}.json")

    def _save(self, res: StageResult):
        if not self.ckpt:
            return
        os.makedirs(self.ckpt, exist_ok=True)
        tmp = self._path(res.stage) + ".tmp"
        with open(tmp, "w") as f:
            json.dump({"seed": self.seed, "spec": asdict(self.stages[res.stage]), "result": asdict(res)}, f)
        os.replace(tmp, self._path(res.stage))

    def _load(self, i) -> StageResult | None:
        p = self._path(i)
        if not p or not os.path.exists(p):
            return None
        with open(p) as f:
            d = json.load(f)
        if d.get("seed") != self.seed or d.get("spec") != json.loads(json.dumps(asdict(self.stages[i]))):
            raise ValueError(f"checkpoint {p} belongs to a different search")
        return StageResult(**d["result"])

    # ---------------------------------------------------------------- all stages
    def run(self, extrinsic: bool = True) -> dict:
        """All stages (resuming from checkpoints); extrinsic: also report the
        amplitudes and extrinsic parameters at the final best point."""
        self.results = []
        for i in range(len(self.stages)):
            res = self._load(i)
            if res is None:
                res = self.run_stage(i)
            self.results.append(res)
        last = self.results[-1]
        k = int(np.argmax(last.winner_f))
        return {"best": last.winners[k], "best_F_hat": last.winner_f[k],
                "extrinsic": self.extrinsic(last.winners[k]) if extrinsic else None,
                "stages": [asdict(r) for r in self.results],
                "seconds": sum(r.seconds for r in self.results)}

    def extrinsic(self, theta) -> dict:
        """Fully coherent amplitudes a (Eq. aandMN3) and (D_L, iota, psi, phi_c)
        (App. B) at the intrinsic parameters theta, computed on the device."""
        import torch
        with torch.cuda.stream(self.plan.stream):
            P = torch.tensor(np.asarray(theta, dtype=np.float64).reshape(1, 6), device="cuda")
            F, a, ext = self.plan.amplitudes(P, 1)
            F, a, ext = F.cpu().numpy(), a.cpu().numpy(), ext.cpu().numpy()
        DL, iota, psi, phic = (float(x) for x in ext[0, 0])
        return {"F": float(F[0]), "a": a[0, 0].tolist(), "D_L": DL, "iota": iota, "psi": psi, "phi_c": phic}
