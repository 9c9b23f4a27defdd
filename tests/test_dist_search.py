"""Multi-process search on the CPU (gloo, 127.0.0.1): the exchange of box
winners between processes and the bench's cross-rank reductions.

The GPU part of a stage (the PSO runs of a block of boxes) is replaced by a
deterministic stand-in that depends only on the stage, the box and its
global index, so a search split over 2 or 3 processes must reproduce the
one-process result exactly: the same boxes, winners and fitness in every
stage, on every process.
"""
import json
import os
import socket
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

from paper_2407_10797_gb300 import search  # noqa: E402
from paper_2407_10797_gb300 import synth as S  # noqa: E402


class StandInSearch(search.HierarchicalSearch):
    def _run_boxes(self, i, boxes, k0, k1):
        win, wf = [], []
        for k in range(k0, k1):
            b = boxes[k]
            u = 0.2 + 0.6 * (((k * 7 + 3 * i) % 5) / 4.0)
            p = search.to_physical(np.full(5, u), b, self.q)
            f = -abs(p[0] - 31.0) - 1e-6 * abs(p[1] - 0.6 * S.YEAR_S) + 0.01 * k
            win.append([float(x) for x in p])
            wf.append(float(f))
        return win, wf, 0


def make_search(comm=None):
    prior = S.Prior(Mc_lo=20.0, Mc_hi=40.0, tc_lo=0.0, tc_hi=S.YEAR_S, e0_hi=0.1)
    plan = types.SimpleNamespace(mode=1, stream=None)
    return StandInSearch(plan, prior, search.default_stages(10), n_boxes=7, runs_per_box=2, n_part=4, seed=5,
                         autotune=False, comm=comm)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = make_search(search.Comm()).run(extrinsic=False)
        # the bench's cross-rank reductions on the same process group
        import bench
        bench.barrier(world)
        mx = bench.allmax(world, float(rank + 1))
        sm = bench.allsum(world, float(rank + 1))
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"res": res, "max": mx, "sum": sm}, f)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_split_search_equals_single_process(tmp_path, world):
    single = make_search().run(extrinsic=False)
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        with open(tmp_path / f"rank{r}.json") as f:
            d = json.load(f)
        got = d["res"]
        assert got["best"] == single["best"] and got["best_F_hat"] == single["best_F_hat"]
        for a, b in zip(got["stages"], single["stages"]):
            assert a["boxes"] == b["boxes"]
            assert a["winners"] == b["winners"] and a["winner_f"] == b["winner_f"]
        assert d["max"] == float(world)
        assert d["sum"] == float(world * (world + 1) // 2)


def test_box_blocks_cover_every_box_once():
    for world in (1, 2, 3, 4, 7, 9):
        seen = []
        for rank in range(world):
            hs = make_search(types.SimpleNamespace(rank=rank, world=world))
            k0, k1 = hs.local_boxes()
            assert 0 <= k0 <= k1 <= 7
            seen.extend(range(k0, k1))
        assert seen == list(range(7))
