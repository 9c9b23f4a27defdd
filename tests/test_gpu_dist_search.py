"""The search split over two processes that share one GPU (gloo for the
winner exchange): the same result as one process, bit for bit.  The two
processes' kernels never wait on each other; they only meet on the host at
the end of each stage."""
import json
import math
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

pytestmark = pytest.mark.gpu


def tc_for(Mc, f, t):
    from paper_2407_10797_gb300 import synth as S
    m = Mc * S.MSUN_S
    return t + 5.0 / 256.0 * m * (np.pi * m * f) ** (-8.0 / 3.0)


def build(comm=None):
    from oracle import oracle as O
    from paper_2407_10797_gb300 import fstat, search
    from paper_2407_10797_gb300 import synth as S
    g = S.tiny_grid(n=30000, f_min=0.02)
    psd = S.lisa_like_psd(g.freqs())
    m = O.OracleModel.from_grid(g)
    truth = np.array([30.0, tc_for(30.0, 0.02 + 15000 * g.df, 0.5 * g.T_obs), 0.4, 2.0, 0.02, 1.0])
    a = O.extrinsic_to_a(1.0, S.INJ_PSI, S.INJ_IOTA, S.INJ_PHIC)
    k0, k1 = O.band(truth, m)
    h = O.inject(truth, m, a, k0, k1 + 1)
    d = S.gaussian_noise(g, psd, 12) + h * (30.0 / math.sqrt(O.inner(h, h, psd, g.df)))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan = fstat.Plan.from_grid(g, mode=fstat.FS_MIXED, stream=s)
        plan.set_data(torch.from_numpy(d).cuda(), torch.from_numpy(psd).cuda())
        plan.set_variant(2)
    prior = S.Prior(Mc_lo=29.0, Mc_hi=31.0, tc_lo=truth[1] - 2e5, tc_hi=truth[1] + 2e5, e0_hi=0.05)
    stages = [search.StageSpec(64, 30, "split_tc"), search.StageSpec(16, 30, "around", (0.4, 4e4, None, None, None)),
              search.StageSpec(1, 30, "around_best_mirror", (0.1, 1e4, 0.2, 0.2, 0.01))]
    hs = search.HierarchicalSearch(plan, prior, stages, n_boxes=4, runs_per_box=2, n_part=40, seed=7,
                                   autotune=False, comm=comm)
    return hs


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, os.getcwd())
    import torch.distributed as dist
    from paper_2407_10797_gb300 import search
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = build(search.Comm()).run()
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump(res, f)
    finally:
        dist.destroy_process_group()


def test_two_processes_one_gpu_equal_one_process(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    single = build().run()
    mp.spawn(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        with open(tmp_path / f"rank{r}.json") as f:
            got = json.load(f)
        assert got["best"] == single["best"] and got["best_F_hat"] == single["best_F_hat"]
        for a, b in zip(got["stages"], single["stages"]):
            assert a["boxes"] == b["boxes"] and a["winners"] == b["winners"] and a["winner_f"] == b["winner_f"]
        assert got["extrinsic"]["a"] == single["extrinsic"]["a"]
