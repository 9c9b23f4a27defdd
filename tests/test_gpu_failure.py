"""Failure detection on the GPU without a fault: a device-side wait that gives
up is reported on the host, and the plan keeps working.

fs_plan_selftest_timeout launches one bounded mbarrier wait that nothing
completes (the same bounded poll the staged FS_MIXED kernel uses for its
copies).  The wait runs out, sets the plan's timeout bit, and the next
fs_plan_check returns FS_ETIMEOUT; the bit is then cleared and later
evaluations on the same plan give the same F as before, bit for bit.
"""
import time

import numpy as np
import pytest

from paper_2407_10797_gb300 import synth as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fst():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_10797_gb300 import fstat
    fstat.load()
    return fstat


@pytest.mark.parametrize("mode", [0, 1])
def test_wait_that_runs_out_is_reported_and_the_plan_recovers(fst, mode):
    g = S.tiny_grid(n=4096, f_min=0.02, stride=8)
    psd = S.lisa_like_psd(g.freqs())
    d = S.gaussian_noise(g, psd, 4)
    P = torch.from_numpy(S.draw_params(S.Prior(tc_lo=0.1 * g.T_obs, tc_hi=0.9 * g.T_obs), 24, 5)).cuda()
    plan = fst.Plan.from_grid(g, mode=mode)
    plan.set_data(torch.from_numpy(d).cuda(), torch.from_numpy(psd).cuda())
    F0 = plan.fstat(P, 4)[0].clone()
    assert plan.check() == 0
    t0 = time.time()
    plan.selftest_timeout()
    with pytest.raises(fst.FstatError) as ei:
        plan.check()
    assert ei.value.status == fst.FS_ETIMEOUT
    assert time.time() - t0 < 10.0
    assert plan.check() == 0   # the bit was cleared
    F1 = plan.fstat(P, 4)[0]
    torch.cuda.synchronize()
    assert torch.equal(F0, F1)
    assert plan.check() == 0
    plan.close()
