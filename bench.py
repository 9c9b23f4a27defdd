#!/usr/bin/env python3
"""Throughput of the batched semi-coherent F-statistic on GB300.

Workload (one step): the paper-scale data set -- 2.5 yr of one TDI channel,
1/T bins over [10, 50) mHz (3,155,760 bins), LISA-like noise plus one
injection at SNR 12.5 -- and one batch of 8 PSO runs x 40 particles (B = 320)
evaluated at N_p = 256, 64, 16 and 1 per-particle segments (one launch each).
Metric: in-band particle*bins per second (a bin counts for a particle when
its stationary-phase time lies in [0, T]).

Arms:
  default           the CUDA library through its C ABI (FP64 mode)
  --impl reference  the CPU oracle on the host cores, on a bounded sample of
                    the same workload per step

Launch: `python bench.py [--gpus N --steps K --warmup W]`; for N > 1 under
torch.distributed.run, one rank per GPU, each with its own batch (weak
scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2407_10797_gb300 import synth as S  # noqa: E402

METRIC = "F-stat particle·bins/s on 1 GB300 (FP64 vs mixed at ≤1e-4 rel err); search wall time"
UNIT = "particle*bins/s"
NP_LIST = (256, 64, 16, 1)

# FP64 operations per in-band particle*bin of the fused kernel (algorithmic
# count of the template + response + reduction arithmetic, FMA = 2, with each
# of the two FP64 trig evaluations counted as 40).
FP64_FLOP_PER_PBIN = 203.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--profile-case", choices=["fp64", "mixed"], default=None,
                    help="one small evaluation for kernel profiling: paper grid, 64 particles, N_p = 16")
    return ap.parse_args()


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(world, x: float) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allsum(world, x: float) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
def workload_inputs(rank: int):
    w = S.paper_workload()
    g = w.grid
    psd = S.lisa_like_psd(g.freqs())
    noise = S.gaussian_noise(g, psd, w.seed + 1000 * rank)
    P = S.draw_params(w.prior, w.B, w.seed + 1000 * rank)
    # injection: a particle drawn from the prior with a long in-band track
    inj = S.draw_params(S.Prior(Mc_lo=20.0, Mc_hi=40.0, tc_lo=0.95 * g.T_obs, tc_hi=1.05 * g.T_obs), 1,
                        w.seed + 1000 * rank, stream=S.STREAM_INJECTION)[0]
    return w, g, psd, noise, P, inj


def extrinsic_amplitudes(iota, psi, phic):
    """Amplitudes a_i of Appendix B, Eq. (B1), at unit distance."""
    c2p, s2p, ci = math.cos(2 * psi), math.sin(2 * psi), math.cos(iota)
    ap = 0.5 * (1 + ci * ci)
    cf, sf = math.cos(phic), math.sin(phic)
    return np.array([c2p * ap * cf - s2p * ci * sf, -(s2p * ap * cf + c2p * ci * sf),
                     -(c2p * ap * sf + s2p * ci * cf), s2p * ap * sf - c2p * ci * cf])


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = os.path.join("/tmp", f"fs_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def fp64_peak_tflops() -> float:
    """FP64 peak from unit counts: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop at the
    2070 MHz maximum SM clock (the nominal 1.26 TFLOP/s)."""
    return 152 * 2 * 2 * 2070e6 / 1e12


# ---------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ---------------------------------------------------------------------------
def oracle_sample(g, P, psd, data, seconds: float, Np: int = 16):
    """Run the oracle on whole particles (all their in-band bins) until about
    `seconds` of wall time; returns (pbins, elapsed s, threads, n particles)."""
    from oracle import oracle as O
    m = O.OracleModel.from_grid(g)
    bands = np.array([O.band(p, m) for p in P])
    nb = np.maximum(bands[:, 1] - bands[:, 0] + 1, 0)
    order = [i for i in np.argsort(nb) if nb[i] > 0]
    threads = O.num_threads()
    # calibrate on the smallest particle with at least 2e4 in-band bins
    big = [i for i in order if nb[i] >= 20000]
    i0 = big[0] if big else order[-1]
    t0 = time.perf_counter()
    O.fstat_batch(P[i0:i0 + 1], m, data, psd, Np, nthreads=1)
    per_bin = (time.perf_counter() - t0) / max(nb[i0], 1)
    budget_bins = seconds * threads / per_bin
    pick, tot = [], 0
    for i in order[len(order) // 4:] + order[:len(order) // 4]:
        if tot + nb[i] > budget_bins and pick:
            continue
        pick.append(i)
        tot += nb[i]
        if tot >= budget_bins:
            break
    t0 = time.perf_counter()
    O.fstat_batch(P[pick], m, data, psd, Np, nthreads=threads)
    el = time.perf_counter() - t0
    return int(nb[pick].sum()), el, threads, len(pick)


def run_reference(args, world, rank):
    if rank != 0:
        return
    w, g, psd, noise, P, inj = workload_inputs(0)
    from oracle import oracle as O
    m = O.OracleModel.from_grid(g)
    a = extrinsic_amplitudes(S.INJ_IOTA, S.INJ_PSI, S.INJ_PHIC)
    k0, k1 = O.band(inj, m)
    h = O.inject(inj, m, a, k0, k1 + 1)
    data = noise + h * (w.snr / math.sqrt(O.inner(h, h, psd, g.df)))
    per_step = max(1.0, min(10.0, 120.0 / max(args.steps + args.warmup, 1)))
    for _ in range(args.warmup):
        oracle_sample(g, P, psd, data, per_step / 2)
    tot_pb, tot_s, thr, npart = 0, 0.0, 1, 0
    for _ in range(args.steps):
        pb, el, thr, npart = oracle_sample(g, P, psd, data, per_step)
        tot_pb += pb
        tot_s += el
    value = tot_pb / tot_s
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n_bins": g.n, "B": w.B, "N_p": [16],
                   "sample": "whole in-band particles of the batch, N_p = 16, about %.0f s per step" % per_step},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": thr, "kind": "oracle",
                         "sample": f"{npart} particles x all their in-band bins per step, N_p = 16"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def time_mode(args, world, plan, P_dev, B, F_out, stream, kernel_prof=True):
    """Warm up, then time `steps` evaluations at every N_p with CUDA events on
    the plan's stream (barrier + synchronize on both sides).  Returns
    (ms for all steps, max over ranks; fused-kernel ms and launches; clocks)."""
    import torch

    def step(params):
        for Np in NP_LIST:
            plan.fstat(params, Np, F=F_out[Np], want_parts=False)

    for _ in range(args.warmup):
        step(P_dev)
    torch.cuda.synchronize()
    for k in ("main", "setup", "reduce"):
        plan.read_profile(k)
    plan.set_profiling(kernel_prof)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        barrier(world)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            step(P_dev)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
    plan.set_profiling(False)
    ms = allmax(world, ev0.elapsed_time(ev1))
    prof = {k: plan.read_profile(k) for k in ("main", "setup", "reduce")}
    return ms, prof, clk.summary(), step


def fp32_peak_tflops() -> float:
    """FP32 peak from unit counts: 152 SMs x 128 FP32 lanes x 2 flop (FMA) at
    2070 MHz (80.5 TFLOP/s)."""
    return 152 * 128 * 2 * 2070e6 / 1e12


# Operations per in-band particle*bin of the mixed kernel's body (algorithmic
# count, FMA = 2): orbital-phase offset 3, antenna pair G1, G2 as degree-6
# polynomials 24, Doppler polynomial 17, phase assembly and reduction 5, SFU
# sincos 3, z = dw e^{i Phi} 6, seven sums 16, fixed-point phase steps 6
# (integer adds counted as one each).
MIXED_FLOP_PER_PBIN = 80.0


def run_gpu(args, world, rank, local):
    import torch
    from paper_2407_10797_gb300 import fstat

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    w, g, psd, noise, P, inj = workload_inputs(rank)
    d_dev = torch.from_numpy(noise).to(dev)
    psd_dev = torch.from_numpy(psd).to(dev)
    plan = fstat.Plan.from_grid(g, mode=fstat.FS_FP64, stream=stream)
    plan.set_data(d_dev, psd_dev)
    # injection through the library's own template generator
    a = extrinsic_amplitudes(S.INJ_IOTA, S.INJ_PSI, S.INJ_PHIC)
    h = torch.zeros_like(d_dev)
    plan.add_signal(inj, a, h)
    hh = float((4.0 * g.df * (h.abs() ** 2) / psd_dev).sum().item())
    d_dev = d_dev + h * (w.snr / math.sqrt(hh))
    plan.set_data(d_dev, psd_dev)
    del h
    B = w.B
    plan.reserve(B, max(NP_LIST))
    P_dev = torch.from_numpy(P).to(dev)
    bands = plan.bands(P_dev).cpu().numpy()
    inband = int(np.maximum(bands[:, 1] - bands[:, 0] + 1, 0).sum())
    pbins_per_step = inband * len(NP_LIST)
    total_pbins = allsum(world, float(pbins_per_step * args.steps))
    F_out = {Np: torch.empty(B, dtype=torch.float64, device=dev) for Np in NP_LIST}

    # ---- FP64 mode (the paper-scale FP64 configuration): device-resident timing
    ms, prof, clocks, step = time_mode(args, world, plan, P_dev, B, F_out, stream)
    value = total_pbins / (ms / 1e3)
    main_ms, main_n = prof["main"]
    F64 = {Np: F_out[Np].cpu().numpy() for Np in NP_LIST}

    # ---- end to end through the C ABI with host buffers (pinned)
    P_host = torch.from_numpy(P).pin_memory()
    F_host = torch.empty(len(NP_LIST), B, dtype=torch.float64).pin_memory()
    P_e2e = torch.empty_like(P_dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        P_e2e.copy_(P_host, non_blocking=True)
        step(P_e2e)
        for i, Np in enumerate(NP_LIST):
            F_host[i].copy_(F_out[Np], non_blocking=True)
        torch.cuda.current_stream().synchronize()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    e2e_ms = allmax(world, e0.elapsed_time(e1))
    e2e_value = total_pbins / (e2e_ms / 1e3)
    plan.close()

    # ---- mixed mode on the same data and particles
    planm = fstat.Plan.from_grid(g, mode=fstat.FS_MIXED, stream=stream)
    planm.set_data(d_dev, psd_dev)
    planm.reserve(B, max(NP_LIST))
    ms_m, prof_m, clocks_m, _ = time_mode(args, world, planm, P_dev, B, F_out, stream)
    value_m = total_pbins / (ms_m / 1e3)
    mix_err = max(float(np.max(np.abs(F_out[Np].cpu().numpy() - F64[Np]) / np.maximum(np.abs(F64[Np]), 2.0 * Np)))
                  for Np in NP_LIST)
    planm.close()

    # ---- roofline of the dominant kernels (average launch duration, live events)
    main_avg_ms = main_ms / max(main_n, 1)
    achieved_tf = FP64_FLOP_PER_PBIN * inband / (main_avg_ms / 1e3) / 1e12
    peak_tf = fp64_peak_tflops()
    mm_ms, mm_n = prof_m["main"]
    mm_avg = mm_ms / max(mm_n, 1)
    ach_m = MIXED_FLOP_PER_PBIN * inband / (mm_avg / 1e3) / 1e12
    peak_m = fp32_peak_tflops()
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            data_h = d_dev.cpu().numpy()
            pb, el, thr, npart = oracle_sample(g, P, psd, data_h, args.cpu_seconds)
            cpu = {"value": pb / el, "unit": UNIT, "cores": thr, "kind": "oracle",
                   "sample": f"{npart} particles x all their in-band bins ({pb} particle*bins), N_p = 16, "
                             f"{el:.1f} s"}
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "n_bins": g.n, "f_band_hz": [0.01, 0.05], "T_obs_s": g.T_obs,
                       "B": B, "runs_x_particles": "8x40", "N_p": list(NP_LIST), "mode": "fp64",
                       "inband_particle_bins_per_launch": inband, "grid_particle_bins_per_launch": B * g.n,
                       "l2": "inputs exceed L2: per-bin tables 227 MB > 129 MB L2", "parallelism": f"dp{world}"},
            "gpu_launches": args.steps * len(NP_LIST) * 5,
            "kernel_ms": {"fused_fp64_avg": main_avg_ms, "setup_avg": prof["setup"][0] / max(prof["setup"][1], 1),
                          "solve_avg": prof["reduce"][0] / max(prof["reduce"][1], 1),
                          "fused_share_of_step": main_ms / max(ms, 1e-9)},
            "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": peak_tf, "unit": "TFLOP/s",
                         "frac": achieved_tf / peak_tf, "traffic": None, "pipe": "fp64",
                         "peak_source": "unit counts: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz",
                         "flop_per_pbin": FP64_FLOP_PER_PBIN},
            "clocks": clocks,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(P.nbytes),
                    "d2h_bytes_per_step": int(8 * B * len(NP_LIST))},
            "mixed": {"value": value_m, "unit": UNIT, "ms_per_step": ms_m / args.steps, "dtype": "f64 anchors + f32",
                      "max_rel_err_vs_fp64": mix_err, "error_metric": "|dF|/max(|F|, 2 N_p)",
                      "kernel_ms": {"fused_mixed_avg": mm_avg, "fused_share_of_step": mm_ms / max(ms_m, 1e-9)},
                      "roofline": {"bound": "alu", "achieved": ach_m, "peak": peak_m, "unit": "TFLOP/s",
                                   "frac": ach_m / peak_m, "traffic": None, "pipe": "fp32",
                                   "peak_source": "unit counts: 152 SMs x 128 lanes x 2 flop x 2.07 GHz",
                                   "flop_per_pbin": MIXED_FLOP_PER_PBIN},
                      "clocks": clocks_m},
            "cpu_baseline": cpu,
        }
        print(json.dumps(out), flush=True)


def run_profile_case(args):
    """Paper-scale grid (tables 227 MB > L2), 64 particles, one N_p = 16 launch
    after one warm-up launch: a short capture target for kernel profilers."""
    import torch
    from paper_2407_10797_gb300 import fstat
    w, g, psd, noise, P, inj = workload_inputs(0)
    mode = fstat.FS_MIXED if args.profile_case == "mixed" else fstat.FS_FP64
    plan = fstat.Plan.from_grid(g, mode=mode)
    plan.set_data(torch.from_numpy(noise).cuda(), torch.from_numpy(psd).cuda())
    P_dev = torch.from_numpy(P[:64] if mode == fstat.FS_FP64 else P).cuda()
    for _ in range(2):
        F, _ = plan.fstat(P_dev, 16, want_parts=False)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": f"paper grid, {args.profile_case}, B={P_dev.shape[0]}, N_p=16",
                      "F_mean": float(F.mean().item())}))
    plan.close()


def main():
    args = parse()
    if args.profile_case:
        run_profile_case(args)
        return
    world, rank, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_gpu(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
