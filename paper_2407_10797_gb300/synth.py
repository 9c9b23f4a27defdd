"""Seeded synthetic inputs: frequency grids, a LISA-like noise PSD, Gaussian
noise realisations and particle draws from the search priors.

This module is shared by the tests, the oracle's callers and the benchmark.
It holds none of the F-statistic's arithmetic (no waveform, no response, no
inner product): only the inputs the method consumes.  All randomness comes
from a counter-based Philox4x32-10 generator (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC 2011), written here in
numpy so the same seed gives the same bits on every machine.

Units follow the paper (G = c = 1, Sec. I): masses and times in seconds,
frequencies in Hz.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------
# Physical constants (one table; the oracle and the CUDA library each keep
# their own copy, and a test checks that the three agree).
# --------------------------------------------------------------------------
MSUN_S = 4.925490947e-6          # G M_sun / c^3 in seconds
YEAR_S = 365.25 * 86400.0        # Julian year, orbital period of the detector
AU_S = 499.004784                # 1 AU / c in seconds
MPC_S = 3.0856775814913673e22 / 299792458.0   # 1 Mpc / c in seconds

# --------------------------------------------------------------------------
# Philox4x32-10
# --------------------------------------------------------------------------
_PHILOX_M0 = np.uint64(0xD2511F53)
_PHILOX_M1 = np.uint64(0xCD9E8D57)
_PHILOX_W0 = np.uint32(0x9E3779B9)
_PHILOX_W1 = np.uint32(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)

# Stream tags keep the different kinds of draws apart under one seed.
STREAM_NOISE = 0x4E4F4953      # "NOIS"
STREAM_PARTICLES = 0x50415254  # "PART"
STREAM_INJECTION = 0x494E4A45  # "INJE"


def philox4x32_10(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    """Philox4x32 with 10 rounds.

    ctr: uint32 array [..., 4]; key: uint32 array [..., 2] (broadcastable).
    Returns uint32 array [..., 4].
    """
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    c0, c1, c2, c3 = (c[..., i].astype(np.uint64) for i in range(4))
    k0 = np.broadcast_to(k[..., 0], c0.shape).astype(np.uint64)
    k1 = np.broadcast_to(k[..., 1], c0.shape).astype(np.uint64)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + np.uint64(_PHILOX_W0)) & _MASK32
            k1 = (k1 + np.uint64(_PHILOX_W1)) & _MASK32
        p0 = _PHILOX_M0 * c0
        p1 = _PHILOX_M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)
    out = np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)
    return out


def _u53(lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    """Uniform double in [0, 1) from two 32-bit words (top 53 of 64 bits)."""
    w = (hi.astype(np.uint64) << np.uint64(32)) | lo.astype(np.uint64)
    return (w >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _key(seed: int, stream: int) -> np.ndarray:
    return np.array([seed & 0xFFFFFFFF, (stream ^ (seed >> 32)) & 0xFFFFFFFF],
                    dtype=np.uint32)


def uniforms(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n uniform doubles in [0, 1): two per Philox block, counter = block id."""
    nb = (n + 1) // 2
    idx = np.arange(offset, offset + nb, dtype=np.uint64)
    ctr = np.zeros((nb, 4), dtype=np.uint32)
    ctr[:, 0] = (idx & _MASK32).astype(np.uint32)
    ctr[:, 1] = (idx >> np.uint64(32)).astype(np.uint32)
    out = philox4x32_10(ctr, _key(seed, stream))
    u = np.empty(2 * nb)
    u[0::2] = _u53(out[:, 0], out[:, 1])
    u[1::2] = _u53(out[:, 2], out[:, 3])
    return u[:n]


def standard_normal_pairs(seed: int, stream: int, n: int) -> tuple[np.ndarray, np.ndarray]:
    """n pairs of independent N(0,1) deviates by the Box-Muller transform."""
    u = uniforms(seed, stream, 2 * n)
    u1 = 1.0 - u[0::2]              # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    return r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)


# --------------------------------------------------------------------------
# Frequency grid, PSD and noise
# --------------------------------------------------------------------------
@dataclass(frozen=True)
class Grid:
    """Uniform one-sided frequency grid f_k = f_min + k*df, k = 0..n-1."""
    f_min: float
    df: float
    n: int
    T_obs: float      # observation time; the data's frequency resolution is 1/T_obs

    def freqs(self) -> np.ndarray:
        return self.f_min + np.arange(self.n, dtype=np.float64) * self.df

    def edge_freqs(self, starts) -> np.ndarray:
        """Edge frequencies half a bin below the given start bins, so that the
        segments between them hold exactly the bins [starts[p], starts[p+1])."""
        k = np.asarray(starts, dtype=np.float64)
        return self.f_min + (k - 0.5) * self.df


def lisa_like_psd(f: np.ndarray) -> np.ndarray:
    """Smooth analytic LISA-like one-sided noise PSD (strain^2/Hz).

    Optical-metrology and test-mass-acceleration terms of the LISA analytic
    noise model (Robson, Cornish, Liu 2019), without the galactic foreground
    and without the sky-averaging factor.  Only its shape matters here: the
    injected signal is rescaled to a target SNR.
    """
    f = np.asarray(f, dtype=np.float64)
    L = 2.5e9
    fstar = 299792458.0 / (2.0 * np.pi * L)
    p_oms = (1.5e-11) ** 2 * (1.0 + (2.0e-3 / f) ** 4)
    p_acc = (3.0e-15) ** 2 * (1.0 + (0.4e-3 / f) ** 2) * (1.0 + (f / 8.0e-3) ** 4)
    return (p_oms + 2.0 * (1.0 + np.cos(f / fstar) ** 2) * p_acc / (2.0 * np.pi * f) ** 4) \
        * (1.0 + 0.6 * (f / fstar) ** 2) / L ** 2


def gaussian_noise(grid: Grid, psd: np.ndarray, seed: int, channel: int = 0) -> np.ndarray:
    """Complex frequency-domain noise: Re and Im of n_k are i.i.d.
    N(0, S_k T/4), so E|n_k|^2 = S_k T/2 (one-sided PSD, bin width 1/T).
    Each channel draws from its own stream, so channels are independent."""
    z0, z1 = standard_normal_pairs(seed, STREAM_NOISE + channel, grid.n)
    sigma = np.sqrt(psd * grid.T_obs / 4.0)
    return sigma * z0 + 1j * (sigma * z1)


TDI_X, TDI_AE = 0, 1


def tdi_psds(f: np.ndarray, tdi: int) -> np.ndarray:
    """One-sided noise PSDs of the channels of a TDI set, [channels, n]: X
    takes the LISA-like model, A and E (responses sqrt(3/2) times a Michelson
    of the same arms, noise-orthogonal) 3/2 of it each, the long-wavelength
    relation S_A = S_E = S_X - S_XY with S_XY = -S_X / 2."""
    sx = lisa_like_psd(f)
    return sx[None, :] if tdi == TDI_X else np.stack([1.5 * sx, 1.5 * sx])


# --------------------------------------------------------------------------
# Priors and particle draws
# --------------------------------------------------------------------------
PARAM_FIELDS = ("Mc", "tc", "lat", "lon", "e0", "q")   # Mc in Msun, tc in s, rad


@dataclass(frozen=True)
class Prior:
    """Search prior: M_c ~ U[Mc_lo, Mc_hi] (Msun), t_c ~ U[tc_lo, tc_hi] (s),
    ecliptic latitude uniform on the sphere (sin(lat) ~ U[-1, 1]), longitude
    ~ U[0, 2 pi), e0 ~ U[0, e0_hi], equal masses (q = 1)."""
    Mc_lo: float = 10.0
    Mc_hi: float = 50.0
    tc_lo: float = 0.0
    tc_hi: float = 1.0
    e0_hi: float = 0.1


def draw_params(prior: Prior, B: int, seed: int, stream: int = STREAM_PARTICLES,
                offset: int = 0) -> np.ndarray:
    """B particles as a float64 array [B, 6] with columns PARAM_FIELDS; with
    `offset` = o they are particles o .. o + B - 1 of one long draw."""
    first = 5 * offset                      # index of the first uniform used
    u = uniforms(seed, stream, 5 * B + 1, offset=first // 2)[first % 2:first % 2 + 5 * B].reshape(B, 5)
    out = np.empty((B, 6))
    out[:, 0] = prior.Mc_lo + (prior.Mc_hi - prior.Mc_lo) * u[:, 0]
    out[:, 1] = prior.tc_lo + (prior.tc_hi - prior.tc_lo) * u[:, 1]
    out[:, 2] = np.arcsin(2.0 * u[:, 2] - 1.0)
    out[:, 3] = 2.0 * np.pi * u[:, 3]
    out[:, 4] = prior.e0_hi * u[:, 4]
    out[:, 5] = 1.0
    return out


# Extrinsic parameters of the injections (Table I of the paper).
INJ_IOTA = 0.5329
INJ_PSI = 1.2501
INJ_PHIC = 0.8419


# --------------------------------------------------------------------------
# Workload presets
# --------------------------------------------------------------------------
@dataclass(frozen=True)
class Workload:
    name: str
    grid: Grid
    prior: Prior
    B: int
    Np_list: tuple
    global_edges: bool
    snr: float
    seed: int = 0
    description: str = ""


def small_workload() -> Workload:
    """2^15 bins over [15, 25) mHz, 1024 particles, 8 global equal-width
    partitions, one injection at SNR 12 in Gaussian noise (seed 0)."""
    n = 1 << 15
    df = 0.01 / n
    grid = Grid(f_min=0.015, df=df, n=n, T_obs=1.0 / df)
    return Workload("fstat_small_2^15bins_B1024_Np8", grid,
                    Prior(tc_lo=0.0, tc_hi=grid.T_obs), 1024, (8,), True, 12.0, 0,
                    "2^15 bins, 15-25 mHz, B=1024, N_p=8 global edges, SNR 12")


def paper_workload() -> Workload:
    """2.5 yr single channel: 1/T bins over [10, 50) mHz (3,155,760 bins),
    8 PSO runs x 40 particles = 320 per launch, per-particle partitions with
    N_p in {256, 64, 16, 1}, one injection at SNR 12.5."""
    T = 2.5 * YEAR_S
    df = 1.0 / T
    n = int(math.floor((0.05 - 0.01) / df))
    grid = Grid(f_min=0.01, df=df, n=n, T_obs=T)
    return Workload("fstat_paper_2.5yr_3.16e6bins_B320", grid,
                    Prior(tc_lo=0.0, tc_hi=T), 320, (256, 64, 16, 1), False, 12.5, 0,
                    "2.5 yr, 10-50 mHz at 1/T, B=320 (8 runs x 40), N_p 256/64/16/1, SNR 12.5")


def tiny_grid(n: int = 4096, f_min: float = 0.02, T_obs: float = 2.5 * YEAR_S,
              stride: int = 1) -> Grid:
    """A short slice of the 2.5 yr grid (or every `stride`-th bin of it) for
    tests that the oracle must finish in seconds."""
    df = stride / T_obs
    return Grid(f_min=f_min, df=df, n=n, T_obs=T_obs)
