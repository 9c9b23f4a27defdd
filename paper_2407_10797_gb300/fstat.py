"""Thin ctypes binding of the C ABI in include/fstat.h.

Argument marshalling only: every step of the F-statistic path runs in the
library's CUDA kernels.  PyTorch provides device memory and the stream; the
binding passes raw device pointers.  There is no CPU fallback: if the shared
library cannot be loaded, or a tensor is not on a CUDA device, the call
raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

FS_OK, FS_EINVAL, FS_ECUDA, FS_ENOMEM, FS_ETIMEOUT, FS_EUNSUPPORTED = 0, -1, -2, -3, -4, -5
FS_FP64, FS_MIXED = 0, 1
FS_TDI_X, FS_TDI_AE = 0, 1
_STATUS = {0: "FS_OK", -1: "FS_EINVAL", -2: "FS_ECUDA", -3: "FS_ENOMEM", -4: "FS_ETIMEOUT",
           -5: "FS_EUNSUPPORTED"}

_lock = threading.Lock()
_lib = None


class FstatError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class fs_params(C.Structure):
    _fields_ = [("Mc", C.c_double), ("tc", C.c_double), ("lat", C.c_double), ("lon", C.c_double),
                ("e0", C.c_double), ("q", C.c_double)]


_vp = C.c_void_p
_dp = C.POINTER(C.c_double)


class fs_sample_ring(C.Structure):
    _fields_ = [("x", _vp), ("f", _vp), ("cap", C.c_int), ("count", _vp), ("dims", C.c_int)]


class fs_swarm(C.Structure):
    _fields_ = [("R", C.c_int), ("n_part", C.c_int), ("x", _vp), ("v", _vp), ("pbest_x", _vp),
                ("pbest_f", _vp), ("fit", _vp), ("box", _vp), ("q", C.c_double), ("iter", _vp), ("run0", C.c_int),
                ("dims", C.c_int)]


def load(build_if_missing: bool = True) -> C.CDLL:
    """Load libfs_gb300.so (compiling it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise ImportError(f"CUDA library {_build.LIB} is missing; run __graft_entry__.build()")
        L = C.CDLL(_build.LIB)
        L.fs_plan_create.argtypes = [C.POINTER(_vp), C.c_int64, C.c_double, C.c_double, C.c_double, C.c_int, _vp]
        L.fs_plan_create_tdi.argtypes = [C.POINTER(_vp), C.c_int64, C.c_double, C.c_double, C.c_double, C.c_int,
                                         C.c_int, _vp]
        L.fs_plan_channels.argtypes = [_vp]
        L.fs_plan_channels.restype = C.c_int
        L.fs_plan_destroy.argtypes = [_vp]
        L.fs_plan_set_data.argtypes = [_vp, _vp, _vp, _vp]
        L.fs_plan_check.argtypes = [_vp, C.POINTER(C.c_int)]
        L.fs_plan_reserve.argtypes = [_vp, C.c_int, C.c_int]
        L.fs_fstat_batch.argtypes = [_vp, _vp, C.c_int, _vp, C.c_int, _vp, _vp]
        L.fs_amplitudes.argtypes = [_vp, _vp, C.c_int, _vp, C.c_int, _vp, _vp, _vp]
        L.fs_add_signal.argtypes = [_vp, C.POINTER(fs_params), _dp, _vp]
        L.fs_constants.argtypes = [_dp]
        L.fs_particle_bands.argtypes = [_vp, _vp, C.c_int, _vp]
        L.fs_mixed_probe.argtypes = [_vp, _vp, C.c_int, _vp, C.c_int, C.c_int, C.c_int64, C.c_int64, _vp]
        L.fs_fstat_batch_noalloc.argtypes = [C.c_int64, C.c_double, C.c_double, C.c_double, _vp, _vp, _vp,
                                             C.c_int, _vp, C.c_int, _vp, _vp, _vp]
        L.fs_plan_set_profiling.argtypes = [_vp, C.c_int]
        L.fs_plan_set_variant.argtypes = [_vp, C.c_int]
        L.fs_plan_set_response.argtypes = [_vp, C.c_int, C.c_int]
        L.fs_plan_get_response.argtypes = [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.fs_plan_set_orbit.argtypes = [_vp, C.c_double]
        L.fs_plan_set_arm.argtypes = [_vp, C.c_double]
        L.fs_plan_get_arm.argtypes = [_vp, C.POINTER(C.c_double)]
        L.fs_plan_selftest_timeout.argtypes = [_vp]
        L.fs_plan_get_orbit.argtypes = [_vp, C.POINTER(C.c_double)]
        L.fs_plan_set_variant_for.argtypes = [_vp, C.c_int, C.c_int, C.c_int]
        L.fs_plan_get_variant.argtypes = [_vp, C.c_int, C.c_int, C.POINTER(C.c_int)]
        L.fs_plan_census.argtypes = [_vp, _vp, C.c_int, _vp, C.c_int, C.POINTER(C.c_int64)]
        L.fs_plan_autotune.argtypes = [_vp, _vp, C.c_int, _vp, C.c_int, C.c_int,
                                       C.POINTER(C.c_int), C.POINTER(C.c_float)]
        _sw = C.POINTER(fs_swarm)
        _ep = _vp   # edge frequencies: device pointer
        L.fs_pso_init.argtypes = [_vp, _sw, C.c_uint64]
        L.fs_pso_evaluate.argtypes = [_vp, _sw, _ep, C.c_int]
        L.fs_pso_autotune.argtypes = [_vp, _sw, _ep, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_float)]
        L.fs_pso_step.argtypes = [_vp, _sw, C.c_uint64, C.c_int, C.c_double, C.c_double, C.c_int, C.c_double,
                                  C.c_double, C.c_double, _vp]
        L.fs_pso_best.argtypes = [_vp, _sw, _vp, _vp]
        L.fs_pso_graph_build.argtypes = [_vp, _sw, _ep, C.c_int, C.c_uint64, C.c_double, C.c_double, C.c_int,
                                         C.c_double, C.c_double, C.c_double, C.POINTER(_vp)]
        L.fs_graph_run.argtypes = [_vp, C.c_int]
        _rp = C.POINTER(fs_sample_ring)
        L.fs_pso_record.argtypes = [_vp, _sw, _rp, C.c_int]
        L.fs_mlp_train_graph_build.argtypes = [C.POINTER(_vp), C.c_int, _rp, C.c_int, C.c_float, C.POINTER(_vp)]
        L.fs_pso_graph_build_ex.argtypes = [_vp, _sw, _ep, C.c_int, C.c_uint64, C.c_double, C.c_double, C.c_int,
                                            C.c_double, C.c_double, C.c_double, C.c_int, _rp, C.c_int,
                                            C.POINTER(_vp), C.c_int, C.c_int, C.POINTER(_vp)]
        L.fs_graph_destroy.argtypes = [_vp]
        L.fs_pso_step_screened.argtypes = [_vp, _sw, C.POINTER(_vp), C.c_int, C.c_int, C.c_uint64, C.c_int,
                                           C.c_double, C.c_double, C.c_int, C.c_double, C.c_double, C.c_double]
        L.fs_mlp_num_params.argtypes = [C.c_int]
        L.fs_mlp_num_params.restype = C.c_int64
        L.fs_mlp_create.argtypes = [C.POINTER(_vp), C.c_int, C.c_int, C.c_uint64, _vp]
        L.fs_mlp_create_group.argtypes = [C.POINTER(_vp), C.c_int, C.c_int, C.c_int, C.c_uint64, _vp]
        L.fs_mlp_groups.argtypes = [_vp]
        L.fs_mlp_groups.restype = C.c_int
        L.fs_mlp_destroy.argtypes = [_vp]
        L.fs_mlp_set_tensor_path.argtypes = [_vp, C.c_int]
        L.fs_mlp_tensor_status.argtypes = [_vp, C.POINTER(C.c_int)]
        L.fs_mlp_set_params.argtypes = [_vp, _vp]
        L.fs_mlp_get_params.argtypes = [_vp, _vp]
        L.fs_mlp_forward.argtypes = [_vp, _vp, C.c_int, _vp]
        L.fs_mlp_loss_grad.argtypes = [_vp, _vp, _vp, C.c_int, _vp, _vp]
        L.fs_mlp_train.argtypes = [_vp, _vp, _vp, C.c_int, C.c_int, C.c_float, _vp]
        L.fs_plan_read_profile.argtypes = [_vp, C.c_int, _dp, C.POINTER(C.c_int64)]
        L.fs_last_error.restype = C.c_char_p
        for name in ("fs_plan_create", "fs_plan_create_tdi", "fs_plan_destroy", "fs_plan_set_data", "fs_plan_check", "fs_plan_reserve",
                     "fs_fstat_batch", "fs_amplitudes", "fs_add_signal", "fs_constants", "fs_particle_bands",
                     "fs_plan_set_profiling", "fs_plan_read_profile", "fs_fstat_batch_noalloc", "fs_mixed_probe",
                     "fs_plan_set_variant", "fs_plan_set_variant_for", "fs_plan_get_variant",
                     "fs_plan_autotune", "fs_pso_autotune", "fs_plan_census", "fs_pso_init", "fs_pso_evaluate", "fs_pso_step", "fs_pso_best",
                     "fs_pso_graph_build", "fs_pso_graph_build_ex", "fs_pso_record", "fs_mlp_train_graph_build",
                     "fs_graph_run", "fs_graph_destroy", "fs_mlp_create", "fs_mlp_create_group",
                     "fs_mlp_destroy", "fs_mlp_set_tensor_path", "fs_mlp_tensor_status", "fs_mlp_set_params", "fs_mlp_get_params", "fs_mlp_forward",
                     "fs_mlp_loss_grad", "fs_mlp_train", "fs_pso_step_screened"):
            getattr(L, name).restype = C.c_int
        _lib = L
        return L


def _check(st: int):
    if st != FS_OK:
        raise FstatError(st, load().fs_last_error().decode())


def constants() -> np.ndarray:
    out = np.zeros(4)
    _check(load().fs_constants(out.ctypes.data_as(_dp)))
    return out


def _cuda_ptr(t, dtype=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _check_size(t, n: int, what: str):
    """The library reads or writes exactly n elements of t: refuse any other size."""
    if t.numel() != n:
        raise ValueError(f"{what} holds {t.numel()} elements, the call needs {n}")


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Plan:
    """One frequency grid + precision mode; wraps fs_plan."""

    def __init__(self, n_bins: int, f_min: float, df: float, T_obs: float, mode: int = FS_FP64, stream=None,
                 tdi: int = FS_TDI_X):
        import torch
        L = load()
        self._L = L
        self.n = int(n_bins)
        self.mode = int(mode)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        _check(L.fs_plan_create_tdi(C.byref(h), self.n, float(f_min), float(df), float(T_obs), int(mode), int(tdi),
                                    _stream_handle(self.stream)))
        self._h = h
        self.nch = L.fs_plan_channels(h)

    @classmethod
    def from_grid(cls, grid, mode: int = FS_FP64, stream=None, tdi: int = FS_TDI_X) -> "Plan":
        return cls(grid.n, grid.f_min, grid.df, grid.T_obs, mode, stream, tdi)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.fs_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_data(self, data, psd, f_grid=None):
        """data: complex128 CUDA tensor [n] (or float64 [n, 2]), [channels, n] for a
        plan with several channels; psd: float64 CUDA tensor [n] ([channels, n]);
        f_grid: optional float64 CUDA tensor [n] of the data's frequencies (must be the
        plan's uniform grid; FstatError FS_EUNSUPPORTED otherwise)."""
        import torch
        if data.dtype == torch.complex128:
            data = torch.view_as_real(data)
        if data.numel() != 2 * self.nch * self.n or psd.numel() != self.nch * self.n or data.shape[-1] != 2:
            raise ValueError(f"data must be [{self.nch}, {self.n}] complex and psd [{self.nch}, {self.n}]")
        if f_grid is not None:
            _check_size(f_grid, self.n, "f_grid")
        # keep the inputs alive until the stream has consumed them
        self._data_keep = data.contiguous()
        self._psd_keep = psd.contiguous()
        _check(self._L.fs_plan_set_data(self._h, _cuda_ptr(self._data_keep, torch.float64),
                                        _cuda_ptr(self._psd_keep, torch.float64),
                                        _cuda_ptr(f_grid.contiguous(), torch.float64) if f_grid is not None
                                        else None))

    def check(self) -> int:
        """fs_plan_check: flag bits the device raised since the last check (raises
        FstatError FS_EINVAL if a call was given invalid partition edges,
        FS_ETIMEOUT if a bounded device-side wait ran out)."""
        f = C.c_int()
        _check(self._L.fs_plan_check(self._h, C.byref(f)))
        return f.value

    def selftest_timeout(self):
        """fs_plan_selftest_timeout: one device wait that runs out by design; the next
        check() raises FstatError FS_ETIMEOUT."""
        _check(self._L.fs_plan_selftest_timeout(self._h))

    def reserve(self, B_max: int, Np_max: int):
        _check(self._L.fs_plan_reserve(self._h, int(B_max), int(Np_max)))

    def fstat(self, params, Np: int, edges=None, F=None, F_part=None, want_parts: bool = True):
        """Semi-coherent F for params (float64 CUDA tensor [B, 6]: Mc, tc, lat, lon, e0, q).
        edges: None (per-particle segments) or N_p + 1 edge frequencies in Hz, best
        as a float64 CUDA tensor (any other array is copied to the device on every call).
        Returns (F [B], F_part [B, Np] or None) as CUDA tensors."""
        import torch
        if params.dim() != 2 or params.shape[1] != 6:
            raise ValueError("params must be [B, 6]")
        B = params.shape[0]
        dev = params.device
        if F is None:
            F = torch.empty(B, dtype=torch.float64, device=dev)
        if want_parts and F_part is None:
            F_part = torch.empty(B, Np, dtype=torch.float64, device=dev)
        _check_size(F, B, "F")
        if F_part is not None:
            _check_size(F_part, B * Np, "F_part")
        self._edges_keep, e = _edges_arg(edges, Np, dev, self.stream)
        _check(self._L.fs_fstat_batch(self._h, _cuda_ptr(params.contiguous(), torch.float64), int(B), e, int(Np),
                                      _cuda_ptr(F, torch.float64),
                                      _cuda_ptr(F_part, torch.float64) if F_part is not None else None))
        return F, F_part

    def amplitudes(self, params, Np: int = 1, edges=None, extrinsic: bool = True):
        """(F [B], a [B, N_p, 4], (D_L, iota, psi, phi_c) [B, N_p, 4] or None):
        maximum-likelihood amplitudes per segment and their extrinsic parameters."""
        import torch
        if params.dim() != 2 or params.shape[1] != 6:
            raise ValueError("params must be [B, 6]")
        B = params.shape[0]
        dev = params.device
        F = torch.empty(B, dtype=torch.float64, device=dev)
        a = torch.empty(B, Np, 4, dtype=torch.float64, device=dev)
        ext = torch.empty(B, Np, 4, dtype=torch.float64, device=dev) if extrinsic else None
        self._edges_keep, e = _edges_arg(edges, Np, dev, self.stream)
        _check(self._L.fs_amplitudes(self._h, _cuda_ptr(params.contiguous(), torch.float64), int(B), e, int(Np),
                                     _cuda_ptr(F, torch.float64), _cuda_ptr(a, torch.float64),
                                     _cuda_ptr(ext, torch.float64) if ext is not None else None))
        return F, a, ext

    def bands(self, params, out=None):
        """Per-particle (first, last) in-band bin, int64 CUDA tensor [B, 2]."""
        import torch
        if params.dim() != 2 or params.shape[1] != 6:
            raise ValueError("params must be [B, 6]")
        B = params.shape[0]
        if out is None:
            out = torch.empty(B, 2, dtype=torch.int64, device=params.device)
        _check_size(out, 2 * B, "out")
        _check(self._L.fs_particle_bands(self._h, _cuda_ptr(params.contiguous(), torch.float64), int(B),
                                         _cuda_ptr(out, torch.int64)))
        return out

    PROBE_FIELDS = ("mode", "k_anchor", "seg", "orb", "dalpha", "dop", "ph", "G1", "G2", "rot_c", "rot_s",
                    "cos", "sin", "tw_re", "tw_im", "tw_W", "t0", "t1", "t2", "t3", "t4", "t5", "t6", "rot_c_lo",
                    "rot_s_lo", "unused0", "unused1", "unused2")

    def mixed_probe(self, params, Np: int, b: int, k0: int, nbins: int, edges=None):
        """fs_mixed_probe: per-bin values of the FS_MIXED body for particle b over
        bins [k0, k0 + nbins); float32 CUDA tensor [nbins, 28] (PROBE_FIELDS)."""
        import torch
        if params.dim() != 2 or params.shape[1] != 6:
            raise ValueError("params must be [B, 6]")
        out = torch.empty(int(nbins), len(self.PROBE_FIELDS), dtype=torch.float32, device=params.device)
        self._edges_keep, e = _edges_arg(edges, Np, params.device, self.stream)
        _check(self._L.fs_mixed_probe(self._h, _cuda_ptr(params.contiguous(), torch.float64), int(params.shape[0]),
                                      e, int(Np), int(b), int(k0), int(nbins),
                                      _cuda_ptr(out, torch.float32) if nbins > 0 else None))
        return out

    KERNELS = {"setup": 0, "main": 1, "reduce": 2, "precompute": 3}

    def set_response(self, filter_order: int = -1, k_max: int = 0):
        """Response model of the FS_FP64 path: -1 the paper's form, 0..2 the series of
        Eq. (freDres) with that filter order and terms up to k_max (0 or 1)."""
        _check(self._L.fs_plan_set_response(self._h, int(filter_order), int(k_max)))

    def get_response(self) -> tuple[int, int]:
        n, k = C.c_int(), C.c_int()
        _check(self._L.fs_plan_get_response(self._h, C.byref(n), C.byref(k)))
        return n.value, k.value

    def set_orbit(self, eccentricity: float = 0.0):
        """Spacecraft orbits of the FS_FP64 path: 0 the rigid constellation, e > 0 the
        orbits to second order in eccentricity e (LISA: 4.824e-3)."""
        _check(self._L.fs_plan_set_orbit(self._h, float(eccentricity)))

    def set_arm(self, arm_seconds: float = 0.0):
        """Arm transfer of the FS_FP64 response: 0 the long-wavelength limit, L > 0 the
        finite-arm TDI response with nominal arm L seconds (LISA: 8.339)."""
        _check(self._L.fs_plan_set_arm(self._h, float(arm_seconds)))

    def get_arm(self) -> float:
        v = C.c_double()
        _check(self._L.fs_plan_get_arm(self._h, C.byref(v)))
        return v.value

    def get_orbit(self) -> float:
        e = C.c_double()
        _check(self._L.fs_plan_get_orbit(self._h, C.byref(e)))
        return e.value

    def set_variant(self, variant: int):
        """Force a launch variant of the fused kernel for every call (-1: per-N_p choice)."""
        _check(self._L.fs_plan_set_variant(self._h, int(variant)))

    def set_variant_for(self, Np: int, variant: int, global_edges: bool = False):
        _check(self._L.fs_plan_set_variant_for(self._h, int(Np), 1 if global_edges else 0, int(variant)))

    def get_variant(self, Np: int, global_edges: bool = False) -> int:
        v = C.c_int()
        _check(self._L.fs_plan_get_variant(self._h, int(Np), 1 if global_edges else 0, C.byref(v)))
        return v.value

    @property
    def n_variants(self) -> int:
        return 5

    def autotune(self, params, Np: int, edges=None, reps: int = 3):
        """Time every launch variant on this batch and keep the fastest for
        (N_p, edge kind).  Returns (variant, [mean ms per call of each variant])."""
        import torch
        self._edges_keep, e = _edges_arg(edges, Np, params.device, self.stream)
        v = C.c_int()
        ms = (C.c_float * 8)()
        _check(self._L.fs_plan_autotune(self._h, _cuda_ptr(params.contiguous(), torch.float64), int(params.shape[0]),
                                        e, int(Np), int(reps), C.byref(v), ms))
        return v.value, [ms[i] for i in range(self.n_variants)]

    def census(self, params, Np: int, edges=None) -> list[int]:
        """In-band particle*bins per anchor mode (fs_plan_census), 9 entries:
        [unused, widest tier or FP32 body, bin-by-bin fallback, tier 3 or the
        mixed low-degree tier, tiers 4, 5 (narrowest), tier 5 with the FP32
        phase remainder, the same with antenna degree 5, with degree 4]."""
        import torch
        self._edges_keep, e = _edges_arg(edges, Np, params.device, self.stream)
        out = (C.c_int64 * 9)()
        _check(self._L.fs_plan_census(self._h, _cuda_ptr(params.contiguous(), torch.float64), int(params.shape[0]),
                                      e, int(Np), out))
        return [int(out[i]) for i in range(9)]

    def set_profiling(self, enable: bool):
        _check(self._L.fs_plan_set_profiling(self._h, 1 if enable else 0))

    def read_profile(self, kernel: str) -> tuple[float, int]:
        """(summed ms, launches) of one kernel kind since the last read; waits for the stream."""
        ms = C.c_double()
        n = C.c_int64()
        _check(self._L.fs_plan_read_profile(self._h, self.KERNELS[kernel], C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def add_signal(self, p, a, data):
        """data += sum_i a_i A^i(p) over the particle's band (data: complex128 CUDA tensor,
        [channels, n] for a plan with several channels, each through its own response)."""
        import torch
        if data.dtype == torch.complex128:
            view = torch.view_as_real(data)
        else:
            view = data
        _check_size(view, 2 * self.nch * self.n, "data (re, im pairs per channel)")
        pp = fs_params(*[float(x) for x in np.asarray(p, dtype=np.float64)[:6]])
        aa = np.ascontiguousarray(a, dtype=np.float64)
        _check(self._L.fs_add_signal(self._h, C.byref(pp), aa.ctypes.data_as(_dp), _cuda_ptr(view, torch.float64)))
        return data


def fstat_batch_noalloc(grid, data, psd, params, Np: int, edges=None, F=None, F_part=None, stream=None):
    """fs_fstat_batch_noalloc: FP64 F-statistic that allocates no device memory
    (workspace in the library's fixed 10 MiB device array; n_bins <= 32768,
    B <= 1024, N_p <= 64).  For callers that cannot allocate device memory; the
    output tensors here are made by the caller (this wrapper creates them with
    torch if not given).  Calls that overlap on the GPU race on the shared
    workspace.  Every tensor must be on one CUDA device; the call is made with
    that device current (the library finds its array on the current device)."""
    import torch
    L = load()
    if data.dtype == torch.complex128:
        data = torch.view_as_real(data)
    if params.dim() != 2 or params.shape[1] != 6:
        raise ValueError("params must be [B, 6]")
    B = params.shape[0]
    dev = params.device
    if F is None:
        F = torch.empty(B, dtype=torch.float64, device=dev)
    _check_size(data, 2 * int(grid.n), "data (re, im pairs)")
    _check_size(psd, int(grid.n), "psd")
    _check_size(F, B, "F")
    if F_part is not None:
        _check_size(F_part, B * Np, "F_part")
    keep, e = _edges_arg(edges, Np, dev, stream)
    for name, t in (("data", data), ("psd", psd), ("F", F), ("F_part", F_part), ("edges", keep)):
        if t is not None and t.device != dev:
            raise ValueError(f"{name} is on {t.device}, params on {dev}: all tensors must share one device")
    with torch.cuda.device(dev):
        _check(L.fs_fstat_batch_noalloc(int(grid.n), float(grid.f_min), float(grid.df), float(grid.T_obs),
                                        _cuda_ptr(data, torch.float64), _cuda_ptr(psd, torch.float64),
                                        _cuda_ptr(params, torch.float64), int(B), e, int(Np),
                                        _cuda_ptr(F, torch.float64),
                                        _cuda_ptr(F_part, torch.float64) if F_part is not None else None,
                                        _stream_handle(stream)))
    return F, F_part


def _edges_arg(edges, Np, device, stream=None):
    """Global segment edges as N_p + 1 frequencies (Hz) in device memory: a float64
    CUDA tensor is passed as it is; other array-likes are copied to `device` on
    the current stream, which `stream` (the stream the library will read them
    on) then waits for.  Returns (tensor to keep alive while the stream or a
    graph reads it, pointer)."""
    if edges is None:
        return None, None
    import torch
    if isinstance(edges, torch.Tensor) and edges.is_cuda:
        t = edges.contiguous()
        if t.dtype != torch.float64:
            raise TypeError("edges must be float64 frequencies")
        if t.device != torch.device(device):
            raise ValueError(f"edges are on {t.device}, the call runs on {device}")
    else:
        t = torch.as_tensor(np.ascontiguousarray(edges, dtype=np.float64)).to(device)
        if stream is not None and stream != torch.cuda.current_stream(device):
            stream.wait_stream(torch.cuda.current_stream(device))
            t.record_stream(stream)
    if t.shape != (Np + 1,):
        raise ValueError("edges must have N_p + 1 entries")
    return t, C.c_void_p(t.data_ptr())


class Swarm:
    """Device state of R PSO runs x n_part particles in [0,1]^D (fs_swarm).

    box: float64 [R, D, 2] search boxes (lo, hi) of (M_c [Msun], t_c [s],
    sin(lat), lon [rad], e0) and, with dims = 6, delta_mu (the mass ratio is
    then each particle's (1 + delta_mu)/(1 - delta_mu) instead of q)."""

    def __init__(self, plan: "Plan", R: int, n_part: int, box, q: float = 1.0, run0: int = 0, dims: int = 5):
        import torch
        if dims not in (5, 6):
            raise ValueError("dims must be 5 or 6")
        self.plan = plan
        self.R, self.n_part, self.dims = int(R), int(n_part), int(dims)
        dev = torch.device("cuda", torch.cuda.current_device())
        z = lambda *shape: torch.zeros(*shape, dtype=torch.float64, device=dev)
        self.x = z(R, n_part, dims)
        self.v = z(R, n_part, dims)
        self.pbest_x = z(R, n_part, dims)
        self.pbest_f = z(R, n_part)
        self.fit = z(R, n_part)
        self.box = torch.as_tensor(np.ascontiguousarray(box, dtype=np.float64)).to(dev).reshape(R, dims, 2).contiguous()
        self.iter = torch.zeros(1, dtype=torch.int32, device=dev)
        self.best_f = z(R)
        self.best_i = torch.zeros(R, dtype=torch.int32, device=dev)
        self.c = fs_swarm(self.R, self.n_part, self.x.data_ptr(), self.v.data_ptr(), self.pbest_x.data_ptr(),
                          self.pbest_f.data_ptr(), self.fit.data_ptr(), self.box.data_ptr(), float(q),
                          self.iter.data_ptr(), int(run0), int(dims))

    def set_box(self, box):
        import torch
        self.box.copy_(torch.as_tensor(np.ascontiguousarray(box, dtype=np.float64)).reshape(self.R, self.dims, 2))

    def init(self, seed: int):
        _check(load().fs_pso_init(self.plan._h, C.byref(self.c), int(seed)))

    def evaluate(self, Np: int, edges=None):
        self._edges_keep, e = _edges_arg(edges, Np, self.x.device, self.plan.stream)
        _check(load().fs_pso_evaluate(self.plan._h, C.byref(self.c), e, int(Np)))

    def autotune(self, Np: int, edges=None, reps: int = 3):
        """fs_pso_autotune: pick the plan's fastest variant on the current positions."""
        self._edges_keep, e = _edges_arg(edges, Np, self.x.device, self.plan.stream)
        v = C.c_int()
        ms = (C.c_float * 8)()
        _check(load().fs_pso_autotune(self.plan._h, C.byref(self.c), e, int(Np), int(reps), C.byref(v), ms))
        return v.value, [ms[i] for i in range(self.plan.n_variants)]

    def step(self, seed: int, iteration: int, w0=0.9, w1=0.4, n_iter=2, c1=2.0, c2=2.0, vmax=0.5, lbest=None):
        import torch
        if lbest is not None:
            _check_size(lbest, self.R * self.n_part, "lbest")
        _check(load().fs_pso_step(self.plan._h, C.byref(self.c), int(seed), int(iteration), float(w0), float(w1),
                                  int(n_iter), float(c1), float(c2), float(vmax),
                                  None if lbest is None else _cuda_ptr(lbest, torch.int32)))

    def step_screened(self, mlp, n_cand: int, seed: int, iteration: int, w0=0.9, w1=0.4, n_iter=2, c1=2.0,
                      c2=2.0, vmax=0.5):
        """Screened step; mlp: one MLP or a list of them (one per equal group of runs)."""
        arr = _mlp_array(mlp)
        _check(load().fs_pso_step_screened(self.plan._h, C.byref(self.c), arr, len(arr), int(n_cand), int(seed),
                                           int(iteration), float(w0), float(w1), int(n_iter), float(c1), float(c2),
                                           float(vmax)))

    def best(self):
        """(best fitness [R], best particle index [R]) as CUDA tensors."""
        _check(load().fs_pso_best(self.plan._h, C.byref(self.c), C.c_void_p(self.best_f.data_ptr()),
                                  C.c_void_p(self.best_i.data_ptr())))
        return self.best_f, self.best_i

    def graph_build(self, Np: int, seed: int, edges=None, w0=0.9, w1=0.4, n_iter=2, c1=2.0, c2=2.0, vmax=0.5):
        """Capture one PSO iteration of this swarm as a CUDA graph (replaces a previous one).
        Edge frequencies are read from device memory each time the graph runs."""
        keep, e = _edges_arg(edges, Np, self.x.device, self.plan.stream)
        self.graph_free()
        h = C.c_void_p()
        _check(load().fs_pso_graph_build(self.plan._h, C.byref(self.c), e, int(Np), int(seed), float(w0),
                                         float(w1), int(n_iter), float(c1), float(c2), float(vmax), C.byref(h)))
        self._graph = h
        self._graph_edges = keep

    def graph_run(self, n: int):
        _check(load().fs_graph_run(self._graph, int(n)))

    def record(self, ring):
        """Append the current (positions, fitness) to a sample ring, or to a list of
        rings (one per equal group of runs) (fs_pso_record)."""
        rings = _ring_array(ring)
        _check(load().fs_pso_record(self.plan._h, C.byref(self.c), rings, len(rings)))

    def graph_build_ex(self, parts: int, Np: int, seed: int, edges=None, ring=None, mlp=None, n_cand: int = 16,
                       w0=0.9, w1=0.4, n_iter=2, c1=2.0, c2=2.0, vmax=0.5) -> "Graph":
        """Capture part of a PSO iteration (fs_pso_graph_build_ex; parts: 1 evaluate,
        2 record to `ring` (one or a list), 4 step, 8 screened step with `mlp` (one or a list))."""
        keep, e = _edges_arg(edges, Np, self.x.device, self.plan.stream)
        rings = _ring_array(ring) if ring is not None else None
        mlps = _mlp_array(mlp) if mlp is not None else None
        h = C.c_void_p()
        _check(load().fs_pso_graph_build_ex(self.plan._h, C.byref(self.c), e, int(Np), int(seed), float(w0),
                                            float(w1), int(n_iter), float(c1), float(c2), float(vmax), int(parts),
                                            rings, 0 if rings is None else len(rings), mlps,
                                            0 if mlps is None else len(mlps), int(n_cand), C.byref(h)))
        return Graph(h, keep)

    def graph_free(self):
        g = getattr(self, "_graph", None)
        if g is not None and g.value:
            load().fs_graph_destroy(g)
        self._graph = None

    def __del__(self):
        try:
            self.graph_free()
        except Exception:
            pass


def _mlp_array(mlp):
    nets = list(mlp) if isinstance(mlp, (list, tuple)) else [mlp]
    return (C.c_void_p * len(nets))(*[n._h.value for n in nets])


def _ring_array(ring):
    rings = list(ring) if isinstance(ring, (list, tuple)) else [ring]
    return (fs_sample_ring * len(rings))(*[r.c for r in rings])


def mlp_train_graph(nets, rings, steps: int, lr: float = 1e-3) -> "Graph":
    """fs_mlp_train_graph_build: `steps` Adam steps of every network on its ring's
    whole contents, captured as one graph."""
    arr = _mlp_array(nets)
    rarr = _ring_array(rings)
    nlist = list(nets) if isinstance(nets, (list, tuple)) else [nets]
    if sum(n.groups for n in nlist) != len(rarr):
        raise ValueError("one ring per network (a batch of G networks takes G rings from SampleRing.batch)")
    h = C.c_void_p()
    _check(load().fs_mlp_train_graph_build(arr, len(arr), rarr, int(steps), float(lr), C.byref(h)))
    return Graph(h)


class Graph:
    """A captured part of a PSO iteration or a training round (fs_graph)."""

    def __init__(self, h, keep=None):
        self._h = h
        self._keep = keep   # device buffers the graph reads when it runs (edge frequencies)

    def run(self, n: int = 1):
        _check(load().fs_graph_run(self._h, int(n)))

    def close(self):
        if self._h is not None and self._h.value:
            load().fs_graph_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SampleRing:
    """Device ring of (position, fitness) training samples (fs_sample_ring);
    dims: the dimensions of the swarms that append to it."""

    def __init__(self, cap: int, device=None, dims: int = 5):
        import torch
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.cap = int(cap)
        self.x = torch.zeros(self.cap, dims, dtype=torch.float32, device=dev)
        self.f = torch.full((self.cap,), float("nan"), dtype=torch.float32, device=dev)
        self.count = torch.zeros(1, dtype=torch.int64, device=dev)
        self.c = fs_sample_ring(self.x.data_ptr(), self.f.data_ptr(), self.cap, self.count.data_ptr(), int(dims))

    @classmethod
    def batch(cls, n: int, cap: int, device=None, dims: int = 5) -> list:
        """n rings of one capacity laid end to end in one buffer (x: [n][cap][dims],
        f: [n][cap]), the layout a batch of n networks trains on."""
        import torch
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        x = torch.zeros(n, int(cap), dims, dtype=torch.float32, device=dev)
        f = torch.full((n, int(cap)), float("nan"), dtype=torch.float32, device=dev)
        count = torch.zeros(n, dtype=torch.int64, device=dev)
        out = []
        for j in range(n):
            r = cls.__new__(cls)
            r.cap = int(cap)
            r.x, r.f, r.count = x[j], f[j], count[j:j + 1]
            r.c = fs_sample_ring(r.x.data_ptr(), r.f.data_ptr(), r.cap, r.count.data_ptr(), int(dims))
            out.append(r)
        return out


def torch_tensor(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()


class MLP:
    """Surrogate network (fs_mlp): 5 -> width^3 -> 1, bf16 tensor-core kernels.

    groups > 1 makes a batch of independent networks (network g seeded
    seed + g) that every kernel evaluates and trains together; its inputs are
    then [groups][N][5], targets and outputs [groups][N], parameters
    [groups][P]."""

    def __init__(self, width: int = 256, max_batch: int = 8192, seed: int = 0, stream=None, groups: int = 1):
        import torch
        self._L = load()
        self.width = int(width)
        self.groups = int(groups)
        self.P = int(self._L.fs_mlp_num_params(self.width))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        if self.groups == 1:
            _check(self._L.fs_mlp_create(C.byref(h), self.width, int(max_batch), int(seed),
                                         _stream_handle(self.stream)))
        else:
            _check(self._L.fs_mlp_create_group(C.byref(h), self.groups, self.width, int(max_batch), int(seed),
                                               _stream_handle(self.stream)))
        self._h = h

    def _rows(self, X):
        """Rows per network of an input batch ([N][5] for one network, [G][N][5] for G)."""
        if X.dim() < 1 or X.shape[-1] != 5:
            raise ValueError("inputs are rows of 5 normalised coordinates")
        if self.groups == 1:
            return int(X.numel() // 5)
        if X.dim() != 3 or X.shape[0] != self.groups:
            raise ValueError(f"a batch of {self.groups} networks takes inputs [{self.groups}][N][5]")
        return int(X.shape[1])

    def _check_len(self, v, n, what):
        """The library reads or writes exactly n floats of v: refuse any other size."""
        if v.numel() != n:
            raise ValueError(f"{what} holds {v.numel()} values, the call needs {n}")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.fs_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tensor_path(self, tcgen05):
        """True or 1: tcgen05 GEMMs (TMEM accumulators; TMA-fed forward layers);
        2: tcgen05 forward layers, mma.sync backward; False or 0: mma.sync GEMMs."""
        path = int(tcgen05) if not isinstance(tcgen05, bool) else (1 if tcgen05 else 0)
        _check(self._L.fs_mlp_set_tensor_path(self._h, path))

    def tensor_status(self) -> bool:
        """True if no tcgen05 GEMM of this network timed out (waits for its stream)."""
        flag = C.c_int()
        st = self._L.fs_mlp_tensor_status(self._h, C.byref(flag))
        return st == FS_OK and flag.value == 0

    def params(self):
        import torch
        out = torch.empty(self.P if self.groups == 1 else (self.groups, self.P), dtype=torch.float32,
                          device="cuda")
        self.stream.synchronize()   # out was made on the current stream; the copy runs on the network's
        _check(self._L.fs_mlp_get_params(self._h, _cuda_ptr(out, torch.float32)))
        self.stream.synchronize()
        return out

    def set_params(self, theta):
        import torch
        theta = theta.to(torch.float32).contiguous()
        self._check_len(theta, self.groups * self.P, "theta")
        _check(self._L.fs_mlp_set_params(self._h, _cuda_ptr(theta, torch.float32)))

    def forward(self, X, y=None):
        import torch
        X = X.to(torch.float32).contiguous()
        n = self._rows(X)
        if y is None:
            y = torch.empty(X.shape[:-1], dtype=torch.float32, device=X.device)
        self._check_len(y, self.groups * n, "y")
        _check(self._L.fs_mlp_forward(self._h, _cuda_ptr(X, torch.float32), n, _cuda_ptr(y, torch.float32)))
        return y

    def loss_grad(self, X, t):
        import torch
        X = X.to(torch.float32).contiguous()
        t = t.to(torch.float32).contiguous()
        self._check_len(t, self.groups * self._rows(X), "t")
        g = torch.empty(self.groups * self.P, dtype=torch.float32, device=X.device)
        L = torch.empty(self.groups, dtype=torch.float32, device=X.device)
        _check(self._L.fs_mlp_loss_grad(self._h, _cuda_ptr(X, torch.float32), _cuda_ptr(t, torch.float32),
                                        self._rows(X), _cuda_ptr(g, torch.float32), _cuda_ptr(L, torch.float32)))
        return L, g

    def train(self, X, t, steps: int, lr: float = 1e-3):
        import torch
        X = X.to(torch.float32).contiguous()
        t = t.to(torch.float32).contiguous()
        self._check_len(t, self.groups * self._rows(X), "t")
        losses = torch.empty(max(int(steps), 1) * self.groups, dtype=torch.float32, device=X.device)
        _check(self._L.fs_mlp_train(self._h, _cuda_ptr(X, torch.float32), _cuda_ptr(t, torch.float32),
                                    self._rows(X), int(steps), float(lr), _cuda_ptr(losses, torch.float32)))
        if self.groups > 1:
            losses = losses.reshape(-1, self.groups)
        return losses
