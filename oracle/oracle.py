"""ctypes front end of the CPU oracle (fstat_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, `__graft_entry__.smoke()` and the
benchmark's CPU-baseline leg may import this module; the product package
never does.  It shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fstat_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FP contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(C.Structure):
    _fields_ = [("Mc", C.c_double), ("tc", C.c_double), ("lat", C.c_double),
                ("lon", C.c_double), ("e0", C.c_double), ("q", C.c_double)]


class Model(C.Structure):
    _fields_ = [("f_min", C.c_double), ("df", C.c_double), ("T_obs", C.c_double),
                ("n", C.c_int64), ("response", C.c_int), ("pn_order", C.c_int),
                ("alpha0", C.c_double), ("orient", C.c_double), ("channel", C.c_int),
                ("mb_order", C.c_int), ("mb_kmax", C.c_int), ("ecc", C.c_double), ("arm_s", C.c_double),
                ("no_doppler", C.c_int)]


_dp = C.POINTER(C.c_double)
_i64p = C.POINTER(C.c_int64)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.or_fstat_batch.argtypes = [C.POINTER(Params), C.c_int, C.POINTER(Model), _dp, _dp, _dp,
                                         _i64p, C.c_int, _dp, _dp, C.c_int]
            L.or_fstat_batch.restype = C.c_int
            L.or_fstat_batch_multi.argtypes = [C.POINTER(Params), C.c_int, C.POINTER(Model), C.c_int, _dp, _dp, _dp,
                                               _i64p, C.c_int, _dp, _dp, C.c_int]
            L.or_fstat_batch_multi.restype = C.c_int
            L.or_segment_sums.argtypes = [C.POINTER(Params), C.POINTER(Model), _dp, _dp, _dp, _i64p,
                                          C.c_int, _dp, _dp, _i64p]
            L.or_edge_starts.argtypes = [C.POINTER(Model), _dp, C.c_int, _i64p]
            L.or_edge_starts.restype = C.c_int
            L.or_segment_F.argtypes = [_dp, _dp, C.c_int64]
            L.or_segment_F.restype = C.c_double
            L.or_basis.argtypes = [C.POINTER(Params), C.POINTER(Model), C.c_int64, C.c_int64, _dp, _dp]
            L.or_band.argtypes = [C.POINTER(Params), C.POINTER(Model), _i64p, _i64p]
            L.or_time_of_freq.argtypes = [C.POINTER(Params), C.POINTER(Model), C.c_double]
            L.or_time_of_freq.restype = C.c_double
            L.or_phase_orb_cycles_d.argtypes = [C.POINTER(Params), C.POINTER(Model), C.c_double]
            L.or_phase_orb_cycles_d.restype = C.c_double
            L.or_phase_frac.argtypes = [C.POINTER(Params), C.POINTER(Model), C.c_double, C.c_double,
                                        C.c_int64]
            L.or_phase_frac.restype = C.c_double
            L.or_antenna_at.argtypes = [C.POINTER(Params), C.POINTER(Model), C.c_double, _dp, _dp]
            L.or_doppler_at.argtypes = [C.POINTER(Params), C.POINTER(Model), C.c_double]
            L.or_doppler_at.restype = C.c_double
            L.or_detector_tensor_at.argtypes = [C.POINTER(Model), C.c_double, _dp]
            L.or_detector_tensor_at.restype = None
            L.or_extrinsic_to_a.argtypes = [C.c_double] * 4 + [_dp]
            L.or_a_to_extrinsic.argtypes = [_dp, _dp, _dp, _dp, _dp]
            L.or_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                           C.POINTER(C.c_uint32)]
            L.or_pso_init.argtypes = [C.c_int, C.c_int, C.c_int, C.c_uint64, _dp, _dp]
            L.or_pso_step.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _dp, _dp, _dp, _dp, C.c_uint64,
                                      C.c_uint32, C.c_double, C.c_double, C.c_double, C.c_double,
                                      C.POINTER(C.c_int)]
            L.or_num_threads.restype = C.c_int
            L.or_mb_weights.argtypes = [C.c_int, _dp, _dp]
            L.or_mb_weights.restype = None
            L.or_mb_response_at.argtypes = [C.POINTER(Params), C.POINTER(Model), C.c_double, _dp]
            L.or_mb_response_at.restype = None
            L.or_doppler_rates_at.argtypes = [C.POINTER(Params), C.POINTER(Model), C.c_double, _dp, _dp]
            L.or_doppler_rates_at.restype = None
            L.or_sc_offset_at.argtypes = [C.POINTER(Model), C.c_int, C.c_double, _dp]
            L.or_sc_offset_at.restype = None
            L.or_tdi_response_at.argtypes = [C.POINTER(Params), C.POINTER(Model), C.c_double, C.c_double, _dp]
            L.or_tdi_response_at.restype = None
            _lib = L
    return _lib


def _ptr(a: np.ndarray, ct=C.c_double):
    return a.ctypes.data_as(C.POINTER(ct))


@dataclass
class OracleModel:
    """Frequency grid and response options of the oracle."""
    f_min: float
    df: float
    n: int
    T_obs: float
    response: int = 0      # 0 LISA response, 1 test mode (F+ = 1, Fx = 0, no Doppler)
    pn_order: int = 4
    alpha0: float = 0.0
    orient: float = 0.0
    channel: int = 0       # TDI channel: 0 X, 1 A, 2 E, 3 T
    mb_order: int = -1     # -1 the paper's response; 0..2 the Eq. (freDres) series with filter order N
    mb_kmax: int = 0       # highest k of that series (0 or 1)
    ecc: float = 0.0       # 0 the rigid constellation; > 0 the orbits to second order in this eccentricity
    arm_s: float = 0.0     # 0 the long-wavelength response; > 0 the finite-arm TDI response, arm length in s
    no_doppler: int = 0    # 1: no Doppler delay of the guiding centre (test knob)

    @staticmethod
    def from_grid(grid, **kw) -> "OracleModel":
        return OracleModel(grid.f_min, grid.df, grid.n, grid.T_obs, **kw)

    def c(self) -> Model:
        return Model(self.f_min, self.df, self.T_obs, self.n, self.response, self.pn_order,
                     self.alpha0, self.orient, self.channel, self.mb_order, self.mb_kmax, self.ecc,
                     self.arm_s, self.no_doppler)


def _params(p) -> Params:
    p = np.asarray(p, dtype=np.float64)
    return Params(*[float(x) for x in p[:6]])


def _params_array(P: np.ndarray):
    P = np.ascontiguousarray(P, dtype=np.float64)
    arr = (Params * len(P))()
    for i, row in enumerate(P):
        arr[i] = Params(*[float(x) for x in row[:6]])
    return arr


def edge_starts(model: OracleModel, edges_hz, Np: int) -> np.ndarray:
    """Segment start bins [Np + 1] of global edge frequencies (Sec. II.B membership rule)."""
    e = np.ascontiguousarray(edges_hz, dtype=np.float64)
    if e.shape != (Np + 1,):
        raise ValueError("edges_hz must have N_p + 1 entries")
    out = np.zeros(Np + 1, dtype=np.int64)
    m = model.c()
    if lib().or_edge_starts(C.byref(m), _ptr(e), int(Np), _ptr(out, C.c_int64)) != 0:
        raise ValueError("edge frequencies must be finite and non-decreasing")
    return out


def fstat_batch(params: np.ndarray, model: OracleModel, data: np.ndarray, psd: np.ndarray,
                Np: int, edges: np.ndarray | None = None, nthreads: int = 0, edges_hz=None):
    """F[b] = sum over segments of F_p and Fpart[b, p] for params [B, 6].
    Global segments as start bins (edges) or as edge frequencies (edges_hz)."""
    if edges_hz is not None:
        edges = edge_starts(model, edges_hz, Np)
    B = len(params)
    d_re = np.ascontiguousarray(data.real, dtype=np.float64)
    d_im = np.ascontiguousarray(data.imag, dtype=np.float64)
    psd = np.ascontiguousarray(psd, dtype=np.float64)
    F = np.zeros(B)
    Fp = np.zeros((B, Np))
    e = None if edges is None else np.ascontiguousarray(edges, dtype=np.int64)
    m = model.c()
    rc = lib().or_fstat_batch(_params_array(params), B, C.byref(m), _ptr(d_re), _ptr(d_im), _ptr(psd),
                              None if e is None else _ptr(e, C.c_int64), Np, _ptr(F), _ptr(Fp),
                              int(nthreads))
    if rc != 0:
        raise ValueError("or_fstat_batch rejected its arguments")
    return F, Fp


def fstat_batch_channels(params: np.ndarray, models, data: np.ndarray, psd: np.ndarray, Np: int,
                         edges: np.ndarray | None = None, nthreads: int = 0, edges_hz=None):
    """F and Fpart for data in several TDI channels: models[c] (same grid, its
    own `channel`), data [nch, n] complex, psd [nch, n]."""
    models = list(models)
    nch = len(models)
    if edges_hz is not None:
        edges = edge_starts(models[0], edges_hz, Np)
    data = np.asarray(data).reshape(nch, -1)
    psd = np.ascontiguousarray(np.asarray(psd, dtype=np.float64).reshape(nch, -1))
    d_re = np.ascontiguousarray(data.real, dtype=np.float64)
    d_im = np.ascontiguousarray(data.imag, dtype=np.float64)
    B = len(params)
    F = np.zeros(B)
    Fp = np.zeros((B, Np))
    e = None if edges is None else np.ascontiguousarray(edges, dtype=np.int64)
    ms = (Model * nch)(*[m.c() for m in models])
    rc = lib().or_fstat_batch_multi(_params_array(params), B, ms, nch, _ptr(d_re), _ptr(d_im), _ptr(psd),
                                    None if e is None else _ptr(e, C.c_int64), Np, _ptr(F), _ptr(Fp), int(nthreads))
    if rc != 0:
        raise ValueError("or_fstat_batch_multi rejected its arguments")
    return F, Fp


def segment_sums(p, model: OracleModel, data, psd, Np, edges=None):
    """Per-segment N [Np, 4], M [Np, 4, 4] and bin counts [Np]."""
    d_re = np.ascontiguousarray(np.real(data), dtype=np.float64)
    d_im = np.ascontiguousarray(np.imag(data), dtype=np.float64)
    psd = np.ascontiguousarray(psd, dtype=np.float64)
    N = np.zeros((Np, 4))
    M = np.zeros((Np, 16))
    nb = np.zeros(Np, dtype=np.int64)
    e = None if edges is None else np.ascontiguousarray(edges, dtype=np.int64)
    m = model.c()
    P = _params(p)
    lib().or_segment_sums(C.byref(P), C.byref(m), _ptr(d_re), _ptr(d_im), _ptr(psd),
                          None if e is None else _ptr(e, C.c_int64), Np, _ptr(N), _ptr(M),
                          _ptr(nb, C.c_int64))
    return N, M.reshape(Np, 4, 4), nb


def segment_F(N, M, nbins) -> float:
    N = np.ascontiguousarray(N, dtype=np.float64)
    M = np.ascontiguousarray(M, dtype=np.float64).reshape(16)
    return lib().or_segment_F(_ptr(N), _ptr(M), int(nbins))


def basis(p, model: OracleModel, k0: int, k1: int) -> np.ndarray:
    """Complex basis waveforms A^i at bins k0..k1-1, shape [4, k1-k0]."""
    n = k1 - k0
    re = np.zeros(4 * n)
    im = np.zeros(4 * n)
    m = model.c()
    P = _params(p)
    lib().or_basis(C.byref(P), C.byref(m), k0, k1, _ptr(re), _ptr(im))
    return (re + 1j * im).reshape(4, n)


def band(p, model: OracleModel) -> tuple[int, int]:
    a = C.c_int64()
    b = C.c_int64()
    m = model.c()
    P = _params(p)
    lib().or_band(C.byref(P), C.byref(m), C.byref(a), C.byref(b))
    return a.value, b.value


def time_of_freq(p, model: OracleModel, f: float) -> float:
    m = model.c()
    P = _params(p)
    return lib().or_time_of_freq(C.byref(P), C.byref(m), float(f))


def phase_orb_cycles(p, model: OracleModel, f: float) -> float:
    m = model.c()
    P = _params(p)
    return lib().or_phase_orb_cycles_d(C.byref(P), C.byref(m), float(f))


def phase_frac(p, model: OracleModel, k: int) -> float:
    m = model.c()
    P = _params(p)
    return lib().or_phase_frac(C.byref(P), C.byref(m), model.f_min, model.df, int(k))


def antenna(p, model: OracleModel, t: float) -> tuple[float, float]:
    a = C.c_double()
    b = C.c_double()
    m = model.c()
    P = _params(p)
    lib().or_antenna_at(C.byref(P), C.byref(m), float(t), C.byref(a), C.byref(b))
    return a.value, b.value


def doppler_delay(p, model: OracleModel, t: float) -> float:
    m = model.c()
    P = _params(p)
    return lib().or_doppler_at(C.byref(P), C.byref(m), float(t))


def detector_tensor(model: OracleModel, t: float) -> np.ndarray:
    """Detector tensor D = (a a - b b)/2 of the Michelson at time t (Sec. IV), 3 x 3."""
    m = model.c()
    out = np.zeros(9)
    lib().or_detector_tensor_at(C.byref(m), float(t), out.ctypes.data_as(_dp))
    return out.reshape(3, 3)


def extrinsic_to_a(DL, psi, iota, phic) -> np.ndarray:
    a = np.zeros(4)
    lib().or_extrinsic_to_a(float(DL), float(psi), float(iota), float(phic), _ptr(a))
    return a


def a_to_extrinsic(a) -> tuple[float, float, float, float]:
    a = np.ascontiguousarray(a, dtype=np.float64)
    out = [C.c_double() for _ in range(4)]
    lib().or_a_to_extrinsic(_ptr(a), *[C.byref(o) for o in out])
    return tuple(o.value for o in out)


def philox(ctr, key) -> np.ndarray:
    c = (C.c_uint32 * 4)(*[int(x) for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) for x in key])
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def pso_init(R, Npart, D, seed):
    x = np.zeros(R * Npart * D)
    v = np.zeros(R * Npart * D)
    lib().or_pso_init(R, Npart, D, int(seed), _ptr(x), _ptr(v))
    return x.reshape(R, Npart, D), v.reshape(R, Npart, D)


def pso_step(x, v, pbest_x, pbest_f, fit, seed, iteration, w, c1=2.0, c2=2.0, vmax=0.5):
    """One PSO iteration in place on float64 arrays x, v, pbest_x [R, Npart, D]
    and pbest_f, fit [R, Npart].  Returns the local-best indices [R, Npart]."""
    R, Npart, D = x.shape
    for a in (x, v, pbest_x, pbest_f):
        assert a.flags.c_contiguous and a.dtype == np.float64
    fit = np.ascontiguousarray(fit, dtype=np.float64)
    lb = np.zeros((R, Npart), dtype=np.int32)
    lib().or_pso_step(R, Npart, D, _ptr(x), _ptr(v), _ptr(pbest_x), _ptr(pbest_f), _ptr(fit),
                      int(seed), int(iteration) & 0xFFFFFFFF, float(w), float(c1), float(c2),
                      float(vmax), lb.ctypes.data_as(C.POINTER(C.c_int)))
    return lb


def num_threads() -> int:
    return lib().or_num_threads()


def inject(p, model: OracleModel, a, k0: int = 0, k1: int | None = None) -> np.ndarray:
    """Signal sum_i a_i A^i over the whole grid (zero outside [k0, k1))."""
    k1 = model.n if k1 is None else k1
    out = np.zeros(model.n, dtype=np.complex128)
    A = basis(p, model, k0, k1)
    out[k0:k1] = np.tensordot(np.asarray(a, dtype=np.float64), A, axes=1)
    return out


def inner(a, b, psd, df) -> float:
    """<a, b> = 4 df Re sum a conj(b) / S  (Eq. inner_product on the grid)."""
    return float(4.0 * df * np.sum((a * np.conj(b)).real / psd))


def mb_weights(N: int) -> np.ndarray:
    """Complex weights a_0..a_N of the filter of order N in Eq. (freDres)."""
    re = np.zeros(3)
    im = np.zeros(3)
    lib().or_mb_weights(int(N), _ptr(re), _ptr(im))
    return (re + 1j * im)[:N + 1]


def mb_response(p, model: OracleModel, f: float):
    """(T+, Tx, D0, T_f) of the Eq. (freDres) response at frequency f; T+ and Tx
    are divided by exp(2 pi i f D0), which the template phase carries."""
    out = np.zeros(6)
    m = model.c()
    P = _params(p)
    lib().or_mb_response_at(C.byref(P), C.byref(m), float(f), _ptr(out))
    return out[0] + 1j * out[1], out[2] + 1j * out[3], out[4], out[5]


def doppler_rates(p, model: OracleModel, t: float) -> tuple[float, float]:
    """First and second time derivatives of the Doppler delay at time t."""
    a = C.c_double()
    b = C.c_double()
    m = model.c()
    P = _params(p)
    lib().or_doppler_rates_at(C.byref(P), C.byref(m), float(t), C.byref(a), C.byref(b))
    return a.value, b.value


def sc_offset(model: OracleModel, n: int, alpha: float) -> np.ndarray:
    """Offset of spacecraft n from the guiding centre at orbital phase alpha, in units of e R."""
    out = np.zeros(3)
    m = model.c()
    lib().or_sc_offset_at(C.byref(m), int(n), float(alpha), _ptr(out))
    return out


def tdi_response(p, model: OracleModel, f: float, t: float):
    """(T+, Tx) of the finite-arm TDI response at frequency f, constellation at time t."""
    out = np.zeros(4)
    m = model.c()
    P = _params(p)
    lib().or_tdi_response_at(C.byref(P), C.byref(m), float(f), float(t), _ptr(out))
    return out[0] + 1j * out[1], out[2] + 1j * out[3]
