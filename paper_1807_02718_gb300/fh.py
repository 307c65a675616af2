"""Thin Python binding of libfh (include/fh.h): argument marshalling only.

Every function has the name of the C entry point it wraps and raises FHError
on a non-zero status.  Every step of the scattering path runs in libfh's CUDA
kernels; nothing here computes.  If libfh.so has not been built (see
paper_1807_02718_gb300.build) the first call raises: there is no CPU fallback.

Device-pointer variants accept torch CUDA tensors (float64, contiguous).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libfh.so")

FH_OK, FH_EINVAL, FH_ENOMEM, FH_ECUDA, FH_ESTATE, FH_ESINGULAR, FH_ENOCONV, FH_ETIMEOUT = range(8)
FH_FP64, FH_MIXED_FP32, FH_MIXED_TF32, FH_MIXED_BF16 = 0, 1, 2, 3
FH_CURVE_CIRCLE, FH_CURVE_KITE, FH_CURVE_STAR = 0, 1, 2
FH_MAX_HARMONICS = 16

STATUS_NAMES = {0: "FH_OK", 1: "FH_EINVAL", 2: "FH_ENOMEM", 3: "FH_ECUDA", 4: "FH_ESTATE",
                5: "FH_ESINGULAR", 6: "FH_ENOCONV", 7: "FH_ETIMEOUT"}

EXPORTED = [
    "fh_create", "fh_destroy", "fh_last_error", "fh_set_stream", "fh_discretize",
    "fh_solve_frequencies", "fh_window_spectra", "fh_window_spectra_dev", "fh_sample",
    "fh_sample_dev", "fh_get_num_windows", "fh_get_window_spectra", "fh_get_geometry",
    "fh_assemble_matrix", "fh_get_density", "fh_set_densities", "fh_get_target_field",
    "fh_synthesize", "fh_set_timing", "fh_get_timings", "fh_probe_fma_peak",
    "fh_eval_bessel", "fh_synthesize_static", "fh_discretize_batch", "fh_num_problems",
    "fh_window_spectra_p", "fh_window_spectra_p_dev", "fh_sample_p", "fh_sample_p_dev",
    "fh_get_density_p", "fh_footprint", "fh_tc_gemm_test", "fh_eval_bessel_df", "fh_set_graphs",
    "fh_get_tuning", "fh_set_tuning", "fh_autotune", "fh_probe_mma_peak",
    "fh_sing_frequencies", "fh_synthesize_sing", "fh_scaled_convolution", "fh_get_window_spectra_p",
    "fh_get_num_windows_p", "fh_resample_p", "fh_resample_p_dev", "fh_device_memory",
]

PHASES = ["geometry", "assemble", "factor", "refine", "spectra", "field", "weights", "contract"]


class fh_curve(C.Structure):
    _fields_ = [("kind", C.c_int), ("r0", C.c_double), ("n_harm", C.c_int),
                ("amp", C.c_double * FH_MAX_HARMONICS), ("phase", C.c_double * FH_MAX_HARMONICS),
                ("center", C.c_double * 2)]


class fh_solve_stats(C.Structure):
    _fields_ = [("n_solves", C.c_int), ("max_N", C.c_int), ("matrix_entries", C.c_longlong),
                ("refine_iters_max", C.c_int), ("residual_max", C.c_double)]


class fh_timings(C.Structure):
    _fields_ = [("ms", C.c_double * len(PHASES)), ("launches", C.c_longlong * len(PHASES)),
                ("events", C.c_longlong * len(PHASES))]


class fh_tuning(C.Structure):
    _fields_ = [("assemble_group", C.c_int), ("field_group", C.c_int), ("field_chunk", C.c_int),
                ("lu_rows_per_cta", C.c_int), ("lu_early", C.c_int), ("contract_tc", C.c_int)]


class FHError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None
_DP = C.POINTER(C.c_double)
_IP = C.POINTER(C.c_int)


def load_library(path: str | None = None):
    """Load libfh.so (raises if it is missing: build it with build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libfh.so not found at {path}; build it first "
                           "(python -m paper_1807_02718_gb300.build)")
    lib = C.CDLL(path)
    vp = C.c_void_p
    sig = {
        "fh_create": (C.c_int, [C.POINTER(vp), C.c_int, C.c_int]),
        "fh_destroy": (None, [vp]),
        "fh_last_error": (C.c_char_p, [vp]),
        "fh_set_stream": (C.c_int, [vp, vp]),
        "fh_discretize": (C.c_int, [vp, C.POINTER(fh_curve), C.c_int, _DP, _IP, C.c_double, _DP]),
        "fh_solve_frequencies": (C.c_int, [vp, _DP, C.POINTER(fh_solve_stats)]),
        "fh_window_spectra": (C.c_int, [vp, _DP, C.c_int, C.c_double, C.c_double, C.c_double]),
        "fh_window_spectra_dev": (C.c_int, [vp, vp, C.c_int, C.c_double, C.c_double, C.c_double]),
        "fh_sample": (C.c_int, [vp, _DP, C.c_int, _DP, C.c_int, _DP]),
        "fh_sample_dev": (C.c_int, [vp, vp, C.c_int, vp, C.c_int, vp]),
        "fh_get_num_windows": (C.c_int, [vp, _IP]),
        "fh_get_window_spectra": (C.c_int, [vp, _DP, _DP]),
        "fh_get_geometry": (C.c_int, [vp, C.c_int, _DP, _DP, _DP]),
        "fh_assemble_matrix": (C.c_int, [vp, C.c_int, C.c_double, _DP, _DP]),
        "fh_get_density": (C.c_int, [vp, C.c_int, _DP]),
        "fh_set_densities": (C.c_int, [vp, _DP]),
        "fh_get_target_field": (C.c_int, [vp, _DP]),
        "fh_synthesize": (C.c_int, [vp, _DP, C.c_int, _DP, C.c_int, _DP]),
        "fh_set_timing": (C.c_int, [vp, C.c_int]),
        "fh_get_timings": (C.c_int, [vp, C.POINTER(fh_timings), C.c_int]),
        "fh_probe_fma_peak": (C.c_int, [C.c_int, C.c_int, C.c_int, _DP]),
        "fh_probe_mma_peak": (C.c_int, [C.c_int, C.c_int, C.c_int, _DP]),
        "fh_sing_frequencies": (C.c_int, [C.c_double, _DP]),
        "fh_synthesize_sing": (C.c_int, [C.c_int, C.c_double, C.c_int, C.c_int, vp, vp, vp, vp, vp, C.c_int,
                                         vp, C.c_int, vp, vp]),
        "fh_scaled_convolution": (C.c_int, [vp, C.c_int, C.c_int, C.c_double, C.c_double, C.c_longlong,
                                            C.c_int, C.c_double, C.c_double, vp, vp]),
        "fh_get_window_spectra_p": (C.c_int, [vp, C.c_int, _DP, _DP]),
        "fh_get_num_windows_p": (C.c_int, [vp, C.c_int, _IP]),
        "fh_resample_p": (C.c_int, [vp, C.c_int, _DP, C.c_int, _DP]),
        "fh_device_memory": (C.c_int, [C.c_int, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
        "fh_resample_p_dev": (C.c_int, [vp, C.c_int, vp, C.c_int, vp]),
        "fh_eval_bessel": (C.c_int, [_DP, C.c_int, _DP]),
        "fh_eval_bessel_df": (C.c_int, [_DP, C.c_int, _DP]),
        "fh_set_graphs": (C.c_int, [vp, C.c_int]),
        "fh_get_tuning": (C.c_int, [vp, C.POINTER(fh_tuning)]),
        "fh_set_tuning": (C.c_int, [vp, C.POINTER(fh_tuning)]),
        "fh_autotune": (C.c_int, [vp, _DP, C.c_int, C.c_int, C.POINTER(fh_tuning), _DP]),
        "fh_discretize_batch": (C.c_int, [vp, C.c_int, C.POINTER(fh_curve), _IP, _DP, _IP, _DP, _DP]),
        "fh_num_problems": (C.c_int, [vp, _IP]),
        "fh_window_spectra_p": (C.c_int, [vp, C.c_int, _DP, C.c_int, C.c_double, C.c_double, C.c_double]),
        "fh_window_spectra_p_dev": (C.c_int, [vp, C.c_int, vp, C.c_int, C.c_double, C.c_double, C.c_double]),
        "fh_sample_p": (C.c_int, [vp, C.c_int, _DP, C.c_int, _DP, C.c_int, _DP]),
        "fh_sample_p_dev": (C.c_int, [vp, C.c_int, vp, C.c_int, vp, C.c_int, vp]),
        "fh_get_density_p": (C.c_int, [vp, C.c_int, C.c_int, _DP]),
        "fh_footprint": (C.c_int, [_IP, _IP, C.c_int, C.c_int, C.POINTER(C.c_longlong)]),
        "fh_tc_gemm_test": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_float),
                                      C.POINTER(C.c_float), C.POINTER(C.c_float)]),
        "fh_synthesize_static": (C.c_int, [C.c_int, C.c_double, C.c_int, vp, vp, vp, C.c_int, vp,
                                           C.c_int, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(_DP)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(ctx, st):
    if st != FH_OK:
        msg = load_library().fh_last_error(ctx).decode() if ctx else ""
        raise FHError(st, msg)


def _dev_ptr(t):
    """Device pointer of a contiguous float64 CUDA tensor."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return C.c_void_p(t.data_ptr())


def make_curve(curve) -> fh_curve:
    """fh_curve from an object with kind, r0, amp, phase, center (e.g. fh_inputs.Curve)."""
    c = fh_curve()
    c.kind = int(curve.kind)
    c.r0 = float(curve.r0)
    amp = list(getattr(curve, "amp", []) or [])
    ph = list(getattr(curve, "phase", []) or [])
    c.n_harm = len(amp)
    for k, (a, p) in enumerate(zip(amp, ph)):
        c.amp[k] = a
        c.phase[k] = p
    c.center[0], c.center[1] = curve.center
    return c


# ---------------------------------------------------------------- entry points

def fh_create(device: int = 0, precision: int = FH_FP64):
    lib = load_library()
    h = C.c_void_p()
    st = lib.fh_create(C.byref(h), device, precision)
    if st != FH_OK:
        raise FHError(st, f"fh_create(device={device}, precision={precision}) failed")
    return h


def fh_destroy(ctx):
    load_library().fh_destroy(ctx)


def fh_last_error(ctx) -> str:
    return load_library().fh_last_error(ctx).decode()


def fh_set_stream(ctx, stream_handle: int | None):
    _check(ctx, load_library().fh_set_stream(ctx, C.c_void_p(stream_handle or 0)))


def fh_discretize(ctx, curve, omega, N=None, c: float = 1.0, p=(1.0, 0.0)):
    om = _f64(omega)
    Nv = None if N is None else np.ascontiguousarray(N, dtype=np.int32)
    cv = curve if isinstance(curve, fh_curve) else make_curve(curve)
    pv = _f64(p)
    _check(ctx, load_library().fh_discretize(ctx, C.byref(cv), om.size, _dp(om),
                                             None if Nv is None else Nv.ctypes.data_as(_IP),
                                             float(c), _dp(pv)))


def fh_solve_frequencies(ctx, eta=None) -> fh_solve_stats:
    st = fh_solve_stats()
    e = None if eta is None else _f64(eta)
    _check(ctx, load_library().fh_solve_frequencies(ctx, _dp(e), C.byref(st)))
    return st


def fh_window_spectra(ctx, a, t0: float, dt: float, H: float = 10.0):
    av = _f64(a)
    _check(ctx, load_library().fh_window_spectra(ctx, _dp(av), av.size, float(t0), float(dt), float(H)))


def fh_window_spectra_dev(ctx, d_a, t0: float, dt: float, H: float = 10.0):
    _check(ctx, load_library().fh_window_spectra_dev(ctx, _dev_ptr(d_a), d_a.numel(), float(t0),
                                                     float(dt), float(H)))


def fh_sample(ctx, x, T, out=None):
    """u(x, T) into a new array, or into `out` (C-contiguous float64 of n_x * n_T
    elements, e.g. a view of page-locked host memory for full-speed copies)."""
    xv, Tv = _f64(x), _f64(T)
    n_x, n_T = xv.size // 2, Tv.size
    if out is None:
        u = np.empty((n_x, n_T), dtype=np.float64)
    else:
        if out.dtype != np.float64 or out.size != n_x * n_T or not out.flags["C_CONTIGUOUS"]:
            raise ValueError("out must be a C-contiguous float64 array of n_x * n_T elements")
        u = out.reshape(n_x, n_T)
    _check(ctx, load_library().fh_sample(ctx, _dp(xv), n_x, _dp(Tv), n_T, _dp(u)))
    return u


def fh_sample_dev(ctx, d_x, d_T, d_u):
    n_x, n_T = d_x.numel() // 2, d_T.numel()
    if d_u.numel() != n_x * n_T:
        raise ValueError("d_u must hold n_x * n_T doubles")
    _check(ctx, load_library().fh_sample_dev(ctx, _dev_ptr(d_x), n_x, _dev_ptr(d_T), n_T,
                                             _dev_ptr(d_u)))


def fh_get_num_windows(ctx) -> int:
    K = C.c_int()
    _check(ctx, load_library().fh_get_num_windows(ctx, C.byref(K)))
    return K.value


def fh_get_window_spectra(ctx, J: int):
    K = fh_get_num_windows(ctx)
    s = np.empty(K)
    B = np.empty((K, J), dtype=np.complex128)
    _check(ctx, load_library().fh_get_window_spectra(ctx, _dp(s), B.ctypes.data_as(_DP)))
    return s, B


def fh_device_memory(device: int = 0):
    """(free, total) device bytes now."""
    f, t = C.c_longlong(), C.c_longlong()
    st = load_library().fh_device_memory(int(device), C.byref(f), C.byref(t))
    if st != FH_OK:
        raise FHError(st, "fh_device_memory failed")
    return f.value, t.value


def fh_resample_p(ctx, problem: int, T, n_x: int, out=None):
    """u at new times T on the resident target fields (n_x targets of the last sample)."""
    Tv = _f64(T)
    u = np.empty((n_x, Tv.size), dtype=np.float64) if out is None else out.reshape(n_x, Tv.size)
    _check(ctx, load_library().fh_resample_p(ctx, int(problem), _dp(Tv), Tv.size, _dp(u)))
    return u


def fh_resample_p_dev(ctx, problem: int, d_T, d_u):
    _check(ctx, load_library().fh_resample_p_dev(ctx, int(problem), _dev_ptr(d_T), d_T.numel(), _dev_ptr(d_u)))


def fh_get_num_windows_p(ctx, problem: int) -> int:
    K = C.c_int()
    _check(ctx, load_library().fh_get_num_windows_p(ctx, int(problem), C.byref(K)))
    return K.value


def fh_get_window_spectra_p(ctx, problem: int, J: int):
    """(s, B) of problem `problem` of a batch (its J frequencies)."""
    lib = load_library()
    K = C.c_int()
    _check(ctx, lib.fh_get_num_windows_p(ctx, int(problem), C.byref(K)))
    s = np.empty(K.value)
    B = np.empty((K.value, J), dtype=np.complex128)
    _check(ctx, lib.fh_get_window_spectra_p(ctx, int(problem), _dp(s), B.ctypes.data_as(_DP)))
    return s, B


def fh_sing_frequencies(omega_c: float) -> np.ndarray:
    """The 24 frequencies of the singular (Filon-Clenshaw-Curtis) quadrature on (0, omega_c]."""
    out = np.empty(24)
    st = load_library().fh_sing_frequencies(float(omega_c), _dp(out))
    if st != FH_OK:
        raise FHError(st, "fh_sing_frequencies failed")
    return out


def fh_synthesize_sing(J: int, W: float, j_c: int, d_s, d_B, d_Bs, d_V, d_Vs, d_T, d_u, stream=None):
    """Split 2D synthesis into d_u (float64 CUDA tensors; complex arrays as
    interleaved doubles: d_B K*J, d_Bs K*24, d_V J*n_x, d_Vs 24*n_x)."""
    K = d_s.numel()
    n_x = d_V.numel() // (2 * J)
    st = load_library().fh_synthesize_sing(int(J), float(W), int(j_c), K, _dev_ptr(d_s), _dev_ptr(d_B),
                                           _dev_ptr(d_Bs), _dev_ptr(d_V), _dev_ptr(d_Vs), n_x, _dev_ptr(d_T),
                                           d_T.numel(), _dev_ptr(d_u), C.c_void_p(stream or 0))
    if st != FH_OK:
        raise FHError(st, "fh_synthesize_sing failed")


def fh_scaled_convolution(d_c, M: int, beta: float, gamma: float, n0: int, L: int, A: float, P: float,
                          d_d, stream=None):
    """Scaled convolutions of the batch of coefficient rows in d_c (batch*M
    complex as doubles) into d_d (batch*L complex as doubles)."""
    batch = d_c.numel() // (2 * M)
    st = load_library().fh_scaled_convolution(_dev_ptr(d_c), int(M), batch, float(beta), float(gamma), int(n0),
                                              int(L), float(A), float(P), _dev_ptr(d_d), C.c_void_p(stream or 0))
    if st != FH_OK:
        raise FHError(st, "fh_scaled_convolution failed")


def fh_get_geometry(ctx, j: int, N: int):
    z = np.empty(N, dtype=np.complex128)
    dz = np.empty(N, dtype=np.complex128)
    ddz = np.empty(N, dtype=np.complex128)
    _check(ctx, load_library().fh_get_geometry(ctx, j, z.ctypes.data_as(_DP), dz.ctypes.data_as(_DP),
                                               ddz.ctypes.data_as(_DP)))
    return z, dz, ddz


def fh_assemble_matrix(ctx, j: int, eta_j: float, N: int):
    A = np.empty((N, N), dtype=np.complex128)
    g = np.empty(N, dtype=np.complex128)
    _check(ctx, load_library().fh_assemble_matrix(ctx, j, float(eta_j), A.ctypes.data_as(_DP),
                                                  g.ctypes.data_as(_DP)))
    return A, g


def fh_get_density(ctx, j: int, N: int):
    psi = np.empty(N, dtype=np.complex128)
    _check(ctx, load_library().fh_get_density(ctx, j, psi.ctypes.data_as(_DP)))
    return psi


def fh_set_densities(ctx, psi_all):
    v = np.ascontiguousarray(psi_all, dtype=np.complex128)
    _check(ctx, load_library().fh_set_densities(ctx, v.ctypes.data_as(_DP)))


def fh_get_target_field(ctx, n_x: int, J: int):
    V = np.empty((n_x, J), dtype=np.complex128)
    _check(ctx, load_library().fh_get_target_field(ctx, V.ctypes.data_as(_DP)))
    return V


def fh_synthesize(ctx, V, T):
    Vv = np.ascontiguousarray(V, dtype=np.complex128)
    Tv = _f64(T)
    n_x = Vv.shape[0]
    u = np.empty((n_x, Tv.size), dtype=np.float64)
    _check(ctx, load_library().fh_synthesize(ctx, Vv.ctypes.data_as(_DP), n_x, _dp(Tv), Tv.size,
                                             _dp(u)))
    return u


def fh_set_graphs(ctx, enable: bool):
    """Run the solve and sample launch sequences as CUDA graphs (default on)."""
    _check(ctx, load_library().fh_set_graphs(ctx, int(bool(enable))))


TUNING_FIELDS = [f for f, _ in fh_tuning._fields_]


def fh_get_tuning(ctx) -> dict:
    t = fh_tuning()
    _check(ctx, load_library().fh_get_tuning(ctx, C.byref(t)))
    return {f: getattr(t, f) for f in TUNING_FIELDS}


def fh_set_tuning(ctx, **values):
    """Set schedule parameters by name (the others keep their values)."""
    cur = fh_get_tuning(ctx)
    unknown = set(values) - set(TUNING_FIELDS)
    if unknown:
        raise ValueError(f"unknown tuning fields {sorted(unknown)}")
    cur.update(values)
    t = fh_tuning(*[int(cur[f]) for f in TUNING_FIELDS])
    _check(ctx, load_library().fh_set_tuning(ctx, C.byref(t)))


def fh_autotune(ctx, x=None, reps: int = 3):
    """Time the schedule candidates on the current discretization (and the
    targets x, n_x x 2) and apply the fastest; returns (tuning, best ms of
    {assemble, factor, field, assemble_factor})."""
    xv = None if x is None else _f64(np.asarray(x, dtype=np.float64).reshape(-1, 2))
    n_x = 0 if xv is None else xv.shape[0]
    t = fh_tuning()
    ms = (C.c_double * 4)()
    _check(ctx, load_library().fh_autotune(ctx, None if xv is None else _dp(xv), n_x, int(reps),
                                           C.byref(t), ms))
    return ({f: getattr(t, f) for f in TUNING_FIELDS},
            {"assemble": ms[0], "factor": ms[1], "field": ms[2], "assemble_factor": ms[3]})


def fh_set_timing(ctx, enable: bool):
    _check(ctx, load_library().fh_set_timing(ctx, 1 if enable else 0))


def fh_get_timings(ctx, reset: bool = False) -> dict:
    t = fh_timings()
    _check(ctx, load_library().fh_get_timings(ctx, C.byref(t), 1 if reset else 0))
    return {name: {"ms": t.ms[i], "launches": t.launches[i], "events": t.events[i]}
            for i, name in enumerate(PHASES)}


def fh_probe_fma_peak(device: int = 0, fp64: bool = True, iters: int = 4096) -> float:
    v = C.c_double()
    st = load_library().fh_probe_fma_peak(device, 1 if fp64 else 0, iters, C.byref(v))
    if st != FH_OK:
        raise FHError(st, "fh_probe_fma_peak failed")
    return v.value


def fh_probe_mma_peak(device: int = 0, kind: int = 2, iters: int = 20000) -> float:
    """Dense tcgen05 throughput in TFLOP/s (kind 1 = BF16, 2 = TF32)."""
    v = C.c_double()
    st = load_library().fh_probe_mma_peak(int(device), int(kind), int(iters), C.byref(v))
    if st != FH_OK:
        raise FHError(st, "fh_probe_mma_peak failed")
    return v.value


def fh_eval_bessel(x):
    """(n, 6) array: J0, Y0, J1, Y1 (joint routine), J0, Y0 (H0 routine)."""
    xv = _f64(x)
    out = np.empty((xv.size, 6))
    st = load_library().fh_eval_bessel(_dp(xv), xv.size, _dp(out))
    if st != FH_OK:
        raise FHError(st, "fh_eval_bessel failed")
    return out


def fh_eval_bessel_df(x):
    """(n, 4) array: J0, Y0, J1, Y1 through the double-float Hankel form (x >= 8)."""
    xv = _f64(x)
    out = np.empty((xv.size, 4))
    st = load_library().fh_eval_bessel_df(_dp(xv), xv.size, _dp(out))
    if st != FH_OK:
        raise FHError(st, "fh_eval_bessel_df failed")
    return out


def fh_synthesize_static(J: int, W: float, d_s, d_B, d_V, d_T, d_u, stream=None):
    """Synthesis into d_u without any allocation (static device scratch).
    d_s (K,), d_B (K*J complex as 2*K*J doubles), d_V (J*n_x complex as doubles,
    frequency-major), d_T (n_T,), d_u (n_x*n_T,): float64 CUDA tensors."""
    K = d_s.numel()
    n_T = d_T.numel()
    n_x = d_V.numel() // (2 * J)
    st = load_library().fh_synthesize_static(
        int(J), float(W), K, _dev_ptr(d_s), _dev_ptr(d_B), _dev_ptr(d_V), n_x, _dev_ptr(d_T), n_T,
        _dev_ptr(d_u), C.c_void_p(stream or 0))
    if st != FH_OK:
        raise FHError(st, "fh_synthesize_static failed")


def fh_discretize_batch(ctx, curves, omegas, Ns=None, cs=None, ps=None):
    """Discretise P problems in one context (lists of curves, omega arrays, N arrays)."""
    P = len(curves)
    arr = (fh_curve * P)(*[c if isinstance(c, fh_curve) else make_curve(c) for c in curves])
    J = np.asarray([len(o) for o in omegas], dtype=np.int32)
    om = _f64(np.concatenate([np.asarray(o, dtype=np.float64) for o in omegas]))
    Nv = None if Ns is None else np.ascontiguousarray(np.concatenate(Ns), dtype=np.int32)
    cv = _f64(np.ones(P) if cs is None else cs)
    pv = _f64(np.tile([1.0, 0.0], P) if ps is None else np.asarray(ps, dtype=np.float64).reshape(-1))
    _check(ctx, load_library().fh_discretize_batch(ctx, P, arr, J.ctypes.data_as(_IP), _dp(om),
                                                   None if Nv is None else Nv.ctypes.data_as(_IP),
                                                   _dp(cv), _dp(pv)))


def fh_num_problems(ctx) -> int:
    P = C.c_int()
    _check(ctx, load_library().fh_num_problems(ctx, C.byref(P)))
    return P.value


def fh_window_spectra_p(ctx, problem: int, a, t0: float, dt: float, H: float = 10.0):
    av = _f64(a)
    _check(ctx, load_library().fh_window_spectra_p(ctx, problem, _dp(av), av.size, float(t0),
                                                   float(dt), float(H)))


def fh_window_spectra_p_dev(ctx, problem: int, d_a, t0: float, dt: float, H: float = 10.0):
    _check(ctx, load_library().fh_window_spectra_p_dev(ctx, problem, _dev_ptr(d_a), d_a.numel(),
                                                       float(t0), float(dt), float(H)))


def fh_sample_p(ctx, problem: int, x, T):
    xv, Tv = _f64(x), _f64(T)
    n_x, n_T = xv.size // 2, Tv.size
    u = np.empty((n_x, n_T), dtype=np.float64)
    _check(ctx, load_library().fh_sample_p(ctx, problem, _dp(xv), n_x, _dp(Tv), n_T, _dp(u)))
    return u


def fh_sample_p_dev(ctx, problem: int, d_x, d_T, d_u):
    n_x, n_T = d_x.numel() // 2, d_T.numel()
    if d_u.numel() != n_x * n_T:
        raise ValueError("d_u must hold n_x * n_T doubles")
    _check(ctx, load_library().fh_sample_p_dev(ctx, problem, _dev_ptr(d_x), n_x, _dev_ptr(d_T), n_T,
                                               _dev_ptr(d_u)))


def fh_get_density_p(ctx, problem: int, j: int, N: int):
    psi = np.empty(N, dtype=np.complex128)
    _check(ctx, load_library().fh_get_density_p(ctx, problem, j, psi.ctypes.data_as(_DP)))
    return psi


def fh_footprint(Js, Ns, precision: int = FH_FP64) -> int:
    J = np.ascontiguousarray(Js, dtype=np.int32)
    N = np.ascontiguousarray(np.concatenate(Ns), dtype=np.int32)
    out = C.c_longlong()
    st = load_library().fh_footprint(J.ctypes.data_as(_IP), N.ctypes.data_as(_IP), J.size,
                                     precision, C.byref(out))
    if st != FH_OK:
        raise FHError(st, "fh_footprint failed")
    return out.value


def fh_tc_gemm_test(kind: int, A, B):
    """C = A B^T on the tensor cores (kind 1: BF16 operands, 2: TF32)."""
    Af = np.ascontiguousarray(A, dtype=np.float32)
    Bf = np.ascontiguousarray(B, dtype=np.float32)
    M, K = Af.shape
    N = Bf.shape[0]
    Cf = np.empty((M, N), dtype=np.float32)
    fp = C.POINTER(C.c_float)
    st = load_library().fh_tc_gemm_test(kind, M, N, K, Af.ctypes.data_as(fp), Bf.ctypes.data_as(fp),
                                        Cf.ctypes.data_as(fp))
    if st != FH_OK:
        raise FHError(st, "fh_tc_gemm_test failed")
    return Cf


class Problem:
    """Owns one context: discretise, solve, window, sample (numpy in/out)."""

    def __init__(self, device: int = 0, precision: int = FH_FP64):
        self.ctx = fh_create(device, precision)
        self.J = 0

    def close(self):
        if self.ctx:
            fh_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def discretize(self, curve, omega, N=None, c=1.0, p=(1.0, 0.0)):
        fh_discretize(self.ctx, curve, omega, N, c, p)
        self.J = len(omega)

    def solve(self, eta=None):
        return fh_solve_frequencies(self.ctx, eta)

    def window_spectra(self, a, t0, dt, H=10.0):
        fh_window_spectra(self.ctx, a, t0, dt, H)

    def sample(self, x, T):
        return fh_sample(self.ctx, x, T)
