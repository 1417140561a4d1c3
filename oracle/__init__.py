"""FP64 CPU oracle for the Lomb-Scargle periodogram -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never routes through it and shares no code with it.

The arithmetic lives in ``lsp_oracle.c`` (plain C, FP64, libm, OpenMP): Eq. 1
(tau) and Eq. 2 (power) of Section 2, evaluated in two scans per frequency,
with the half-open grid of Section 2, the first-maximum argmax of Section 3.3,
and the lsp-c parallel schedules of Section 4.5.  This module only marshals
numpy arrays through ctypes.  ``gls_batch`` is the generalized periodogram of
Section 4.11 (weighted three-parameter least squares); ``oracle.learned``
holds the oracle of the learned-proposal stage.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lsp_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liblsp_oracle.so")
_lock = threading.Lock()
_lib = None

FLAG_FEW_OBS = 1
FLAG_ZERO_VAR = 2
FLAG_NONFINITE = 4


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (IEEE semantics, no fast-math)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_SRC32 = os.path.join(_HERE, "lsp_cpu_fp32.c")
_LIB32_PATH = os.path.join(_HERE, "_build", "liblsp_cpu_fp32.so")
_lib32 = None


def build_fp32(force: bool = False) -> str:
    """Compile the FP32 CPU configuration (timing context, not an oracle)."""
    os.makedirs(os.path.dirname(_LIB32_PATH), exist_ok=True)
    stale = (not os.path.exists(_LIB32_PATH)) or os.path.getmtime(_LIB32_PATH) < os.path.getmtime(_SRC32)
    if force or stale:
        tmp = _LIB32_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC32, "-o", tmp, "-lm"],
                       check=True)
        os.replace(tmp, _LIB32_PATH)
    return _LIB32_PATH


def _load32():
    global _lib32
    with _lock:
        if _lib32 is None:
            build_fp32()
            lib = ctypes.CDLL(_LIB32_PATH)
            P, d, i64 = ctypes.c_void_p, ctypes.c_double, ctypes.c_int64
            lib.cpu32_lsp_batch_argmax.argtypes = [P, P, P, i64, d, d, i64, P, P]
            lib.cpu32_lsp_batch_argmax.restype = ctypes.c_int
            lib.cpu32_lsp_single.argtypes = [P, P, i64, d, d, i64, P, i64, P]
            lib.cpu32_lsp_single.restype = ctypes.c_int
            _lib32 = lib
    return _lib32


def fp32_batch_argmax(t, y, offsets, f_min, f_max, n_f):
    """The paper's FP32 CPU configuration (two-scan Eq. 1-2 in single precision),
    batch mode: first maximum of P_n per object.  Timing context only."""
    t, y = _f64(t), _f64(y)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    n_obj = off.size - 1
    idx = np.empty(n_obj, dtype=np.int64)
    pw = np.empty(n_obj, dtype=np.float32)
    if _load32().cpu32_lsp_batch_argmax(_ptr(t), _ptr(y), _ptr(off), n_obj, float(f_min), float(f_max),
                                        int(n_f), _ptr(idx), _ptr(pw)):
        raise MemoryError("cpu32_lsp_batch_argmax")
    return idx, pw


def fp32_single(t, y, f_min, f_max, n_f, k_sel):
    """FP32 CPU configuration, one object, P_n at the indices ``k_sel``."""
    t, y = _f64(t), _f64(y)
    ks = np.ascontiguousarray(k_sel, dtype=np.int64)
    out = np.empty(ks.size, dtype=np.float32)
    if _load32().cpu32_lsp_single(_ptr(t), _ptr(y), t.size, float(f_min), float(f_max), int(n_f), _ptr(ks),
                                  ks.size, _ptr(out)):
        raise MemoryError("cpu32_lsp_single")
    return out


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int
            P = ctypes.c_void_p
            lib.oracle_lsp_single.argtypes = [P, P, i64, d, d, i64, i32, i32, P, i64, P]
            lib.oracle_lsp_single.restype = i32
            lib.oracle_lsp_single_ld.argtypes = [P, P, i64, d, d, i64, i32, P, i64, P]
            lib.oracle_lsp_single_ld.restype = i32
            lib.oracle_lsp_batch.argtypes = [P, P, P, i64, d, d, i64, i32, i32, i32, P, P, P, P, P, P]
            lib.oracle_lsp_batch.restype = i32
            lib.oracle_argmax.argtypes = [P, i64]
            lib.oracle_argmax.restype = i64
            lib.oracle_top_local_maxima.argtypes = [P, i64, i32, P, P]
            lib.oracle_top_local_maxima.restype = i32
            lib.oracle_num_threads.restype = i32
            lib.oracle_gls_batch.argtypes = [P, P, P, P, i64, d, d, i64, i32, P, P, P, P]
            lib.oracle_gls_batch.restype = i32
            _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def num_threads() -> int:
    """OpenMP threads the oracle runs with (OMP_NUM_THREADS or all cores)."""
    return int(_load().oracle_num_threads())


def grid_freqs(f_min: float, f_max: float, n_f: int) -> np.ndarray:
    """Half-open evenly spaced grid of Section 2: f_k = f_min + k (f_max - f_min) / N_f."""
    df = (f_max - f_min) / float(n_f)
    return f_min + np.arange(n_f, dtype=np.float64) * df


def lsp_single(t, y, f_min, f_max, n_f, *, norm=1, center=True, k_sel=None):
    """Power of one object on the grid (or at the indices ``k_sel``).

    Returns ``(power, flags)``; ``norm=1`` gives P_n = 2P / sum(y_c^2),
    ``norm=0`` the P of Eq. 2.
    """
    t, y = _f64(t), _f64(y)
    assert t.shape == y.shape and t.ndim == 1
    ks = None if k_sel is None else np.ascontiguousarray(k_sel, dtype=np.int64)
    n_out = n_f if ks is None else ks.size
    out = np.empty(n_out, dtype=np.float64)
    fl = _load().oracle_lsp_single(_ptr(t), _ptr(y), t.size, float(f_min), float(f_max), int(n_f),
                                   int(norm), int(bool(center)), _ptr(ks), 0 if ks is None else ks.size,
                                   _ptr(out))
    return out, int(fl)


def lsp_single_ld(t, y, f_min, f_max, n_f, k_sel, *, norm=1):
    """Extended-precision (long double) recomputation at a few frequencies."""
    t, y = _f64(t), _f64(y)
    ks = np.ascontiguousarray(k_sel, dtype=np.int64)
    out = np.empty(ks.size, dtype=np.float64)
    _load().oracle_lsp_single_ld(_ptr(t), _ptr(y), t.size, float(f_min), float(f_max), int(n_f),
                                 int(norm), _ptr(ks), ks.size, _ptr(out))
    return out


def lsp_batch(t, y, offsets, f_min, f_max, n_f, *, norm=1, center=True, top_k=1, return_power=False):
    """Batch mode (Section 3.4) over CSR ``offsets``.

    Returns a dict with ``arg_idx``, ``arg_pow``, ``top_idx``/``top_pow``
    (n_obj x top_k), ``flags`` and, if requested, ``power`` (n_obj x n_f).
    """
    t, y = _f64(t), _f64(y)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    n_obj = off.size - 1
    top_k = max(1, min(3, int(top_k)))
    power = np.empty((n_obj, n_f), dtype=np.float64) if return_power else None
    arg_idx = np.empty(n_obj, dtype=np.int64)
    arg_pow = np.empty(n_obj, dtype=np.float64)
    top_idx = np.empty((n_obj, top_k), dtype=np.int64)
    top_pow = np.empty((n_obj, top_k), dtype=np.float64)
    flags = np.empty(n_obj, dtype=np.int32)
    _load().oracle_lsp_batch(_ptr(t), _ptr(y), _ptr(off), n_obj, float(f_min), float(f_max), int(n_f),
                             int(norm), int(bool(center)), top_k, _ptr(power), _ptr(arg_idx),
                             _ptr(arg_pow), _ptr(top_idx), _ptr(top_pow), _ptr(flags))
    res = dict(arg_idx=arg_idx, arg_pow=arg_pow, top_idx=top_idx, top_pow=top_pow, flags=flags)
    if return_power:
        res["power"] = power
    return res


def gls_batch(t, y, dy, offsets, f_min, f_max, n_f, *, norm=1, return_power=True):
    """Generalized periodogram (Section 4.11): weighted 3-parameter least squares.

    ``dy`` None means unit weights.  Returns a dict with ``power`` (if
    requested), ``arg_idx``, ``arg_pow`` and ``flags``.
    """
    t, y = _f64(t), _f64(y)
    dyv = None if dy is None else _f64(dy)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    n_obj = off.size - 1
    power = np.empty((n_obj, n_f), dtype=np.float64) if return_power else None
    arg_idx = np.empty(n_obj, dtype=np.int64)
    arg_pow = np.empty(n_obj, dtype=np.float64)
    flags = np.empty(n_obj, dtype=np.int32)
    _load().oracle_gls_batch(_ptr(t), _ptr(y), _ptr(dyv), _ptr(off), n_obj, float(f_min), float(f_max), int(n_f),
                             int(norm), _ptr(power), _ptr(arg_idx), _ptr(arg_pow), _ptr(flags))
    res = dict(arg_idx=arg_idx, arg_pow=arg_pow, flags=flags)
    if return_power:
        res["power"] = power
    return res


def argmax(p) -> int:
    """First maximum (Section 3.3, thrust::max_element semantics)."""
    p = _f64(p)
    return int(_load().oracle_argmax(_ptr(p), p.size))


def top_local_maxima(p, k_top=3):
    """The k_top largest local maxima, ordered by power, ties to the lower index."""
    p = _f64(p)
    idx = np.empty(k_top, dtype=np.int64)
    pw = np.empty(k_top, dtype=np.float64)
    _load().oracle_top_local_maxima(_ptr(p), p.size, int(k_top), _ptr(idx), _ptr(pw))
    return idx, pw


def period_of(f_min, f_max, n_f, k):
    """Period (1/f) of grid bin k; Section 3.3 gives the angular form 2 pi / w_k."""
    return 1.0 / (f_min + k * (f_max - f_min) / float(n_f))
