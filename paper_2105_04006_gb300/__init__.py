"""Python binding of the GB300 Lomb-Scargle library (``include/lsp.h``).

Argument marshalling only: every step of the periodogram runs in the CUDA
library ``_build/liblsp.so`` (built by ``paper_2105_04006_gb300.build``).
PyTorch supplies device memory and the current stream.  If the library is
missing, importing works but every call raises ``LibraryNotBuilt`` -- there
is no CPU fallback.

Names follow the C ABI: ``periodogram`` (single object, Section 3.3),
``batch`` (ragged CSR batch, Section 3.4), ``argmax_period`` (the period of a
stored periodogram), ``Plan`` (tuned, graph-captured repeats).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "liblsp.so")

FP32, FP64 = 0, 1
NORM_PSD, NORM_STANDARD = 0, 1
FLAG_FEW_OBS, FLAG_ZERO_VAR, FLAG_NONFINITE, FLAG_BAD_OFFSETS = 1, 2, 4, 8

PEAK_DTYPE = np.dtype([("idx", "<i8"), ("power", "<f8"), ("freq", "<f8"), ("period", "<f8"),
                       ("flags", "<i4"), ("reserved", "<i4")])
assert PEAK_DTYPE.itemsize == 40


class LibraryNotBuilt(RuntimeError):
    pass


class LSPError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"lsp status {status}: {message}")
        self.status = status


class Grid(ctypes.Structure):
    """Half-open grid [f_min, f_max) of n_f frequencies (cycles per unit of t)."""
    _fields_ = [("f_min", ctypes.c_double), ("f_max", ctypes.c_double), ("n_f", ctypes.c_int64)]

    @property
    def df(self) -> float:
        return (self.f_max - self.f_min) / float(self.n_f)

    def freqs(self) -> np.ndarray:
        return self.f_min + np.arange(self.n_f, dtype=np.float64) * self.df


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("norm", ctypes.c_int32), ("center_y", ctypes.c_int32),
                ("top_k", ctypes.c_int32), ("k_reseed", ctypes.c_int32),
                ("freqs_per_thread", ctypes.c_int32), ("block_threads", ctypes.c_int32),
                ("obs_split", ctypes.c_int32)]


class Config(ctypes.Structure):
    _fields_ = [("k_reseed", ctypes.c_int32), ("freqs_per_thread", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("obs_split", ctypes.c_int32),
                ("packed", ctypes.c_int32), ("trig", ctypes.c_int32), ("staging", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return dict(k_reseed=self.k_reseed, freqs_per_thread=self.freqs_per_thread,
                    block_threads=self.block_threads, obs_split=self.obs_split, packed=self.packed,
                    trig=self.trig, staging=self.staging)


class Trial(ctypes.Structure):
    _fields_ = [("config", Config), ("ms", ctypes.c_float), ("max_err", ctypes.c_float),
                ("passed", ctypes.c_int32), ("worst_object", ctypes.c_int32)]


TUNE_ABLATIONS = 1


_lib = None
_lock = threading.Lock()

EXPORTS = [
    "lsp_status_string", "lsp_last_error", "lsp_default_opts", "lsp_version", "lsp_workspace_size",
    "lsp_periodogram", "lsp_batch", "lsp_argmax_period", "lsp_plan_create", "lsp_plan_execute",
    "lsp_plan_execute_host", "lsp_plan_autotune", "lsp_plan_get_config", "lsp_plan_set_config",
    "lsp_plan_destroy", "lsp_plan_enable_timing", "lsp_plan_main_kernel_ms", "lsp_plan_kernel_count",
    "lsp_batch_noalloc", "lsp_grid_for_span",
    "lsp_mlp_param_count", "lsp_mlp_workspace_size", "lsp_featurize", "lsp_mlp_forward",
    "lsp_mlp_loss_grad", "lsp_mlp_adamw", "lsp_to_bf16", "lsp_top_classes", "lsp_refine_workspace_size",
    "lsp_refine_windows", "lsp_batch_gls", "lsp_periodogram_gls", "lsp_workspace_size_gls",
    "lsp_probe_fma_rates", "lsp_plan_autotune_ex", "lsp_plan_set_host_parts", "lsp_plan_get_host_parts",
    "lsp_propose_refine", "lsp_propose_refine_workspace_size", "lsp_window_labels", "lsp_noalloc_prepare",
    "lsp_plan_gate_report", "lsp_probe_sincos_fixed64", "lsp_mlp_gemm_timeouts",
    "lsp_mlp_gemm_wait_test",
]


class MlpDims(ctypes.Structure):
    _fields_ = [("in_dim", ctypes.c_int32), ("hidden", ctypes.c_int32), ("n_hidden", ctypes.c_int32),
                ("n_classes", ctypes.c_int32)]


class Proposer(ctypes.Structure):
    """lsp_proposer: the learned stage's network and refine settings."""
    _fields_ = [("dims", MlpDims), ("params", ctypes.c_void_p), ("params_bf16", ctypes.c_void_p),
                ("window", ctypes.c_int64), ("stride", ctypes.c_int64), ("lag_max", ctypes.c_float),
                ("k_windows", ctypes.c_int32), ("stop_power", ctypes.c_float), ("fallback_power", ctypes.c_float),
                ("inconclusive_fallback", ctypes.c_int32), ("norm", ctypes.c_int32)]


def lib():
    """The loaded CUDA library (raises LibraryNotBuilt if it was never built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise LibraryNotBuilt(
                    f"{LIB_PATH} is missing: build it with `python -m paper_2105_04006_gb300.build` "
                    "(or __graft_entry__.build()); there is no CPU fallback")
            L = ctypes.CDLL(LIB_PATH)
            P, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
            GP, OP = ctypes.POINTER(Grid), ctypes.POINTER(Opts)
            L.lsp_status_string.argtypes = [i32]
            L.lsp_status_string.restype = ctypes.c_char_p
            L.lsp_last_error.restype = ctypes.c_char_p
            L.lsp_default_opts.restype = Opts
            L.lsp_version.restype = i32
            L.lsp_workspace_size.argtypes = [i64, i64, GP, OP, ctypes.POINTER(sz)]
            L.lsp_periodogram.argtypes = [P, P, i64, GP, OP, P, P, P, sz, P]
            L.lsp_batch.argtypes = [P, P, P, i64, i64, GP, OP, P, P, P, sz, P]
            L.lsp_argmax_period.argtypes = [P, i64, i64, GP, i32, P, P]
            L.lsp_batch_noalloc.argtypes = [P, P, P, i64, i64, GP, OP, P, P, P]
            L.lsp_batch_gls.argtypes = [P, P, P, P, i64, i64, GP, OP, P, P, P, sz, P]
            L.lsp_workspace_size_gls.argtypes = [i64, i64, GP, OP, ctypes.POINTER(sz)]
            L.lsp_periodogram_gls.argtypes = [P, P, P, i64, GP, OP, P, P, P, sz, P]
            L.lsp_grid_for_span.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, GP]
            L.lsp_plan_create.argtypes = [ctypes.POINTER(P), i64, i64, GP, OP]
            L.lsp_plan_execute.argtypes = [P, P, P, P, P, P, P]
            L.lsp_plan_execute_host.argtypes = [P, P, P, P, P, P, P]
            L.lsp_plan_autotune.argtypes = [P, P, P, P, ctypes.c_char_p, P]
            L.lsp_plan_autotune_ex.argtypes = [P, P, P, P, ctypes.c_char_p, i32, P, i32, P, P]
            L.lsp_plan_get_config.argtypes = [P, ctypes.POINTER(Config)]
            L.lsp_plan_set_config.argtypes = [P, ctypes.POINTER(Config)]
            L.lsp_plan_enable_timing.argtypes = [P, i32]
            L.lsp_plan_main_kernel_ms.argtypes = [P, ctypes.POINTER(ctypes.c_float)]
            L.lsp_plan_kernel_count.argtypes = [P, ctypes.POINTER(i32)]
            L.lsp_plan_set_host_parts.argtypes = [P, i32]
            L.lsp_plan_get_host_parts.argtypes = [P, i64, ctypes.POINTER(i32)]
            DP = ctypes.POINTER(MlpDims)
            f32 = ctypes.c_float
            L.lsp_mlp_param_count.argtypes = [DP, ctypes.POINTER(i64)]
            L.lsp_mlp_workspace_size.argtypes = [DP, i64, ctypes.POINTER(sz)]
            L.lsp_featurize.argtypes = [P, P, P, i64, i64, GP, f32, P, P, P]
            L.lsp_mlp_forward.argtypes = [DP, P, P, P, i64, P, P, sz, P]
            L.lsp_mlp_loss_grad.argtypes = [DP, P, P, P, P, i64, P, P, P, sz, P]
            L.lsp_mlp_adamw.argtypes = [i64, P, P, P, P, P, i64, f32, f32, f32, f32, f32, P]
            L.lsp_to_bf16.argtypes = [P, P, i64, P]
            L.lsp_mlp_gemm_timeouts.argtypes = [ctypes.POINTER(ctypes.c_uint32)]
            L.lsp_mlp_gemm_wait_test.argtypes = [P, sz, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(i32), P]
            L.lsp_top_classes.argtypes = [P, i64, i32, i32, P, P]
            L.lsp_refine_workspace_size.argtypes = [i64, i64, GP, ctypes.POINTER(sz)]
            L.lsp_refine_windows.argtypes = [P, P, P, i64, i64, GP, i32, P, i32, i64, i64, f32, f32, i32, P,
                                             P, P, sz, P]
            PP = ctypes.POINTER(Proposer)
            L.lsp_propose_refine_workspace_size.argtypes = [PP, i64, i64, GP, ctypes.POINTER(sz)]
            L.lsp_propose_refine.argtypes = [PP, P, P, P, i64, i64, GP, P, P, P, P, sz, P]
            L.lsp_window_labels.argtypes = [P, i64, i64, i32, P, P]
            L.lsp_noalloc_prepare.argtypes = []
            L.lsp_plan_gate_report.argtypes = [P, P, P, i32, ctypes.POINTER(i32)]
            L.lsp_probe_sincos_fixed64.argtypes = [i64, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double), P]
            L.lsp_plan_destroy.argtypes = [P]
            L.lsp_plan_destroy.restype = None
            for name in EXPORTS:
                if name not in ("lsp_status_string", "lsp_last_error", "lsp_default_opts",
                                "lsp_version", "lsp_plan_destroy"):
                    getattr(L, name).restype = i32
            _lib = L
    return _lib


def _check(status: int):
    if status != 0:
        msg = lib().lsp_last_error().decode()
        raise LSPError(status, msg)


def _torch():
    import torch
    return torch


def _stream_handle(device):
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _ptr(x):
    return ctypes.c_void_p(0 if x is None else x.data_ptr())


def _require(x, name, dtype, device=None, numel=None, host_ok=False):
    """A contiguous tensor of `dtype` (and, if given, exactly `numel` elements:
    the library reads or writes that many) on a CUDA device; host_ok also
    admits page-locked host memory, which the kernels address directly."""
    torch = _torch()
    if not isinstance(x, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if x.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {x.dtype}")
    if not x.is_cuda and not (host_ok and x.is_pinned()):
        raise TypeError(f"{name} must be a CUDA tensor" + (" or page-locked host memory" if host_ok else ""))
    if device is not None and x.is_cuda and x.device != device:
        raise ValueError(f"{name} is on {x.device}, expected {device}")
    if not x.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and x.numel() != numel:
        raise ValueError(f"{name} has {x.numel()} elements, expected {numel}")


def make_opts(precision="fp32", norm="standard", center=True, top_k=1, k_reseed=0,
              freqs_per_thread=0, block_threads=0, obs_split=0) -> Opts:
    prec = {"fp32": FP32, "fp64": FP64, FP32: FP32, FP64: FP64}[precision]
    nrm = {"standard": NORM_STANDARD, "psd": NORM_PSD, NORM_PSD: NORM_PSD,
           NORM_STANDARD: NORM_STANDARD}[norm]
    return Opts(prec, nrm, int(bool(center)), int(top_k), int(k_reseed), int(freqs_per_thread),
                int(block_threads), int(obs_split))


def _dtypes(opts: Opts):
    torch = _torch()
    return torch.float64 if opts.precision == FP64 else torch.float32


def grid_for_span(f_min: float, f_max: float, t_span: float) -> Grid:
    """Section 4.3's grid: df = 0.1 / t_span cycles per unit time, n_f = round(range / df)."""
    g = Grid()
    _check(lib().lsp_grid_for_span(float(f_min), float(f_max), float(t_span), ctypes.byref(g)))
    return g


def probe_fma_rates(device=None) -> dict:
    """Measured FMA-pipe rates of the current GPU, in lane-operations per second
    for the whole device: scalar FP32, packed f32x2 (two per instruction) and
    FP64.  Register-only probe kernels in the library; the ceilings for the
    trig-sum kernels' roofline fractions."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    r32, r2, r64 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    with torch.cuda.device(dev):
        _check(lib().lsp_probe_fma_rates(ctypes.byref(r32), ctypes.byref(r2), ctypes.byref(r64),
                                         _stream_handle(dev)))
    return {"f32": r32.value, "f32x2": r2.value, "f64": r64.value}


def workspace_size(n_obj, total_nt, grid: Grid, opts: Opts) -> int:
    n = ctypes.c_size_t(0)
    _check(lib().lsp_workspace_size(int(n_obj), int(total_nt), ctypes.byref(grid), ctypes.byref(opts),
                                    ctypes.byref(n)))
    return int(n.value)


def peaks_to_numpy(peaks) -> np.ndarray:
    """Copy a peaks buffer (uint8 tensor of 40-byte records) to a structured array."""
    host = peaks.detach().to("cpu").numpy() if hasattr(peaks, "detach") else np.asarray(peaks)
    return host.view(PEAK_DTYPE).reshape(-1)


def periodogram(t, y, grid: Grid, *, return_power=True, workspace=None, **kw):
    """Single-object periodogram on the GPU.

    t: float64 CUDA tensor [n_t]; y: float32 (fp32) or float64 (fp64) [n_t].
    Returns (power or None, peaks) with peaks a uint8 tensor of top_k records
    (``peaks_to_numpy`` decodes them).
    """
    torch = _torch()
    opts = make_opts(**kw)
    _require(t, "t", torch.float64)
    _require(y, "y", _dtypes(opts), t.device)
    n_t = t.numel()
    if y.numel() != n_t:
        raise ValueError("t and y differ in length")
    ws_bytes = workspace_size(1, n_t, grid, opts)
    ws = workspace if workspace is not None else torch.empty(max(ws_bytes, 256), dtype=torch.uint8,
                                                                device=t.device)
    power = torch.empty(grid.n_f, dtype=_dtypes(opts), device=t.device) if return_power else None
    peaks = torch.empty(opts.top_k * 40, dtype=torch.uint8, device=t.device)
    _check(lib().lsp_periodogram(_ptr(t), _ptr(y), n_t, ctypes.byref(grid), ctypes.byref(opts),
                                 _ptr(power), _ptr(peaks), _ptr(ws), ws.numel(), _stream_handle(t.device)))
    return power, peaks


def batch(t, y, offsets, grid: Grid, *, return_power=False, workspace=None, **kw):
    """Ragged batch (CSR offsets, int64 CUDA tensor of n_obj + 1) on the GPU.

    Returns (power [n_obj, n_f] or None, peaks uint8 tensor of n_obj*top_k records).
    """
    torch = _torch()
    opts = make_opts(**kw)
    _require(t, "t", torch.float64)
    _require(y, "y", _dtypes(opts), t.device, numel=t.numel())
    _require(offsets, "offsets", torch.int64, t.device)
    n_obj = offsets.numel() - 1
    total = t.numel()
    ws_bytes = workspace_size(n_obj, total, grid, opts)
    ws = workspace if workspace is not None else torch.empty(max(ws_bytes, 256), dtype=torch.uint8,
                                                                device=t.device)
    power = (torch.empty((n_obj, grid.n_f), dtype=_dtypes(opts), device=t.device)
             if return_power else None)
    peaks = torch.empty(max(n_obj, 0) * opts.top_k * 40, dtype=torch.uint8, device=t.device)
    _check(lib().lsp_batch(_ptr(t), _ptr(y), _ptr(offsets), n_obj, total, ctypes.byref(grid),
                           ctypes.byref(opts), _ptr(power), _ptr(peaks), _ptr(ws), ws.numel(),
                           _stream_handle(t.device)))
    return power, peaks


def workspace_size_gls(n_obj, total_nt, grid: Grid, opts: Opts) -> int:
    n = ctypes.c_size_t(0)
    _check(lib().lsp_workspace_size_gls(int(n_obj), int(total_nt), ctypes.byref(grid), ctypes.byref(opts),
                                        ctypes.byref(n)))
    return int(n.value)


def periodogram_gls(t, y, dy, grid: Grid, *, return_power=True, workspace=None, **kw):
    """Generalized periodogram of one object (photometric errors dy, floating
    mean), split over its observations like ``periodogram``.  Returns (power or
    None, peaks)."""
    torch = _torch()
    opts = make_opts(**kw)
    _require(t, "t", torch.float64)
    _require(y, "y", _dtypes(opts), t.device)
    if dy is not None:
        _require(dy, "dy", _dtypes(opts), t.device)
    n_t = t.numel()
    if y.numel() != n_t or (dy is not None and dy.numel() != n_t):
        raise ValueError("t, y and dy differ in length")
    ws_bytes = workspace_size_gls(1, n_t, grid, opts)
    ws = workspace if workspace is not None else torch.empty(max(ws_bytes, 256), dtype=torch.uint8,
                                                                device=t.device)
    power = torch.empty(grid.n_f, dtype=_dtypes(opts), device=t.device) if return_power else None
    peaks = torch.empty(opts.top_k * 40, dtype=torch.uint8, device=t.device)
    _check(lib().lsp_periodogram_gls(_ptr(t), _ptr(y), _ptr(dy), n_t, ctypes.byref(grid), ctypes.byref(opts),
                                     _ptr(power), _ptr(peaks), _ptr(ws), ws.numel(), _stream_handle(t.device)))
    return power, peaks


def batch_gls(t, y, dy, offsets, grid: Grid, *, return_power=False, workspace=None, **kw):
    """Generalized periodogram of a CSR batch (photometric errors dy, floating mean).

    dy: tensor like y, or None for unit weights.  Returns (power or None, peaks).
    """
    torch = _torch()
    opts = make_opts(**kw)
    _require(t, "t", torch.float64)
    _require(y, "y", _dtypes(opts), t.device, numel=t.numel())
    if dy is not None:
        _require(dy, "dy", _dtypes(opts), t.device, numel=t.numel())
    _require(offsets, "offsets", torch.int64, t.device)
    n_obj = offsets.numel() - 1
    ws_bytes = workspace_size_gls(n_obj, t.numel(), grid, opts)
    ws = workspace if workspace is not None else torch.empty(max(ws_bytes, 256), dtype=torch.uint8,
                                                                device=t.device)
    power = (torch.empty((n_obj, grid.n_f), dtype=_dtypes(opts), device=t.device)
             if return_power else None)
    peaks = torch.empty(max(n_obj, 0) * opts.top_k * 40, dtype=torch.uint8, device=t.device)
    _check(lib().lsp_batch_gls(_ptr(t), _ptr(y), _ptr(dy), _ptr(offsets), n_obj, t.numel(), ctypes.byref(grid),
                               ctypes.byref(opts), _ptr(power), _ptr(peaks), _ptr(ws), ws.numel(),
                               _stream_handle(t.device)))
    return power, peaks


def argmax_period(power, grid: Grid):
    """First maximum of each row of a stored periodogram (float32 or float64 CUDA tensor)."""
    torch = _torch()
    if power.dtype not in (torch.float32, torch.float64):
        raise TypeError("power must be float32 or float64")
    _require(power, "power", power.dtype)
    p2 = power.reshape(-1, grid.n_f)
    n_obj = p2.shape[0]
    peaks = torch.empty(n_obj * 40, dtype=torch.uint8, device=power.device)
    prec = FP64 if power.dtype == torch.float64 else FP32
    _check(lib().lsp_argmax_period(_ptr(p2), n_obj, grid.n_f, ctypes.byref(grid), prec, _ptr(peaks),
                                   _stream_handle(power.device)))
    return peaks


class Plan:
    """A tuned, graph-captured periodogram job for one shape (``lsp_plan_*``)."""

    def __init__(self, n_obj: int, total_nt: int, grid: Grid, **kw):
        self.opts = make_opts(**kw)
        self.grid = grid
        self.n_obj = int(n_obj)
        self.total_nt = int(total_nt)
        h = ctypes.c_void_p()
        _check(lib().lsp_plan_create(ctypes.byref(h), self.n_obj, self.total_nt, ctypes.byref(grid),
                                     ctypes.byref(self.opts)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().lsp_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def config(self) -> dict:
        c = Config()
        _check(lib().lsp_plan_get_config(self._h, ctypes.byref(c)))
        return c.as_dict()

    def set_config(self, **cfg):
        c = Config()
        _check(lib().lsp_plan_get_config(self._h, ctypes.byref(c)))
        for k, v in cfg.items():
            setattr(c, k, int(v))
        _check(lib().lsp_plan_set_config(self._h, ctypes.byref(c)))

    def enable_timing(self, on: bool = True):
        """Record events around the main kernel of every execution (re-captures)."""
        _check(lib().lsp_plan_enable_timing(self._h, int(bool(on))))

    def main_kernel_ms(self) -> float:
        """Main-kernel duration of the last execution (waits for it)."""
        v = ctypes.c_float()
        _check(lib().lsp_plan_main_kernel_ms(self._h, ctypes.byref(v)))
        return float(v.value)

    @property
    def kernel_count(self) -> int:
        v = ctypes.c_int32()
        _check(lib().lsp_plan_kernel_count(self._h, ctypes.byref(v)))
        return int(v.value)

    def set_host_parts(self, parts: int):
        """Object groups of execute_host (0: by size, 1: one pass, n: n groups
        whose input and periodogram copies overlap the other groups' kernels)."""
        _check(lib().lsp_plan_set_host_parts(self._h, int(parts)))

    def host_parts(self, power: bool = True) -> int:
        """The group count execute_host uses for a call that returns this plan's
        full periodogram (power=True) or peaks only (power=False)."""
        v = ctypes.c_int32()
        nbytes = self.n_obj * self.grid.n_f * (8 if self.opts.precision == FP64 else 4) if power else 0
        _check(lib().lsp_plan_get_host_parts(self._h, nbytes, ctypes.byref(v)))
        return int(v.value)

    def peaks_buffer(self, device):
        torch = _torch()
        return torch.empty(self.n_obj * self.opts.top_k * 40, dtype=torch.uint8, device=device)

    def execute(self, t, y, offsets=None, power=None, peaks=None):
        """Run on device tensors; returns the peaks tensor (allocated if not given)."""
        torch = _torch()
        _require(t, "t", torch.float64, numel=self.total_nt)
        _require(y, "y", _dtypes(self.opts), t.device, numel=self.total_nt)
        if offsets is not None:
            _require(offsets, "offsets", torch.int64, t.device, numel=self.n_obj + 1)
        elif self.n_obj > 1:
            raise ValueError("a batch plan needs offsets")
        if power is not None:  # device memory, or page-locked host memory written directly
            _require(power, "power", _dtypes(self.opts), t.device, numel=self.n_obj * self.grid.n_f,
                     host_ok=True)
        if peaks is None:
            peaks = self.peaks_buffer(t.device)
        else:
            _require(peaks, "peaks", torch.uint8, t.device, numel=self.n_obj * self.opts.top_k * 40, host_ok=True)
        _check(lib().lsp_plan_execute(self._h, _ptr(t), _ptr(y), _ptr(offsets), _ptr(power), _ptr(peaks),
                                      _stream_handle(t.device)))
        return peaks

    def execute_host(self, t, y, offsets=None, power=None, peaks=None, device=None):
        """End-to-end on host buffers (numpy arrays or CPU tensors, pinned is fastest).

        Copies inputs in, runs, copies the peaks (and power if given) out, and
        synchronises.  Returns the peaks as a structured numpy array.
        """
        torch = _torch()
        tdt = {np.float64: torch.float64, np.float32: torch.float32, np.int64: torch.int64}

        def hptr(a, dtype, n, name):
            # the library reads or writes exactly n elements of `dtype` here
            if a is None:
                return ctypes.c_void_p(0)
            if isinstance(a, np.ndarray):
                if a.dtype != dtype or not a.flags.c_contiguous:
                    raise TypeError(f"{name} must be a contiguous {np.dtype(dtype).name} array")
                if a.size != n:
                    raise ValueError(f"{name} has {a.size} elements, the plan needs {n}")
                return ctypes.c_void_p(a.ctypes.data)
            if a.is_cuda or not a.is_contiguous() or a.dtype != tdt[dtype]:
                raise TypeError(f"{name} must be a contiguous CPU tensor of {tdt[dtype]}")
            if a.numel() != n:
                raise ValueError(f"{name} has {a.numel()} elements, the plan needs {n}")
            return ctypes.c_void_p(a.data_ptr())

        ydt = np.float64 if self.opts.precision == FP64 else np.float32
        n_pk = self.n_obj * self.opts.top_k
        if peaks is None:
            peaks = np.empty(n_pk, dtype=PEAK_DTYPE)
        if isinstance(peaks, np.ndarray):
            if peaks.dtype != PEAK_DTYPE or not peaks.flags.c_contiguous or peaks.size != n_pk:
                raise TypeError(f"peaks must be a contiguous array of {n_pk} PEAK_DTYPE records")
            pk_ptr = ctypes.c_void_p(peaks.ctypes.data)
        else:
            if peaks.is_cuda or not peaks.is_contiguous() or peaks.numel() * peaks.element_size() != n_pk * 40:
                raise TypeError(f"peaks must be a contiguous CPU tensor of {n_pk * 40} bytes")
            pk_ptr = ctypes.c_void_p(peaks.data_ptr())
        if self.n_obj > 1 and offsets is None:
            raise ValueError("a batch plan needs offsets")
        args = (hptr(t, np.float64, self.total_nt, "t"), hptr(y, ydt, self.total_nt, "y"),
                hptr(offsets, np.int64, self.n_obj + 1, "offsets"),
                hptr(power, ydt, self.n_obj * self.grid.n_f, "power"), pk_ptr)
        dev = device or torch.device("cuda", torch.cuda.current_device())
        _check(lib().lsp_plan_execute_host(self._h, *args, _stream_handle(dev)))
        return peaks

    def autotune(self, t, y, offsets=None, cache_path=None, ablations=False, return_trials=False):
        """Pick the fastest configuration within the FP32 error gate.  ablations:
        also measure the trig/staging ablation kernels.  return_trials: return
        (config, [trial dicts]) with every measured candidate."""
        torch = _torch()
        _require(t, "t", torch.float64, numel=self.total_nt)
        _require(y, "y", _dtypes(self.opts), t.device, numel=self.total_nt)
        if offsets is not None:
            _require(offsets, "offsets", torch.int64, t.device, numel=self.n_obj + 1)
        elif self.n_obj > 1:
            raise ValueError("a batch plan needs offsets")
        cp = cache_path.encode() if cache_path else None
        if not (ablations or return_trials):
            _check(lib().lsp_plan_autotune(self._h, _ptr(t), _ptr(y), _ptr(offsets), cp,
                                           _stream_handle(t.device)))
            return self.config
        buf = (Trial * 64)()
        n = ctypes.c_int32(0)
        _check(lib().lsp_plan_autotune_ex(self._h, _ptr(t), _ptr(y), _ptr(offsets), cp,
                                          TUNE_ABLATIONS if ablations else 0, buf, 64, ctypes.byref(n),
                                          _stream_handle(t.device)))
        trials = [dict(config=buf[i].config.as_dict(), ms=float(buf[i].ms), max_err=float(buf[i].max_err),
                       passed=bool(buf[i].passed), worst_object=int(buf[i].worst_object))
                  for i in range(min(n.value, 64))]
        return (self.config, trials) if return_trials else self.config

    def gate_report(self):
        """The last autotune's error gate: [(object index, max |P_n - P_n(FP64)|)] for the chosen configuration."""
        objs = (ctypes.c_int64 * 8)()
        errs = (ctypes.c_float * 8)()
        n = ctypes.c_int32(0)
        _check(lib().lsp_plan_gate_report(self._h, objs, errs, 8, ctypes.byref(n)))
        return [(int(objs[i]), float(errs[i])) for i in range(min(n.value, 8))]
