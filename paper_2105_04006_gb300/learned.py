"""Learned proposal stage: featurize -> MLP -> top-k windows -> refine -> fallback.

Binding-level orchestration only: every numeric step (features, GEMMs,
loss, gradients, AdamW, top-k, the windowed direct method, the full-grid
fallback) runs in the CUDA library through ``include/lsp.h``.  Torch holds
the device memory.  The paper has no learned component; see the design
notes for the readings this stage rests on.

Windows: class c of a grid of n_f bins covers the 2048 bins centred on
c * 1024 + 512 (stride 1024), so consecutive windows overlap by half and the
bin of any maximum lies well inside some window.  The network is trained to
name the class of the full-grid maximum computed by lsp_batch.
"""
from __future__ import annotations

import ctypes
import math
import time

import numpy as np

from . import FP32, Grid, MlpDims, NORM_STANDARD, PEAK_DTYPE, _check, _ptr, _require, _stream_handle, batch, \
    lib, peaks_to_numpy
from . import Proposer as _ProposerStruct

FEAT_DIM = 512
LAG_MAX = 16.0
WINDOW = 2048
STRIDE = 1024
REFINE_FALLBACK = 256  # bit of the refine's info word (LSP_REFINE_FALLBACK)


def n_classes(n_f: int, stride: int = STRIDE) -> int:
    return (int(n_f) + stride - 1) // stride


def featurize(t, y, offsets, grid: Grid, lag_max: float = LAG_MAX, want_f32: bool = False):
    """bfloat16 features (n_obj x 512) [and FP32 copy] of a CSR batch on the device."""
    import torch
    _require(t, "t", torch.float64)
    _require(y, "y", torch.float32, t.device, numel=t.numel())
    _require(offsets, "offsets", torch.int64, t.device)
    n_obj = offsets.numel() - 1
    f16 = torch.empty((n_obj, FEAT_DIM), dtype=torch.bfloat16, device=t.device)
    f32 = torch.empty((n_obj, FEAT_DIM), dtype=torch.float32, device=t.device) if want_f32 else None
    _check(lib().lsp_featurize(_ptr(t), _ptr(y), _ptr(offsets), n_obj, t.numel(), ctypes.byref(grid),
                               float(lag_max), _ptr(f16), _ptr(f32), _stream_handle(t.device)))
    return (f16, f32) if want_f32 else f16


def he_init(dims: MlpDims, seed: int) -> np.ndarray:
    """He-uniform weights and zero biases, drawn on the host (a Philox stream keyed by seed)."""
    g = np.random.Generator(np.random.Philox(key=[seed, 0xA11CE]))
    widths = [dims.in_dim] + [dims.hidden] * dims.n_hidden + [dims.n_classes]
    parts = []
    for a, b in zip(widths[:-1], widths[1:]):
        lim = math.sqrt(6.0 / a)
        parts.append(g.uniform(-lim, lim, a * b))
        parts.append(np.zeros(b))
    return np.concatenate(parts)


class Proposer:
    """The MLP proposal network, its AdamW state and the refine settings."""

    def __init__(self, n_f: int, device, hidden: int = 256, n_hidden: int = 3, seed: int = 1,
                 k_windows: int = 8, stop_power: float = 0.5, fallback_power: float = 0.3,
                 inconclusive_fallback: bool = True):
        import torch
        device = torch.device(device)
        if device.type == "cuda" and device.index is None:
            device = torch.device("cuda", torch.cuda.current_device())
        self.device = device
        self.n_f = int(n_f)
        self.dims = MlpDims(FEAT_DIM, hidden, n_hidden, n_classes(n_f))
        cnt = ctypes.c_int64()
        _check(lib().lsp_mlp_param_count(ctypes.byref(self.dims), ctypes.byref(cnt)))
        self.n_params = int(cnt.value)
        theta = he_init(self.dims, seed)
        assert theta.size == self.n_params
        self.params = torch.tensor(theta, dtype=torch.float32, device=device)
        self.params16 = torch.empty(self.n_params, dtype=torch.bfloat16, device=device)
        self.grad = torch.zeros(self.n_params, dtype=torch.float32, device=device)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step = 0
        self.k_windows = k_windows
        self.stop_power = stop_power
        self.fallback_power = fallback_power
        self.inconclusive_fallback = inconclusive_fallback
        self._ws = None
        self._ws_batch = 0
        self._loss = torch.zeros(1, dtype=torch.float32, device=device)
        self.refresh_bf16()

    # -- parameters ---------------------------------------------------------
    def refresh_bf16(self):
        _check(lib().lsp_to_bf16(_ptr(self.params), _ptr(self.params16), self.n_params,
                                 _stream_handle(self.device)))

    def _workspace(self, batch_size):
        import torch
        if self._ws is None or self._ws_batch < batch_size:
            n = ctypes.c_size_t()
            _check(lib().lsp_mlp_workspace_size(ctypes.byref(self.dims), int(batch_size), ctypes.byref(n)))
            self._ws = torch.empty(int(n.value), dtype=torch.uint8, device=self.device)
            self._ws_batch = batch_size
        return self._ws

    # -- network ------------------------------------------------------------
    def _require_x(self, x16):
        import torch
        if x16.dim() != 2 or x16.shape[1] != self.dims.in_dim:
            raise ValueError(f"x16 must be (batch, {self.dims.in_dim}), got {tuple(x16.shape)}")
        _require(x16, "x16", torch.bfloat16, self.device)

    def forward(self, x16):
        import torch
        self._require_x(x16)
        b = x16.shape[0]
        logits = torch.empty((b, self.dims.n_classes), dtype=torch.float32, device=self.device)
        ws = self._workspace(b)
        _check(lib().lsp_mlp_forward(ctypes.byref(self.dims), _ptr(self.params), _ptr(self.params16), _ptr(x16),
                                     b, _ptr(logits), _ptr(ws), ws.numel(), _stream_handle(self.device)))
        return logits

    def loss_grad(self, x16, labels):
        """Mean cross-entropy (device scalar) and the gradient (in self.grad)."""
        import torch
        self._require_x(x16)
        b = x16.shape[0]
        _require(labels, "labels", torch.int32, self.device, numel=b)
        ws = self._workspace(b)
        _check(lib().lsp_mlp_loss_grad(ctypes.byref(self.dims), _ptr(self.params), _ptr(self.params16),
                                       _ptr(x16), _ptr(labels), b, _ptr(self._loss), _ptr(self.grad), _ptr(ws),
                                       ws.numel(), _stream_handle(self.device)))
        return self._loss

    def train_step(self, x16, labels, lr=1e-3, weight_decay=1e-4):
        loss = self.loss_grad(x16, labels)
        self.step += 1
        _check(lib().lsp_mlp_adamw(self.n_params, _ptr(self.params), _ptr(self.params16), _ptr(self.grad),
                                   _ptr(self.m), _ptr(self.v), self.step, float(lr), 0.9, 0.999, 1e-8,
                                   float(weight_decay), _stream_handle(self.device)))
        return loss

    def propose(self, x16, k=None):
        """Top-k window classes per row, best first (int32, n x k)."""
        import torch
        k = int(k or self.k_windows)
        logits = self.forward(x16)
        cls = torch.empty((x16.shape[0], k), dtype=torch.int32, device=self.device)
        _check(lib().lsp_top_classes(_ptr(logits), x16.shape[0], self.dims.n_classes, k, _ptr(cls),
                                     _stream_handle(self.device)))
        return cls

    def as_struct(self, window=WINDOW, stride=STRIDE, lag_max=LAG_MAX, norm=NORM_STANDARD):
        """The lsp_proposer record of this network (pointers into its device tensors)."""
        return _ProposerStruct(self.dims, self.params.data_ptr(), self.params16.data_ptr(), int(window),
                               int(stride), float(lag_max), int(self.k_windows), float(self.stop_power),
                               float(self.fallback_power), int(bool(self.inconclusive_fallback)), int(norm))

    # -- checkpoints --------------------------------------------------------
    def state_dict(self):
        return {"params": self.params.detach().cpu(), "m": self.m.detach().cpu(), "v": self.v.detach().cpu(),
                "step": self.step, "dims": (self.dims.in_dim, self.dims.hidden, self.dims.n_hidden,
                                            self.dims.n_classes),
                "n_f": self.n_f, "k_windows": self.k_windows, "stop_power": self.stop_power,
                "fallback_power": self.fallback_power, "inconclusive_fallback": self.inconclusive_fallback}

    def load_state_dict(self, sd):
        dims = tuple(sd["dims"])
        if dims != (self.dims.in_dim, self.dims.hidden, self.dims.n_hidden, self.dims.n_classes):
            raise ValueError(f"checkpoint dims {dims} do not match")
        self.params.copy_(sd["params"].to(self.device))
        self.m.copy_(sd["m"].to(self.device))
        self.v.copy_(sd["v"].to(self.device))
        self.step = int(sd["step"])
        self.k_windows = int(sd["k_windows"])
        self.stop_power = float(sd["stop_power"])
        self.fallback_power = float(sd["fallback_power"])
        self.inconclusive_fallback = bool(sd.get("inconclusive_fallback", True))
        self.refresh_bf16()

    def save(self, path, extra=None):
        import torch
        sd = self.state_dict()
        if extra:
            sd["extra"] = extra
        torch.save(sd, path)

    def save_npz(self, path, **meta):
        """The network alone (FP32 parameters and settings, no optimizer state)
        as a compressed numpy archive; `meta` adds string or number fields."""
        d = dict(params=self.params.detach().cpu().numpy().astype(np.float32),
                 dims=np.array([self.dims.in_dim, self.dims.hidden, self.dims.n_hidden, self.dims.n_classes]),
                 n_f=np.array(self.n_f), k_windows=np.array(self.k_windows),
                 stop_power=np.array(self.stop_power), fallback_power=np.array(self.fallback_power),
                 inconclusive_fallback=np.array(int(bool(self.inconclusive_fallback))), step=np.array(self.step))
        for k, v in meta.items():
            d["meta_" + k] = np.array(v)
        np.savez_compressed(path, **d)

    @classmethod
    def load_npz(cls, path, device):
        """A network written by save_npz; returns (proposer, metadata dict)."""
        import torch
        with np.load(path) as z:
            dims = [int(v) for v in z["dims"]]
            p = cls(int(z["n_f"]), device, hidden=dims[1], n_hidden=dims[2], k_windows=int(z["k_windows"]),
                    stop_power=float(z["stop_power"]), fallback_power=float(z["fallback_power"]),
                    inconclusive_fallback=bool(int(z["inconclusive_fallback"])))
            if dims != [p.dims.in_dim, p.dims.hidden, p.dims.n_hidden, p.dims.n_classes]:
                raise ValueError(f"checkpoint dims {dims} do not match")
            p.params.copy_(torch.from_numpy(z["params"]).to(p.device))
            p.step = int(z["step"])
            meta = {k[5:]: z[k].item() for k in z.files if k.startswith("meta_")}
        p.refresh_bf16()
        return p, meta

    @classmethod
    def load(cls, path, device):
        import torch
        sd = torch.load(path, map_location="cpu")
        d = sd["dims"]
        p = cls(sd["n_f"], device, hidden=d[1], n_hidden=d[2])
        p.load_state_dict(sd)
        return p, sd.get("extra")


def refine(t, y, offsets, grid: Grid, classes, k_windows, stop_power, fallback_power,
           inconclusive_fallback=True, window=WINDOW, stride=STRIDE, norm=NORM_STANDARD, workspace=None):
    """Windowed direct method with full-grid fallback; returns (peaks uint8 tensor, info int32)."""
    import torch
    _require(t, "t", torch.float64)
    _require(y, "y", torch.float32, t.device, numel=t.numel())
    _require(offsets, "offsets", torch.int64, t.device)
    n_obj = offsets.numel() - 1
    _require(classes, "classes", torch.int32, t.device, numel=n_obj * int(k_windows))
    n = ctypes.c_size_t()
    _check(lib().lsp_refine_workspace_size(n_obj, t.numel(), ctypes.byref(grid), ctypes.byref(n)))
    ws = workspace if workspace is not None else torch.empty(max(int(n.value), 256), dtype=torch.uint8,
                                                                device=t.device)
    peaks = torch.empty(n_obj * 40, dtype=torch.uint8, device=t.device)
    info = torch.empty(n_obj, dtype=torch.int32, device=t.device)
    _check(lib().lsp_refine_windows(_ptr(t), _ptr(y), _ptr(offsets), n_obj, t.numel(), ctypes.byref(grid),
                                    int(norm), _ptr(classes), int(k_windows), int(window), int(stride),
                                    float(stop_power), float(fallback_power), int(bool(inconclusive_fallback)),
                                    _ptr(peaks), _ptr(info), _ptr(ws),
                                    ws.numel(), _stream_handle(t.device)))
    return peaks, info


class LearnedPath:
    """The learned path as one library call (lsp_propose_refine) on a CSR batch
    on the device, with its workspace kept between calls of the same shape."""

    def __init__(self, proposer: Proposer):
        self.proposer = proposer
        self._ws = None

    def __call__(self, t, y, offsets, grid: Grid, classes_out=None):
        """(peaks uint8 tensor of n_obj records, info int32 tensor)."""
        import torch
        _require(t, "t", torch.float64)
        _require(y, "y", torch.float32, t.device, numel=t.numel())
        _require(offsets, "offsets", torch.int64, t.device)
        n_obj = offsets.numel() - 1
        net = self.proposer.as_struct()
        n = ctypes.c_size_t()
        _check(lib().lsp_propose_refine_workspace_size(ctypes.byref(net), n_obj, t.numel(), ctypes.byref(grid),
                                                       ctypes.byref(n)))
        if self._ws is None or self._ws.numel() < int(n.value) or self._ws.device != t.device:
            self._ws = torch.empty(max(int(n.value), 256), dtype=torch.uint8, device=t.device)
        if classes_out is not None:
            _require(classes_out, "classes_out", torch.int32, t.device, numel=n_obj * net.k_windows)
        peaks = torch.empty(n_obj * 40, dtype=torch.uint8, device=t.device)
        info = torch.empty(n_obj, dtype=torch.int32, device=t.device)
        _check(lib().lsp_propose_refine(ctypes.byref(net), _ptr(t), _ptr(y), _ptr(offsets), n_obj, t.numel(),
                                        ctypes.byref(grid), _ptr(peaks), _ptr(info), _ptr(classes_out),
                                        _ptr(self._ws), self._ws.numel(), _stream_handle(t.device)))
        return peaks, info


def propose_and_refine(proposer: Proposer, t, y, offsets, grid: Grid):
    """The whole learned path for a CSR batch on the device, one library call: (peaks, info)."""
    return LearnedPath(proposer)(t, y, offsets, grid)


def window_labels(peaks, n_obj, n_cls, stride=STRIDE):
    """Training labels: the window class of each object's full-grid first maximum."""
    import torch
    _require(peaks, "peaks", torch.uint8, numel=n_obj * 40)
    labels = torch.empty(n_obj, dtype=torch.int32, device=peaks.device)
    _check(lib().lsp_window_labels(_ptr(peaks), n_obj, int(stride), int(n_cls), _ptr(labels),
                                   _stream_handle(peaks.device)))
    return labels


# --------------------------------------------------------------- training data
def labelled_set(n_obj, device, which="learned_train", part=0, grid=None):
    """A survey-shaped set on the device, its features and full-grid labels.

    The labels are the window classes of the first maximum of each object's
    full-grid periodogram, computed by the direct method (lsp_batch).
    """
    import torch
    import synth
    b = synth.learned_set(n_obj, which=which, part=part, grid=grid)
    g = Grid(b.grid.f_min, b.grid.f_max, b.grid.n_f)
    t = torch.tensor(b.t, dtype=torch.float64, device=device)
    y = torch.tensor(b.y.astype(np.float32), device=device)
    off = torch.tensor(b.offsets, dtype=torch.int64, device=device)
    _, peaks = batch(t, y, off, g)
    idx = torch.from_numpy(peaks_to_numpy(peaks)["idx"].copy()).to(device)
    labels = window_labels(peaks, b.n_obj, n_classes(g.n_f))
    x16 = featurize(t, y, off, g)
    return dict(batch=b, grid=g, t=t, y=y, off=off, x16=x16, labels=labels, full_idx=idx)


def train(proposer: Proposer, sets, epochs=4, batch_size=4096, lr=2e-3, seed=0, log=None):
    """Mini-batch AdamW over the labelled sets (lists of dicts from labelled_set)."""
    import torch
    x = torch.cat([s["x16"] for s in sets])
    lab = torch.cat([s["labels"] for s in sets])
    n = x.shape[0]
    g = np.random.Generator(np.random.Philox(key=[seed, 0x7A1]))
    hist = []
    steps_per_epoch = max(1, n // batch_size)
    total = epochs * steps_per_epoch
    for ep in range(epochs):
        perm = torch.from_numpy(g.permutation(n)).to(x.device)
        for i in range(steps_per_epoch):
            sel = perm[i * batch_size:(i + 1) * batch_size]
            # cosine learning-rate decay over the whole run
            frac = (ep * steps_per_epoch + i) / max(1, total - 1)
            loss = proposer.train_step(x[sel].contiguous(), lab[sel].contiguous(),
                                       lr=lr * 0.5 * (1 + math.cos(math.pi * frac)))
        hist.append(float(loss.item()))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.4f}")
    return hist


def evaluate(proposer: Proposer, s, stop_power=None, fallback_power=None, k_windows=None,
             inconclusive_fallback=None):
    """Run the learned path on a labelled set: recovery against the full grid and cost."""
    kw = k_windows or proposer.k_windows
    cls = proposer.propose(s["x16"], kw)
    sp = proposer.stop_power if stop_power is None else stop_power
    fp = proposer.fallback_power if fallback_power is None else fallback_power
    inc = proposer.inconclusive_fallback if inconclusive_fallback is None else inconclusive_fallback
    peaks, info = refine(s["t"], s["y"], s["off"], s["grid"], cls, kw, sp, fp, inc)
    pk = peaks_to_numpy(peaks)
    info = info.cpu().numpy()
    full = s["full_idx"].cpu().numpy()
    ok = np.abs(pk["idx"] - full) <= 1
    fb = (info & 256) != 0
    rounds = info & 255
    n_f = s["grid"].n_f
    b = s["batch"]
    nt = b.n_t
    pairs = float(np.sum(nt * (rounds * WINDOW + fb * n_f)))
    return dict(recovery=float(ok.mean()), fallback=float(fb.mean()), mean_windows=float(rounds.mean()),
                pair_fraction=pairs / float(b.pairs), n=int(b.n_obj))
