"""CPU oracle of the learned-proposal stage -- TEST INFRASTRUCTURE.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may use
this module.  The paper has no learned component; the stage and its
definitions below are this project's (the design notes list them as
readings).  Plain numpy in FP64, with no blocking or reordering.

Featurizer (512 values per light curve):
  z_j = (y_j - mean(y)) / rms(y - mean(y));
  pairs: every i < j with |t_j - t_i| < LAG_MAX;
  D[c] = sum_pairs z_i z_j cos(2 pi f_c |t_j - t_i|),
         f_c = f_min + (c + 1/2)(f_max - f_min)/256, c = 0..255;
  feat[c]       = D[c] / (P + 1), P = number of pairs;
  feat[256 + l] = log(1 + #pairs with |dt| in [l, l+1) * LAG_MAX / 256).
D is the periodogram of the light curve restricted to short lags: it has
resolution 1/LAG_MAX in frequency, enough to point at the window that holds
the full periodogram's peak.

MLP: x (512) -> 3 x [Linear(256) + ReLU] -> Linear(n_classes).  Parameters
are one flat vector in the order W1, b1, W2, b2, W3, b3, W4, b4 with W_l of
shape (fan_in, fan_out), row-major.  Loss: mean softmax cross-entropy.
``bf16=True`` rounds to bfloat16 (nearest-even) exactly where the GPU
kernels store bfloat16: inputs, weights, hidden activations, and the
back-propagated gradients of the pre-activations.

Refinement windows and the refine rule (this project's reading of the
"top-k windows, refine, fall back" workload):
  class c covers the ``window`` bins starting at c*stride + stride/2 - window/2,
  moved inside the grid [0, n_f);
  the proposed windows of an object are evaluated in rank order; each gives
  the first maximum of the periodogram over its bins; the running best keeps
  the larger power (the lower bin on a tie); evaluation stops once the best
  power reaches stop_power or the windows run out;
  the object falls back to the full grid when its best power is below
  fallback_power or, with ``inconclusive``, when no window reached stop_power.
"""
from __future__ import annotations

import math

import numpy as np

FEAT_DIM = 512
N_COARSE = 256
N_LAG = 256
LAG_MAX = 16.0  # days


def featurize(t, y, f_min, f_max, lag_max=LAG_MAX):
    """512 features of one light curve (see the module docstring)."""
    t = np.asarray(t, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    out = np.zeros(FEAT_DIM)
    n = t.size
    if n < 2:
        return out
    yc = y - y.mean()
    rms = math.sqrt(np.mean(yc * yc))
    if not rms > 0:
        return out
    z = yc / rms
    i, j = np.triu_indices(n, k=1)
    dt = np.abs(t[j] - t[i])
    keep = dt < lag_max
    dt, w = dt[keep], (z[i] * z[j])[keep]
    fc = f_min + (np.arange(N_COARSE) + 0.5) * (f_max - f_min) / N_COARSE
    d = np.cos(2 * math.pi * np.outer(fc, dt)) @ w
    out[:N_COARSE] = d / (dt.size + 1)
    lag_bin = np.minimum((dt * (N_LAG / lag_max)).astype(np.int64), N_LAG - 1)
    out[N_COARSE:] = np.log1p(np.bincount(lag_bin, minlength=N_LAG))
    return out


def featurize_batch(t, y, offsets, f_min, f_max, lag_max=LAG_MAX):
    off = np.asarray(offsets, dtype=np.int64)
    return np.stack([featurize(t[off[o]:off[o + 1]], y[off[o]:off[o + 1]], f_min, f_max, lag_max)
                     for o in range(off.size - 1)])


# ------------------------------------------------------------------ bf16
def bf16(x):
    """Round FP32 values to bfloat16, nearest-even, returned as float64."""
    a = np.asarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


# ------------------------------------------------------------------- MLP
def layer_shapes(in_dim=FEAT_DIM, hidden=256, n_hidden=3, n_classes=98):
    dims = [in_dim] + [hidden] * n_hidden + [n_classes]
    return [(dims[l], dims[l + 1]) for l in range(len(dims) - 1)]


def n_params(shapes):
    return sum(a * b + b for a, b in shapes)


def unpack(theta, shapes):
    """Views (W_l, b_l) of the flat parameter vector."""
    out, at = [], 0
    for a, b in shapes:
        w = theta[at:at + a * b].reshape(a, b)
        at += a * b
        bias = theta[at:at + b]
        at += b
        out.append((w, bias))
    return out


def forward(theta, x, shapes, bf16_mode=False):
    """Logits and the per-layer activations (inputs of each layer)."""
    rnd = bf16 if bf16_mode else (lambda v: np.asarray(v, dtype=np.float64))
    params = unpack(np.asarray(theta, dtype=np.float64), shapes)
    a = rnd(x)
    acts = [a]
    for l, (w, b) in enumerate(params):
        z = a @ rnd(w) + b
        if l + 1 < len(params):
            a = rnd(np.maximum(z, 0.0))
            acts.append(a)
        else:
            return z, acts
    raise AssertionError


def loss_and_grad(theta, x, labels, shapes, bf16_mode=False, return_intermediates=False):
    """Mean softmax cross-entropy and its gradient w.r.t. the flat parameters.

    With ``return_intermediates`` a third value holds, per layer l, the layer's
    input ``acts[l]``, its weights as used ``w[l]``, its pre-activation ``z[l]``
    and the gradient of the loss with respect to ``z[l]`` as used ``dz[l]``
    (rounded to bfloat16 in ``bf16_mode``, like the stored copies).
    """
    rnd = bf16 if bf16_mode else (lambda v: np.asarray(v, dtype=np.float64))
    theta = np.asarray(theta, dtype=np.float64)
    params = unpack(theta, shapes)
    logits, acts = forward(theta, x, shapes, bf16_mode)
    bsz = logits.shape[0]
    m = logits.max(axis=1, keepdims=True)
    e = np.exp(logits - m)
    sm = e / e.sum(axis=1, keepdims=True)
    lab = np.asarray(labels, dtype=np.int64)
    loss = float(np.mean(np.log(e.sum(axis=1)) + m[:, 0] - logits[np.arange(bsz), lab]))
    dz = sm.copy()
    dz[np.arange(bsz), lab] -= 1.0
    dz = rnd(dz / bsz)
    grads = [None] * len(params)
    dzs = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        w, _ = params[l]
        a_in = acts[l]
        dzs[l] = dz
        grads[l] = (a_in.T @ dz, dz.sum(axis=0))
        if l > 0:
            da = dz @ rnd(w).T
            dz = rnd(da * (acts[l] > 0))
    flat = np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in grads])
    if not return_intermediates:
        return loss, flat
    zs = [acts[l] @ rnd(w) + b for l, (w, b) in enumerate(params)]
    inter = dict(acts=acts, w=[rnd(w) for w, _ in params], z=zs, dz=dzs)
    return loss, flat, inter


def init_params(shapes, seed):
    """He-uniform weights, zero biases (deterministic in the seed)."""
    g = np.random.Generator(np.random.Philox(key=[seed, 0xA11CE]))
    parts = []
    for a, b in shapes:
        lim = math.sqrt(6.0 / a)
        parts.append(g.uniform(-lim, lim, a * b))
        parts.append(np.zeros(b))
    return np.concatenate(parts)


def adamw_step(theta, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0):
    """One AdamW update (step counts from 1), returning new (theta, m, v)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    theta = theta - lr * (mh / (np.sqrt(vh) + eps) + wd * theta)
    return theta, m, v


# ------------------------------------------------------- refine windows
def window_start(c, n_f, window=2048, stride=1024):
    """First bin of window class c: c*stride + stride/2 - window/2, moved inside [0, n_f)."""
    s = int(c) * int(stride) + int(stride) // 2 - int(window) // 2
    s = min(s, int(n_f) - int(window))
    return max(s, 0)


def window_bins(c, n_f, window=2048, stride=1024):
    """Grid indices of window class c (at most n_f of them)."""
    s = window_start(c, n_f, window, stride)
    return np.arange(s, min(s + int(window), int(n_f)), dtype=np.int64)


def first_max(power, bins):
    """(power, bin) of the first maximum of ``power`` over ``bins`` (bins ascending)."""
    p = np.asarray(power, dtype=np.float64)
    i = int(np.argmax(p))  # numpy's argmax returns the first of equal maxima
    return float(p[i]), int(bins[i])


def refine_replay(window_maxima, stop_power, fallback_power, inconclusive=True):
    """The refine rule over one object's ranked windows.

    ``window_maxima`` lists, in rank order, the (power, bin) first maximum of
    every proposed window (as if all were evaluated).  Returns rounds (windows
    evaluated), stopped, fallback and the best (power, bin) of the evaluated
    windows.
    """
    best_p, best_k = 0.0, -1
    rounds, stopped = 0, False
    for p, k in window_maxima:
        rounds += 1
        if k >= 0 and (p > best_p or (p == best_p and (best_k < 0 or k < best_k))):
            best_p, best_k = float(p), int(k)
        stopped = best_p >= stop_power
        if stopped:
            break
    fallback = best_p < fallback_power or (bool(inconclusive) and not stopped)
    return dict(rounds=rounds, stopped=stopped, fallback=fallback, best_p=best_p, best_k=best_k)
