"""Element-wise tolerances for comparing the GPU MLP with the FP64 oracle.

The GPU stores inputs, weights, hidden activations and back-propagated
pre-activation gradients in bfloat16 and accumulates products in FP32; the
oracle (oracle/learned.py, ``bf16_mode=True``) rounds at the same points but
accumulates in FP64.

The gradient comparison uses parameters and inputs on a dyadic lattice
(few-bit multiples of powers of two), chosen so that every forward sum is
exact in FP32: ``lattice_exact`` checks that premise on the oracle's own
values.  The forward pass is then identical on both sides, bit for bit.
The backward pass starts from the softmax, which FP32 and FP64 evaluate
differently, so each stored bfloat16 gradient either equals the oracle's or
-- where the oracle's unrounded value lies within the FP32 error of a
bfloat16 rounding midpoint -- may differ by about one bfloat16 ulp.
``grad_bound`` finds those ambiguous elements layer by layer, propagates
their possible difference to the later layers and to the parameter
gradients, and adds the FP32 accumulation error gamma(K) = K * 2^-23 times the
sum of absolute products wherever a sum is not exact in FP32.  The result is one bound per gradient element:
a wrong sign, a swapped operand or a dropped term changes an element by O(1)
of its size and exceeds it.
"""
from __future__ import annotations

import numpy as np

EPS32 = 2.0 ** -24


def gamma(k):
    return k * 2.0 ** -23


def bf16_ulp(v):
    """Spacing of bfloat16 values at |v| (8 significant bits)."""
    a = np.abs(np.asarray(v, dtype=np.float64))
    e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    return np.where(a > 0, 2.0 ** (e - 7), 0.0)


def midpoint_distance(v):
    """Distance of v from the nearest bfloat16 rounding midpoint."""
    u = bf16_ulp(v)
    a = np.abs(np.asarray(v, dtype=np.float64))
    frac = np.where(u > 0, a / np.where(u > 0, u, 1.0), 0.0)
    return np.abs(frac - np.floor(frac) - 0.5) * u


def _granularity(v):
    """Largest power of two dividing every non-zero entry of each row of v (FP64 values)."""
    a = np.abs(np.asarray(v, dtype=np.float64))
    m, e = np.frexp(a)  # a = m 2^e, m in [0.5, 1)
    # trailing zero bits of the 53-bit significand give the last set bit
    sig = (m * 2.0 ** 53).astype(np.uint64)
    tz = np.zeros(sig.shape, dtype=np.int64)
    s = sig.copy()
    for _ in range(53):
        z = (s & np.uint64(1)) == 0
        z &= s != 0
        tz += z
        s = np.where(z, s >> np.uint64(1), s)
    last = np.where(a > 0, e - 53 + tz, 1 << 20)
    return last.min(axis=-1)


def lattice_exact(inter, biases):
    """True when every forward sum (inputs times weights plus bias, per output)
    has terms on a common power-of-two grid 2^g and absolute values adding up
    to less than 2^(g + 24): such a sum is exact in FP32 in any order.  Also
    returns, per layer, (g, the largest sum over 2^(g + 24))."""
    acts, w = inter["acts"], inter["w"]
    ok, info = True, []
    for l in range(len(w)):
        ga = _granularity(acts[l].reshape(1, -1))[0]
        gw = _granularity(w[l].reshape(1, -1))[0]
        gb = _granularity(np.asarray(biases[l], dtype=np.float64).reshape(1, -1))[0]
        g = int(min(ga + gw, gb))
        total = np.abs(acts[l]) @ np.abs(w[l]) + np.abs(biases[l])
        ratio = float(total.max() / 2.0 ** (g + 24))
        ok &= ratio < 1.0
        info.append((g, ratio))
    return ok, info


def _exact_rows(terms_abs_sum, g_row):
    """True where a sum whose terms are multiples of 2^g_row and whose absolute
    values add to terms_abs_sum is exact in FP32 whatever the order."""
    return terms_abs_sum < 2.0 ** (g_row + 24)


def grad_bound(inter, labels):
    """Bound on |grad_gpu - grad_oracle| per element (layout W1, b1, ...),
    valid when the forward pass is exact on both sides (lattice_exact), and
    the number of bfloat16 gradient elements whose rounding is ambiguous."""
    acts, w, z, dz = inter["acts"], inter["w"], inter["z"], inter["dz"]
    n = len(w)
    logits = z[-1]
    bsz, n_cls = logits.shape
    p = np.exp(logits - logits.max(axis=1, keepdims=True))
    p /= p.sum(axis=1, keepdims=True)
    onehot = np.zeros_like(p)
    onehot[np.arange(bsz), np.asarray(labels, dtype=np.int64)] = 1.0
    pre = (p - onehot) / bsz
    # FP32 softmax of one row: exponentials, subtraction and scaling within a
    # few ulp, the row's sum within (n_cls / 32 + 5) ulp (32 lanes, then a
    # 5-level tree); allowed twice over
    delta = (8 + n_cls / 32 + 5) * 2 * EPS32 * (p + np.abs(p - onehot)) / bsz
    ed = [None] * n
    n_amb = 0

    def stored_error(v, d, live=True):
        nonlocal n_amb
        amb = live & (d > 0) & ((midpoint_distance(v) <= d) | (np.abs(v) <= d))
        n_amb += int(amb.sum())
        return np.where(amb, d + bf16_ulp(np.abs(v) + d), 0.0)

    ed[-1] = stored_error(pre, delta)
    for l in range(n - 1, 0, -1):
        aw = np.abs(w[l]).T
        da_pre = dz[l] @ w[l].T
        # products of stored bfloat16 gradients and lattice weights: where the
        # row's sum is exact in FP32 only the differing inputs contribute
        g_row = _granularity(dz[l]) + int(_granularity(w[l].T.reshape(1, -1))[0])
        tot = (np.abs(dz[l]) + ed[l]) @ aw
        acc = np.where(_exact_rows(tot, g_row[:, None]), 0.0, gamma(w[l].shape[1]) * tot)
        d = ed[l] @ aw + acc
        mask = acts[l] > 0
        ed[l - 1] = stored_error(da_pre * mask, d, mask)
    parts = []
    for l in range(n):
        a = np.abs(acts[l])
        gw = a.T @ ed[l] + gamma(bsz) * (a.T @ (np.abs(dz[l]) + ed[l]))
        gb = ed[l].sum(axis=0) + gamma(bsz) * (np.abs(dz[l]) + ed[l]).sum(axis=0)
        parts += [gw.ravel(), gb]
    return np.concatenate(parts), n_amb


def dyadic_problem(shapes, batch, seed):
    """Parameters and bfloat16 inputs on a dyadic lattice: weights in
    {-1, 0, 1} / 16 (half of them zero), biases in {-4..4} / 512, inputs in
    {-2..2} / 4.  Exact in FP32 and in bfloat16."""
    g = np.random.default_rng(seed)
    parts = []
    for a, b in shapes:
        wv = g.integers(-1, 2, a * b) * (g.random(a * b) < 0.5)
        parts += [wv / 16.0, g.integers(-4, 5, b) / 512.0]
    theta = np.concatenate(parts)
    x = g.integers(-2, 3, (batch, shapes[0][0])) / 4.0
    labels = g.integers(0, shapes[-1][1], batch)
    return theta, x, labels
