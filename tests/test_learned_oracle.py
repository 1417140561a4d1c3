"""Pins of the learned-stage oracle (oracle/learned.py), CPU only.

* Gradients: the analytic back-propagation equals central finite
  differences of the FP64 loss.
* Featurizer: closed forms (one pair of observations; evenly spaced lag
  counts), invariance to time shift / y shift and scale / permutation, and
  its purpose -- the short-lag periodogram peaks in the coarse bin of an
  injected frequency.
* bfloat16 rounding equals torch's float32 -> bfloat16 conversion.
* AdamW equals torch.optim.AdamW on the same step.
"""
import math

import numpy as np
import pytest
import torch

from oracle import learned as L


def test_finite_difference_gradients():
    shapes = L.layer_shapes(in_dim=7, hidden=6, n_hidden=3, n_classes=5)
    g = np.random.default_rng(0)
    theta = L.init_params(shapes, seed=3) + g.normal(0, 0.05, L.n_params(shapes))
    x = g.normal(0, 1, (9, 7))
    lab = g.integers(0, 5, 9)
    loss, grad = L.loss_and_grad(theta, x, lab, shapes)
    h = 1e-6
    idx = g.choice(theta.size, 60, replace=False)
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (L.loss_and_grad(tp, x, lab, shapes)[0] - L.loss_and_grad(tm, x, lab, shapes)[0]) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, grad[i])


def test_one_pair_closed_form():
    # two observations: z = (+1, -1) after standardisation, one pair at lag dt
    dt = 3.7
    f = L.featurize([60000.0, 60000.0 + dt], [2.0, 1.0], 0.24, 12.0)
    fc = 0.24 + (np.arange(256) + 0.5) * (12.0 - 0.24) / 256
    np.testing.assert_allclose(f[:256], -np.cos(2 * math.pi * fc * dt) / 2, atol=1e-12)
    expect = np.zeros(256)
    expect[int(dt * 256 / 16.0)] = math.log(2.0)
    np.testing.assert_allclose(f[256:], expect, atol=1e-12)


def test_even_spacing_lag_counts():
    # n evenly spaced points at spacing h: m*h lags occur n - m times
    n, h = 40, 0.7
    t = 60000.0 + h * np.arange(n)
    f = L.featurize(t, np.sin(np.arange(n)), 0.24, 12.0)
    expect = np.zeros(256)
    for m in range(1, n):
        if m * h < 16.0:
            expect[int(m * h * 256 / 16.0)] += n - m
    np.testing.assert_allclose(f[256:], np.log1p(expect), atol=1e-12)


def test_featurizer_invariances():
    g = np.random.default_rng(4)
    t = np.sort(g.uniform(60000, 60400, 120))
    y = np.sin(2 * math.pi * 2.3 * t) + g.normal(0, 0.3, 120)
    base = L.featurize(t, y, 0.24, 12.0)
    np.testing.assert_allclose(L.featurize(t + 1000.0, y, 0.24, 12.0), base, atol=1e-9)
    np.testing.assert_allclose(L.featurize(t, 3.0 * y - 7.0, 0.24, 12.0), base, atol=1e-12)
    p = g.permutation(120)
    np.testing.assert_allclose(L.featurize(t[p], y[p], 0.24, 12.0), base, atol=1e-12)


@pytest.mark.parametrize("f0", [0.7, 3.3, 9.1, 11.5])
def test_short_lag_periodogram_points_at_the_signal(f0):
    g = np.random.default_rng(int(f0 * 10))
    t = np.sort(g.uniform(60000, 60060, 300))  # dense: many short-lag pairs
    y = np.sin(2 * math.pi * f0 * t + 1.0) + g.normal(0, 0.2, 300)
    f = L.featurize(t, y, 0.24, 12.0)
    c0 = int((f0 - 0.24) / ((12.0 - 0.24) / 256))
    assert abs(int(np.argmax(f[:256])) - c0) <= 1


def test_bf16_rounding_matches_torch():
    g = np.random.default_rng(5)
    x = np.concatenate([g.normal(0, 1, 5000), g.normal(0, 1e-3, 1000), [0.0, -0.0, 1.0, 3.0e38]])
    x = x.astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(L.bf16(x), ref)


def test_adamw_matches_torch():
    g = np.random.default_rng(6)
    theta = g.normal(0, 1, 50)
    p = torch.nn.Parameter(torch.tensor(theta))
    opt = torch.optim.AdamW([p], lr=3e-3, betas=(0.9, 0.999), eps=1e-8, weight_decay=0.01)
    m = np.zeros(50)
    v = np.zeros(50)
    th = theta.copy()
    for step in range(1, 4):
        grad = g.normal(0, 1, 50)
        p.grad = torch.tensor(grad)
        opt.step()
        th, m, v = L.adamw_step(th, grad, m, v, step, lr=3e-3, wd=0.01)
    np.testing.assert_allclose(th, p.detach().numpy(), rtol=1e-12, atol=1e-12)


def test_intermediates_are_consistent_with_the_pinned_gradient():
    # the finite-difference-pinned bias gradients are the batch sums of dz,
    # and each hidden layer's input is the ReLU of the previous pre-activation
    shapes = L.layer_shapes(in_dim=7, hidden=6, n_hidden=3, n_classes=5)
    g = np.random.default_rng(1)
    theta = L.init_params(shapes, seed=4) + g.normal(0, 0.05, L.n_params(shapes))
    x = g.normal(0, 1, (9, 7))
    lab = g.integers(0, 5, 9)
    loss, grad, inter = L.loss_and_grad(theta, x, lab, shapes, return_intermediates=True)
    at = 0
    for l, (a, b) in enumerate(shapes):
        at += a * b
        np.testing.assert_allclose(inter["dz"][l].sum(axis=0), grad[at:at + b], atol=1e-14)
        at += b
        if l + 1 < len(shapes):
            np.testing.assert_array_equal(inter["acts"][l + 1], np.maximum(inter["z"][l], 0.0))
    logits, _ = L.forward(theta, x, shapes)
    np.testing.assert_allclose(inter["z"][-1], logits, atol=1e-14)


def test_windows_cover_the_grid_and_overlap_by_half():
    n_f, win, stride = 100_000, 2048, 1024
    n_cls = (n_f + stride - 1) // stride
    covered = np.zeros(n_f, dtype=bool)
    starts = [L.window_start(c, n_f, win, stride) for c in range(n_cls)]
    for c in range(n_cls):
        b = L.window_bins(c, n_f, win, stride)
        assert b.size == win and b[0] == starts[c] and b[-1] < n_f
        covered[b] = True
    assert covered.all()
    assert starts[0] == 0 and starts[-1] + win == n_f  # edge windows moved inside the grid
    for c in range(1, n_cls - 2):  # interior: centred on c*stride + stride/2, half-overlapping
        assert starts[c] + win // 2 == c * stride + stride // 2
        assert starts[c + 1] - starts[c] == stride
    # a grid narrower than one window: the whole grid
    np.testing.assert_array_equal(L.window_bins(3, 1500, win, stride), np.arange(1500))


def _replay_by_enumeration(wm, stop, fb, inconclusive):
    # the smallest prefix whose best power reaches stop (else all windows),
    # and the first maximum over the union of that prefix's window maxima
    n = len(wm)
    rounds = n
    for r in range(1, n + 1):
        if max([p for p, k in wm[:r] if k >= 0] + [0.0]) >= stop:
            rounds = r
            break
    cand = [(p, k) for p, k in wm[:rounds] if k >= 0]
    if cand:
        best_p = max(p for p, _ in cand)
        best_k = min(k for p, k in cand if p == best_p)
    else:
        best_p, best_k = 0.0, -1
    stopped = best_p >= stop
    return dict(rounds=rounds, stopped=stopped, fallback=best_p < fb or (inconclusive and not stopped),
                best_p=best_p, best_k=best_k)


def test_refine_rule_equals_enumeration():
    g = np.random.default_rng(9)
    levels = np.array([0.0, 0.1, 0.29, 0.3, 0.31, 0.45, 0.5, 0.7, 0.7])  # repeats make ties
    for _ in range(3000):
        n = int(g.integers(1, 6))
        wm = [(float(g.choice(levels)), int(g.integers(-1, 50)) if g.random() > 0.1 else -1)
              for _ in range(n)]
        wm = [(p if k >= 0 else 0.0, k) for p, k in wm]
        for inc in (False, True):
            assert L.refine_replay(wm, 0.5, 0.3, inc) == _replay_by_enumeration(wm, 0.5, 0.3, inc), wm


def test_refine_rule_special_cases():
    # stops at the first window that reaches the stop power
    r = L.refine_replay([(0.2, 10), (0.6, 900), (0.9, 5)], 0.5, 0.3)
    assert (r["rounds"], r["stopped"], r["fallback"], r["best_k"]) == (2, True, False, 900)
    # equal powers in two windows: the lower bin
    r = L.refine_replay([(0.4, 700), (0.4, 300)], 0.5, 0.3, inconclusive=False)
    assert (r["rounds"], r["best_k"], r["fallback"]) == (2, 300, False)
    # weak everywhere: full grid; inconclusive alone also falls back
    assert L.refine_replay([(0.1, 1), (0.2, 2)], 0.5, 0.3, False)["fallback"]
    assert L.refine_replay([(0.4, 1), (0.45, 2)], 0.5, 0.3, True)["fallback"]
    assert not L.refine_replay([(0.4, 1), (0.45, 2)], 0.5, 0.3, False)["fallback"]
