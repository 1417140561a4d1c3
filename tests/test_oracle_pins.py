"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Every test here is CPU-only.  None re-types the oracle's formula: each checks
the oracle against an independent statement of the same quantity --

* Section 2 / Eq. 2 equals half the chi-square reduction of a least-squares
  fit of a cos(wt) + b sin(wt) (numpy lstsq, i.e. an SVD solve);
* on evenly sampled data at Fourier frequencies, Eq. 2 equals |DFT|^2 / N
  (numpy FFT);
* with two observations the 2-parameter fit is exact, so P = sum(y^2)/2;
* a noiseless sinusoid on the grid has normalised power exactly 1;
* reversing time, permuting, negating or scaling the data leaves P_n fixed;
* 0 <= P_n <= 1;
* an injected high-SNR period is recovered within one bin;
* an extended-precision recomputation agrees to 1e-12;
* argmax / top-k semantics against brute force (Section 3.3, first maximum).
"""
import math

import numpy as np
import pytest

import synth


def _lsq_power(t, y, f):
    """Half the chi-square reduction of the 2-parameter sinusoid fit (no offset)."""
    w = 2 * math.pi * f
    X = np.stack([np.cos(w * t), np.sin(w * t)], axis=1)
    beta, *_ = np.linalg.lstsq(X, y, rcond=None)
    resid = y - X @ beta
    return 0.5 * (np.dot(y, y) - np.dot(resid, resid))


@pytest.mark.parametrize("n_t", [3, 4, 5, 8, 16])
def test_least_squares_reduction(oracle_mod, n_t):
    g = np.random.default_rng(100 + n_t)
    for trial in range(5):
        t = np.sort(g.uniform(60000, 60030, n_t))
        y = g.normal(0, 1, n_t)
        yc = y - y.mean()
        f_min, f_max, n_f = 0.3, 4.0, 37
        ks = g.integers(0, n_f, 6)
        p, fl = oracle_mod.lsp_single(t, y, f_min, f_max, n_f, norm=0, k_sel=ks)
        assert fl == 0
        fk = oracle_mod.grid_freqs(f_min, f_max, n_f)[ks]
        ref = np.array([_lsq_power(t - t[0], yc, f) for f in fk])
        np.testing.assert_allclose(p, ref, rtol=1e-9, atol=1e-12)


def test_two_observations_closed_form(oracle_mod):
    # With N_t = 2 the two-parameter fit reproduces the data exactly.
    t = np.array([60000.125, 60003.7])
    y = np.array([0.3, -1.1])
    p, fl = oracle_mod.lsp_single(t, y, 0.21, 3.3, 11, norm=0)
    yc = y - y.mean()
    np.testing.assert_allclose(p, 0.5 * np.dot(yc, yc), rtol=1e-10)


def test_fft_even_sampling(oracle_mod):
    n, dt = 64, 0.37
    g = np.random.default_rng(7)
    t = 60000.0 + dt * np.arange(n)
    y = g.normal(0, 1, n)
    yc = y - y.mean()
    df = 1.0 / (n * dt)
    n_f = n // 2 - 1  # m = 1 .. n/2 - 1
    p, fl = oracle_mod.lsp_single(t, y, df, df * (n_f + 1), n_f, norm=0)
    ref = np.abs(np.fft.fft(yc)[1:n_f + 1]) ** 2 / n
    np.testing.assert_allclose(p, ref, rtol=1e-9, atol=1e-12)


def test_exact_fit_power_one(oracle_mod):
    g = np.random.default_rng(11)
    t = np.sort(g.uniform(60000, 61000, 200))
    f_min, f_max, n_f = 0.1, 10.0, 1000
    k0 = 437
    f0 = oracle_mod.grid_freqs(f_min, f_max, n_f)[k0]
    y = 0.7 * np.cos(2 * math.pi * f0 * (t - 60000) + 0.4)
    # no centring: the pure sinusoid is exactly the two-parameter model
    p, fl = oracle_mod.lsp_single(t, y, f_min, f_max, n_f, norm=1, center=False, k_sel=[k0])
    assert abs(p[0] - 1.0) < 1e-11


def test_invariances(oracle_mod):
    g = np.random.default_rng(12)
    n = 150
    t = np.sort(g.uniform(60000, 62000, n))
    y = 0.4 * np.sin(2 * math.pi * 1.7 * t) + g.normal(0, 0.3, n)
    args = (0.2, 8.0, 4000)
    base, _ = oracle_mod.lsp_single(t, y, *args, norm=1)
    # time reversal: the oracle's internal shift differs, tau changes sign
    rev, _ = oracle_mod.lsp_single(-t[::-1], y[::-1], *args, norm=1)
    np.testing.assert_allclose(rev, base, rtol=0, atol=1e-10)
    # time shift by a non-representable amount
    sh, _ = oracle_mod.lsp_single(t + 12345.678, y, *args, norm=1)
    np.testing.assert_allclose(sh, base, rtol=0, atol=1e-8)
    # permutation
    perm = g.permutation(n)
    pm, _ = oracle_mod.lsp_single(t[perm], y[perm], *args, norm=1)
    np.testing.assert_allclose(pm, base, rtol=0, atol=1e-12)
    # sign and scale: P_n unchanged, P scales with a^2
    neg, _ = oracle_mod.lsp_single(t, -y, *args, norm=1)
    np.testing.assert_allclose(neg, base, rtol=0, atol=1e-12)
    p0, _ = oracle_mod.lsp_single(t, y, *args, norm=0)
    p3, _ = oracle_mod.lsp_single(t, 3.0 * y, *args, norm=0)
    np.testing.assert_allclose(p3, 9.0 * p0, rtol=1e-11)
    s3, _ = oracle_mod.lsp_single(t, 3.0 * y, *args, norm=1)
    np.testing.assert_allclose(s3, base, rtol=0, atol=1e-12)


def test_normalised_power_bounds(oracle_mod):
    b = synth.ragged_survey(40, seed=5, grid=synth.Grid(0.24, 12.0, 3000))
    res = oracle_mod.lsp_batch(b.t, b.y, b.offsets, 0.24, 12.0, 3000, norm=1, return_power=True)
    assert (res["flags"] == 0).all()
    assert res["power"].min() >= 0.0
    assert res["power"].max() <= 1.0 + 1e-12


def test_injected_period_recovery(oracle_mod):
    # Section 4.2: the L-S peak finds the injected period.  High SNR, N_t >= 200.
    # One 180-day season, so the peak (width ~1/180 c/d) spans ~10 bins of the
    # grid and sits within one bin of the injected frequency.
    grid = synth.Grid(0.24, 12.0, 20000)
    g = np.random.default_rng(77)
    n_obj, n_t = 24, 300
    f0 = np.exp(g.uniform(np.log(0.3), np.log(11.5), n_obj))
    ts, ys = [], []
    for o in range(n_obj):
        t = np.sort(g.uniform(60000.0, 60180.0, n_t))
        ts.append(t)
        ys.append(0.5 * np.sin(2 * math.pi * f0[o] * t + g.uniform(0, 6.28)) + g.normal(0, 0.03, n_t))
    off = np.arange(n_obj + 1, dtype=np.int64) * n_t
    res = oracle_mod.lsp_batch(np.concatenate(ts), np.concatenate(ys), off,
                               grid.f_min, grid.f_max, grid.n_f, norm=1)
    k_true = (f0 - grid.f_min) / grid.df
    assert np.all(np.abs(res["arg_idx"] - k_true) <= 1.0)


def test_extended_precision_bound(oracle_mod):
    b = synth.single_small()
    g = b.grid
    ks = np.linspace(0, g.n_f - 1, 24).astype(np.int64)
    p, _ = oracle_mod.lsp_single(b.t, b.y, g.f_min, g.f_max, g.n_f, norm=1, k_sel=ks)
    pl = oracle_mod.lsp_single_ld(b.t, b.y, g.f_min, g.f_max, g.n_f, ks, norm=1)
    assert np.max(np.abs(p - pl)) < 1e-12


def _brute_top(p, k):
    n = len(p)
    cand = [i for i in range(n)
            if (i == 0 or p[i] > p[i - 1]) and (i == n - 1 or p[i] >= p[i + 1])]
    cand.sort(key=lambda i: (-p[i], i))
    cand = cand[:k]
    return cand + [-1] * (k - len(cand))


def test_argmax_and_top_k_semantics(oracle_mod):
    cases = [
        [1.0], [1.0, 1.0], [0.0, 2.0], [3.0, 1.0, 3.0], [1, 2, 2, 1, 5, 5, 0],
        [0, 0, 0, 0], [5, 4, 3, 2, 1], [1, 3, 2, 3, 2, 3, 1], [2, 1, 2, 1, 2],
    ]
    g = np.random.default_rng(3)
    cases += [list(g.integers(0, 4, n).astype(float)) for n in range(1, 40)]
    for c in cases:
        p = np.array(c, dtype=np.float64)
        assert oracle_mod.argmax(p) == int(np.argmax(p))  # numpy: first maximum
        idx, pw = oracle_mod.top_local_maxima(p, 3)
        assert list(idx) == _brute_top(list(p), 3), c
        # the first maximum is always a local maximum, and the top one
        assert idx[0] == int(np.argmax(p))


def test_batch_equals_singles_and_flags(oracle_mod):
    b = synth.ragged_survey(6, seed=9, grid=synth.Grid(0.24, 12.0, 500))
    t = b.t.copy()
    y = b.y.copy()
    # plant degenerate objects: empty, one observation, zero variance, NaN
    lens = list(b.n_t[:6])
    segs_t = [t[b.offsets[i]:b.offsets[i + 1]] for i in range(6)]
    segs_y = [y[b.offsets[i]:b.offsets[i + 1]] for i in range(6)]
    segs_t += [np.zeros(0), np.array([60000.0]), np.array([60000.0, 60001.0, 60002.5]), np.array([60000.0, 60003.0])]
    segs_y += [np.zeros(0), np.array([1.0]), np.array([2.0, 2.0, 2.0]), np.array([1.0, np.nan])]
    tt = np.concatenate(segs_t)
    yy = np.concatenate(segs_y)
    off = np.concatenate([[0], np.cumsum([len(s) for s in segs_t])]).astype(np.int64)
    res = oracle_mod.lsp_batch(tt, yy, off, 0.24, 12.0, 500, norm=1, top_k=3, return_power=True)
    for o in range(6):
        p, fl = oracle_mod.lsp_single(segs_t[o], segs_y[o], 0.24, 12.0, 500, norm=1)
        assert fl == 0
        np.testing.assert_array_equal(res["power"][o], p)
        assert res["arg_idx"][o] == int(np.argmax(p))
    assert res["flags"][6] & oracle_mod.FLAG_FEW_OBS
    assert res["flags"][7] & oracle_mod.FLAG_FEW_OBS
    assert res["flags"][8] & oracle_mod.FLAG_ZERO_VAR
    assert res["flags"][9] & oracle_mod.FLAG_NONFINITE
    assert (res["arg_idx"][6:] == -1).all()
    assert (res["power"][6:] == 0).all()


# ---------------------------------------------- generalized periodogram (Section 4.11)
def _wlsq_power(t, y, dy, f):
    """Fraction of the weighted variance explained by a cos + b sin + c (numpy lstsq)."""
    w = 1.0 / dy ** 2
    sw = np.sqrt(w)
    wt = 2 * math.pi * f
    X = np.stack([np.cos(wt * t), np.sin(wt * t), np.ones_like(t)], axis=1)
    beta, *_ = np.linalg.lstsq(X * sw[:, None], y * sw, rcond=None)
    chi2 = np.sum(w * (y - X @ beta) ** 2)
    ybar = np.sum(w * y) / np.sum(w)
    chi0 = np.sum(w * (y - ybar) ** 2)
    return 1.0 - chi2 / chi0


@pytest.mark.parametrize("n_t", [4, 7, 12, 40])
def test_gls_weighted_least_squares(oracle_mod, n_t):
    g = np.random.default_rng(200 + n_t)
    t = np.sort(g.uniform(60000, 60030, n_t))
    y = g.normal(0, 1, n_t)
    dy = g.uniform(0.05, 0.5, n_t)
    res = oracle_mod.gls_batch(t, y, dy, [0, n_t], 0.3, 4.0, 37)
    fk = oracle_mod.grid_freqs(0.3, 4.0, 37)
    ref = np.array([_wlsq_power(t - t[0], y, dy, f) for f in fk])
    np.testing.assert_allclose(res["power"][0], ref, rtol=1e-8, atol=1e-10)
    # the non-normalised form is half the chi-square reduction
    res0 = oracle_mod.gls_batch(t, y, dy, [0, n_t], 0.3, 4.0, 37, norm=0)
    w = 1 / dy ** 2
    chi0 = np.sum(w * (y - np.sum(w * y) / np.sum(w)) ** 2)
    np.testing.assert_allclose(res0["power"][0], 0.5 * chi0 * ref, rtol=1e-8, atol=1e-10)


def test_gls_exact_fit_and_bounds(oracle_mod):
    g = np.random.default_rng(21)
    t = np.sort(g.uniform(60000, 61000, 80))
    k0, f_min, f_max, n_f = 123, 0.1, 5.0, 500
    f0 = oracle_mod.grid_freqs(f_min, f_max, n_f)[k0]
    y = 0.4 * np.cos(2 * math.pi * f0 * t + 1.1) + 3.0
    dy = g.uniform(0.01, 0.3, 80)
    res = oracle_mod.gls_batch(t, y, dy, [0, 80], f_min, f_max, n_f)
    assert abs(res["power"][0, k0] - 1.0) < 1e-9
    yn = y + g.normal(0, 0.2, 80)
    p = oracle_mod.gls_batch(t, yn, dy, [0, 80], f_min, f_max, n_f)["power"][0]
    assert p.min() >= -1e-12 and p.max() <= 1 + 1e-12


def test_gls_unit_weights_fourier_frequencies_equal_fft(oracle_mod):
    # at Fourier frequencies of even sampling, cos/sin are orthogonal to the
    # constant, so the floating mean changes nothing: P = 2 |DFT_m|^2 / (N sum yc^2)
    n, dt = 48, 0.25
    g = np.random.default_rng(22)
    t = 60000.0 + dt * np.arange(n)
    y = g.normal(0, 1, n) + 5.0
    df = 1.0 / (n * dt)
    n_f = n // 2 - 1
    p = oracle_mod.gls_batch(t, y, None, [0, n], df, df * (n_f + 1), n_f)["power"][0]
    yc = y - y.mean()
    ref = 2 * np.abs(np.fft.fft(yc)[1:n_f + 1]) ** 2 / (n * np.dot(yc, yc))
    np.testing.assert_allclose(p, ref, rtol=1e-9, atol=1e-12)


def test_gls_invariances_and_flags(oracle_mod):
    g = np.random.default_rng(23)
    t = np.sort(g.uniform(60000, 60500, 60))
    y = np.sin(2 * math.pi * 1.3 * t) + g.normal(0, 0.3, 60)
    dy = g.uniform(0.1, 0.4, 60)
    args = ([0, 60], 0.2, 6.0, 800)
    base = oracle_mod.gls_batch(t, y, dy, *args)["power"][0]
    for tt, yy, ee in [(t + 777.7, y, dy), (t, -2.0 * y + 9.0, dy), (t, y, 3.0 * dy)]:
        np.testing.assert_allclose(oracle_mod.gls_batch(tt, yy, ee, *args)["power"][0], base, atol=1e-8)
    off = np.array([0, 2, 5, 8], dtype=np.int64)
    tt = np.array([0.0, 1.0, 0.0, 1.0, 2.0, 0.0, 1.0, 2.0]) + 60000
    yy = np.array([1.0, 2.0, 1.0, 1.0, 1.0, 1.0, 2.0, 3.0])
    ee = np.array([1.0, 1.0, 1.0, 1.0, 1.0, 1.0, -1.0, 1.0])
    fl = oracle_mod.gls_batch(tt, yy, ee, off, 0.2, 6.0, 10)["flags"]
    assert fl[0] & oracle_mod.FLAG_FEW_OBS and fl[1] & oracle_mod.FLAG_ZERO_VAR and fl[2] & oracle_mod.FLAG_NONFINITE


def test_fp32_cpu_configuration_tracks_the_oracle(oracle_mod):
    oracle = oracle_mod
    # the FP32 CPU configuration timed beside the oracle computes the same
    # periodogram to FP32 accuracy (it is timing context, not a reference)
    b = synth.ragged_survey(6, seed=77, grid=synth.Grid(0.24, 12.0, 3001))
    ref = oracle.lsp_batch(b.t, b.y, b.offsets, 0.24, 12.0, 3001, return_power=True)
    idx, pw = oracle.fp32_batch_argmax(b.t, b.y, b.offsets, 0.24, 12.0, 3001)
    for o in range(b.n_obj):
        assert abs(float(pw[o]) - ref["arg_pow"][o]) < 5e-3
        assert ref["power"][o][idx[o]] >= ref["arg_pow"][o] - 5e-3
    s = synth.single_small(n_t=300, grid=synth.Grid(0.1, 10.0, 2000))
    ks = np.arange(0, 2000, 7)
    p32 = oracle.fp32_single(s.t, s.y, 0.1, 10.0, 2000, ks)
    p64 = oracle.lsp_single(s.t, s.y, 0.1, 10.0, 2000, k_sel=ks)[0]
    assert np.max(np.abs(p32 - p64)) < 5e-3
