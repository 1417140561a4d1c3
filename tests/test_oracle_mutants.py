"""The oracle's pins must catch plausible mistakes.

Each mutant below is a one-line edit of a copy of ``oracle/lsp_oracle.c``
(a dropped term, a wrong sign, a wrong factor, a swapped operand, a wrong
grid, a missing centring, a last-maximum argmax).  The copy is compiled on
the CPU into a temporary directory and the independent checks of
``test_oracle_pins`` -- least squares, FFT, exact fit, bounds, argmax -- are
run against it; every mutant must fail at least one of them.
"""
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lsp_oracle.c")

MUTANTS = {
    "drop_sin_term": ("if (ss > eps) p += xs * xs / ss;", ""),
    "tau_sign": ("double tau = atan2(s2, c2) / (2.0 * w);", "double tau = -atan2(s2, c2) / (2.0 * w);"),
    "tau_swapped_args": ("double tau = atan2(s2, c2) / (2.0 * w);", "double tau = atan2(c2, s2) / (2.0 * w);"),
    "tau_missing_two": ("double tau = atan2(s2, c2) / (2.0 * w);", "double tau = atan2(s2, c2) / w;"),
    "eq1_single_angle": ("s2 += sin(2.0 * w * ts[j]);", "s2 += sin(w * ts[j]);"),
    "missing_half": ("return 0.5 * p;", "return p;"),
    "norm_factor": ("out[i] = norm ? 2.0 * p / sum_x2 : p;", "out[i] = norm ? p / sum_x2 : p;"),
    "closed_grid": ("double df = (f_max - f_min) / (double)n_f;", "double df = (f_max - f_min) / (double)(n_f - 1);"),
    "no_centring": ("mean /= (double)n;", "mean = 0.0;"),
    "last_maximum": ("if (p[k] > p[best]) best = k;", "if (p[k] >= p[best]) best = k;"),
    "cos_sin_swapped": ("xc += x[j] * c;", "xc += x[j] * s;"),
}

# mutants of the generalized periodogram and the check that must catch them
GLS_MUTANTS = {
    "gls_no_offset_column": ("double phi[3] = {cos(wv * ts[j]), sin(wv * ts[j]), 1.0};",
                             "double phi[3] = {cos(wv * ts[j]), sin(wv * ts[j]), 0.0};"),
    "gls_weight_not_squared": ("w[j] = 1.0 / (e * e);", "w[j] = 1.0 / e;"),
    "gls_unweighted_mean": ("double ybar = swy / sw;", "double ybar = swy / (double)n;"),
    "gls_wrong_normalisation": ("return norm ? red / chi2_0 : 0.5 * red;", "return norm ? red / syy : 0.5 * red;"),
}


def _compile(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique/absent"
    path = os.path.join(tmp_path, f"{name}.c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    so = os.path.join(tmp_path, f"{name}.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", path, "-o", so, "-lm"], check=True)
    lib = ctypes.CDLL(so)
    P, d, i64, i32 = ctypes.c_void_p, ctypes.c_double, ctypes.c_int64, ctypes.c_int
    lib.oracle_lsp_single.argtypes = [P, P, i64, d, d, i64, i32, i32, P, i64, P]
    lib.oracle_lsp_single.restype = i32
    lib.oracle_argmax.argtypes = [P, i64]
    lib.oracle_argmax.restype = i64
    return lib


def _single(lib, t, y, f_min, f_max, n_f, norm, center=True):
    t = np.ascontiguousarray(t, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    out = np.empty(n_f)
    lib.oracle_lsp_single(t.ctypes.data, y.ctypes.data, t.size, f_min, f_max, n_f, norm, int(center),
                          None, 0, out.ctypes.data)
    return out


def _pins_hold(lib) -> bool:
    """True if every independent check passes for this library."""
    g = np.random.default_rng(5)
    ok = True
    # least squares on tiny inputs
    for n_t in (4, 9):
        t = np.sort(g.uniform(60000, 60030, n_t))
        y = g.normal(0, 1, n_t)
        yc = y - y.mean()
        p = _single(lib, t, y, 0.3, 4.0, 37, 0)
        fk = 0.3 + np.arange(37) * (3.7 / 37)
        for k in (0, 5, 17, 36):
            w = 2 * math.pi * fk[k]
            X = np.stack([np.cos(w * (t - t[0])), np.sin(w * (t - t[0]))], axis=1)
            beta, *_ = np.linalg.lstsq(X, yc, rcond=None)
            r = yc - X @ beta
            ok &= abs(p[k] - 0.5 * (yc @ yc - r @ r)) <= 1e-9 * max(1.0, abs(p[k]))
    # FFT at Fourier frequencies
    n, dt = 32, 0.5
    t = 60000.0 + dt * np.arange(n)
    y = g.normal(0, 1, n)
    df = 1.0 / (n * dt)
    p = _single(lib, t, y, df, df * (n // 2), n // 2 - 1, 0)
    ref = np.abs(np.fft.fft(y - y.mean())[1:n // 2]) ** 2 / n
    ok &= np.allclose(p, ref, rtol=1e-9, atol=1e-12)
    # exact fit -> normalised power 1
    t = np.sort(g.uniform(60000, 61000, 100))
    f0 = 0.1 + 437 * (9.9 / 1000)
    y = 0.7 * np.cos(2 * math.pi * f0 * (t - 60000) + 0.4)
    p = _single(lib, t, y, 0.1, 10.0, 1000, 1, center=False)
    ok &= abs(p[437] - 1.0) < 1e-9
    # first maximum
    arr = np.array([1.0, 3.0, 2.0, 3.0])
    ok &= lib.oracle_argmax(arr.ctypes.data, 4) == 1
    return bool(ok)


def test_unmutated_copy_passes(tmp_path):
    lib = _compile(str(tmp_path), "identity", "int oracle_version(void) { return 1; }",
                   "int oracle_version(void) { return 1; }")
    assert _pins_hold(lib)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    lib = _compile(str(tmp_path), name, old, new)
    assert not _pins_hold(lib), f"mutant {name} survived the pins"


def _gls_holds(lib) -> bool:
    P, d, i64, i32 = ctypes.c_void_p, ctypes.c_double, ctypes.c_int64, ctypes.c_int
    lib.oracle_gls_batch.argtypes = [P, P, P, P, i64, d, d, i64, i32, P, P, P, P]
    g = np.random.default_rng(8)
    ok = True
    for n in (6, 15):
        t = np.sort(g.uniform(60000, 60030, n))
        y = g.normal(0, 1, n) + 2.0
        dy = g.uniform(0.05, 0.5, n)
        off = np.array([0, n], dtype=np.int64)
        out = np.empty(20)
        ai, ap, fl = np.empty(1, np.int64), np.empty(1), np.empty(1, np.int32)
        lib.oracle_gls_batch(t.ctypes.data, y.ctypes.data, dy.ctypes.data, off.ctypes.data, 1, 0.3, 4.0, 20, 1,
                             out.ctypes.data, ai.ctypes.data, ap.ctypes.data, fl.ctypes.data)
        fk = 0.3 + np.arange(20) * (3.7 / 20)
        w = 1 / dy ** 2
        for k in (0, 7, 19):
            wt = 2 * math.pi * fk[k]
            X = np.stack([np.cos(wt * (t - t[0])), np.sin(wt * (t - t[0])), np.ones(n)], axis=1)
            beta, *_ = np.linalg.lstsq(X * np.sqrt(w)[:, None], y * np.sqrt(w), rcond=None)
            chi2 = np.sum(w * (y - X @ beta) ** 2)
            chi0 = np.sum(w * (y - np.sum(w * y) / np.sum(w)) ** 2)
            ok &= abs(out[k] - (1 - chi2 / chi0)) <= 1e-8
    return bool(ok)


def test_gls_unmutated_passes(tmp_path):
    lib = _compile(str(tmp_path), "gls_identity", "int oracle_version(void) { return 1; }",
                   "int oracle_version(void) { return 1; }")
    assert _gls_holds(lib)


@pytest.mark.parametrize("name", sorted(GLS_MUTANTS))
def test_gls_mutant_is_caught(tmp_path, name):
    old, new = GLS_MUTANTS[name]
    lib = _compile(str(tmp_path), name, old, new)
    assert not _gls_holds(lib), f"mutant {name} survived the pins"
