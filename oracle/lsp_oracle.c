/*
 * lsp_oracle.c -- FP64 CPU oracle for the Lomb-Scargle periodogram.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * restatement of what the GPU path computes.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or constant with the CUDA library and neither includes
 * nor links the other.
 *
 * What it computes (Gowanlock et al. 2021, arXiv:2105.04006):
 *   - Section 2, Eq. 1: the time offset tau from
 *         tan(2 w tau) = sum_j sin(2 w t_j) / sum_j cos(2 w t_j)
 *   - Section 2, Eq. 2: the (non-normalised) L-S power
 *         P(f) = 1/2 ( [sum_j X_j cos w(t_j - tau)]^2 / sum_j cos^2 w(t_j - tau)
 *                    + [sum_j X_j sin w(t_j - tau)]^2 / sum_j sin^2 w(t_j - tau) )
 *     with w = 2 pi f.  This is the two-scan form that Section 2 describes
 *     (first scan: tau; second scan: the four tau-shifted sums); it is
 *     deliberately NOT the single-scan refactoring the GPU kernels use.
 *   - Section 2: X has zero mean (the data are mean-subtracted first) and the
 *     grid is evenly spaced and half-open, [f_min, f_max), with
 *     df = (f_max - f_min) / N_f and f_k = f_min + k df.
 *   - Section 3.3: the period comes from the index of the first maximum of the
 *     periodogram (thrust::max_element semantics: ties go to the lowest index).
 *   - Section 3.4: batch mode computes one periodogram per object over a
 *     shared grid.
 *   - Section 4.5 (lsp-c): batches are parallelised per object with a dynamic
 *     OpenMP schedule, single objects per frequency with a static schedule.
 *
 * Readings where the paper is silent (each is listed with the others in the
 * design notes):
 *   - Frequencies are in cycles per unit time (cycles/day); w = 2 pi f and the
 *     period is 1/f.  The paper's own grid is angular (Appendix A); the two
 *     differ only by the factor 2 pi.
 *   - Normalisation: norm=0 returns P of Eq. 2; norm=1 returns the standard
 *     normalisation P_n = 2 P / sum_j X_j^2, which lies in [0, 1].
 *   - t is shifted by its minimum before the phases are formed (the power is
 *     invariant under a common time shift; the shift only keeps w t small).
 *   - A denominator of Eq. 2 at or below 1e-12 N_t drops its term (atan2(0,0)
 *     is 0).  An object with fewer than two observations, or whose centred
 *     magnitudes are all zero, gets power 0 and a nonzero flag.
 *   - "Top-k peaks" are the k largest local maxima, where bin k is a local
 *     maximum when P[k] > P[k-1] and P[k] >= P[k+1] (a grid end compares with
 *     its one neighbour only); ordered by power, ties to the lower index.
 *
 * Parity pins (see tests/test_oracle_pins.py): least-squares chi-square
 * reduction on tiny inputs, |DFT|^2/N on evenly sampled data at Fourier
 * frequencies, exact fit of a noiseless sinusoid, invariance to time shift,
 * permutation, sign and scale, P_n in [0, 1], injected-period recovery, and
 * an extended-precision recomputation bounding the oracle's own rounding.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_TWO_PI 6.283185307179586476925286766559

/* Per-object flags, reported next to the peak. */
#define ORACLE_FLAG_FEW_OBS 1   /* fewer than two observations */
#define ORACLE_FLAG_ZERO_VAR 2  /* centred magnitudes all zero */
#define ORACLE_FLAG_NONFINITE 4 /* a NaN or Inf in t or y */

int oracle_version(void) { return 1; }

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Frequency k of the half-open grid of Section 2. */
static double grid_freq(double f_min, double f_max, int64_t n_f, int64_t k) {
  double df = (f_max - f_min) / (double)n_f;
  return f_min + (double)k * df;
}

/*
 * Eq. 1 then Eq. 2 at one frequency f (cycles per unit time), two scans over
 * the data.  ts[j] are the (shifted) times, x[j] the zero-mean magnitudes.
 */
static double lsp_power_eq2(const double* ts, const double* x, int64_t n, double f) {
  double w = ORACLE_TWO_PI * f;

  /* Eq. 1: tan(2 w tau) = sum sin(2 w t) / sum cos(2 w t). */
  double s2 = 0.0, c2 = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    s2 += sin(2.0 * w * ts[j]);
    c2 += cos(2.0 * w * ts[j]);
  }
  double tau = atan2(s2, c2) / (2.0 * w);

  /* Eq. 2: the four tau-shifted sums. */
  double xc = 0.0, xs = 0.0, cc = 0.0, ss = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    double arg = w * (ts[j] - tau);
    double c = cos(arg);
    double s = sin(arg);
    xc += x[j] * c;
    xs += x[j] * s;
    cc += c * c;
    ss += s * s;
  }
  double eps = 1e-12 * (double)n;
  double p = 0.0;
  if (cc > eps) p += xc * xc / cc;
  if (ss > eps) p += xs * xs / ss;
  return 0.5 * p;
}

/*
 * Centre the magnitudes (Section 2 assumes zero mean) and shift the times.
 * Returns the flags and writes sum x^2 of the centred magnitudes.
 */
static int prepare_object(const double* t, const double* y, int64_t n, int center,
                          double* ts, double* x, double* sum_x2) {
  int flags = 0;
  *sum_x2 = 0.0;
  if (n < 2) flags |= ORACLE_FLAG_FEW_OBS;
  for (int64_t j = 0; j < n; ++j)
    if (!isfinite(t[j]) || !isfinite(y[j])) flags |= ORACLE_FLAG_NONFINITE;
  if (n == 0 || (flags & ORACLE_FLAG_NONFINITE)) return flags;

  double mean = 0.0;
  if (center) {
    for (int64_t j = 0; j < n; ++j) mean += y[j];
    mean /= (double)n;
  }
  double tmin = t[0];
  for (int64_t j = 1; j < n; ++j)
    if (t[j] < tmin) tmin = t[j];
  for (int64_t j = 0; j < n; ++j) {
    ts[j] = t[j] - tmin;
    x[j] = y[j] - mean;
    *sum_x2 += x[j] * x[j];
  }
  if (!(*sum_x2 > 0.0)) flags |= ORACLE_FLAG_ZERO_VAR;
  return flags;
}

/* Section 3.3: first maximum (lowest index on ties). */
int64_t oracle_argmax(const double* p, int64_t n) {
  if (n <= 0) return -1;
  int64_t best = 0;
  for (int64_t k = 1; k < n; ++k)
    if (p[k] > p[best]) best = k;
  return best;
}

/*
 * The k_top largest local maxima (reading above), written to idx[]/pw[];
 * missing entries get idx -1 and power 0.  Returns how many were found.
 */
int oracle_top_local_maxima(const double* p, int64_t n, int k_top, int64_t* idx, double* pw) {
  for (int i = 0; i < k_top; ++i) {
    idx[i] = -1;
    pw[i] = 0.0;
  }
  int found = 0;
  for (int64_t k = 0; k < n; ++k) {
    int left_ok = (k == 0) || (p[k] > p[k - 1]);
    int right_ok = (k == n - 1) || (p[k] >= p[k + 1]);
    if (!(left_ok && right_ok)) continue;
    /* insert into the sorted list: higher power first, lower index first */
    int pos = found < k_top ? found : k_top;
    while (pos > 0 && p[k] > pw[pos - 1]) --pos;
    if (pos >= k_top) continue;
    for (int i = (found < k_top ? found : k_top - 1); i > pos; --i) {
      idx[i] = idx[i - 1];
      pw[i] = pw[i - 1];
    }
    idx[pos] = k;
    pw[pos] = p[k];
    if (found < k_top) ++found;
  }
  return found;
}

/*
 * Single object (Section 3.3): power at every frequency of the grid, or, when
 * k_sel is not NULL, only at the n_sel listed frequency indices (out[i] is the
 * power at k_sel[i]).  Parallel over frequencies with a static schedule
 * (Section 4.5).  Returns the object's flags.
 */
int oracle_lsp_single(const double* t, const double* y, int64_t n_t, double f_min,
                      double f_max, int64_t n_f, int norm, int center,
                      const int64_t* k_sel, int64_t n_sel, double* out) {
  int64_t n_out = k_sel ? n_sel : n_f;
  double* ts = (double*)malloc(sizeof(double) * (size_t)(n_t > 0 ? n_t : 1));
  double* x = (double*)malloc(sizeof(double) * (size_t)(n_t > 0 ? n_t : 1));
  double sum_x2 = 0.0;
  int flags = prepare_object(t, y, n_t, center, ts, x, &sum_x2);
  if (flags) {
    for (int64_t i = 0; i < n_out; ++i) out[i] = 0.0;
  } else {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n_out; ++i) {
      int64_t k = k_sel ? k_sel[i] : i;
      double p = lsp_power_eq2(ts, x, n_t, grid_freq(f_min, f_max, n_f, k));
      out[i] = norm ? 2.0 * p / sum_x2 : p;
    }
  }
  free(ts);
  free(x);
  return flags;
}

/*
 * Batch (Section 3.4): objects o = 0..n_obj-1 own t/y[offsets[o] .. offsets[o+1]).
 * Per object it writes the argmax index and power (Section 3.3 semantics),
 * the top_k (<= 3) local maxima, the flags, and -- when power is not NULL --
 * the whole periodogram at power[o * n_f ...].  Parallel over objects with a
 * dynamic schedule (Section 4.5).
 */
int oracle_lsp_batch(const double* t, const double* y, const int64_t* offsets, int64_t n_obj,
                     double f_min, double f_max, int64_t n_f, int norm, int center, int top_k,
                     double* power, int64_t* arg_idx, double* arg_pow, int64_t* top_idx,
                     double* top_pow, int32_t* flags_out) {
  if (top_k < 1) top_k = 1;
  if (top_k > 3) top_k = 3;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t o = 0; o < n_obj; ++o) {
    int64_t b = offsets[o], n = offsets[o + 1] - offsets[o];
    double* pg = power ? power + o * n_f : (double*)malloc(sizeof(double) * (size_t)n_f);
    double* ts = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* x = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double sum_x2 = 0.0;
    int fl = prepare_object(t + b, y + b, n, center, ts, x, &sum_x2);
    for (int64_t k = 0; k < n_f; ++k) {
      if (fl) {
        pg[k] = 0.0;
        continue;
      }
      double p = lsp_power_eq2(ts, x, n, grid_freq(f_min, f_max, n_f, k));
      pg[k] = norm ? 2.0 * p / sum_x2 : p;
    }
    if (fl) {
      arg_idx[o] = -1;
      arg_pow[o] = 0.0;
      for (int i = 0; i < top_k; ++i) {
        if (top_idx) top_idx[o * top_k + i] = -1;
        if (top_pow) top_pow[o * top_k + i] = 0.0;
      }
    } else {
      arg_idx[o] = oracle_argmax(pg, n_f);
      arg_pow[o] = pg[arg_idx[o]];
      if (top_idx && top_pow)
        oracle_top_local_maxima(pg, n_f, top_k, top_idx + o * top_k, top_pow + o * top_k);
    }
    if (flags_out) flags_out[o] = fl;
    free(ts);
    free(x);
    if (!power) free(pg);
  }
  return 0;
}

/*
 * The same Eq. 1 / Eq. 2 evaluation carried out in long double (80-bit on
 * x86-64, binary128 on AArch64), for a handful of frequencies.  It exists only
 * to bound the FP64 oracle's own rounding error in the tests.
 */
int oracle_lsp_single_ld(const double* t, const double* y, int64_t n_t, double f_min,
                         double f_max, int64_t n_f, int norm, const int64_t* k_sel,
                         int64_t n_sel, double* out) {
  if (n_t < 2) return ORACLE_FLAG_FEW_OBS;
  long double mean = 0.0L, tmin = t[0];
  for (int64_t j = 0; j < n_t; ++j) {
    mean += y[j];
    if (t[j] < tmin) tmin = t[j];
  }
  mean /= (long double)n_t;
  long double sum_x2 = 0.0L;
  for (int64_t j = 0; j < n_t; ++j) sum_x2 += ((long double)y[j] - mean) * ((long double)y[j] - mean);
  const long double two_pi = 6.283185307179586476925286766559005768L;
  for (int64_t i = 0; i < n_sel; ++i) {
    long double df = ((long double)f_max - (long double)f_min) / (long double)n_f;
    long double w = two_pi * ((long double)f_min + (long double)k_sel[i] * df);
    long double s2 = 0.0L, c2 = 0.0L;
    for (int64_t j = 0; j < n_t; ++j) {
      long double a = 2.0L * w * ((long double)t[j] - tmin);
      s2 += sinl(a);
      c2 += cosl(a);
    }
    long double tau = atan2l(s2, c2) / (2.0L * w);
    long double xc = 0, xs = 0, cc = 0, ss = 0;
    for (int64_t j = 0; j < n_t; ++j) {
      long double a = w * ((long double)t[j] - tmin - tau);
      long double c = cosl(a), s = sinl(a), xv = (long double)y[j] - mean;
      xc += xv * c;
      xs += xv * s;
      cc += c * c;
      ss += s * s;
    }
    long double p = 0.5L * (xc * xc / cc + xs * xs / ss);
    out[i] = (double)(norm ? 2.0L * p / sum_x2 : p);
  }
  return 0;
}

/*
 * Generalized L-S periodogram (Section 4.11: photometric errors and a
 * floating mean).  The paper gives no formula; its plain definition is used:
 * at each frequency the weighted least-squares fit of
 *     y(t) ~ a cos(w t) + b sin(w t) + c,   weights 1 / dy^2,
 * and the power
 *     P = 1 - chi2_min(w) / chi2_0,   chi2_0 = sum_j w_j (y_j - ybar_w)^2,
 * the fraction of the weighted variance the sinusoid explains (in [0, 1]).
 * norm = 0 returns (chi2_0 - chi2_min) / 2 instead, the generalized
 * counterpart of Eq. 2's P.  The 3x3 normal equations are solved by Gaussian
 * elimination with partial pivoting in FP64.  dy NULL means unit weights.
 * Objects with fewer than three observations, zero weighted variance or a
 * non-positive / non-finite error get power 0 and a flag.
 */
static double gls_power(const double* ts, const double* y, const double* w, int64_t n, double f,
                        double chi2_0, int norm) {
  double wv = ORACLE_TWO_PI * f;
  double m[3][4] = {{0}};
  double syy = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    double phi[3] = {cos(wv * ts[j]), sin(wv * ts[j]), 1.0};
    for (int r = 0; r < 3; ++r) {
      for (int c = 0; c < 3; ++c) m[r][c] += w[j] * phi[r] * phi[c];
      m[r][3] += w[j] * phi[r] * y[j];
    }
    syy += w[j] * y[j] * y[j];
  }
  double rhs[3] = {m[0][3], m[1][3], m[2][3]};
  for (int col = 0; col < 3; ++col) {
    int piv = col;
    for (int r = col + 1; r < 3; ++r)
      if (fabs(m[r][col]) > fabs(m[piv][col])) piv = r;
    if (fabs(m[piv][col]) <= 1e-300) return 0.0;
    if (piv != col)
      for (int c = 0; c < 4; ++c) {
        double tmp = m[col][c];
        m[col][c] = m[piv][c];
        m[piv][c] = tmp;
      }
    for (int r = col + 1; r < 3; ++r) {
      double fct = m[r][col] / m[col][col];
      for (int c = col; c < 4; ++c) m[r][c] -= fct * m[col][c];
    }
  }
  double beta[3];
  for (int r = 2; r >= 0; --r) {
    double acc = m[r][3];
    for (int c = r + 1; c < 3; ++c) acc -= m[r][c] * beta[c];
    beta[r] = acc / m[r][r];
  }
  double chi2_min = syy;
  for (int r = 0; r < 3; ++r) chi2_min -= beta[r] * rhs[r];
  double red = chi2_0 - chi2_min;
  return norm ? red / chi2_0 : 0.5 * red;
}

static int prepare_gls(const double* t, const double* y, const double* dy, int64_t n, double* ts,
                       double* w, double* chi2_0) {
  int flags = 0;
  *chi2_0 = 0.0;
  if (n < 3) flags |= ORACLE_FLAG_FEW_OBS;
  for (int64_t j = 0; j < n; ++j) {
    double e = dy ? dy[j] : 1.0;
    if (!isfinite(t[j]) || !isfinite(y[j]) || !isfinite(e) || !(e > 0.0)) flags |= ORACLE_FLAG_NONFINITE;
  }
  if (n == 0 || (flags & ORACLE_FLAG_NONFINITE)) return flags;
  double tmin = t[0], sw = 0.0, swy = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    if (t[j] < tmin) tmin = t[j];
    double e = dy ? dy[j] : 1.0;
    w[j] = 1.0 / (e * e);
    sw += w[j];
    swy += w[j] * y[j];
  }
  double ybar = swy / sw;
  for (int64_t j = 0; j < n; ++j) {
    ts[j] = t[j] - tmin;
    *chi2_0 += w[j] * (y[j] - ybar) * (y[j] - ybar);
  }
  if (!(*chi2_0 > 0.0)) flags |= ORACLE_FLAG_ZERO_VAR;
  return flags;
}

int oracle_gls_batch(const double* t, const double* y, const double* dy, const int64_t* offsets,
                     int64_t n_obj, double f_min, double f_max, int64_t n_f, int norm, double* power,
                     int64_t* arg_idx, double* arg_pow, int32_t* flags_out) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t o = 0; o < n_obj; ++o) {
    int64_t b = offsets[o], n = offsets[o + 1] - offsets[o];
    double* pg = power ? power + o * n_f : (double*)malloc(sizeof(double) * (size_t)n_f);
    double* ts = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* w = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double chi2_0 = 0.0;
    int fl = prepare_gls(t + b, y + b, dy ? dy + b : NULL, n, ts, w, &chi2_0);
    for (int64_t k = 0; k < n_f; ++k)
      pg[k] = fl ? 0.0 : gls_power(ts, y + b, w, n, grid_freq(f_min, f_max, n_f, k), chi2_0, norm);
    arg_idx[o] = fl ? -1 : oracle_argmax(pg, n_f);
    arg_pow[o] = fl ? 0.0 : pg[arg_idx[o]];
    if (flags_out) flags_out[o] = fl;
    free(ts);
    free(w);
    if (!power) free(pg);
  }
  return 0;
}
