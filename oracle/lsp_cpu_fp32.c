/*
 * lsp_cpu_fp32.c -- the paper's FP32 CPU configuration, for timing context.
 *
 * TEST INFRASTRUCTURE ONLY, and not an oracle: the benchmark's CPU leg times
 * it beside the FP64 oracle, as the paper times its C/OpenMP reference in
 * FP32 and FP64 (Section 4.5, lsp-c).  It restates the same two-scan Eq. 1 /
 * Eq. 2 as lsp_oracle.c in single precision (times shifted by their minimum
 * in FP64, then stored in FP32, as the paper's FP32 mode stores them; the
 * mean is subtracted in FP64), with the same OpenMP schedules: dynamic over
 * objects for batches, static over frequencies for one object.  It shares
 * no code with the CUDA library.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define CPU32_TWO_PI 6.2831853071795864769f

/* Eq. 1 then Eq. 2 at one frequency, FP32, two scans. */
static float power_eq2_f32(const float* ts, const float* x, int64_t n, float f) {
  const float w = CPU32_TWO_PI * f;
  float s2 = 0.0f, c2 = 0.0f;
  for (int64_t j = 0; j < n; ++j) {
    s2 += sinf(2.0f * w * ts[j]);
    c2 += cosf(2.0f * w * ts[j]);
  }
  const float tau = atan2f(s2, c2) / (2.0f * w);
  float xc = 0.0f, xs = 0.0f, cc = 0.0f, ss = 0.0f;
  for (int64_t j = 0; j < n; ++j) {
    const float arg = w * (ts[j] - tau);
    const float c = cosf(arg), s = sinf(arg);
    xc += x[j] * c;
    xs += x[j] * s;
    cc += c * c;
    ss += s * s;
  }
  const float eps = 1e-6f * (float)n;
  float p = 0.0f;
  if (cc > eps) p += xc * xc / cc;
  if (ss > eps) p += xs * xs / ss;
  return 0.5f * p;
}

/* Shifted FP32 times, centred FP32 magnitudes; returns sum x^2 (0: degenerate). */
static float prepare_f32(const double* t, const double* y, int64_t n, float* ts, float* x) {
  if (n < 2) return 0.0f;
  double mean = 0.0, tmin = t[0];
  for (int64_t j = 0; j < n; ++j) {
    mean += y[j];
    if (t[j] < tmin) tmin = t[j];
  }
  mean /= (double)n;
  float s = 0.0f;
  for (int64_t j = 0; j < n; ++j) {
    ts[j] = (float)(t[j] - tmin);
    x[j] = (float)(y[j] - mean);
    s += x[j] * x[j];
  }
  return s;
}

/* Batch: the first maximum of P_n per object (dynamic schedule over objects). */
int cpu32_lsp_batch_argmax(const double* t, const double* y, const int64_t* offsets, int64_t n_obj,
                           double f_min, double f_max, int64_t n_f, int64_t* arg_idx, float* arg_pow) {
  const double df = (f_max - f_min) / (double)n_f;
  int rc = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t o = 0; o < n_obj; ++o) {
    const int64_t b = offsets[o], n = offsets[o + 1] - offsets[o];
    float* ts = (float*)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    float* x = (float*)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    if (!ts || !x) {
      rc = -1;
    } else {
      const float sx2 = prepare_f32(t + b, y + b, n, ts, x);
      int64_t best = -1;
      float bp = 0.0f;
      if (sx2 > 0.0f)
        for (int64_t k = 0; k < n_f; ++k) {
          const float p = 2.0f * power_eq2_f32(ts, x, n, (float)(f_min + (double)k * df)) / sx2;
          if (best < 0 || p > bp) {
            bp = p;
            best = k;
          }
        }
      arg_idx[o] = best;
      arg_pow[o] = bp;
    }
    free(ts);
    free(x);
  }
  return rc;
}

/* One object, P_n at the grid indices k_sel[0..n_sel) (static schedule). */
int cpu32_lsp_single(const double* t, const double* y, int64_t n, double f_min, double f_max, int64_t n_f,
                     const int64_t* k_sel, int64_t n_sel, float* out) {
  float* ts = (float*)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
  float* x = (float*)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
  if (!ts || !x) {
    free(ts);
    free(x);
    return -1;
  }
  const float sx2 = prepare_f32(t, y, n, ts, x);
  const double df = (f_max - f_min) / (double)n_f;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n_sel; ++i)
    out[i] = sx2 > 0.0f ? 2.0f * power_eq2_f32(ts, x, n, (float)(f_min + (double)k_sel[i] * df)) / sx2 : 0.0f;
  free(ts);
  free(x);
  return 0;
}
