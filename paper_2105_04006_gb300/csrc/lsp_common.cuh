// lsp_common.cuh -- data layout and device helpers shared by the kernels of
// the GB300 Lomb-Scargle library (internal; not part of the C ABI).
//
// HBM layout of one call's workspace (all sections 256-byte aligned):
//   ObjInfo  obj[n_obj]                 per-object statistics (prologue)
//   Rec      rec[total_nt]              per-observation records (prologue)
//   int32    order[n_obj]               objects by decreasing N_t (LPT queue)
//   uint32   hist[LSP_HIST_BINS + 1]    counting-sort scratch
//   uint32   queue[4]                   persistent-kernel work counter
//   ChunkBest best[n_obj * n_chunks]    first maximum of each frequency chunk
//   ChunkCand cand[n_obj * n_chunks]    top-3 local maxima + edge bins (top_k > 1)
//   partial  part[split * n_f]          split-N_t partial sums (single object)
#pragma once

#include <type_traits>

#include <cstdint>
#include <cuda_runtime.h>

#define LSP_HIST_BINS 4096
#define LSP_TILE_OBS 256

namespace lsp {

// Per-object statistics written by the prologue (Section 2: zero-mean y).
struct __align__(16) ObjInfo {
  double t0;         // midpoint of the object's time span; phases use t - t0
  double ymean;      // FP64 mean of y (0 when centring is off)
  double sum_y2;     // FP64 sum of the centred y^2
  int64_t begin;     // offsets[o]
  int32_t n;         // N_t (0 for an object with bad offsets)
  int32_t flags;     // LSP_FLAG_*
  double norm_scale; // 2 / sum_y2 (standard normalisation) or 1 (PSD); generalized: 1 or sum_y2 / 2
  float norm_scale_f; // the same, rounded to FP32 (the FP32 kernels never touch FP64)
  float wsum_f;       // generalized periodogram: sum of the weights 1/dy^2 (FP32)
  double wsum;        // the same in FP64
};

// Generalized periodogram (Section 4.11): the records hold u = w (y - ybar_w)
// in the y slot and the weight w = 1/dy^2 in the spare word (pad / pad bits),
// with ybar_w the weighted mean; ObjInfo.sum_y2 is then sum w (y - ybar_w)^2.

// FP32 path record, 32 bytes.  Phase of frequency k at this observation, in
// cycles, is frac(a + k b) with a = f_min (t - t0) and b = df (t - t0), both
// held as 64-bit fixed point (2^64 = one cycle).  (cr, sr) rotate the phase
// by one grid step: cos/sin(2 pi df (t - t0)).
struct __align__(16) RecF32 {
  float y;   // centred magnitude
  float cr;  // cos(2 pi b)
  float sr;  // sin(2 pi b)
  uint32_t a_hi;
  uint32_t b_hi;
  uint32_t b_lo;
  uint32_t a_lo;
  uint32_t pad;
};

// FP64 path record, 48 bytes.
struct __align__(16) RecF64 {
  double y;
  double cr;
  double sr;
  uint64_t a;
  uint64_t b;
  uint64_t pad;
};

// First maximum of one frequency chunk (lowest index on ties).
struct __align__(16) ChunkBest {
  double p;
  int64_t k;  // -1: empty chunk
};

// Top-3 interior local maxima of a chunk plus its edge bins, from which the
// finalize kernel resolves maxima that straddle chunk boundaries.
struct __align__(16) ChunkCand {
  double p[3];
  int64_t k[3];      // -1: none
  double first[2];   // powers of the chunk's first two bins
  double last[2];    // powers of the last bin and the one before it
  int64_t k_first;   // index of the first bin
  int32_t nvalid;    // bins of the chunk inside the grid
  int32_t pad;
};

// Main-kernel parameters.
template <typename Rec, typename Real>
struct MainParams {
  const Rec* rec;
  const ObjInfo* obj;
  const int32_t* order;  // LPT object order (nullptr: identity)
  Real* power_out;       // nullable, n_obj x n_f
  Real* part;            // split partials (4 per frequency), nullable
  ChunkBest* best;
  ChunkCand* cand;       // nullable: only with top_k > 1
  uint32_t* queue;
  int64_t n_f;
  int32_t n_chunks;      // frequency chunks per object
  int32_t split;         // observation splits per chunk (1 = fused epilogue)
  int64_t n_items;       // n_obj * n_chunks * split
  // Optional: the number of items read from device memory at kernel start
  // (work lists built on the device), and per-object window origins (the
  // learned stage's refinement windows: one chunk per listed object, bins
  // [win_start[o], win_start[o] + win_len) of the grid).
  const uint32_t* n_items_dev;
  const int32_t* win_start;
  int32_t win_len;
};

// ---------------------------------------------------------------- f32x2 ops
// Packed FP32 pairs (two reseed chains side by side).  Each instruction does
// two FP32 operations, halving the issue slots of the hot loop.
typedef unsigned long long f2_t;

__device__ __forceinline__ f2_t f2_pack(float lo, float hi) {
  f2_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2_unpack(f2_t v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c) {
  f2_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f2_t f2_mul(f2_t a, f2_t b) {
  f2_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// ------------------------------------------------------------ phase seeds
// High 32 bits of (a + k b) mod 2^64 from a_hi, b_hi, b_lo: the fraction of
// a cycle as a 32-bit fixed-point number (the carry out of the low word is
// dropped: error <= 2^-32 cycle).
__device__ __forceinline__ uint32_t phase_hi32(uint32_t a_hi, uint32_t b_hi, uint32_t b_lo,
                                               uint32_t k) {
  return a_hi + k * b_hi + __umulhi(k, b_lo);
}

// (cos, sin) of a 32-bit fixed-point phase, on the SFU.  The phase is read as
// a signed fraction in [-1/2, 1/2) cycle so the hardware sine sees an
// argument in [-pi, pi), where its absolute error is about 2^-21.4.
__device__ __forceinline__ void seed_sincos_f32(uint32_t ph, float& c, float& s) {
  const float scale = 6.28318530717958647692f * 2.3283064365386963e-10f;  // 2 pi / 2^32
  float x = __int2float_rn((int)ph) * scale;
  __sincosf(x, &s, &c);
}

// (cos, sin) of a 64-bit fixed-point phase (2^64 = one cycle) in FP64,
// without a library call.  The phase's top 8 bits pick e^{2 pi i j / 256}
// from a table (correctly rounded, lsp_twiddles.inc); the remaining 56 bits
// are an angle x < 2 pi / 256 = 0.0245 rad whose cosine and sine come from
// their Taylor series, 1 - x^2/2 + x^4/24 - x^6/720 and x - x^3/6 + x^5/120 -
// x^7/5040 (the first omitted terms, x^8/8! and x^9/9!, are below 4e-18);
// the two are combined by the angle-addition formulas.  About a dozen FP64
// operations against a library sincos's few dozen, at an error of a few
// 1e-16 (checked against sincospi by lsp_probe_sincos_fixed64).
__device__ const double2 kTwiddle256[256] = {
#include "lsp_twiddles.inc"
};

__device__ __forceinline__ void sincos_fixed64(uint64_t ph, double& c, double& s) {
  const double2 t = __ldg(&kTwiddle256[ph >> 56]);
  const double x = (double)(ph & 0x00FFFFFFFFFFFFFFull) * 3.4061215800865545e-19;  // 2 pi / 2^64
  const double x2 = x * x;
  const double cx = fma(x2, fma(x2, fma(x2, -1.0 / 720.0, 1.0 / 24.0), -0.5), 1.0);
  const double sx = fma(x * x2, fma(x2, fma(x2, -1.0 / 5040.0, 1.0 / 120.0), -1.0 / 6.0), x);
  c = fma(t.x, cx, -(t.y * sx));
  s = fma(t.y, cx, t.x * sx);
}

// (cos, sin) of a 64-bit fixed-point phase in FP64.
__device__ __forceinline__ void seed_sincos_f64(uint64_t ph, double& c, double& s) { sincos_fixed64(ph, c, s); }

// --------------------------------------------------------- power (Eq. 1-2)
// Eq. 2 evaluated from single-scan sums (the refactoring of Section 2):
//   Z = XC + i XS = sum y e^{i phi},  W = (2 CC - N) + i 2 CS = sum e^{2 i phi}.
// With R = |W|, Eq. 1's tau satisfies e^{2 i w tau} = W / R, the tau-shifted
// denominators are (N + R)/2 and (N - R)/2, and with Q = Re(Z^2 conj(W)) / R
// the tau-shifted numerators are (|Z|^2 + Q)/2 and (|Z|^2 - Q)/2, so
//   P = 1/2 [ (|Z|^2 + Q) / (N + R) + (|Z|^2 - Q) / (N - R) ].
// A term whose denominator (N +- R)/2 is at or below eps_rel * N is dropped
// (the Eq. 2 sum vanishes there); atan2(0, 0) = 0 corresponds to Q = 0.
template <typename Real>
__device__ __forceinline__ Real lsp_power(Real xc, Real xs, Real cc, Real cs, Real n,
                                          Real eps_rel) {
  Real c2 = Real(2) * cc - n;
  Real s2 = Real(2) * cs;
  Real r = sqrt(c2 * c2 + s2 * s2);
  Real z2 = xc * xc + xs * xs;
  Real q = r > Real(0) ? ((xc * xc - xs * xs) * c2 + Real(2) * xc * xs * s2) / r : Real(0);
  Real eps = eps_rel * n;
  Real p = Real(0);
  Real d1 = n + r, d2 = n - r;
  Real n1 = z2 + q, n2 = z2 - q;
  if (Real(0.5) * d1 > eps) p += (n1 > Real(0) ? n1 : Real(0)) / d1;
  if (Real(0.5) * d2 > eps) p += (n2 > Real(0) ? n2 : Real(0)) / d2;
  return Real(0.5) * p;
}

// The FP32 sums determine Eq. 2's smaller denominator, (N - R)/2, only to
// about 1e-6 N absolute (phase and rounding errors of N unit terms), so the
// power's relative error grows like 1e-6 N / (N - R).  Where (N - R) falls
// below this fraction of N (all doubled phases nearly aligned, e.g. a daily
// alias of a narrow nightly window, or N_t of 2-3), the FP32 kernels
// re-evaluate the bin in FP64 (exact_power_warp).
constexpr float kIllConditioned = 0.05f;

__device__ __forceinline__ bool ill_conditioned_f32(float cc, float cs, float n) {
  const float c2 = 2.0f * cc - n, s2 = 2.0f * cs;
  const float r = sqrtf(c2 * c2 + s2 * s2);
  return n - r < kIllConditioned * n;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Power at frequency k from FP64 sums over the object's records, evaluated by
// the whole warp (lanes stride the observations).  Phases are exact:
// frac(a + k b) from the 64-bit fixed-point record words.  Every lane returns
// the same value.  Must be called by all 32 lanes.
static __device__ __noinline__ double exact_power_warp(const RecF32* __restrict__ rec, int64_t begin, int n,
                                                uint32_t k, double norm_scale);

template <typename Real> struct EpsRel;
template <> struct EpsRel<float> { static constexpr float v = 1e-6f; };
template <> struct EpsRel<double> { static constexpr double v = 1e-12; };

static __device__ __noinline__ double exact_power_warp(const RecF32* __restrict__ rec, int64_t begin, int n,
                                                uint32_t k, double norm_scale) {
  double xc = 0.0, xs = 0.0, cc = 0.0, cs = 0.0;
  for (int j = threadIdx.x & 31; j < n; j += 32) {
    const RecF32 r = rec[begin + j];
    const uint64_t a = ((uint64_t)r.a_hi << 32) | r.a_lo;
    const uint64_t b = ((uint64_t)r.b_hi << 32) | r.b_lo;
    double c, s;
    seed_sincos_f64(a + (uint64_t)k * b, c, s);
    const double y = (double)r.y;
    xc = fma(y, c, xc);
    xs = fma(y, s, xs);
    cc = fma(c, c, cc);
    cs = fma(c, s, cs);
  }
  xc = warp_sum_d(xc);
  xs = warp_sum_d(xs);
  cc = warp_sum_d(cc);
  cs = warp_sum_d(cs);
  return norm_scale * lsp_power<double>(xc, xs, cc, cs, (double)n, EpsRel<double>::v);
}

// The same power evaluated by one lane alone, over the observations in
// order: for objects of at most kLaneExactMaxObs observations a warp per bin
// would leave most lanes idle and spend more on its FP64 shuffles than on
// the sums, so the lanes re-evaluate their own bins side by side instead.
constexpr int kLaneExactMaxObs = 64;
static __device__ __noinline__ double exact_power_lane(const RecF32* __restrict__ rec, int64_t begin, int n,
                                                       uint32_t k, double norm_scale) {
  double xc = 0.0, xs = 0.0, cc = 0.0, cs = 0.0;
  for (int j = 0; j < n; ++j) {
    const RecF32 r = rec[begin + j];
    const uint64_t a = ((uint64_t)r.a_hi << 32) | r.a_lo;
    const uint64_t b = ((uint64_t)r.b_hi << 32) | r.b_lo;
    double c, s;
    seed_sincos_f64(a + (uint64_t)k * b, c, s);
    const double y = (double)r.y;
    xc = fma(y, c, xc);
    xs = fma(y, s, xs);
    cc = fma(c, c, cc);
    cs = fma(c, s, cs);
  }
  return norm_scale * lsp_power<double>(xc, xs, cc, cs, (double)n, EpsRel<double>::v);
}

// ---------------------------------------- generalized periodogram (Section 4.11)
// Power of the weighted fit y ~ a cos + b sin + c from the six weighted sums
// (y centred on its weighted mean, u = w y'):  YC = sum u c, YS = sum u s,
// C = sum w c, S = sum w s, CCw = sum w c^2, CSw = sum w c s; W = sum w and
// YY = sum w y'^2 per object.  Eliminating the offset c,
//   CC = CCw - C^2/W,  SS = (W - CCw) - S^2/W,  CS = CSw - C S / W,
//   D = CC SS - CS^2,  P = (SS YC^2 + CC YS^2 - 2 CS YC YS) / (YY D),
// the fraction of the weighted variance the sinusoid explains.  `ill`
// reports a Gram determinant D below 0.8 % of its largest value W^2/4
// (D < 0.002 W^2): an FP32 emulation of these sums, each cos/sin off by up
// to 2e-6 and accumulated in FP32, keeps |P_n - P_n(FP64)| below 6e-5 down to
// D = 3e-4 W^2 on short light curves with weights spanning 225x, so only
// the bins below the threshold are re-evaluated in FP64.
template <typename Real>
__device__ __forceinline__ Real gls_power(Real yc, Real ys, Real c, Real s, Real ccw, Real csw, Real w,
                                          Real yy, Real eps_rel, bool& ill) {
  const Real iw = Real(1) / w;
  const Real cc = ccw - c * c * iw;
  const Real ss = (w - ccw) - s * s * iw;
  const Real cs = csw - c * s * iw;
  const Real d = cc * ss - cs * cs;
  ill = d < Real(0.002) * w * w;
  if (!(d > eps_rel * w * w) || !(yy > Real(0))) return Real(0);
  const Real num = ss * yc * yc + cc * ys * ys - Real(2) * cs * yc * ys;
  if constexpr (std::is_same<Real, float>::value)  // the SFU's fast division (relative error ~1e-7)
    return __fdividef(num > 0.0f ? num : 0.0f, yy * d);
  else
    return (num > Real(0) ? num : Real(0)) / (yy * d);
}

// FP64 re-evaluation of a generalized bin by the whole warp (exact phases).
static __device__ __noinline__ double exact_gls_power_warp(const RecF32* __restrict__ rec, int64_t begin,
                                                           int n, uint32_t k, double wsum, double yy,
                                                           double norm_scale) {
  double xc = 0.0, xs = 0.0, c1 = 0.0, s1 = 0.0, cc = 0.0, cs = 0.0;
  for (int j = threadIdx.x & 31; j < n; j += 32) {
    const RecF32 r = rec[begin + j];
    const uint64_t a = ((uint64_t)r.a_hi << 32) | r.a_lo;
    const uint64_t b = ((uint64_t)r.b_hi << 32) | r.b_lo;
    double c, s;
    seed_sincos_f64(a + (uint64_t)k * b, c, s);
    const double u = (double)r.y, w = (double)__uint_as_float(r.pad);
    xc = fma(u, c, xc);
    xs = fma(u, s, xs);
    c1 = fma(w, c, c1);
    s1 = fma(w, s, s1);
    cc = fma(w * c, c, cc);
    cs = fma(w * c, s, cs);
  }
  xc = warp_sum_d(xc);
  xs = warp_sum_d(xs);
  c1 = warp_sum_d(c1);
  s1 = warp_sum_d(s1);
  cc = warp_sum_d(cc);
  cs = warp_sum_d(cs);
  bool ill;
  return norm_scale * gls_power<double>(xc, xs, c1, s1, cc, cs, wsum, yy, EpsRel<double>::v, ill);
}

// exact_gls_power_warp by one lane alone (see exact_power_lane).
static __device__ __noinline__ double exact_gls_power_lane(const RecF32* __restrict__ rec, int64_t begin, int n,
                                                           uint32_t k, double wsum, double yy, double norm_scale) {
  double xc = 0.0, xs = 0.0, c1 = 0.0, s1 = 0.0, cc = 0.0, cs = 0.0;
  for (int j = 0; j < n; ++j) {
    const RecF32 r = rec[begin + j];
    const uint64_t a = ((uint64_t)r.a_hi << 32) | r.a_lo;
    const uint64_t b = ((uint64_t)r.b_hi << 32) | r.b_lo;
    double c, s;
    seed_sincos_f64(a + (uint64_t)k * b, c, s);
    const double u = (double)r.y, w = (double)__uint_as_float(r.pad);
    xc = fma(u, c, xc);
    xs = fma(u, s, xs);
    c1 = fma(w, c, c1);
    s1 = fma(w, s, s1);
    cc = fma(w * c, c, cc);
    cs = fma(w * c, s, cs);
  }
  bool ill;
  return norm_scale * gls_power<double>(xc, xs, c1, s1, cc, cs, wsum, yy, EpsRel<double>::v, ill);
}

template <int F>
__device__ __forceinline__ void fix_ill_conditioned_gls(float (&pv)[F], uint32_t bad, uint32_t k0,
                                                        const RecF32* __restrict__ rec, const ObjInfo& oi) {
  if (!__any_sync(0xffffffffu, bad != 0u)) return;
  if (oi.n <= kLaneExactMaxObs) {
    // a short object: each lane re-evaluates its own flagged bins, lowest
    // first, one per round, so every lane with a bin left works in each
    // round (the rounds: the most bins any lane flagged)
    while (__any_sync(0xffffffffu, bad != 0u)) {
      if (bad) {
        const int m = __ffs(bad) - 1;
        bad &= bad - 1u;
        const float p = (float)exact_gls_power_lane(rec, oi.begin, oi.n, k0 + (uint32_t)m, oi.wsum, oi.sum_y2,
                                                    oi.norm_scale);
#pragma unroll
        for (int mm = 0; mm < F; ++mm)
          if (mm == m) pv[mm] = p;
      }
    }
    return;
  }
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int m = 0; m < F; ++m) {
    unsigned mask = __ballot_sync(0xffffffffu, (bad >> m) & 1u);
    while (mask) {
      const int l = __ffs(mask) - 1;
      mask &= mask - 1;
      const uint32_t k = __shfl_sync(0xffffffffu, k0 + (uint32_t)m, l);
      const double p = exact_gls_power_warp(rec, oi.begin, oi.n, k, oi.wsum, oi.sum_y2, oi.norm_scale);
      if (lane == l) pv[m] = (float)p;
    }
  }
}

// Replace the ill-conditioned bins (bit m of `bad`: bin k0 + m) of every lane
// of the warp by their FP64 re-evaluation.  Called by all 32 lanes.
template <int F>
__device__ __forceinline__ void fix_ill_conditioned(float (&pv)[F], uint32_t bad, uint32_t k0,
                                                    const RecF32* __restrict__ rec, int64_t begin,
                                                    int n, double norm_scale) {
  if (!__any_sync(0xffffffffu, bad != 0u)) return;
  if (n <= kLaneExactMaxObs) {  // a short object: lanes in rounds, as in fix_ill_conditioned_gls
    while (__any_sync(0xffffffffu, bad != 0u)) {
      if (bad) {
        const int m = __ffs(bad) - 1;
        bad &= bad - 1u;
        const float p = (float)exact_power_lane(rec, begin, n, k0 + (uint32_t)m, norm_scale);
#pragma unroll
        for (int mm = 0; mm < F; ++mm)
          if (mm == m) pv[mm] = p;
      }
    }
    return;
  }
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int m = 0; m < F; ++m) {
    unsigned mask = __ballot_sync(0xffffffffu, (bad >> m) & 1u);
    while (mask) {
      const int l = __ffs(mask) - 1;
      mask &= mask - 1;
      const uint32_t k = __shfl_sync(0xffffffffu, k0 + (uint32_t)m, l);
      const double p = exact_power_warp(rec, begin, n, k, norm_scale);
      if (lane == l) pv[m] = (float)p;
    }
  }
}

// ------------------------------------------------------ chunk reductions
// (p, k) pair ordering: higher power first, lower index on ties.
__device__ __forceinline__ bool better(double pa, int64_t ka, double pb, int64_t kb) {
  if (ka < 0) return false;
  if (kb < 0) return true;
  return pa > pb || (pa == pb && ka < kb);
}

__device__ __forceinline__ void warp_best(double& p, int64_t& k) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    double po = __shfl_xor_sync(0xffffffffu, p, off);
    long long ko = __shfl_xor_sync(0xffffffffu, (long long)k, off);
    if (better(po, ko, p, k)) {
      p = po;
      k = ko;
    }
  }
}

// Block-wide best (p, k); every thread gets the result.  `red` needs
// 2 * (blockDim.x / 32) 8-byte slots.  Contains __syncthreads.
__device__ __forceinline__ void block_best(double& p, int64_t& k, double* red_p, int64_t* red_k) {
  warp_best(p, k);
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == 0) {
    red_p[warp] = p;
    red_k[warp] = k;
  }
  __syncthreads();
  p = lane < nw ? red_p[lane] : 0.0;
  k = lane < nw ? red_k[lane] : -1;
  warp_best(p, k);
  __syncthreads();
}

// Reduce the chunk's powers (each thread holds NP consecutive bins starting
// at k0, `nv` of them inside the grid) to its first maximum and, when cand
// is not null, to its top-3 interior local maxima and edge bins.  `pw` is a
// shared buffer of blockDim.x * NP floats/doubles (only used with cand).
template <typename Real, int NP>
__device__ void chunk_results(const Real (&pv)[NP], int64_t k0, int64_t k_chunk0, int64_t n_f,
                              ChunkBest* best_out, ChunkCand* cand_out, Real* pw, double* red_p,
                              int64_t* red_k) {
  double bp = 0.0;
  int64_t bk = -1;
#pragma unroll
  for (int m = 0; m < NP; ++m) {
    int64_t k = k0 + m;
    if (k < n_f && better((double)pv[m], k, bp, bk)) {
      bp = (double)pv[m];
      bk = k;
    }
  }
  if (cand_out == nullptr) {
    block_best(bp, bk, red_p, red_k);
    if (threadIdx.x == 0) *best_out = ChunkBest{bp, bk};
    return;
  }
  // top-k path: stage the chunk's powers in shared memory
  const int chunk_len = blockDim.x * NP;
  int64_t nvalid64 = n_f - k_chunk0;
  int nvalid = nvalid64 < chunk_len ? (int)nvalid64 : chunk_len;
  int base = threadIdx.x * NP;
#pragma unroll
  for (int m = 0; m < NP; ++m) pw[base + m] = pv[m];
  __syncthreads();
  // per-thread top-3 of interior local maxima (bins 1 .. nvalid-2 of the chunk)
  double tp[3] = {0.0, 0.0, 0.0};
  int64_t tk[3] = {-1, -1, -1};
#pragma unroll
  for (int m = 0; m < NP; ++m) {
    int i = base + m;
    if (i >= 1 && i <= nvalid - 2) {
      Real v = pw[i];
      if (v > pw[i - 1] && v >= pw[i + 1]) {
        double dv = (double)v;
        int64_t k = k_chunk0 + i;
        if (better(dv, k, tp[0], tk[0])) {
          tp[2] = tp[1]; tk[2] = tk[1]; tp[1] = tp[0]; tk[1] = tk[0]; tp[0] = dv; tk[0] = k;
        } else if (better(dv, k, tp[1], tk[1])) {
          tp[2] = tp[1]; tk[2] = tk[1]; tp[1] = dv; tk[1] = k;
        } else if (better(dv, k, tp[2], tk[2])) {
          tp[2] = dv; tk[2] = k;
        }
      }
    }
  }
  // three rounds of block arg-best, each removing the winner from its owner
  ChunkCand out;
  for (int r = 0; r < 3; ++r) {
    double p = tp[0];
    int64_t k = tk[0];
    block_best(p, k, red_p, red_k);
    out.p[r] = p;
    out.k[r] = k;
    if (k >= 0 && tk[0] == k) {
      tp[0] = tp[1]; tk[0] = tk[1]; tp[1] = tp[2]; tk[1] = tk[2]; tp[2] = 0.0; tk[2] = -1;
    }
  }
  // the chunk's first maximum over all its bins
  block_best(bp, bk, red_p, red_k);
  if (threadIdx.x == 0) {
    *best_out = ChunkBest{bp, bk};
    out.k_first = k_chunk0;
    out.nvalid = nvalid;
    out.pad = 0;
    out.first[0] = nvalid > 0 ? (double)pw[0] : 0.0;
    out.first[1] = nvalid > 1 ? (double)pw[1] : 0.0;
    out.last[0] = nvalid > 0 ? (double)pw[nvalid - 1] : 0.0;
    out.last[1] = nvalid > 1 ? (double)pw[nvalid - 2] : 0.0;
    *cand_out = out;
  }
  __syncthreads();
}

// ------------------------------------------- FP32 chunk reductions (keys)
// In the FP32 kernels a (power, index) pair is one 64-bit key,
//   key = (bits(P) << 32) | (0xFFFFFFFF - k),
// whose unsigned order is "higher power, then lower index" for P >= 0 (the
// kernels' powers are never negative or NaN).  Key 0 means "no bin".  This
// keeps the FP64 pipe (about 1/64 of the FP32 rate on GB300) out of the
// epilogue.
__device__ __forceinline__ unsigned long long pkey(float p, uint32_t k) {
  return ((unsigned long long)__float_as_uint(p) << 32) | (unsigned long long)(0xFFFFFFFFu - k);
}
__device__ __forceinline__ float key_power(unsigned long long key) { return __uint_as_float((uint32_t)(key >> 32)); }
__device__ __forceinline__ int64_t key_index(unsigned long long key) {
  return key ? (int64_t)(0xFFFFFFFFu - (uint32_t)key) : -1;
}
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
  return a > b ? a : b;
}
__device__ __forceinline__ unsigned long long warp_max_key(unsigned long long v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = umax64(v, __shfl_xor_sync(0xffffffffu, v, off));
  return v;
}
// Block-wide maximum key, returned to every thread; `red` holds blockDim/32 keys.
__device__ __forceinline__ unsigned long long block_max_key(unsigned long long v, unsigned long long* red) {
  v = warp_max_key(v);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  v = lane < nw ? red[lane] : 0ull;
  v = warp_max_key(v);
  __syncthreads();
  return v;
}

// FP32 counterpart of chunk_results: first maximum and (with cand) the top-3
// interior local maxima and edge bins of the chunk.  Thread t holds the NP
// bins from chunk index t NP (k0 = k_chunk0 + t NP).  `pw` is a shared
// buffer of at least 4 (blockDim.x / 32) + 2 floats and `red` of 32 keys.
//
// The top-k path keeps the chunk in registers.  Each thread tests its own
// bins for interior local maxima (neighbours in registers, the adjacent
// lanes' by shuffle) and keeps the best of them; a warp takes its three best
// in three rounds of a warp-wide maximum, the winning lane re-scanning its
// bins without the taken one; the two bins at each boundary between warps
// are tested by warp 0 from the first and last two bins each warp publishes,
// and warp 0 merges the warps' lists.  The chunk's first maximum is the best
// of its first bin, its best interior local maximum and its last bin (an
// interior first maximum is a local maximum: its left neighbour is lower,
// its right one not higher).  Ties go to the lower bin throughout: lanes
// and bins are scanned in increasing order with strict comparisons.  One
// barrier; on return only warp 0 may still read the shared buffers, and the
// callers pass a barrier before writing them again.
template <int NP>
__device__ void chunk_results_f32(const float (&pv)[NP], uint32_t k0, int64_t k_chunk0, int64_t n_f,
                                  ChunkBest* best_out, ChunkCand* cand_out, float* pw,
                                  unsigned long long* red) {
  static_assert(NP >= 1 && NP <= 32, "bins per thread");
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int chunk_len = blockDim.x * NP;
  const int64_t nvalid64 = n_f - k_chunk0;
  const int nvalid = nvalid64 < chunk_len ? (int)nvalid64 : chunk_len;
  const int base = tid * NP;
  if (cand_out == nullptr) {
    const int nv = nvalid - base;  // this thread's bins inside the grid (may be <= 0)
    float bp = -1.0f;              // powers are >= 0: the first valid bin always enters
    int bm = -1;
#pragma unroll
    for (int m = 0; m < NP; ++m)
      if (m < nv && pv[m] > bp) {
        bp = pv[m];
        bm = m;
      }
    unsigned long long best = bm >= 0 ? pkey(bp, k0 + (uint32_t)bm) : 0ull;
    best = block_max_key(best, red);
    if (tid == 0) *best_out = ChunkBest{(double)key_power(best), key_index(best)};
    return;
  }
  // interior local maxima among this thread's bins; a warp's first and last
  // bins are left to warp 0 (or are the chunk's edges)
  const int lo = lane == 0 ? 1 : 0;
  const int hi_w = lane == 31 ? NP - 2 : NP - 1;
  const int hi_v = nvalid - 2 - base;
  const int hi = hi_w < hi_v ? hi_w : hi_v;
  const float left_in = __shfl_up_sync(0xffffffffu, pv[NP - 1], 1);
  const float right_in = __shfl_down_sync(0xffffffffu, pv[0], 1);
  uint32_t mask = 0u;
  float bp = 0.0f;  // a local maximum exceeds its left neighbour (>= 0): bp > 0 marks a candidate
  int bm = -1;
#pragma unroll
  for (int m = 0; m < NP; ++m) {
    const float v = pv[m];
    const float l = m > 0 ? pv[m > 0 ? m - 1 : 0] : left_in;
    const float r = m + 1 < NP ? pv[m + 1 < NP ? m + 1 : m] : right_in;
    const bool loc = m >= lo && m <= hi && v > l && v >= r;
    if (loc) mask |= 1u << m;
    if (loc && v > bp) {
      bp = v;
      bm = m;
    }
  }
  // the warp's three best
  unsigned long long wk[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const uint32_t hb = __float_as_uint(bp);
    const uint32_t top = __reduce_max_sync(0xffffffffu, hb);
    const uint32_t ball = __ballot_sync(0xffffffffu, hb == top);
    const int win = __ffs(ball) - 1;  // the lowest lane: the lowest bin among equal powers
    const uint32_t kw = __shfl_sync(0xffffffffu, k0 + (uint32_t)bm, win);
    wk[r] = top ? (((unsigned long long)top << 32) | (unsigned long long)(0xFFFFFFFFu - kw)) : 0ull;
    if (r < 2 && top && lane == win) {
      mask &= ~(1u << bm);
      bp = 0.0f;
      bm = -1;
#pragma unroll
      for (int m = 0; m < NP; ++m)
        if (((mask >> m) & 1u) && pv[m] > bp) {
          bp = pv[m];
          bm = m;
        }
    }
  }
  // publish: the list, the warp's first two and last two bins, and the
  // chunk's last two bins where the chunk ends inside a warp
  if (lane == 0) {
    red[3 * warp] = wk[0];
    red[3 * warp + 1] = wk[1];
    red[3 * warp + 2] = wk[2];
    pw[4 * warp] = pv[0];
    if (NP >= 2) pw[4 * warp + 1] = pv[NP >= 2 ? 1 : 0];
  }
  if (NP == 1 && lane == 1) pw[4 * warp + 1] = pv[0];
  if (NP == 1 && lane == 30) pw[4 * warp + 2] = pv[0];
  if (lane == 31) {
    if (NP >= 2) pw[4 * warp + 2] = pv[NP >= 2 ? NP - 2 : 0];
    pw[4 * warp + 3] = pv[NP - 1];
  }
  if (nvalid < chunk_len) {
    const int j0 = nvalid - 1 - base, j1 = nvalid - 2 - base;
    if ((unsigned)j0 < (unsigned)NP || (unsigned)j1 < (unsigned)NP) {
#pragma unroll
      for (int m = 0; m < NP; ++m) {
        if (m == j0) pw[4 * nw] = pv[m];
        if (m == j1) pw[4 * nw + 1] = pv[m];
      }
    }
  }
  __syncthreads();
  if (warp != 0) return;
  // lane w < nw: warp w's list with the two bins at its boundary with warp w - 1
  unsigned long long c0 = 0ull, c1 = 0ull, c2 = 0ull;
  if (lane < nw) {
    c0 = red[3 * lane];
    c1 = red[3 * lane + 1];
    c2 = red[3 * lane + 2];
    if (lane > 0) {
      const int i = lane * 32 * NP;  // chunk index of warp `lane`'s first bin
      const float f0 = pw[4 * lane], f1 = pw[4 * lane + 1];
      const float l1 = pw[4 * lane - 2], l0 = pw[4 * lane - 1];
      unsigned long long e[2] = {0ull, 0ull};
      if (i - 1 <= nvalid - 2 && l0 > l1 && l0 >= f0) e[0] = pkey(l0, (uint32_t)(k_chunk0 + i - 1));
      if (i <= nvalid - 2 && f0 > l0 && f0 >= f1) e[1] = pkey(f0, (uint32_t)(k_chunk0 + i));
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const unsigned long long x = e[q];
        if (x > c0) {
          c2 = c1;
          c1 = c0;
          c0 = x;
        } else if (x > c1) {
          c2 = c1;
          c1 = x;
        } else if (x > c2) {
          c2 = x;
        }
      }
    }
  }
  unsigned long long top3[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const uint32_t h = (uint32_t)(c0 >> 32);
    const uint32_t th = __reduce_max_sync(0xffffffffu, h);
    const uint32_t tl = __reduce_max_sync(0xffffffffu, h == th ? (uint32_t)c0 : 0u);
    const unsigned long long t = ((unsigned long long)th << 32) | tl;
    top3[r] = t;
    if (t && c0 == t) {  // keys of distinct bins differ: one lane holds it
      c0 = c1;
      c1 = c2;
      c2 = 0ull;
    }
  }
  if (lane == 0) {
    const bool full = nvalid == chunk_len;
    const float first0 = pw[0], first1 = pw[1];
    const float last0 = full ? pw[4 * nw - 1] : pw[4 * nw];
    const float last1 = full ? pw[4 * nw - 2] : pw[4 * nw + 1];
    unsigned long long best = top3[0];
    if (nvalid > 0) best = umax64(best, pkey(first0, (uint32_t)k_chunk0));
    if (nvalid > 1) best = umax64(best, pkey(last0, (uint32_t)(k_chunk0 + nvalid - 1)));
    *best_out = ChunkBest{(double)key_power(best), key_index(best)};
    ChunkCand out;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      out.p[r] = (double)key_power(top3[r]);
      out.k[r] = key_index(top3[r]);
    }
    out.k_first = k_chunk0;
    out.nvalid = nvalid;
    out.pad = 0;
    out.first[0] = nvalid > 0 ? (double)first0 : 0.0;
    out.first[1] = nvalid > 1 ? (double)first1 : 0.0;
    out.last[0] = nvalid > 0 ? (double)last0 : 0.0;
    out.last[1] = nvalid > 1 ? (double)last1 : 0.0;
    *cand_out = out;
  }
}

// chunk_results_f32 with the chunk staged in shared memory: the same
// results (first maximum, top-3 interior local maxima, edge bins), found by
// a scan of the staged powers and block-wide key reductions.  The
// generalized periodogram's kernels use it: with the register version their
// main loop compiled measurably slower (0.745 against 0.792 of the bound on
// the lognormal batch), more than its cheaper epilogue won back.  `pw` is a
// shared buffer of blockDim.x * (NP + 1) floats (top-k only).
template <int NP>
__device__ void chunk_results_f32_staged(const float (&pv)[NP], uint32_t k0, int64_t k_chunk0, int64_t n_f,
                                  ChunkBest* best_out, ChunkCand* cand_out, float* pw,
                                  unsigned long long* red) {
  unsigned long long best = 0ull;
#pragma unroll
  for (int m = 0; m < NP; ++m)
    if ((int64_t)k0 + m < n_f) best = umax64(best, pkey(pv[m], k0 + (uint32_t)m));
  if (cand_out == nullptr) {
    best = block_max_key(best, red);
    if (threadIdx.x == 0) *best_out = ChunkBest{(double)key_power(best), key_index(best)};
    return;
  }
  const int chunk_len = blockDim.x * NP;
  const int64_t nvalid64 = n_f - k_chunk0;
  const int nvalid = nvalid64 < chunk_len ? (int)nvalid64 : chunk_len;
  // bin i of the chunk at pw[i + i / NP]: one padding word per thread, so a
  // warp's stores and neighbour reads fall in distinct banks (without it, a
  // stride of NP = 32 floats puts all 32 lanes on one bank)
  const int base = threadIdx.x * NP;
  const int pbase = threadIdx.x * (NP + 1);
#pragma unroll
  for (int m = 0; m < NP; ++m) pw[pbase + m] = pv[m];
  __syncthreads();
  unsigned long long t0 = 0ull, t1 = 0ull, t2 = 0ull;  // this thread's top-3 interior maxima
#pragma unroll
  for (int m = 0; m < NP; ++m) {
    const int i = base + m;
    if (i >= 1 && i <= nvalid - 2) {
      const float v = pw[pbase + m];
      if (v > pw[(i - 1) + (i - 1) / NP] && v >= pw[(i + 1) + (i + 1) / NP]) {
        const unsigned long long key = pkey(v, (uint32_t)(k_chunk0 + i));
        if (key > t0) { t2 = t1; t1 = t0; t0 = key; }
        else if (key > t1) { t2 = t1; t1 = key; }
        else if (key > t2) { t2 = key; }
      }
    }
  }
  ChunkCand out;
  for (int r = 0; r < 3; ++r) {
    const unsigned long long w = block_max_key(t0, red);
    out.p[r] = (double)key_power(w);
    out.k[r] = key_index(w);
    if (w && t0 == w) { t0 = t1; t1 = t2; t2 = 0ull; }
  }
  best = block_max_key(best, red);
  if (threadIdx.x == 0) {
    *best_out = ChunkBest{(double)key_power(best), key_index(best)};
    out.k_first = k_chunk0;
    out.nvalid = nvalid;
    out.pad = 0;
    out.first[0] = nvalid > 0 ? (double)pw[0] : 0.0;
    out.first[1] = nvalid > 1 ? (double)pw[1 + 1 / NP] : 0.0;
    out.last[0] = nvalid > 0 ? (double)pw[(nvalid - 1) + (nvalid - 1) / NP] : 0.0;
    out.last[1] = nvalid > 1 ? (double)pw[(nvalid - 2) + (nvalid - 2) / NP] : 0.0;
    *cand_out = out;
  }
  __syncthreads();
}

// Eq. 2 from the FP32 single-scan sums, its two terms over one denominator:
// with W = (2 CC - N) + i 2 CS and Z = XC + i XS as in lsp_power,
// (N + R)(N - R) = N^2 - |W|^2 and Q R = Re(Z^2 conj W), so
//   P = (N |Z|^2 - Re(Z^2 conj W)) / (N^2 - |W|^2),
// one fast division (relative error ~1e-7) and no square root.  Its
// denominator is N^2 - R^2 = (N + R)(N - R) >= N (N - R), so where the bin
// is well conditioned (N - R >= 5 % N, ill_conditioned below) it is at
// least 0.05 N^2; the ill-conditioned bins, R = N included, are re-evaluated
// in FP64 by the callers.  `ill` is N - R < 5 % N, tested as R^2 > 0.95^2 N^2.
constexpr float kIllR2 = (1.0f - kIllConditioned) * (1.0f - kIllConditioned);

__device__ __forceinline__ float lsp_power_f32(float xc, float xs, float cc, float cs, float n, bool& ill) {
  const float c2 = fmaf(2.0f, cc, -n);
  const float s2 = 2.0f * cs;
  const float r2 = fmaf(c2, c2, s2 * s2);
  const float nn = n * n;
  const float z2 = fmaf(xc, xc, xs * xs);
  const float re = fmaf((xc - xs) * (xc + xs), c2, 2.0f * xc * xs * s2);  // Re(Z^2 conj W)
  const float num = fmaf(n, z2, -re);
  const float den = nn - r2;
  ill = r2 > kIllR2 * nn;
  return den > 0.0f ? __fdividef(fmaxf(num, 0.0f), den) : 0.0f;
}

}  // namespace lsp
