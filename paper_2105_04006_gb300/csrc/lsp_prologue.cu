// lsp_prologue.cu -- per-object statistics and per-observation records.
//
// Section 2 assumes zero-mean magnitudes; the paper excludes this step from
// its timings (Section 4.1).  Here it runs on the GPU in FP64:
//   stats:   mean of y, sum of centred y^2, time span (t0 = midpoint), flags
//            (one pass of shifted sums);
//   records: y - mean, and the phase data of the grid recurrences:
//            a = frac(f_min (t - t0)), b = frac(df (t - t0)) as 64-bit fixed
//            point (2^64 = one cycle), and (cos, sin)(2 pi b).
// Subtracting t0 keeps |t - t0| <= half the span, so the FP64 products carry
// about 1e-13 cycle of error before they are reduced; the fixed-point form
// then makes the phase of any grid frequency k, frac(a + k b), exact up to
// k * 2^-64 cycle with integer arithmetic only.
#include <cmath>

#include "../../include/lsp.h"
#include "lsp_launch.h"

namespace lsp {
namespace {

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, off));
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  return v;
}

// Block reductions through shared memory (blockDim.x <= 1024).  Results are
// broadcast to all threads.  Each contains two __syncthreads.
__device__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = l < nw ? sh[l] : 0.0;
  v = warp_sum(v);
  __syncthreads();
  return v;
}
__device__ double block_min(double v, double* sh) {
  v = warp_min(v);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = l < nw ? sh[l] : INFINITY;
  v = warp_min(v);
  __syncthreads();
  return v;
}
__device__ double block_max(double v, double* sh) {
  v = warp_max(v);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = l < nw ? sh[l] : -INFINITY;
  v = warp_max(v);
  __syncthreads();
  return v;
}

// Per-object statistics in one pass over the observations: with a shift K
// (the object's first magnitude, so that the sums are about the mean's
// order), sy = sum w (y - K), sw = sum w, s2 = sum w (y - K)^2, the time span
// and a non-finite flag.  The centred sum of squares then follows exactly in
// real arithmetic as s2 - 2 d sy + d^2 sw with d = mean - K; in FP64 the
// shift keeps the cancellation to a few digits of the 16.  GLS: w = 1/dy^2
// (dy NULL: unit weights) for the generalized periodogram.
//
// GB300 runs FP64 at 1/64 of the FP32 rate, so only the two (GLS: three)
// sums use FP64 arithmetic: the time span is kept as order-preserving 64-bit
// integer keys of the FP64 times (exact min/max on the integer pipe), and
// without weights sw is the observation count, supplied at the end.
struct StatAcc {
  double sy, sw, s2;
  unsigned long long tmin, tmax;  // time_key of the earliest / latest time
  unsigned long long bad;         // non-zero: a NaN or Inf was seen
};
constexpr int kStatSlice = 256;  // observations (and threads) per CTA of the one-object pass

// An unsigned key that orders like the FP64 value (finite values and infinities).
__device__ __forceinline__ unsigned long long time_key(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double time_of_key(unsigned long long k) {
  const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double((long long)b);
}

__device__ __forceinline__ StatAcc stat_identity() { return StatAcc{0.0, 0.0, 0.0, ~0ull, 0ull, 0ull}; }

template <bool GLS>
__device__ __forceinline__ void stat_merge(StatAcc& a, const StatAcc& b) {
  a.sy += b.sy;
  if (GLS) a.sw += b.sw;
  a.s2 += b.s2;
  a.tmin = b.tmin < a.tmin ? b.tmin : a.tmin;
  a.tmax = b.tmax > a.tmax ? b.tmax : a.tmax;
  a.bad |= b.bad;
}

template <bool GLS>
__device__ __forceinline__ void stat_warp_merge(StatAcc& a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    StatAcc b;
    b.sy = __shfl_xor_sync(0xffffffffu, a.sy, o);
    b.sw = GLS ? __shfl_xor_sync(0xffffffffu, a.sw, o) : 0.0;
    b.s2 = __shfl_xor_sync(0xffffffffu, a.s2, o);
    b.tmin = __shfl_xor_sync(0xffffffffu, a.tmin, o);
    b.tmax = __shfl_xor_sync(0xffffffffu, a.tmax, o);
    b.bad = __shfl_xor_sync(0xffffffffu, a.bad, o);
    stat_merge<GLS>(a, b);
  }
}

// Block reduction of StatAcc; the result is valid in thread 0.  sh holds one
// StatAcc per warp.
template <bool GLS>
__device__ __forceinline__ StatAcc stat_block_merge(StatAcc a, StatAcc* sh) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  stat_warp_merge<GLS>(a);
  if (l == 0) sh[w] = a;
  __syncthreads();
  if (w == 0) {
    a = l < nw ? sh[l] : stat_identity();
    stat_warp_merge<GLS>(a);
  }
  __syncthreads();
  return a;
}

template <typename YT, bool GLS>
__device__ __forceinline__ void stat_accumulate(const double* __restrict__ t, const YT* __restrict__ y,
                                                const YT* __restrict__ dy, int64_t b, int64_t e, double K,
                                                StatAcc& a) {
  for (int64_t j = b + threadIdx.x; j < e; j += blockDim.x) {
    const double tj = t[j], yj = (double)y[j];
    double wj = 1.0;
    if (GLS && dy) {
      const double ej = (double)dy[j];
      if (!isfinite(ej) || !(ej > 0.0)) a.bad = 1ull;
      wj = 1.0 / (ej * ej);
    }
    if (!isfinite(tj) || !isfinite(yj)) a.bad = 1ull;
    const double d = yj - K;
    if (GLS) {
      a.sy = fma(wj, d, a.sy);
      a.sw += wj;
      a.s2 = fma(wj * d, d, a.s2);
    } else {
      a.sy += d;
      a.s2 = fma(d, d, a.s2);
    }
    const unsigned long long k = time_key(tj);
    a.tmin = k < a.tmin ? k : a.tmin;
    a.tmax = k > a.tmax ? k : a.tmax;
  }
}

template <bool GLS>
__device__ __forceinline__ ObjInfo stat_finish(const StatAcc& acc, double K, int64_t b, int64_t n, int flags,
                                               int center) {
  StatAcc a = acc;
  if (!GLS) a.sw = (double)n;  // unit weights: the sum of weights is the count
  const double mean = ((GLS || center) && n > 0 && a.sw > 0.0) ? K + a.sy / a.sw : 0.0;
  const double d = mean - K;
  const double s2 = n > 0 ? a.s2 - 2.0 * d * a.sy + d * d * a.sw : 0.0;
  if (a.bad) flags |= LSP_FLAG_NONFINITE;
  if (n < (GLS ? 3 : 2)) flags |= LSP_FLAG_FEW_OBS;
  if (!(flags & LSP_FLAG_NONFINITE) && n > 0 && !(s2 > 0.0)) flags |= LSP_FLAG_ZERO_VAR;
  ObjInfo oi;
  oi.t0 = n > 0 ? 0.5 * (time_of_key(a.tmin) + time_of_key(a.tmax)) : 0.0;
  oi.ymean = mean;
  oi.sum_y2 = s2;
  oi.begin = b;
  oi.n = (int32_t)n;
  oi.flags = flags;
  oi.wsum = a.sw;
  oi.wsum_f = (float)a.sw;
  return oi;
}

__device__ __forceinline__ void stat_norm(ObjInfo& oi, int norm, bool gls) {
  if (gls)  // the generalized power is normalised in the kernel; PSD form = P * sum_y2 / 2
    oi.norm_scale = norm ? 1.0 : 0.5 * oi.sum_y2;
  else
    oi.norm_scale = (norm && oi.sum_y2 > 0.0) ? 2.0 / oi.sum_y2 : 1.0;
  oi.norm_scale_f = (float)oi.norm_scale;
}

// Batches: one CTA per object.
template <typename YT, bool GLS>
__global__ void stats_kernel(const double* __restrict__ t, const YT* __restrict__ y,
                             const YT* __restrict__ dy, const int64_t* __restrict__ offsets,
                             int64_t total_nt, int center, int norm, ObjInfo* __restrict__ obj) {
  __shared__ StatAcc sh[32];
  const int64_t o = blockIdx.x;
  int64_t b = 0, e = total_nt;
  int flags = 0;
  if (offsets) {
    b = offsets[o];
    e = offsets[o + 1];
    if (b < 0 || e < b || e > total_nt || e - b > (int64_t)INT32_MAX) {
      flags |= LSP_FLAG_BAD_OFFSETS;
      b = e = 0;
    }
  }
  const int64_t n = e - b;
  const double K = n > 0 ? (double)y[b] : 0.0;
  StatAcc a = stat_identity();
  stat_accumulate<YT, GLS>(t, y, dy, b, e, K, a);
  a = stat_block_merge<GLS>(a, sh);
  if (threadIdx.x == 0) {
    ObjInfo oi = stat_finish<GLS>(a, K, b, n, flags, center);
    stat_norm(oi, norm, GLS);
    obj[o] = oi;
  }
}

// One object: CTAs reduce slices of `slice` observations into part[]; the
// last CTA to finish (ticket, zero on entry) merges the partials in index
// order, so the result does not depend on which CTA finished last.
template <typename YT, bool GLS>
__global__ void stats_slices_kernel(const double* __restrict__ t, const YT* __restrict__ y,
                                    const YT* __restrict__ dy, int64_t n, int64_t slice, int center, int norm,
                                    StatAcc* __restrict__ part, uint32_t* __restrict__ ticket,
                                    ObjInfo* __restrict__ obj) {
  __shared__ StatAcc sh[32];
  __shared__ bool s_last;
  const double K = n > 0 ? (double)y[0] : 0.0;
  const int64_t b = (int64_t)blockIdx.x * slice;
  const int64_t e = b + slice < n ? b + slice : n;
  StatAcc a = stat_identity();
  stat_accumulate<YT, GLS>(t, y, dy, b, e, K, a);
  a = stat_block_merge<GLS>(a, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = a;
    __threadfence();
    s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last || threadIdx.x >= 32) return;
  __threadfence();
  StatAcc r = stat_identity();
  for (unsigned s = threadIdx.x; s < gridDim.x; s += 32) {
    const double* q = reinterpret_cast<const double*>(part + s);
    const unsigned long long* u = reinterpret_cast<const unsigned long long*>(part + s);
    StatAcc v{__ldcg(q), __ldcg(q + 1), __ldcg(q + 2), __ldcg(u + 3), __ldcg(u + 4), __ldcg(u + 5)};
    stat_merge<GLS>(r, v);
  }
  stat_warp_merge<GLS>(r);
  if (threadIdx.x == 0) {
    ObjInfo oi = stat_finish<GLS>(r, K, 0, n, n > (int64_t)INT32_MAX ? LSP_FLAG_BAD_OFFSETS : 0, center);
    stat_norm(oi, norm, GLS);
    obj[0] = oi;
  }
}

// frac(f * x) as 64-bit fixed point.  f * x = p + e exactly (FMA two-product);
// frac(p) is exact in FP64; e adds the bits p dropped.
__device__ __forceinline__ uint64_t frac_fixed64(double f, double x) {
  double p = f * x;
  double e = fma(f, x, -p);
  double r = p - floor(p);  // exact, in [0, 1)
  uint64_t u = __double2ull_rz(r * 18446744073709551616.0);
  long long corr = __double2ll_rn(e * 18446744073709551616.0);
  return u + (uint64_t)corr;
}

// The record of observation j of an object (statistics oi).
template <typename YT, typename Rec, bool GLS>
__device__ __forceinline__ void make_record(const double* __restrict__ t, const YT* __restrict__ y,
                                            const YT* __restrict__ dy, int64_t j, const ObjInfo& oi, double f_min,
                                            double df, Rec* __restrict__ rec) {
  const double tp = t[j] - oi.t0;
  const uint64_t a = frac_fixed64(f_min, tp);
  const uint64_t bb = frac_fixed64(df, tp);
  const double xb = (double)(int64_t)bb * 5.421010862427522e-20;  // 2^-64: cycles in [-1/2, 1/2)
  double s, c;
  if constexpr (sizeof(Rec) == sizeof(RecF32)) {
    // FP32 rotation: sincospi of the fraction's leading float, corrected to
    // first order for the remainder (|lo| < 2^-25 cycle): accurate to about
    // one FP32 ulp without an FP64 transcendental (GB300's FP64 pipe is
    // 1/64 of its FP32 rate).
    const float hi = (float)xb;
    const float lo = (float)(xb - (double)hi);
    float sh, ch;
    sincospif(2.0f * hi, &sh, &ch);
    const float d = 6.28318530717958647692f * lo;
    c = (double)fmaf(-sh, d, ch);
    s = (double)fmaf(ch, d, sh);
  } else {
    sincospi(2.0 * xb, &s, &c);
  }
  double w = 1.0;
  if (GLS && dy) {
    const double ej = (double)dy[j];
    w = 1.0 / (ej * ej);
  }
  const double yc = (GLS ? w : 1.0) * ((double)y[j] - oi.ymean);
  Rec r;
  if constexpr (sizeof(Rec) == sizeof(RecF32)) {
    r.y = (float)yc;
    r.cr = (float)c;
    r.sr = (float)s;
    r.a_hi = (uint32_t)(a >> 32);
    r.a_lo = (uint32_t)a;
    r.b_hi = (uint32_t)(bb >> 32);
    r.b_lo = (uint32_t)bb;
    r.pad = GLS ? __float_as_uint((float)w) : 0u;
  } else {
    r.y = yc;
    r.cr = c;
    r.sr = s;
    r.a = a;
    r.b = bb;
    r.pad = GLS ? (uint64_t)__double_as_longlong(w) : 0ull;
  }
  rec[j] = r;
}

// grid.x: object; grid.y: slices of a single large object's observations.
template <typename YT, typename Rec, bool GLS>
__global__ void records_kernel(const double* __restrict__ t, const YT* __restrict__ y,
                               const YT* __restrict__ dy, const ObjInfo* __restrict__ obj,
                               int64_t slice, double f_min, double df, Rec* __restrict__ rec) {
  const ObjInfo oi = obj[blockIdx.x];
  if (oi.flags & (LSP_FLAG_BAD_OFFSETS | LSP_FLAG_NONFINITE)) return;
  const int64_t lo = oi.begin + (int64_t)blockIdx.y * slice;
  int64_t hi = lo + slice;
  if (hi > oi.begin + oi.n) hi = oi.begin + oi.n;
  for (int64_t j = lo + threadIdx.x; j < hi; j += blockDim.x) make_record<YT, Rec, GLS>(t, y, dy, j, oi, f_min, df, rec);
}

// One object of at most kFusedMaxNt observations in one launch: every CTA
// computes the object's statistics itself (the same one-pass sums over all
// observations, in the same order, so every CTA gets the same bits), CTA 0
// stores them and clears the four work-counter words, and each CTA writes
// the records of its slice of kStatSlice observations.
template <typename YT, typename Rec, bool GLS>
__global__ void __launch_bounds__(kStatSlice) single_prologue_kernel(
    const double* __restrict__ t, const YT* __restrict__ y, const YT* __restrict__ dy, int64_t n, int center,
    int norm, double f_min, double df, ObjInfo* __restrict__ obj, Rec* __restrict__ rec,
    uint32_t* __restrict__ queue) {
  __shared__ StatAcc sh[32];
  __shared__ ObjInfo s_oi;
  const double K = n > 0 ? (double)y[0] : 0.0;
  StatAcc a = stat_identity();
  stat_accumulate<YT, GLS>(t, y, dy, 0, n, K, a);
  a = stat_block_merge<GLS>(a, sh);
  if (threadIdx.x == 0) {
    ObjInfo oi = stat_finish<GLS>(a, K, 0, n, 0, center);
    stat_norm(oi, norm, GLS);
    s_oi = oi;
    if (blockIdx.x == 0) {
      obj[0] = oi;
      queue[0] = queue[1] = queue[2] = queue[3] = 0u;
    }
  }
  __syncthreads();
  const ObjInfo oi = s_oi;
  if (oi.flags & (LSP_FLAG_BAD_OFFSETS | LSP_FLAG_NONFINITE)) return;
  const int64_t j = (int64_t)blockIdx.x * kStatSlice + threadIdx.x;
  if (j < n) make_record<YT, Rec, GLS>(t, y, dy, j, oi, f_min, df, rec);
}

__global__ void hist_kernel(const ObjInfo* __restrict__ obj, int64_t n_obj, uint32_t* hist) {
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n_obj;
       o += (int64_t)gridDim.x * blockDim.x) {
    int n = obj[o].n;
    int bin = LSP_HIST_BINS - 1 - (n < LSP_HIST_BINS - 1 ? n : LSP_HIST_BINS - 1);
    atomicAdd(&hist[bin], 1u);
  }
}

// Exclusive scan of LSP_HIST_BINS counters by one CTA of 1024 threads.
__global__ void scan_kernel(uint32_t* hist) {
  __shared__ uint32_t part[1024];
  constexpr int per = LSP_HIST_BINS / 1024;
  uint32_t loc[per];
  uint32_t s = 0;
  for (int i = 0; i < per; ++i) {
    loc[i] = hist[threadIdx.x * per + i];
    s += loc[i];
  }
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    uint32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  uint32_t run = part[threadIdx.x] - s;
  for (int i = 0; i < per; ++i) {
    hist[threadIdx.x * per + i] = run;
    run += loc[i];
  }
}

// Queue position of the object with the r-th most observations: the longest
// and the shortest alternate (r = 0, n-1, 1, n-2, ...), so the items resident
// on an SM at any time mix long objects with short ones, whose fixed costs
// (queue, staging and epilogue latency) the long ones' arithmetic hides; the
// queue still ends with objects of middling length.
__device__ __forceinline__ int64_t interleaved_pos(int64_t r, int64_t n) {
  const int64_t half = (n + 1) / 2;
  return r < half ? 2 * r : 2 * (n - 1 - r) + 1;
}

__global__ void scatter_kernel(const ObjInfo* __restrict__ obj, int64_t n_obj, uint32_t* start,
                               int32_t* order) {
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n_obj;
       o += (int64_t)gridDim.x * blockDim.x) {
    int n = obj[o].n;
    int bin = LSP_HIST_BINS - 1 - (n < LSP_HIST_BINS - 1 ? n : LSP_HIST_BINS - 1);
    uint32_t pos = atomicAdd(&start[bin], 1u);
    order[interleaved_pos((int64_t)pos, n_obj)] = (int32_t)o;
  }
}

}  // namespace

size_t stats_slices_bytes(int64_t total_nt) {
  const int64_t slices = (total_nt + kStatSlice - 1) / kStatSlice;
  return (size_t)(slices > 0 ? slices : 1) * sizeof(StatAcc);
}

cudaError_t launch_stats(const double* t, const void* y, bool y64, const int64_t* offsets,
                         int64_t n_obj, int64_t total_nt, int center, int norm, ObjInfo* obj,
                         cudaStream_t stream, bool gls, const void* dy, void* slices_ws, uint32_t* ticket) {
  if (n_obj <= 0) return cudaSuccess;
  if (n_obj == 1 && !offsets && slices_ws && ticket) {
    // one object without offsets: spread the pass over CTAs of kStatSlice observations
    int64_t g64 = (total_nt + kStatSlice - 1) / kStatSlice;
    const unsigned g = (unsigned)(g64 > 0 ? g64 : 1);
    StatAcc* part = (StatAcc*)slices_ws;
#define LSP_STATS_SLICES(YT, G)                                                                              \
  stats_slices_kernel<YT, G><<<g, kStatSlice, 0, stream>>>(t, (const YT*)y, (const YT*)dy, total_nt, kStatSlice, \
                                                            center, norm, part, ticket, obj)
    if (y64) {
      if (gls) LSP_STATS_SLICES(double, true); else LSP_STATS_SLICES(double, false);
    } else {
      if (gls) LSP_STATS_SLICES(float, true); else LSP_STATS_SLICES(float, false);
    }
#undef LSP_STATS_SLICES
    return cudaGetLastError();
  }
  const int threads = n_obj == 1 ? 1024 : 128;
  const unsigned g = (unsigned)n_obj;
  if (y64) {
    if (gls)
      stats_kernel<double, true><<<g, threads, 0, stream>>>(t, (const double*)y, (const double*)dy, offsets,
                                                             total_nt, center, norm, obj);
    else
      stats_kernel<double, false><<<g, threads, 0, stream>>>(t, (const double*)y, nullptr, offsets,
                                                              total_nt, center, norm, obj);
  } else {
    if (gls)
      stats_kernel<float, true><<<g, threads, 0, stream>>>(t, (const float*)y, (const float*)dy, offsets,
                                                            total_nt, center, norm, obj);
    else
      stats_kernel<float, false><<<g, threads, 0, stream>>>(t, (const float*)y, nullptr, offsets, total_nt,
                                                             center, norm, obj);
  }
  return cudaGetLastError();
}

cudaError_t launch_records(const double* t, const void* y, bool y64, const ObjInfo* obj,
                           int64_t n_obj, int64_t max_nt_single, double f_min, double df,
                           bool rec64, void* rec, cudaStream_t stream, bool gls, const void* dy) {
  if (n_obj <= 0) return cudaSuccess;
  int64_t slice = INT64_MAX / 4;
  unsigned gy = 1;
  int threads = 128;
  if (n_obj == 1) {  // spread one object over many CTAs (FP64 work is slow per SM)
    slice = 256;
    gy = (unsigned)((max_nt_single + slice - 1) / slice);
    if (gy == 0) gy = 1;
    threads = 128;
  }
  dim3 grid((unsigned)n_obj, gy);
#define LSP_REC(YT, REC, G)                                                                        \
  records_kernel<YT, REC, G><<<grid, threads, 0, stream>>>(t, (const YT*)y, (const YT*)dy, obj, slice, \
                                                            f_min, df, (REC*)rec)
  if (rec64) {
    if (y64) {
      if (gls) LSP_REC(double, RecF64, true); else LSP_REC(double, RecF64, false);
    } else {
      if (gls) LSP_REC(float, RecF64, true); else LSP_REC(float, RecF64, false);
    }
  } else {
    if (y64) {
      if (gls) LSP_REC(double, RecF32, true); else LSP_REC(double, RecF32, false);
    } else {
      if (gls) LSP_REC(float, RecF32, true); else LSP_REC(float, RecF32, false);
    }
  }
#undef LSP_REC
  return cudaGetLastError();
}

cudaError_t launch_single_prologue(const double* t, const void* y, bool y64, int64_t n, int center, int norm,
                                   double f_min, double df, bool rec64, ObjInfo* obj, void* rec, uint32_t* queue,
                                   cudaStream_t stream, bool gls, const void* dy) {
  if (n < 0 || n > kFusedMaxNt) return cudaErrorInvalidValue;
  const unsigned g = (unsigned)(n > 0 ? (n + kStatSlice - 1) / kStatSlice : 1);
#define LSP_SP(YT, REC, G)                                                                                       \
  single_prologue_kernel<YT, REC, G><<<g, kStatSlice, 0, stream>>>(t, (const YT*)y, (const YT*)dy, n, center, norm, \
                                                                  f_min, df, obj, (REC*)rec, queue)
  if (rec64) {
    if (y64) {
      if (gls) LSP_SP(double, RecF64, true); else LSP_SP(double, RecF64, false);
    } else {
      if (gls) LSP_SP(float, RecF64, true); else LSP_SP(float, RecF64, false);
    }
  } else {
    if (y64) {
      if (gls) LSP_SP(double, RecF32, true); else LSP_SP(double, RecF32, false);
    } else {
      if (gls) LSP_SP(float, RecF32, true); else LSP_SP(float, RecF32, false);
    }
  }
#undef LSP_SP
  return cudaGetLastError();
}

cudaError_t launch_lpt_order(const ObjInfo* obj, int64_t n_obj, uint32_t* hist, int32_t* order,
                             cudaStream_t stream) {
  if (n_obj <= 0) return cudaSuccess;
  cudaError_t err = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * LSP_HIST_BINS, stream);
  if (err != cudaSuccess) return err;
  int blocks = (int)((n_obj + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  hist_kernel<<<blocks, 256, 0, stream>>>(obj, n_obj, hist);
  scan_kernel<<<1, 1024, 0, stream>>>(hist);
  scatter_kernel<<<blocks, 256, 0, stream>>>(obj, n_obj, hist, order);
  return cudaGetLastError();
}

}  // namespace lsp
