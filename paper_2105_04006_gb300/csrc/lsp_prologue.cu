// lsp_prologue.cu -- per-object statistics and per-observation records.
//
// Section 2 assumes zero-mean magnitudes; the paper excludes this step from
// its timings (Section 4.1).  Here it runs on the GPU in FP64:
//   stats:   mean of y, sum of centred y^2, time span (t0 = midpoint), flags;
//   records: y - mean, and the phase data of the rotation recurrence:
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

// One CTA per object.  GLS: weighted statistics with w = 1/dy^2 (dy NULL:
// unit weights) for the generalized periodogram.
template <typename YT, bool GLS>
__global__ void stats_kernel(const double* __restrict__ t, const YT* __restrict__ y,
                             const YT* __restrict__ dy, const int64_t* __restrict__ offsets,
                             int64_t total_nt, int center, int norm, ObjInfo* __restrict__ obj) {
  __shared__ double sh[32];
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
  double sy = 0.0, sw = 0.0, tmin = INFINITY, tmax = -INFINITY, bad = 0.0;
  for (int64_t j = b + threadIdx.x; j < e; j += blockDim.x) {
    double tj = t[j], yj = (double)y[j];
    double wj = 1.0;
    if (GLS && dy) {
      const double ej = (double)dy[j];
      if (!isfinite(ej) || !(ej > 0.0)) bad = 1.0;
      wj = 1.0 / (ej * ej);
    }
    if (!isfinite(tj) || !isfinite(yj)) bad = 1.0;
    sy += wj * yj;
    sw += wj;
    tmin = fmin(tmin, tj);
    tmax = fmax(tmax, tj);
  }
  sy = block_sum(sy, sh);
  sw = block_sum(sw, sh);
  tmin = block_min(tmin, sh);
  tmax = block_max(tmax, sh);
  bad = block_sum(bad, sh);
  const double mean = ((GLS || center) && n > 0 && sw > 0.0) ? sy / sw : 0.0;
  double s2 = 0.0;
  for (int64_t j = b + threadIdx.x; j < e; j += blockDim.x) {
    double d = (double)y[j] - mean;
    double wj = 1.0;
    if (GLS && dy) {
      const double ej = (double)dy[j];
      wj = 1.0 / (ej * ej);
    }
    s2 += wj * d * d;
  }
  s2 = block_sum(s2, sh);
  if (threadIdx.x == 0) {
    if (bad > 0.0) flags |= LSP_FLAG_NONFINITE;
    if (n < (GLS ? 3 : 2)) flags |= LSP_FLAG_FEW_OBS;
    if (!(flags & LSP_FLAG_NONFINITE) && n > 0 && !(s2 > 0.0)) flags |= LSP_FLAG_ZERO_VAR;
    ObjInfo oi;
    oi.t0 = n > 0 ? 0.5 * (tmin + tmax) : 0.0;
    oi.ymean = mean;
    oi.sum_y2 = s2;
    oi.begin = b;
    oi.n = (int32_t)n;
    oi.flags = flags;
    if (GLS)  // the generalized power is normalised in the kernel; PSD form = P * sum_y2 / 2
      oi.norm_scale = norm ? 1.0 : 0.5 * s2;
    else
      oi.norm_scale = (norm && s2 > 0.0) ? 2.0 / s2 : 1.0;
    oi.norm_scale_f = (float)oi.norm_scale;
    oi.wsum = sw;
    oi.wsum_f = (float)sw;
    obj[o] = oi;
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
  for (int64_t j = lo + threadIdx.x; j < hi; j += blockDim.x) {
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

__global__ void scatter_kernel(const ObjInfo* __restrict__ obj, int64_t n_obj, uint32_t* start,
                               int32_t* order) {
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n_obj;
       o += (int64_t)gridDim.x * blockDim.x) {
    int n = obj[o].n;
    int bin = LSP_HIST_BINS - 1 - (n < LSP_HIST_BINS - 1 ? n : LSP_HIST_BINS - 1);
    uint32_t pos = atomicAdd(&start[bin], 1u);
    order[pos] = (int32_t)o;
  }
}

}  // namespace

cudaError_t launch_stats(const double* t, const void* y, bool y64, const int64_t* offsets,
                         int64_t n_obj, int64_t total_nt, int center, int norm, ObjInfo* obj,
                         cudaStream_t stream, bool gls, const void* dy) {
  if (n_obj <= 0) return cudaSuccess;
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
