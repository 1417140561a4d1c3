// lsp_post.cu -- split-N_t combine, per-object peaks, stored-periodogram argmax.
#include <cmath>
#include <type_traits>

#include "../../include/lsp.h"
#include "lsp_launch.h"

namespace lsp {

bool main_variant_exists_f32(int packed, int k, int fpt, int gls, int abl);
bool main_variant_exists_f64(int k, int fpt, int gls);
int main_blocks_per_sm_f32(int packed, int k, int fpt, int threads, int top, int gls, int abl);
int main_blocks_per_sm_f64(int k, int fpt, int threads, int top, int gls);
cudaError_t launch_main_f32(const MainLaunch& ml, cudaStream_t stream);
cudaError_t launch_main_f64(const MainLaunch& ml, cudaStream_t stream);

size_t main_dyn_smem(int prec, int fpt, int threads, int top) {
  // FP32: one padding word per thread (chunk_results_f32)
  return top ? (size_t)threads * (prec ? fpt * sizeof(double) : (fpt + 1) * sizeof(float)) : 0;
}

bool main_variant_exists(int prec, int packed, int k, int fpt, int gls, int abl) {
  return prec ? (!packed && !abl && main_variant_exists_f64(k, fpt, gls))
              : main_variant_exists_f32(packed, k, fpt, gls, abl);
}

int main_blocks_per_sm(int prec, int packed, int k, int fpt, int threads, int top, int gls, int abl) {
  if (!main_variant_exists(prec, packed, k, fpt, gls, abl)) return 0;
  return prec ? main_blocks_per_sm_f64(k, fpt, threads, top, gls)
              : main_blocks_per_sm_f32(packed, k, fpt, threads, top, gls, abl);
}

cudaError_t launch_main(const MainLaunch& ml, cudaStream_t stream) {
  return ml.prec ? launch_main_f64(ml, stream) : launch_main_f32(ml, stream);
}

namespace {

__device__ __forceinline__ lsp_peak make_peak(int64_t k, double p, double f_min, double df,
                                              int flags) {
  lsp_peak pk;
  pk.flags = flags;
  pk.reserved = 0;
  if (flags || k < 0) {
    pk.idx = -1;
    pk.power = 0.0;
    pk.freq = 0.0;
    pk.period = 0.0;
  } else {
    pk.idx = k;
    pk.power = p;
    pk.freq = __dadd_rn(f_min, __dmul_rn((double)k, df));  // f_min + k df, two roundings
    pk.period = 1.0 / pk.freq;
  }
  return pk;
}

// ------------------------------------------------------------- combine
// Split-N_t single object: sum the S partial sums of each frequency in the
// fixed order s = 0..S-1 (deterministic), then Eq. 2 and the chunk results.
// With peaks (first maximum only), the last CTA to finish (ticket, zero on
// entry) also reduces all chunk results in index order and writes the peak,
// so no separate finalize launch follows.  GLS: the six weighted sums of the
// generalized periodogram (Section 4.11) in stride-8 slots, and its power.
template <typename Real, bool GLS>
__global__ void __launch_bounds__(kCombineThreads) combine_kernel(
    const Real* __restrict__ part, int split, int64_t n_f, const ObjInfo* __restrict__ obj,
    const RecF32* __restrict__ rec, Real* __restrict__ power_out, ChunkBest* __restrict__ best,
    ChunkCand* __restrict__ cand, lsp_peak* __restrict__ peaks, double f_min, double df,
    uint32_t* __restrict__ ticket) {
  constexpr int NP = kCombinePerThread;
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  Real* s_pw = reinterpret_cast<Real*>(dyn_smem);
  __shared__ double red_p[32];
  __shared__ int64_t red_k[32];
  const ObjInfo oi = obj[0];
  const int64_t kc0 = (int64_t)blockIdx.x * blockDim.x * NP;
  const int64_t k0 = kc0 + (int64_t)threadIdx.x * NP;
  const Real nf = (Real)oi.n, scale = (Real)oi.norm_scale;
  Real pv[NP];
  uint32_t bad = 0u;
#pragma unroll
  for (int m = 0; m < NP; ++m) {
    const int64_t k = k0 + m;
    if constexpr (GLS) {
      Real v[6] = {0, 0, 0, 0, 0, 0};
      if (k < n_f && !oi.flags) {
        for (int s = 0; s < split; ++s) {
          const Real* q = part + ((int64_t)s * n_f + k) * 8;
#pragma unroll
          for (int j = 0; j < 6; ++j) v[j] += q[j];
        }
      }
      bool ill;
      if constexpr (std::is_same<Real, float>::value) {
        pv[m] = oi.norm_scale_f * gls_power<float>(v[0], v[1], v[2], v[3], v[4], v[5], oi.wsum_f,
                                                   (float)oi.sum_y2, EpsRel<float>::v, ill);
        if (k < n_f && !oi.flags && ill) bad |= 1u << m;
      } else {
        pv[m] = oi.norm_scale * gls_power<double>(v[0], v[1], v[2], v[3], v[4], v[5], oi.wsum, oi.sum_y2,
                                                  EpsRel<double>::v, ill);
      }
      continue;
    }
    Real xc = 0, xs = 0, cc = 0, cs = 0;
    if (k < n_f && !oi.flags) {
      for (int s = 0; s < split; ++s) {
        const Real* q = part + ((int64_t)s * n_f + k) * 4;
        xc += q[0];
        xs += q[1];
        cc += q[2];
        cs += q[3];
      }
    }
    if constexpr (std::is_same<Real, float>::value) {
      bool ill;
      pv[m] = oi.flags ? 0.0f : oi.norm_scale_f * lsp_power_f32(xc, xs, cc, cs, nf, ill);
      if (k < n_f && !oi.flags && ill) bad |= 1u << m;
    } else {
      pv[m] = oi.flags ? Real(0) : scale * lsp_power<Real>(xc, xs, cc, cs, nf, EpsRel<Real>::v);
    }
  }
  if constexpr (std::is_same<Real, float>::value) {
    if constexpr (GLS)
      fix_ill_conditioned_gls<NP>(pv, bad, (uint32_t)k0, rec, oi);
    else
      fix_ill_conditioned<NP>(pv, bad, (uint32_t)k0, rec, oi.begin, oi.n, oi.norm_scale);
  }
  if (power_out) {
#pragma unroll
    for (int m = 0; m < NP; ++m)
      if (k0 + m < n_f) power_out[k0 + m] = pv[m];
  }
  if constexpr (std::is_same<Real, float>::value)
    chunk_results_f32<NP>(pv, (uint32_t)k0, kc0, n_f, best + blockIdx.x, cand ? cand + blockIdx.x : nullptr,
                          reinterpret_cast<float*>(s_pw), reinterpret_cast<unsigned long long*>(red_p));
  else
    chunk_results<Real, NP>(pv, k0, kc0, n_f, best + blockIdx.x, cand ? cand + blockIdx.x : nullptr,
                            s_pw, red_p, red_k);
  if (!peaks) return;
  __shared__ bool s_last;
  if (threadIdx.x == 0) {  // thread 0 wrote this CTA's chunk result
    __threadfence();
    s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // the whole last CTA merges the chunk results (first maximum: the larger
  // power, the lower bin on a tie, so the order of merging does not matter)
  double p = 0.0;
  int64_t k = -1;
  for (unsigned c = threadIdx.x; c < gridDim.x; c += blockDim.x) {
    const double bp = __ldcg(&best[c].p);
    const int64_t bk = __ldcg(&best[c].k);
    if (better(bp, bk, p, k)) {
      p = bp;
      k = bk;
    }
  }
  warp_best(p, k);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red_p[w] = p;
    red_k[w] = k;
  }
  __syncthreads();
  if (threadIdx.x >= 32) return;
  p = threadIdx.x < (blockDim.x >> 5) ? red_p[threadIdx.x] : 0.0;
  k = threadIdx.x < (blockDim.x >> 5) ? red_k[threadIdx.x] : -1;
  warp_best(p, k);
  if (threadIdx.x == 0) peaks[0] = make_peak(k, p, f_min, df, oi.flags);
}

// First maximum per object: one warp per object, lanes stride the chunks.
__global__ void finalize_top1(const ObjInfo* __restrict__ obj, const ChunkBest* __restrict__ best,
                              int64_t n_obj, int n_chunks, double f_min, double df,
                              lsp_peak* __restrict__ peaks) {
  const int64_t o = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (o >= n_obj) return;
  double p = 0.0;
  int64_t k = -1;
  for (int c = lane; c < n_chunks; c += 32) {
    const ChunkBest b = best[o * n_chunks + c];
    if (better(b.p, b.k, p, k)) {
      p = b.p;
      k = b.k;
    }
  }
  warp_best(p, k);
  if (lane == 0) peaks[o] = make_peak(k, p, f_min, df, obj[o].flags);
}

__device__ __forceinline__ void top_insert(double (&tp)[3], int64_t (&tk)[3], double p, int64_t k) {
  if (better(p, k, tp[0], tk[0])) {
    tp[2] = tp[1]; tk[2] = tk[1]; tp[1] = tp[0]; tk[1] = tk[0]; tp[0] = p; tk[0] = k;
  } else if (better(p, k, tp[1], tk[1])) {
    tp[2] = tp[1]; tk[2] = tk[1]; tp[1] = p; tk[1] = k;
  } else if (better(p, k, tp[2], tk[2])) {
    tp[2] = p; tk[2] = k;
  }
}

// Top-k local maxima per object: merge the chunks' interior candidates and
// resolve each chunk's first and last bin against its neighbour chunks.  A
// bin is a local maximum when P[k] > P[k-1] and P[k] >= P[k+1]; the grid
// ends compare with their one neighbour.
__global__ void finalize_topk(const ObjInfo* __restrict__ obj, const ChunkCand* __restrict__ cand,
                              int64_t n_obj, int n_chunks, int top_k, double f_min, double df,
                              lsp_peak* __restrict__ peaks) {
  const int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (o >= n_obj) return;
  const ChunkCand* cc = cand + o * n_chunks;
  double tp[3] = {0.0, 0.0, 0.0};
  int64_t tk[3] = {-1, -1, -1};
  const double lo_inf = -INFINITY;
  for (int c = 0; c < n_chunks; ++c) {
    const ChunkCand x = cc[c];
    if (x.nvalid <= 0) continue;
    for (int r = 0; r < 3; ++r)
      if (x.k[r] >= 0) top_insert(tp, tk, x.p[r], x.k[r]);
    const double next_first = (c + 1 < n_chunks && cc[c + 1].nvalid > 0) ? cc[c + 1].first[0] : lo_inf;
    const double prev_last = c > 0 ? cc[c - 1].last[0] : lo_inf;
    // first bin of the chunk
    {
      const double v = x.first[0];
      const double right = x.nvalid >= 2 ? x.first[1] : next_first;
      if (v > prev_last && v >= right) top_insert(tp, tk, v, x.k_first);
    }
    // last bin of the chunk
    if (x.nvalid >= 2) {
      const double v = x.last[0];
      if (v > x.last[1] && v >= next_first) top_insert(tp, tk, v, x.k_first + x.nvalid - 1);
    }
  }
  const int flags = obj[o].flags;
  for (int r = 0; r < top_k; ++r) peaks[o * top_k + r] = make_peak(tk[r], tp[r], f_min, df, flags);
}

// ------------------------------------------- argmax of a stored periodogram
// Section 3.3 computes the period with a separate reduction over the stored
// periodogram.  The reduction state lives in the output records: pass 1 takes
// the maximum of an order-preserving 64-bit key of each power (in the
// power field), pass 2 the minimum index attaining it (in the idx field).
__device__ __forceinline__ unsigned long long order_key(double v) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double key_value(unsigned long long key) {
  unsigned long long b = (key >> 63) ? (key & 0x7fffffffffffffffull) : ~key;
  return __longlong_as_double((long long)b);
}

__global__ void am_init(int64_t n_obj, lsp_peak* peaks) {
  const int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (o >= n_obj) return;
  lsp_peak pk;
  pk.idx = INT64_MAX;
  pk.power = __longlong_as_double(0);  // key 0: below every non-NaN value
  pk.freq = 0.0;
  pk.period = 0.0;
  pk.flags = 0;
  pk.reserved = 0;
  peaks[o] = pk;
}

template <typename Real>
__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long v, unsigned long long* sh) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    unsigned long long w = __shfl_xor_sync(0xffffffffu, v, off);
    v = w > v ? w : v;
  }
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  v = lane < nw ? sh[lane] : 0ull;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    unsigned long long w = __shfl_xor_sync(0xffffffffu, v, off);
    v = w > v ? w : v;
  }
  return v;
}

// grid: (row blocks, object slices); each CTA reduces a contiguous row range.
template <typename Real, int PASS>
__global__ void am_pass(const Real* __restrict__ power, int64_t n_obj, int64_t n_f, int64_t per_cta,
                        lsp_peak* peaks) {
  __shared__ unsigned long long sh[32];
  for (int64_t o = blockIdx.y; o < n_obj; o += gridDim.y) {
    const Real* row = power + o * n_f;
    const int64_t lo = (int64_t)blockIdx.x * per_cta;
    int64_t hi = lo + per_cta;
    if (hi > n_f) hi = n_f;
    unsigned long long* keyp = reinterpret_cast<unsigned long long*>(&peaks[o].power);
    if (PASS == 1) {
      unsigned long long best = 0ull;
      for (int64_t k = lo + threadIdx.x; k < hi; k += blockDim.x) {
        const double v = (double)row[k];
        if (!isnan(v)) {
          const unsigned long long key = order_key(v);
          best = key > best ? key : best;
        }
      }
      best = block_max_u64<Real>(best, sh);
      if (threadIdx.x == 0 && best) atomicMax(keyp, best);
    } else {
      const unsigned long long target = *keyp;
      unsigned long long mk = ~0ull;  // minimum index, as the max of its complement
      for (int64_t k = lo + threadIdx.x; k < hi; k += blockDim.x) {
        const double v = (double)row[k];
        if (!isnan(v) && order_key(v) == target) {
          mk = (unsigned long long)k < mk ? (unsigned long long)k : mk;
        }
      }
      unsigned long long inv = block_max_u64<Real>(~mk, sh);
      if (threadIdx.x == 0 && inv) atomicMin(reinterpret_cast<unsigned long long*>(&peaks[o].idx), ~inv);
    }
    __syncthreads();
  }
}

__global__ void am_decode(int64_t n_obj, double f_min, double df, lsp_peak* peaks) {
  const int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (o >= n_obj) return;
  lsp_peak pk = peaks[o];
  const unsigned long long key = (unsigned long long)__double_as_longlong(pk.power);
  if (pk.idx == INT64_MAX || key == 0ull) {
    peaks[o] = make_peak(-1, 0.0, f_min, df, 0);
    return;
  }
  peaks[o] = make_peak(pk.idx, key_value(key), f_min, df, 0);
}

__global__ void f32_to_f64_kernel(const float* __restrict__ a, double* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}

// max_i |a_i - b_i| into *out (a non-negative double updated through its bits).
__global__ void max_abs_diff_kernel(const float* __restrict__ a, const double* __restrict__ b, int64_t n,
                                    unsigned long long* out) {
  __shared__ unsigned long long sh[32];
  unsigned long long m = 0ull;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double d = fabs((double)a[i] - b[i]);
    if (isnan(d)) d = INFINITY;
    unsigned long long v = (unsigned long long)__double_as_longlong(d);
    m = v > m ? v : m;
  }
  m = block_max_u64<double>(m, sh);
  if (threadIdx.x == 0) atomicMax(out, m);
}

// Per row of n values: max_i |a_i - b_i| into out[row] (bits of a non-negative double).
__global__ void row_max_abs_diff_kernel(const float* __restrict__ a, const double* __restrict__ b, int64_t n,
                                        unsigned long long* out) {
  __shared__ unsigned long long sh[32];
  const int64_t row = blockIdx.y;
  const float* ar = a + row * n;
  const double* br = b + row * n;
  unsigned long long m = 0ull;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double d = fabs((double)ar[i] - br[i]);
    if (isnan(d)) d = INFINITY;
    const unsigned long long v = (unsigned long long)__double_as_longlong(d);
    m = v > m ? v : m;
  }
  m = block_max_u64<double>(m, sh);
  if (threadIdx.x == 0) atomicMax(out + row, m);
}

// Conditioning of Eq. 2's denominators for object i of a list: the largest
// R / N over the grid, R = |sum_j exp(2 pi i (2 f_k) t_j)| (the spectral
// window at twice the frequency).  Where R approaches N, one of the two
// tau-shifted sums of squares, (N - R)/2, is small and FP32 sums lose
// relative accuracy.  Phases are reduced in FP64 against the object's first
// time (R does not depend on the origin); sin/cos and the sums are FP32.
__global__ void window_score_kernel(const double* __restrict__ t, const int64_t* __restrict__ begin,
                                    const int64_t* __restrict__ count, double f_min, double df, int64_t n_f,
                                    unsigned int* __restrict__ score_bits) {
  __shared__ unsigned long long sh[32];
  const int i = blockIdx.y;
  const int64_t b = begin[i], n = count[i];
  const double t_ref = n > 0 ? t[b] : 0.0;
  float best = 0.0f;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_f; k += (int64_t)gridDim.x * blockDim.x) {
    const double f2 = 2.0 * (f_min + (double)k * df);
    float c = 0.0f, s = 0.0f;
    for (int64_t j = 0; j < n; ++j) {
      double ph = f2 * (t[b + j] - t_ref);
      ph -= rint(ph);
      float sj, cj;
      sincospif((float)(2.0 * ph), &sj, &cj);
      c += cj;
      s += sj;
    }
    const float r = n > 0 ? sqrtf(c * c + s * s) / (float)n : 0.0f;
    best = r > best ? r : best;
  }
  unsigned long long m = (unsigned long long)__float_as_uint(best);  // non-negative: bits order as values
  m = block_max_u64<double>(m, sh);
  if (threadIdx.x == 0) atomicMax(score_bits + i, (unsigned int)m);
}

}  // namespace

cudaError_t launch_row_max_abs_diff(const float* a, const double* b, int64_t rows, int64_t n, double* out,
                                    cudaStream_t stream) {
  if (rows <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(out, 0, (size_t)rows * sizeof(double), stream);
  if (e != cudaSuccess || n <= 0) return e;
  const int64_t per = (n + 255) / 256;
  dim3 grid((unsigned)(per < 128 ? per : 128), (unsigned)rows);
  row_max_abs_diff_kernel<<<grid, 256, 0, stream>>>(a, b, n, reinterpret_cast<unsigned long long*>(out));
  return cudaGetLastError();
}

cudaError_t launch_window_score(const double* t, const int64_t* begin, const int64_t* count, int n_list,
                                double f_min, double df, int64_t n_f, float* score, cudaStream_t stream) {
  if (n_list <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(score, 0, (size_t)n_list * sizeof(float), stream);
  if (e != cudaSuccess || n_f <= 0) return e;
  const int64_t per = (n_f + 255) / 256;
  dim3 grid((unsigned)(per < 64 ? per : 64), (unsigned)n_list);
  window_score_kernel<<<grid, 256, 0, stream>>>(t, begin, count, f_min, df, n_f,
                                                reinterpret_cast<unsigned int*>(score));
  return cudaGetLastError();
}

cudaError_t launch_f32_to_f64(const float* a, double* b, int64_t n, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  f32_to_f64_kernel<<<1024, 256, 0, stream>>>(a, b, n);
  return cudaGetLastError();
}

cudaError_t launch_max_abs_diff(const float* a, const double* b, int64_t n, double* out, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), stream);
  if (e != cudaSuccess || n <= 0) return e;
  max_abs_diff_kernel<<<512, 256, 0, stream>>>(a, b, n, reinterpret_cast<unsigned long long*>(out));
  return cudaGetLastError();
}

cudaError_t launch_combine(int prec, const void* part, int split, int64_t n_f, const ObjInfo* obj,
                           const void* rec, void* power_out, ChunkBest* best, ChunkCand* cand,
                           cudaStream_t stream, lsp_peak* peaks, double f_min, double df, uint32_t* ticket,
                           bool gls) {
  const int64_t per_cta = (int64_t)kCombineThreads * kCombinePerThread;
  const unsigned grid = (unsigned)((n_f + per_cta - 1) / per_cta);
  // chunk_results keeps the chunk's powers in shared memory (FP32: one
  // padding word per thread)
  const size_t dyn = cand ? (prec ? (size_t)per_cta * 8 : (size_t)kCombineThreads * (kCombinePerThread + 1) * 4) : 0;
  if (cand || !ticket) peaks = nullptr;  // top-k peaks: the separate finalize
  auto go = [&](auto kern, const auto* pt, const RecF32* r, auto* pw) {
    kern<<<grid, kCombineThreads, dyn, stream>>>(pt, split, n_f, obj, r, pw, best, cand, peaks, f_min, df,
                                                 ticket);
  };
  if (prec) {
    if (gls)
      go(combine_kernel<double, true>, (const double*)part, nullptr, (double*)power_out);
    else
      go(combine_kernel<double, false>, (const double*)part, nullptr, (double*)power_out);
  } else {
    if (gls)
      go(combine_kernel<float, true>, (const float*)part, (const RecF32*)rec, (float*)power_out);
    else
      go(combine_kernel<float, false>, (const float*)part, (const RecF32*)rec, (float*)power_out);
  }
  return cudaGetLastError();
}

cudaError_t launch_finalize(const ObjInfo* obj, const ChunkBest* best, const ChunkCand* cand,
                            int64_t n_obj, int n_chunks, int top_k, double f_min, double df,
                            lsp_peak* peaks, cudaStream_t stream) {
  if (n_obj <= 0 || peaks == nullptr) return cudaSuccess;
  if (top_k <= 1 || cand == nullptr) {
    const int64_t threads = 256, warps_per_cta = threads / 32;
    const unsigned grid = (unsigned)((n_obj + warps_per_cta - 1) / warps_per_cta);
    finalize_top1<<<grid, (unsigned)threads, 0, stream>>>(obj, best, n_obj, n_chunks, f_min, df, peaks);
  } else {
    const unsigned grid = (unsigned)((n_obj + 127) / 128);
    finalize_topk<<<grid, 128, 0, stream>>>(obj, cand, n_obj, n_chunks, top_k, f_min, df, peaks);
  }
  return cudaGetLastError();
}

cudaError_t launch_argmax_period(const void* power, bool p64, int64_t n_obj, int64_t n_f,
                                 double f_min, double df, lsp_peak* peaks, cudaStream_t stream) {
  if (n_obj <= 0) return cudaSuccess;
  const unsigned g1 = (unsigned)((n_obj + 255) / 256);
  am_init<<<g1, 256, 0, stream>>>(n_obj, peaks);
  const int threads = 256;
  int64_t per_cta = 8192;
  int64_t gx = (n_f + per_cta - 1) / per_cta;
  if (gx > 65535) {
    gx = 65535;
    per_cta = (n_f + gx - 1) / gx;
  }
  const unsigned gy = (unsigned)(n_obj < 65535 ? n_obj : 65535);
  dim3 grid((unsigned)gx, gy);
  if (p64) {
    am_pass<double, 1><<<grid, threads, 0, stream>>>((const double*)power, n_obj, n_f, per_cta, peaks);
    am_pass<double, 2><<<grid, threads, 0, stream>>>((const double*)power, n_obj, n_f, per_cta, peaks);
  } else {
    am_pass<float, 1><<<grid, threads, 0, stream>>>((const float*)power, n_obj, n_f, per_cta, peaks);
    am_pass<float, 2><<<grid, threads, 0, stream>>>((const float*)power, n_obj, n_f, per_cta, peaks);
  }
  am_decode<<<g1, 256, 0, stream>>>(n_obj, f_min, df, peaks);
  return cudaGetLastError();
}

}  // namespace lsp
