// lsp_probe.cu -- calibration probe of the FMA pipes (lsp_probe_fma_rates).
//
// The trig-sum kernels are bound by the FP32 FMA pipe (FP64 pipe for the
// FP64 path).  The roofline bound of the library is the nominal unit count,
// 128 FP32 lanes per SM per clock (2 FP64 FMA); this probe measures what the
// pipes deliver to a register-only stream of independent FMAs, which is the
// ceiling any real kernel sees.  The paper has no counterpart.
#include <cstdio>

#include "../../include/lsp.h"
#include "lsp_common.cuh"

namespace lsp {
void set_last_error(const char* msg);
}

namespace {

constexpr int kChains = 8;     // independent accumulation chains per thread
constexpr int kThreads = 256;  // per CTA
constexpr int kCtasPerSm = 8;  // 64 warps per SM: latency fully hidden

__global__ void __launch_bounds__(kThreads) probe_ffma(float* out, int iters) {
  float a[kChains];
  for (int i = 0; i < kChains; ++i) a[i] = threadIdx.x * 1e-3f + i;
  const float b = 0.999f, c = 1e-4f;
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], b, c);
  float s = 0.f;
  for (int i = 0; i < kChains; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) probe_ffma2(float* out, int iters) {
  lsp::f2_t a[kChains];
  for (int i = 0; i < kChains; ++i) a[i] = lsp::f2_pack(threadIdx.x * 1e-3f + i, (float)i);
  const lsp::f2_t b = lsp::f2_pack(0.999f, 0.998f), c = lsp::f2_pack(1e-4f, 2e-4f);
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = lsp::f2_fma(a[i], b, c);
  float s = 0.f;
  for (int i = 0; i < kChains; ++i) {
    float lo, hi;
    lsp::f2_unpack(a[i], lo, hi);
    s += lo + hi;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) probe_dfma(float* out, int iters) {
  double a[kChains];
  for (int i = 0; i < kChains; ++i) a[i] = threadIdx.x * 1e-3 + i;
  const double b = 0.999, c = 1e-4;
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
  double s = 0.0;
  for (int i = 0; i < kChains; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

// Lane operations per second of one probe: a short warm launch, then a timed
// launch of `iters` iterations bracketed by events on `stream`.
template <typename Kern>
cudaError_t rate(Kern kern, int blocks, int iters, int lanes_per_fma, float* out, cudaStream_t stream,
                 cudaEvent_t e0, cudaEvent_t e1, double* per_s) {
  kern<<<blocks, kThreads, 0, stream>>>(out, 16);
  cudaEventRecord(e0, stream);
  kern<<<blocks, kThreads, 0, stream>>>(out, iters);
  cudaEventRecord(e1, stream);
  cudaError_t e = cudaEventSynchronize(e1);
  if (e != cudaSuccess) return e;
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  float ms = 0.f;
  e = cudaEventElapsedTime(&ms, e0, e1);
  if (e != cudaSuccess) return e;
  *per_s = (double)blocks * kThreads * iters * kChains * lanes_per_fma / (ms * 1e-3);
  return cudaSuccess;
}

}  // namespace

extern "C" lsp_status lsp_probe_fma_rates(double* f32_per_s, double* f32x2_per_s, double* f64_per_s,
                                          lsp_stream_t stream_) {
  cudaStream_t stream = (cudaStream_t)stream_;
  int dev = 0, n_sm = 0;
  char msg[160];
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = n_sm * kCtasPerSm;
  float* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  // one float per thread of the probe grid
  if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(float) * (size_t)blocks * kThreads);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  double r32 = 0.0, r2 = 0.0, r64 = 0.0;
  if (e == cudaSuccess) e = rate(probe_ffma, blocks, 4000, 1, out, stream, e0, e1, &r32);
  if (e == cudaSuccess) e = rate(probe_ffma2, blocks, 4000, 2, out, stream, e0, e1, &r2);
  if (e == cudaSuccess) e = rate(probe_dfma, blocks, 100, 1, out, stream, e0, e1, &r64);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  if (e != cudaSuccess) {
    snprintf(msg, sizeof msg, "lsp_probe_fma_rates: %s", cudaGetErrorString(e));
    lsp::set_last_error(msg);
    return LSP_E_CUDA;
  }
  if (f32_per_s) *f32_per_s = r32;
  if (f32x2_per_s) *f32x2_per_s = r2;
  if (f64_per_s) *f64_per_s = r64;
  return LSP_OK;
}

// ------------------------------------------------------------------------
// Accuracy probe of sincos_fixed64 (the FP64 seeds' sin/cos): n phases from a
// counter-based hash (splitmix64 of seed + i, so every bit pattern can occur,
// plus the 256 table points and their neighbours), each evaluated both ways;
// the largest |difference| of cos and of sin against CUDA's sincospi.
namespace {

__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void probe_sincos_kernel(int64_t n, uint64_t seed, unsigned long long* max_bits) {
  __shared__ unsigned long long sh[32];
  double worst = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t ph;
    if (i < 768) {  // the table points and their neighbours
      ph = ((uint64_t)(i / 3) << 56) + (uint64_t)(i % 3) - 1ull;
    } else {
      ph = splitmix64(seed + (uint64_t)i);
    }
    double c, s, cr, sr;
    lsp::sincos_fixed64(ph, c, s);
    const double x = (double)(int64_t)ph * 5.421010862427522e-20;  // cycles in [-1/2, 1/2)
    sincospi(2.0 * x, &sr, &cr);
    worst = fmax(worst, fmax(fabs(c - cr), fabs(s - sr)));
  }
  unsigned long long m = (unsigned long long)__double_as_longlong(worst);
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, m, off);
    m = o > m ? o : m;
  }
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = sh[w] > m ? sh[w] : m;
    atomicMax(max_bits, m);
  }
}

}  // namespace

extern "C" lsp_status lsp_probe_sincos_fixed64(int64_t n, uint64_t seed, double* max_abs_err, lsp_stream_t stream_) {
  cudaStream_t stream = (cudaStream_t)stream_;
  if (n < 1 || !max_abs_err) {
    lsp::set_last_error("lsp_probe_sincos_fixed64: n must be >= 1 and max_abs_err not NULL");
    return LSP_E_ARG;
  }
  unsigned long long* d = nullptr;
  unsigned long long h = 0ull;
  cudaError_t e = cudaMalloc(&d, sizeof h);
  if (e == cudaSuccess) e = cudaMemsetAsync(d, 0, sizeof h, stream);
  if (e == cudaSuccess) {
    probe_sincos_kernel<<<1024, 256, 0, stream>>>(n, seed, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof h, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (d) cudaFree(d);
  if (e != cudaSuccess) {
    char msg[160];
    snprintf(msg, sizeof msg, "lsp_probe_sincos_fixed64: %s", cudaGetErrorString(e));
    lsp::set_last_error(msg);
    return LSP_E_CUDA;
  }
  *max_abs_err = __builtin_bit_cast(double, h);
  return LSP_OK;
}
