// lsp_learned.cu -- the learned-proposal stage: featurizer, MLP forward /
// backward / AdamW on the tensor cores, proposal of refinement windows, and
// the windowed refine + full-grid fallback built on the main kernel.
//
// The paper has no learned component.  The stage proposes, for each light
// curve, the grid windows most likely to hold the periodogram's maximum; the
// direct method then refines only those windows and falls back to the full
// grid when the refined peak is weak.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cuda_bf16.h>
#include <mutex>

#include "../../include/lsp.h"
#include "lsp_launch.h"
#include "lsp_umma.cuh"

namespace lsp {
void set_last_error(const char* msg);
}

using namespace lsp;

namespace {

typedef __nv_bfloat16 bf16;

lsp_status err_arg(const char* msg) {
  set_last_error(msg);
  return LSP_E_ARG;
}
lsp_status err_cuda(cudaError_t e, const char* what) {
  char buf[256];
  snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  set_last_error(buf);
  return LSP_E_CUDA;
}
#define LEARN_CUDA(call, what)                        \
  do {                                                \
    cudaError_t e__ = (call);                         \
    if (e__ != cudaSuccess) return err_cuda(e__, what); \
  } while (0)

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// =============================================================== featurizer
// One CTA of 256 threads per light curve.  For a time-sorted light curve each
// thread walks the band of observations after its own until the lag reaches
// lag_max, four candidates per step; otherwise all n^2 candidate pairs are
// scanned in flat blocks of 1024.  Pairs with |t_j - t_i| < lag_max go to a
// shared buffer in scan order (a block-wide prefix sum keeps the order, and so
// the float sums, deterministic).  Warp w then takes buffered pairs w, w + 8,
// ...; lane l adds w cos(2 pi f_c dt) of each to coarse bins 8l .. 8l + 7:
// two cosines from the SFU (bins 8l and 8l + 1, the second one grid step of
// phase after the first) and the other six from the three-term recurrence
// cos(x + d) = 2 cos(d) cos(x) - cos(x - d), whose error grows at most
// linearly over the six steps.  The eight warps' partial sums of each bin are
// added in warp order at the end.  The lag histogram counts pairs per lag
// bin.
constexpr int kFeatThreads = 256;
constexpr int kCoarse = 256;
constexpr int kLagBins = 256;
constexpr int kPairBlock = 4 * kFeatThreads;
constexpr int kBinsPerLane = kCoarse / 32;
static_assert(kBinsPerLane == 8, "the featurizer's lanes take eight coarse bins each");

__global__ void __launch_bounds__(kFeatThreads, 6) featurize_kernel(
    const double* __restrict__ t, const float* __restrict__ y, const int64_t* __restrict__ offsets,
    int64_t total_nt, double f_min, double f_max, float lag_max, bf16* __restrict__ feat16,
    float* __restrict__ feat32) {
  __shared__ float4 s_pair[kPairBlock];  // dt, weight, grid step of phase (cycles), 2 cos(step)
  __shared__ float s_part[kFeatThreads / 32][kCoarse];
  __shared__ uint32_t s_hist[kLagBins];
  __shared__ int s_scan[kFeatThreads / 32];
  __shared__ double s_red[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t o = blockIdx.x;
  int64_t b = offsets[o], e = offsets[o + 1];
  if (b < 0 || e < b || e > total_nt) b = e = 0;
  const int n = (int)(e - b);
  s_hist[tid] = 0u;
  // mean and rms of y (FP64)
  double sy = 0.0;
  for (int j = tid; j < n; j += kFeatThreads) sy += (double)y[b + j];
  for (int off = 16; off > 0; off >>= 1) sy += __shfl_xor_sync(0xffffffffu, sy, off);
  if (lane == 0) s_red[warp] = sy;
  __syncthreads();
  double tot = 0.0;
  for (int w = 0; w < kFeatThreads / 32; ++w) tot += s_red[w];
  const double mean = n > 0 ? tot / n : 0.0;
  __syncthreads();
  double s2 = 0.0;
  for (int j = tid; j < n; j += kFeatThreads) {
    const double d = (double)y[b + j] - mean;
    s2 += d * d;
  }
  for (int off = 16; off > 0; off >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, off);
  if (lane == 0) s_red[warp] = s2;
  __syncthreads();
  double var = 0.0;
  for (int w = 0; w < kFeatThreads / 32; ++w) var += s_red[w];
  var = n > 0 ? var / n : 0.0;
  const bool ok = n >= 2 && var > 0.0;
  const float rstd = ok ? (float)(1.0 / sqrt(var)) : 0.0f;
  constexpr float kTwoPi = 6.28318530717958647692f;
  const float fc0 = (float)(f_min + (kBinsPerLane * lane + 0.5) * (f_max - f_min) / kCoarse);
  const float dfc = (float)((f_max - f_min) / kCoarse);
  const float lag_scale = kLagBins / lag_max;
  float acc8[kBinsPerLane];
#pragma unroll
  for (int k = 0; k < kBinsPerLane; ++k) acc8[k] = 0.0f;
  uint32_t n_pairs = 0u;
  // time-sorted light curves (the usual case) only need the short-lag band
  // after each observation; others are scanned over all n^2 candidates
  int unsorted = 0;
  for (int j = tid + 1; j < n; j += kFeatThreads) unsorted |= t[b + j] < t[b + j - 1];
  const bool sorted = !__syncthreads_or(unsorted);

  // Buffers the (up to four) pairs each thread found, in flat order, then
  // adds every buffered pair to this thread's coarse bin.
  auto flush = [&](int cnt, const float (&dt)[4], const float (&w)[4]) {
    int incl = cnt;
    for (int off = 1; off < 32; off <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += v;
    }
    if (lane == 31) s_scan[warp] = incl;
    __syncthreads();
    int wbase = 0, total = 0;
    for (int ww = 0; ww < kFeatThreads / 32; ++ww) {
      if (ww < warp) wbase += s_scan[ww];
      total += s_scan[ww];
    }
    const int at = wbase + incl - cnt;
    for (int q = 0; q < cnt; ++q) {
      const float pb = dfc * dt[q];  // one grid step of phase, cycles
      const float step = pb - rintf(pb);
      s_pair[at + q] = make_float4(dt[q], w[q], step, 2.0f * __cosf(kTwoPi * step));
      int lb = (int)(dt[q] * lag_scale);
      lb = lb < kLagBins - 1 ? lb : kLagBins - 1;
      atomicAdd(&s_hist[lb], 1u);
    }
    __syncthreads();
    for (int q = warp; q < total; q += kFeatThreads / 32) {
      const float4 pr = s_pair[q];
      const float ph = fc0 * pr.x;  // cycles; |ph| < 12 * 16
      const float x0 = ph - rintf(ph);
      float x1 = x0 + pr.z;
      x1 -= rintf(x1);
      float cm = __cosf(kTwoPi * x0), c = __cosf(kTwoPi * x1);
      acc8[0] = fmaf(pr.y, cm, acc8[0]);
      acc8[1] = fmaf(pr.y, c, acc8[1]);
#pragma unroll
      for (int k = 2; k < kBinsPerLane; ++k) {
        const float cn = fmaf(pr.w, c, -cm);
        cm = c;
        c = cn;
        acc8[k] = fmaf(pr.y, c, acc8[k]);
      }
    }
    n_pairs += (uint32_t)total;
    __syncthreads();
  };
  auto pair_of = [&](int i, int j, float (&dt)[4], float (&w)[4], int& cnt) {
    const double d = fabs(t[b + j] - t[b + i]);
    if (d < (double)lag_max) {
      dt[cnt] = (float)d;
      w[cnt] = (float)(((double)y[b + i] - mean) * ((double)y[b + j] - mean)) * rstd * rstd;
      ++cnt;
    }
    return d;
  };

  if (ok && sorted) {
    for (int ib = 0; ib < n; ib += kFeatThreads) {
      const int i = ib + tid;
      bool more = true;
      for (int q = 0;; ++q) {
        float dt[4] = {0.f, 0.f, 0.f, 0.f}, w[4] = {0.f, 0.f, 0.f, 0.f};
        int cnt = 0;
        if (i < n && more) {
          for (int r = 0; r < 4; ++r) {
            const int j = i + 1 + 4 * q + r;
            if (j >= n || pair_of(i, j, dt, w, cnt) >= (double)lag_max) {
              more = false;
              break;
            }
          }
        } else {
          more = false;
        }
        flush(cnt, dt, w);
        if (!__syncthreads_or(more)) break;
      }
    }
  } else if (ok) {
    const int64_t n_cand = (int64_t)n * n;
    for (int64_t base = 0; base < n_cand; base += kPairBlock) {
      float dt[4] = {0.f, 0.f, 0.f, 0.f}, w[4] = {0.f, 0.f, 0.f, 0.f};
      int cnt = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t flat = base + (int64_t)tid * 4 + q;
        if (flat < n_cand) {
          const int i = (int)(flat / n), j = (int)(flat % n);
          if (j > i) pair_of(i, j, dt, w, cnt);
        }
      }
      flush(cnt, dt, w);
    }
  }
#pragma unroll
  for (int k = 0; k < kBinsPerLane; ++k) s_part[warp][kBinsPerLane * lane + k] = acc8[k];
  __syncthreads();
  float acc = 0.0f;
  for (int ww = 0; ww < kFeatThreads / 32; ++ww) acc += s_part[ww][tid];
  const float f_c = ok ? acc / (float)(n_pairs + 1u) : 0.0f;
  const float f_l = ok ? log1pf((float)s_hist[tid]) : 0.0f;
  feat16[o * LSP_FEAT_DIM + tid] = __float2bfloat16_rn(f_c);
  feat16[o * LSP_FEAT_DIM + kCoarse + tid] = __float2bfloat16_rn(f_l);
  if (feat32) {
    feat32[o * LSP_FEAT_DIM + tid] = f_c;
    feat32[o * LSP_FEAT_DIM + kCoarse + tid] = f_l;
  }
}

// ===================================================================== GEMM
// The network's products run on the tcgen05 tensor cores (lsp_umma.cuh):
// C[M, N] = A[M, K] B[N, K]^T with both operands K-contiguous bfloat16, read
// by TMA through tensor maps encoded here.  The forward pass multiplies the
// activations by the transposed weights (prepared once per call), the input
// gradient multiplies dZ by the weights, and the weight gradient multiplies
// the transposed activations by the transposed dZ (both written in that
// layout by the producing kernels), split over K = batch with a fixed-order
// reduction of the partial tiles.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    cudaGetLastError();
  });
  return fn;
}

int64_t ld8(int64_t n) { return (n + 7) / 8 * 8; }  // row pitch (elements) of a TMA-read bfloat16 matrix

// rows x k bfloat16 matrix, K contiguous, pitch ld elements: boxes of
// box_rows rows x 64 K-elements with the 128-byte swizzle.
lsp_status make_map(CUtensorMap* map, const bf16* base, int64_t rows, int64_t k, int64_t ld, int box_rows,
                    const char* what) {
  EncodeTiledFn enc = encode_tiled();
  if (!enc) {
    set_last_error("cuTensorMapEncodeTiled is not available from the driver");
    return LSP_E_CUDA;
  }
  if (((uintptr_t)base) % 16 || (ld * 2) % 16 || ld < k) {
    char buf[200];
    snprintf(buf, sizeof buf, "%s: operand not 16-byte aligned or its row pitch not a multiple of 8 elements", what);
    set_last_error(buf);
    return LSP_E_ARG;
  }
  cuuint64_t dims[2] = {(cuuint64_t)k, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {(cuuint32_t)umma::BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    char buf[200];
    snprintf(buf, sizeof buf, "%s: cuTensorMapEncodeTiled failed (%d)", what, (int)r);
    set_last_error(buf);
    return LSP_E_CUDA;
  }
  return LSP_OK;
}

struct Gemm {
  int M, N, K;
  const bf16* A;  // [M][lda], K contiguous
  int64_t lda;
  const bf16* B;  // [N][ldb], K contiguous
  int64_t ldb;
  const float* bias;
  int relu;
  const bf16* mask;
  int64_t ldm;
  float* C32;
  int64_t ldc32;
  bf16* C16;
  int64_t ldc16;
  bf16* C16T;
  int64_t ldt;
  int splits;     // K split: partial FP32 tiles at part + z M N (pitch N), summed into C32 in order of z
  float* part;
};

// Split count for a weight-gradient GEMM: about one CTA per SM, at most
// kMaxSplits partial tiles.
constexpr int kMaxSplits = 16;

int k_splits(int M, int N, int K) {
  const int tiles = ((M + umma::BM - 1) / umma::BM) * ((N + umma::MAX_BN - 1) / umma::MAX_BN);
  const int kb = (K + umma::BK - 1) / umma::BK;
  int s = 148 / (tiles > 0 ? tiles : 1);
  s = s < 1 ? 1 : (s > kMaxSplits ? kMaxSplits : s);
  return s < kb ? s : kb;
}

__global__ void splitk_reduce_kernel(const float* __restrict__ part, int splits, int64_t mn, int n,
                                     float* __restrict__ out, int64_t ldo) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < mn; i += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int z = 0; z < splits; ++z) s += part[z * mn + i];
    out[(i / n) * ldo + i % n] = s;
  }
}

// dst[c][r] = src[r][c] for a rows x cols bfloat16 matrix (32 x 32 tiles).
__global__ void transpose_bf16_kernel(const bf16* __restrict__ src, int64_t rows, int64_t cols, int64_t lds,
                                      bf16* __restrict__ dst, int64_t ldd) {
  __shared__ bf16 tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32, c0 = (int64_t)blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t r = r0 + i, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[i][threadIdx.x] = src[r * lds + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t c = c0 + i, r = r0 + threadIdx.x;
    if (c < cols && r < rows) dst[c * ldd + r] = tile[threadIdx.x][i];
  }
}

// dst[r][c] = src[r][c] with a new row pitch.
__global__ void repitch_bf16_kernel(const bf16* __restrict__ src, int64_t rows, int64_t cols, int64_t lds,
                                    bf16* __restrict__ dst, int64_t ldd) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows * cols;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[(i / cols) * ldd + i % cols] = src[(i / cols) * lds + i % cols];
}

cudaError_t transpose_bf16(const bf16* src, int64_t rows, int64_t cols, int64_t lds, bf16* dst, int64_t ldd,
                           cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  dim3 grid((unsigned)((rows + 31) / 32), (unsigned)((cols + 31) / 32));
  transpose_bf16_kernel<<<grid, dim3(32, 8), 0, s>>>(src, rows, cols, lds, dst, ldd);
  return cudaGetLastError();
}

cudaError_t repitch_bf16(const bf16* src, int64_t rows, int64_t cols, int64_t lds, bf16* dst, int64_t ldd,
                         cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  repitch_bf16_kernel<<<1024, 256, 0, s>>>(src, rows, cols, lds, dst, ldd);
  return cudaGetLastError();
}

// Shared-memory attributes of the GEMM kernel, once per device: its dynamic
// size, and the largest carveout so that two CTAs share an SM.
lsp_status gemm_attributes() {
  static std::mutex mu;
  static uint64_t done_mask = 0;
  int dev = 0;
  LEARN_CUDA(cudaGetDevice(&dev), "GEMM device");
  std::lock_guard<std::mutex> lk(mu);
  if (dev >= 0 && dev < 64 && (done_mask >> dev) & 1u) return LSP_OK;
  LEARN_CUDA(cudaFuncSetAttribute(umma::gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, umma::SMEM_BYTES),
             "GEMM shared memory");
  LEARN_CUDA(cudaFuncSetAttribute(umma::gemm_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  cudaSharedmemCarveoutMaxShared),
             "GEMM shared-memory carveout");
  if (dev >= 0 && dev < 64) done_mask |= (uint64_t)1 << dev;
  return LSP_OK;
}

lsp_status gemm(const Gemm& q, cudaStream_t s) {
  if (q.M <= 0 || q.N <= 0 || q.K <= 0) return LSP_OK;
  const int n_tile = q.N >= umma::MAX_BN ? umma::MAX_BN : (q.N + 15) / 16 * 16;
  CUtensorMap ma, mb;
  lsp_status st = make_map(&ma, q.A, q.M, q.K, q.lda, umma::BM, "GEMM operand A");
  if (st) return st;
  if ((st = make_map(&mb, q.B, q.N, q.K, q.ldb, n_tile, "GEMM operand B"))) return st;
  const int kb = (q.K + umma::BK - 1) / umma::BK;
  int splits = q.splits < 1 ? 1 : q.splits;
  const int kb_per = (kb + splits - 1) / splits;
  splits = (kb + kb_per - 1) / kb_per;  // every split gets at least one K slice
  umma::Args a;
  memset(&a, 0, sizeof a);
  a.M = q.M;
  a.N = q.N;
  a.K = q.K;
  a.n_tile = n_tile;
  a.kb_per_split = kb_per;
  a.bias = q.bias;
  a.relu = q.relu;
  a.mask = q.mask;
  a.ldm = q.ldm;
  a.C16 = q.C16;
  a.ldc16 = q.ldc16;
  a.C16T = q.C16T;
  a.ldt = q.ldt;
  if (splits > 1) {
    if (!q.part || q.bias || q.relu || q.mask || q.C16 || q.C16T || !q.C32) {
      set_last_error("GEMM: a split product takes an FP32 output only");
      return LSP_E_ARG;
    }
    a.C32 = q.part;
    a.ldc32 = q.N;
    a.split_stride = (int64_t)q.M * q.N;
  } else {
    a.C32 = q.C32;
    a.ldc32 = q.ldc32;
  }
  if ((st = gemm_attributes())) return st;
  dim3 grid((unsigned)((q.M + umma::BM - 1) / umma::BM), (unsigned)((q.N + n_tile - 1) / n_tile), (unsigned)splits);
  umma::gemm_kernel<<<grid, umma::THREADS, umma::SMEM_BYTES, s>>>(ma, mb, a);
  LEARN_CUDA(cudaGetLastError(), "GEMM launch");
  if (splits > 1) {
    const int64_t mn = (int64_t)q.M * q.N;
    splitk_reduce_kernel<<<(unsigned)((mn + 255) / 256 < 1024 ? (mn + 255) / 256 : 1024), 256, 0, s>>>(
        q.part, splits, mn, q.N, q.C32, q.ldc32);
    LEARN_CUDA(cudaGetLastError(), "GEMM split reduction");
  }
  return LSP_OK;
}

// ============================================ loss, reductions, optimizer
// One warp per row: mean softmax cross-entropy terms and dZ = (softmax -
// onehot) / batch in bf16 (row pitch ldz).
__global__ void xent_kernel(const float* __restrict__ logits, const int32_t* __restrict__ labels,
                            int64_t batch, int n_cls, float* __restrict__ row_loss,
                            bf16* __restrict__ dz, int64_t ldz) {
  const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= batch) return;
  const float* z = logits + r * n_cls;
  float m = -INFINITY;
  for (int c = lane; c < n_cls; c += 32) m = fmaxf(m, z[c]);
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
  float s = 0.0f;
  for (int c = lane; c < n_cls; c += 32) s += expf(z[c] - m);
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  int lab = labels[r];
  lab = lab < 0 ? 0 : (lab >= n_cls ? n_cls - 1 : lab);
  const float inv_b = 1.0f / (float)batch;
  for (int c = lane; c < n_cls; c += 32) {
    const float p = expf(z[c] - m) / s;
    dz[r * ldz + c] = __float2bfloat16_rn((p - (c == lab ? 1.0f : 0.0f)) * inv_b);
  }
  if (lane == 0) row_loss[r] = logf(s) + m - z[lab];
}

// Deterministic mean of n values (one CTA).
__global__ void mean_kernel(const float* __restrict__ v, int64_t n, float* out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += (double)v[i];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    *out = (float)(t / (double)(n > 0 ? n : 1));
  }
}

// Row sums of a bf16 [rows x cols] matrix of row pitch ld: the bias
// gradients from the transposed dZ (features x batch).  One warp per row,
// lanes along it, a fixed shuffle tree: the same order on every call.
__global__ void rowsum_kernel(const bf16* __restrict__ m, int rows, int64_t cols, int64_t ld,
                              float* __restrict__ out) {
  const int row = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= rows) return;
  float s = 0.0f;
  for (int64_t c = lane; c < cols; c += 32) s += __bfloat162float(m[row * ld + c]);
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) out[row] = s;
}

__global__ void adamw_kernel(int64_t n, float* __restrict__ p, bf16* __restrict__ p16,
                             const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                             float lr, float b1, float b2, float eps, float wd, float bc1, float bc2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float upd = (mi / bc1) / (sqrtf(vi / bc2) + eps) + wd * p[i];
    const float pi = p[i] - lr * upd;
    p[i] = pi;
    p16[i] = __float2bfloat16_rn(pi);
  }
}

__global__ void to_bf16_kernel(int64_t n, const float* __restrict__ a, bf16* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = __float2bfloat16_rn(a[i]);
}

// Top-k classes per row of logits (k <= 16), ties to the lower class.
__global__ void topk_kernel(const float* __restrict__ logits, int64_t rows, int n_cls, int k,
                            int32_t* __restrict__ out) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= rows) return;
  float tv[16];
  int tc[16];
  for (int i = 0; i < k; ++i) {
    tv[i] = -INFINITY;
    tc[i] = -1;
  }
  const float* z = logits + r * n_cls;
  for (int c = 0; c < n_cls; ++c) {
    const float v = z[c];
    if (tc[k - 1] >= 0 && !(v > tv[k - 1])) continue;
    int at = k - 1;
    while (at > 0 && (tc[at - 1] < 0 || v > tv[at - 1])) {
      tv[at] = tv[at - 1];
      tc[at] = tc[at - 1];
      --at;
    }
    tv[at] = v;
    tc[at] = c;
  }
  for (int i = 0; i < k; ++i) out[r * k + i] = tc[i];
}

// Window class of each object's full-grid first maximum: the training label.
__global__ void labels_kernel(const lsp_peak* __restrict__ peaks, int64_t n_obj, int64_t stride, int n_cls,
                              int32_t* __restrict__ labels) {
  const int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (o >= n_obj) return;
  const int64_t k = peaks[o].idx;
  int64_t c = k > 0 ? k / stride : 0;
  labels[o] = (int32_t)(c < n_cls ? c : n_cls - 1);
}

// ===================================================== refine + fallback
// Per-object refinement state (in the workspace).
struct RefineState {
  double best_p;    // best refined power so far
  int64_t best_k;   // its bin (-1: none)
  int32_t rounds;   // windows evaluated
  int16_t active;   // still refining
  int16_t stopped;  // a window reached stop_power
};

// Full grid for objects whose refined peak is weak or, optionally, that
// evaluated every proposed window without reaching stop_power.
__device__ __forceinline__ bool needs_fallback(const RefineState& s, int flags, float fallback_power,
                                               int inconclusive) {
  return !flags && (s.best_p < (double)fallback_power || (inconclusive && !s.stopped));
}

// Window of class c: bins [c * stride + stride/2 - win/2, ... + win), moved
// inside the grid.
__device__ __forceinline__ int32_t window_start(int32_t c, int64_t stride, int64_t win, int64_t n_f) {
  int64_t s = (int64_t)c * stride + stride / 2 - win / 2;
  if (s + win > n_f) s = n_f - win;
  if (s < 0) s = 0;
  return (int32_t)s;
}

__global__ void refine_init(int64_t n_obj, const ObjInfo* __restrict__ obj, RefineState* st) {
  const int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (o >= n_obj) return;
  RefineState s;
  s.best_p = 0.0;
  s.best_k = -1;
  s.rounds = 0;
  s.active = obj[o].flags ? 0 : 1;
  s.stopped = 0;
  st[o] = s;
}

// List the active objects of round r and place their windows.
__global__ void refine_list(int64_t n_obj, int r, int k_win, const int32_t* __restrict__ classes,
                            int64_t stride, int64_t win, int64_t n_f, const RefineState* __restrict__ st,
                            int32_t* __restrict__ win_start, int32_t* __restrict__ list,
                            uint32_t* __restrict__ count) {
  const int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (o >= n_obj) return;
  if (!st[o].active) return;
  int32_t c = classes[o * k_win + r];
  if (c < 0) c = 0;
  win_start[o] = window_start(c, stride, win, n_f);
  const uint32_t at = atomicAdd(count, 1u);
  list[at] = (int32_t)o;
}

__global__ void refine_merge(int64_t n_obj, int r, int k_win, float stop_power,
                             const ChunkBest* __restrict__ round_best, RefineState* st) {
  const int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (o >= n_obj) return;
  RefineState s = st[o];
  if (!s.active) return;
  const ChunkBest b = round_best[o];
  if (b.k >= 0 && (b.p > s.best_p || (b.p == s.best_p && (s.best_k < 0 || b.k < s.best_k)))) {
    s.best_p = b.p;
    s.best_k = b.k;
  }
  s.rounds = r + 1;
  s.stopped = s.best_p >= (double)stop_power ? 1 : 0;
  s.active = (!s.stopped && r + 1 < k_win) ? 1 : 0;
  st[o] = s;
}

// Objects whose refined peak stays below fallback_power, and their item count.
__global__ void fallback_list(int64_t n_obj, float fallback_power, int inconclusive,
                              const ObjInfo* __restrict__ obj, const RefineState* __restrict__ st,
                              int32_t* __restrict__ list, uint32_t* __restrict__ count) {
  const int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (o >= n_obj) return;
  if (!needs_fallback(st[o], obj[o].flags, fallback_power, inconclusive)) return;
  const uint32_t at = atomicAdd(count, 1u);
  list[at] = (int32_t)o;
}

__global__ void items_from_count(const uint32_t* count, uint32_t per, uint32_t* items) {
  *items = *count * per;
}

__global__ void refine_finalize(int64_t n_obj, const ObjInfo* __restrict__ obj,
                                const RefineState* __restrict__ st, float fallback_power, int inconclusive,
                                const ChunkBest* __restrict__ full_best, int n_chunks, double f_min,
                                double df, lsp_peak* __restrict__ peaks, int32_t* __restrict__ info) {
  const int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (o >= n_obj) return;
  const RefineState s = st[o];
  const int flags = obj[o].flags;
  double p = s.best_p;
  int64_t k = s.best_k;
  const bool fb = needs_fallback(s, flags, fallback_power, inconclusive);
  if (fb) {  // full grid: first maximum over the chunks
    p = 0.0;
    k = -1;
    for (int c = 0; c < n_chunks; ++c) {
      const ChunkBest b = full_best[o * n_chunks + c];
      if (b.k >= 0 && (k < 0 || b.p > p || (b.p == p && b.k < k))) {
        p = b.p;
        k = b.k;
      }
    }
  }
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
    pk.freq = __dadd_rn(f_min, __dmul_rn((double)k, df));
    pk.period = 1.0 / pk.freq;
  }
  peaks[o] = pk;
  if (info) info[o] = s.rounds | (fb ? LSP_REFINE_FALLBACK : 0);
}

// Flat parameter layout (see lsp.h): W1, b1, W2, b2, ..., W_L, b_L.
struct Layers {
  int n;
  int in[8], out[8];
  int64_t w_off[8], b_off[8];
  int64_t total;
};

lsp_status make_layers(const lsp_mlp_dims* d, Layers* L) {
  if (!d || d->in_dim < 1 || d->hidden < 1 || d->n_hidden < 1 || d->n_hidden > 6 || d->n_classes < 1)
    return err_arg("bad MLP dimensions");
  L->n = d->n_hidden + 1;
  int64_t at = 0;
  for (int l = 0; l < L->n; ++l) {
    L->in[l] = l == 0 ? d->in_dim : d->hidden;
    L->out[l] = l + 1 == L->n ? d->n_classes : d->hidden;
    L->w_off[l] = at;
    at += (int64_t)L->in[l] * L->out[l];
    L->b_off[l] = at;
    at += L->out[l];
  }
  L->total = at;
  return LSP_OK;
}

// MLP scratch.  bfloat16 matrices the GEMMs read through TMA have row
// pitches rounded up to 8 elements (16 bytes).
//   wt[l]  (out x in)  transposed weights: forward B operand
//   act[l] (batch x out) hidden activations; logits (batch x n_cls, FP32)
//   xin    (batch x in) padded copy of the input when in_dim % 8 != 0
// training only:
//   wp[l]  (in x out)  weights at a padded pitch: input-gradient B operand
//   xT, actT[l] (features x batch) transposed inputs / activations and
//   dzT[2] (features x batch) transposed dZ: weight-gradient operands
//   dz[2]  (batch x width) dZ of the current and the previous layer
//   part   split-K partial weight-gradient tiles; row_loss (batch)
struct MlpWs {
  bf16* wt[8];
  bf16* act[8];
  float* logits;
  bf16* xin;
  bf16* wp[8];
  bf16* xT;
  bf16* actT[8];
  bf16* dz[2];
  bf16* dzT[2];
  float* part;
  float* row_loss;
  int64_t ldb;  // pitch of the transposed (features x batch) matrices
  size_t total;
};

void mlp_ws_layout(const Layers& L, int64_t batch, bool training, char* base, MlpWs* w) {
  memset(w, 0, sizeof *w);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* at = base ? base + off : nullptr;
    off = align256(off + bytes);
    return at;
  };
  int maxw = 0;
  int64_t max_mn = 0;
  for (int l = 0; l < L.n; ++l) {
    maxw = L.out[l] > maxw ? L.out[l] : maxw;
    max_mn = (int64_t)L.in[l] * L.out[l] > max_mn ? (int64_t)L.in[l] * L.out[l] : max_mn;
  }
  w->ldb = ld8(batch);
  for (int l = 0; l < L.n; ++l) w->wt[l] = (bf16*)take((size_t)L.out[l] * ld8(L.in[l]) * sizeof(bf16));
  for (int l = 0; l + 1 < L.n; ++l) w->act[l] = (bf16*)take((size_t)batch * ld8(L.out[l]) * sizeof(bf16));
  w->logits = (float*)take((size_t)batch * L.out[L.n - 1] * sizeof(float));
  if (L.in[0] % 8) w->xin = (bf16*)take((size_t)batch * ld8(L.in[0]) * sizeof(bf16));
  if (training) {
    for (int l = 1; l < L.n; ++l) w->wp[l] = (bf16*)take((size_t)L.in[l] * ld8(L.out[l]) * sizeof(bf16));
    w->xT = (bf16*)take((size_t)L.in[0] * w->ldb * sizeof(bf16));
    for (int l = 0; l + 1 < L.n; ++l) w->actT[l] = (bf16*)take((size_t)L.out[l] * w->ldb * sizeof(bf16));
    for (int i = 0; i < 2; ++i) {
      w->dz[i] = (bf16*)take((size_t)batch * ld8(maxw) * sizeof(bf16));
      w->dzT[i] = (bf16*)take((size_t)maxw * w->ldb * sizeof(bf16));
    }
    w->part = (float*)take((size_t)kMaxSplits * max_mn * sizeof(float));
    w->row_loss = (float*)take((size_t)batch * sizeof(float));
  }
  w->total = off;
}

// Transposed weights of every layer (the forward GEMMs' B operands).
lsp_status prep_forward_weights(const Layers& L, const bf16* p16, const MlpWs& w, cudaStream_t s) {
  for (int l = 0; l < L.n; ++l)
    LEARN_CUDA(transpose_bf16(p16 + L.w_off[l], L.in[l], L.out[l], L.out[l], w.wt[l], ld8(L.in[l]), s),
               "MLP weight transpose");
  return LSP_OK;
}

// Logits of `batch` rows of x (row pitch in_dim).  With `training`, every
// layer's output is also written transposed (the weight-gradient operands).
lsp_status mlp_forward_impl(const Layers& L, const float* p32, const bf16* x, int64_t batch, const MlpWs& w,
                            bool training, cudaStream_t s) {
  const bf16* a = x;
  int64_t lda = L.in[0];
  if (w.xin) {
    LEARN_CUDA(repitch_bf16(x, batch, L.in[0], L.in[0], w.xin, ld8(L.in[0]), s), "MLP input copy");
    a = w.xin;
    lda = ld8(L.in[0]);
  }
  for (int l = 0; l < L.n; ++l) {
    Gemm g;
    memset(&g, 0, sizeof g);
    g.M = (int)batch;
    g.N = L.out[l];
    g.K = L.in[l];
    g.A = a;
    g.lda = lda;
    g.B = w.wt[l];
    g.ldb = ld8(L.in[l]);
    g.bias = p32 + L.b_off[l];
    g.splits = 1;
    if (l + 1 < L.n) {
      g.relu = 1;
      g.C16 = w.act[l];
      g.ldc16 = ld8(L.out[l]);
      if (training) {
        g.C16T = w.actT[l];
        g.ldt = w.ldb;
      }
      a = w.act[l];
      lda = ld8(L.out[l]);
    } else {
      g.C32 = w.logits;
      g.ldc32 = L.out[l];
    }
    lsp_status st = gemm(g, s);
    if (st) return st;
  }
  return LSP_OK;
}

lsp_status check_x(const uint16_t* x, int in_dim) {
  if (in_dim % 8 == 0 && ((uintptr_t)x) % 16) return err_arg("x_bf16 must be 16-byte aligned");
  return LSP_OK;
}

}  // namespace

// ======================================================================= C ABI
extern "C" {

lsp_status lsp_mlp_param_count(const lsp_mlp_dims* dims, int64_t* count) {
  if (!count) return err_arg("count is NULL");
  Layers L;
  lsp_status st = make_layers(dims, &L);
  if (st) return st;
  *count = L.total;
  return LSP_OK;
}

lsp_status lsp_mlp_workspace_size(const lsp_mlp_dims* dims, int64_t batch, size_t* bytes) {
  if (!bytes || batch < 1) return err_arg("bad batch or NULL bytes");
  Layers L;
  lsp_status st = make_layers(dims, &L);
  if (st) return st;
  MlpWs w;
  mlp_ws_layout(L, batch, true, nullptr, &w);
  *bytes = w.total;
  return LSP_OK;
}
lsp_status lsp_featurize(const double* t, const float* y, const int64_t* offsets, int64_t n_obj,
                         int64_t total_nt, const lsp_grid* grid, float lag_max, uint16_t* feat_bf16,
                         float* feat_f32, lsp_stream_t stream) {
  if (n_obj < 0 || n_obj > INT32_MAX || total_nt < 0) return err_arg("bad n_obj or total_nt");
  if (n_obj == 0) return LSP_OK;
  if (!grid || !(grid->f_max > grid->f_min)) return err_arg("bad grid");
  if (!(lag_max > 0.0f)) return err_arg("lag_max must be > 0");
  if (!offsets || !feat_bf16 || (total_nt > 0 && (!t || !y))) return err_arg("NULL array");
  featurize_kernel<<<(unsigned)n_obj, kFeatThreads, 0, (cudaStream_t)stream>>>(
      t, y, offsets, total_nt, grid->f_min, grid->f_max, lag_max, (bf16*)feat_bf16, feat_f32);
  LEARN_CUDA(cudaGetLastError(), "featurize");
  return LSP_OK;
}

lsp_status lsp_mlp_forward(const lsp_mlp_dims* dims, const float* params, const uint16_t* params_bf16,
                           const uint16_t* x_bf16, int64_t batch, float* logits, void* workspace,
                           size_t ws_bytes, lsp_stream_t stream) {
  Layers L;
  lsp_status st = make_layers(dims, &L);
  if (st) return st;
  if (batch < 1 || !params || !params_bf16 || !x_bf16 || !logits) return err_arg("NULL argument");
  if (batch > LSP_MLP_MAX_BATCH) return err_arg("batch exceeds LSP_MLP_MAX_BATCH rows");
  if ((st = check_x(x_bf16, L.in[0]))) return st;
  MlpWs w;
  mlp_ws_layout(L, batch, false, (char*)workspace, &w);
  if (!workspace || ws_bytes < w.total) return err_arg("MLP workspace too small");
  w.logits = logits;
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = prep_forward_weights(L, (const bf16*)params_bf16, w, s))) return st;
  return mlp_forward_impl(L, params, (const bf16*)x_bf16, batch, w, false, s);
}

lsp_status lsp_mlp_loss_grad(const lsp_mlp_dims* dims, const float* params, const uint16_t* params_bf16,
                             const uint16_t* x_bf16, const int32_t* labels, int64_t batch, float* loss,
                             float* grad, void* workspace, size_t ws_bytes, lsp_stream_t stream) {
  Layers L;
  lsp_status st = make_layers(dims, &L);
  if (st) return st;
  if (batch < 1 || !params || !params_bf16 || !x_bf16 || !labels || !loss || !grad)
    return err_arg("NULL argument");
  if (batch > LSP_MLP_MAX_BATCH) return err_arg("batch exceeds LSP_MLP_MAX_BATCH rows");
  if ((st = check_x(x_bf16, L.in[0]))) return st;
  MlpWs w;
  mlp_ws_layout(L, batch, true, (char*)workspace, &w);
  if (!workspace || ws_bytes < w.total) return err_arg("MLP workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  const bf16* p16 = (const bf16*)params_bf16;
  const bf16* x = (const bf16*)x_bf16;
  if ((st = prep_forward_weights(L, p16, w, s))) return st;
  for (int l = 1; l < L.n; ++l)
    LEARN_CUDA(repitch_bf16(p16 + L.w_off[l], L.in[l], L.out[l], L.out[l], w.wp[l], ld8(L.out[l]), s),
               "MLP weight copy");
  LEARN_CUDA(transpose_bf16(x, batch, L.in[0], L.in[0], w.xT, w.ldb, s), "MLP input transpose");
  if ((st = mlp_forward_impl(L, params, x, batch, w, true, s))) return st;
  const int n_cls = L.out[L.n - 1];
  const int64_t warps_per_cta = 8;
  xent_kernel<<<(unsigned)((batch + warps_per_cta - 1) / warps_per_cta), 256, 0, s>>>(
      w.logits, labels, batch, n_cls, w.row_loss, w.dz[0], ld8(n_cls));
  mean_kernel<<<1, 1024, 0, s>>>(w.row_loss, batch, loss);
  LEARN_CUDA(cudaGetLastError(), "loss");
  LEARN_CUDA(transpose_bf16(w.dz[0], batch, n_cls, ld8(n_cls), w.dzT[0], w.ldb, s), "dZ transpose");
  int cur = 0;
  for (int l = L.n - 1; l >= 0; --l) {
    // dW_l = A_in^T dZ_l  (in x out): both operands transposed, K = batch
    Gemm g;
    memset(&g, 0, sizeof g);
    g.M = L.in[l];
    g.N = L.out[l];
    g.K = (int)batch;
    g.A = l == 0 ? w.xT : w.actT[l - 1];
    g.lda = w.ldb;
    g.B = w.dzT[cur];
    g.ldb = w.ldb;
    g.C32 = grad + L.w_off[l];
    g.ldc32 = L.out[l];
    g.splits = k_splits(g.M, g.N, g.K);
    g.part = w.part;
    if ((st = gemm(g, s))) return st;
    rowsum_kernel<<<(L.out[l] + 7) / 8, 256, 0, s>>>(w.dzT[cur], L.out[l], batch, w.ldb, grad + L.b_off[l]);
    LEARN_CUDA(cudaGetLastError(), "bias gradient");
    if (l > 0) {
      // dZ_{l-1} = (dZ_l W_l^T) * (A_{l-1} > 0), also written transposed
      Gemm h;
      memset(&h, 0, sizeof h);
      h.M = (int)batch;
      h.N = L.in[l];
      h.K = L.out[l];
      h.A = w.dz[cur];
      h.lda = ld8(L.out[l]);
      h.B = w.wp[l];
      h.ldb = ld8(L.out[l]);
      h.mask = w.act[l - 1];
      h.ldm = ld8(L.in[l]);
      h.C16 = w.dz[1 - cur];
      h.ldc16 = ld8(L.in[l]);
      h.C16T = w.dzT[1 - cur];
      h.ldt = w.ldb;
      h.splits = 1;
      if ((st = gemm(h, s))) return st;
      cur = 1 - cur;
    }
  }
  return LSP_OK;
}

lsp_status lsp_mlp_gemm_wait_test(void* workspace, size_t ws_bytes, uint32_t* timeouts, int32_t* nan_outputs,
                                  lsp_stream_t stream) {
  if (!workspace || ws_bytes < LSP_MLP_WAIT_TEST_BYTES || ((uintptr_t)workspace) % 256 || !timeouts ||
      !nan_outputs)
    return err_arg("wait test: NULL argument or workspace smaller than LSP_MLP_WAIT_TEST_BYTES");
  cudaStream_t s = (cudaStream_t)stream;
  // one 128 x 16 tile over one K slice of 64: A 16 KiB, B 2 KiB, C 8 KiB
  char* ws = (char*)workspace;
  bf16* A = (bf16*)ws;
  bf16* B = (bf16*)(ws + 16384);
  float* C = (float*)(ws + 16384 + 2048);
  LEARN_CUDA(cudaMemsetAsync(ws, 0, 16384 + 2048, s), "wait test inputs");
  uint32_t before = 0;
  lsp_status st = lsp_mlp_gemm_timeouts(&before);  // clears the count
  if (st) return st;
  CUtensorMap ma, mb;
  if ((st = make_map(&ma, A, 128, 64, 64, umma::BM, "wait test A"))) return st;
  if ((st = make_map(&mb, B, 16, 64, 64, 16, "wait test B"))) return st;
  if ((st = gemm_attributes())) return st;
  umma::Args a;
  memset(&a, 0, sizeof a);
  a.M = 128;
  a.N = 16;
  a.K = 64;
  a.n_tile = 16;
  a.kb_per_split = 1;
  a.C32 = C;
  a.ldc32 = 16;
  a.withhold_first_load = 1;
  umma::gemm_kernel<<<1, umma::THREADS, umma::SMEM_BYTES, s>>>(ma, mb, a);
  LEARN_CUDA(cudaGetLastError(), "wait test launch");
  LEARN_CUDA(cudaStreamSynchronize(s), "wait test");
  float host[128 * 16];
  LEARN_CUDA(cudaMemcpy(host, C, sizeof host, cudaMemcpyDeviceToHost), "wait test result");
  int32_t nans = 0;
  for (int i = 0; i < 128 * 16; ++i) nans += host[i] != host[i];
  *nan_outputs = nans;
  return lsp_mlp_gemm_timeouts(timeouts);
}

lsp_status lsp_mlp_gemm_timeouts(uint32_t* count) {
  if (!count) return err_arg("count is NULL");
  unsigned int v = 0;
  LEARN_CUDA(cudaMemcpyFromSymbol(&v, umma::g_umma_timeouts, sizeof v), "reading the GEMM wait counter");
  const unsigned int zero = 0;
  LEARN_CUDA(cudaMemcpyToSymbol(umma::g_umma_timeouts, &zero, sizeof zero), "clearing the GEMM wait counter");
  *count = v;
  return LSP_OK;
}

lsp_status lsp_mlp_adamw(int64_t n, float* params, uint16_t* params_bf16, const float* grad, float* m,
                         float* v, int64_t step, float lr, float beta1, float beta2, float eps,
                         float weight_decay, lsp_stream_t stream) {
  if (n < 1 || !params || !params_bf16 || !grad || !m || !v || step < 1) return err_arg("bad argument");
  // bias corrections 1 - beta^step in FP64, rounded once: in FP32 the
  // subtraction cancels (1 - 0.999^2 keeps only a few correct bits)
  const float bc1 = (float)(1.0 - pow((double)beta1, (double)step));
  const float bc2 = (float)(1.0 - pow((double)beta2, (double)step));
  adamw_kernel<<<1024, 256, 0, (cudaStream_t)stream>>>(n, params, (bf16*)params_bf16, grad, m, v, lr, beta1,
                                                       beta2, eps, weight_decay, bc1, bc2);
  LEARN_CUDA(cudaGetLastError(), "AdamW");
  return LSP_OK;
}

lsp_status lsp_to_bf16(const float* a, uint16_t* b, int64_t n, lsp_stream_t stream) {
  if (n < 0 || (n > 0 && (!a || !b))) return err_arg("bad argument");
  if (n == 0) return LSP_OK;
  to_bf16_kernel<<<1024, 256, 0, (cudaStream_t)stream>>>(n, a, (bf16*)b);
  LEARN_CUDA(cudaGetLastError(), "to_bf16");
  return LSP_OK;
}

lsp_status lsp_top_classes(const float* logits, int64_t rows, int32_t n_classes, int32_t k,
                           int32_t* classes, lsp_stream_t stream) {
  if (rows < 0 || n_classes < 1 || k < 1 || k > 16 || k > n_classes) return err_arg("bad argument");
  if (rows == 0) return LSP_OK;
  if (!logits || !classes) return err_arg("NULL argument");
  topk_kernel<<<(unsigned)((rows + 127) / 128), 128, 0, (cudaStream_t)stream>>>(logits, rows, n_classes,
                                                                                 k, classes);
  LEARN_CUDA(cudaGetLastError(), "top classes");
  return LSP_OK;
}

}  // extern "C"

// The refine entry point needs the library's prologue and main kernel; it
// lives here with its own workspace layout.
namespace {
struct RefineLayout {
  size_t off_obj, off_rec, off_state, off_best, off_full, off_win, off_list, off_cnt, total;
  int n_chunks;
};
// The refine kernel's configuration: 64 threads x 32 frequencies = 2048 bins
// per item (K = 16 packed chains; the fastest shape measured on GB300 for
// 2048-bin chunks).  lsp_batch with k_reseed 16, freqs_per_thread 32 and
// block_threads 64 runs the same kernel on the same chunks.
constexpr int kRefineK = 16;
constexpr int kRefineThreads = 64;

void refine_layout(int64_t n_obj, int64_t total_nt, int64_t n_f, RefineLayout* r) {
  size_t off = 0;
  auto take = [&](size_t b) {
    size_t at = off;
    off = align256(off + b);
    return at;
  };
  const int64_t chunk = (int64_t)kRefineThreads * 2 * kRefineK;
  r->n_chunks = (int)((n_f + chunk - 1) / chunk);
  r->off_obj = take((size_t)n_obj * sizeof(ObjInfo));
  r->off_rec = take((size_t)total_nt * sizeof(RecF32));
  r->off_state = take((size_t)n_obj * sizeof(RefineState));
  r->off_best = take((size_t)n_obj * sizeof(ChunkBest));
  r->off_full = take((size_t)n_obj * r->n_chunks * sizeof(ChunkBest));
  r->off_win = take((size_t)n_obj * sizeof(int32_t));
  r->off_list = take((size_t)n_obj * sizeof(int32_t));
  r->off_cnt = take(64);
  r->total = off;
}
}  // namespace

extern "C" {

lsp_status lsp_refine_workspace_size(int64_t n_obj, int64_t total_nt, const lsp_grid* grid, size_t* bytes) {
  if (!bytes || !grid || n_obj < 0 || total_nt < 0 || grid->n_f < 1) return err_arg("bad argument");
  RefineLayout r;
  refine_layout(n_obj, total_nt, grid->n_f, &r);
  *bytes = r.total;
  return LSP_OK;
}

}  // extern "C"

namespace {

lsp_status check_refine_args(const double* t, const float* y, const int64_t* offsets, int64_t n_obj,
                             int64_t total_nt, const lsp_grid* grid, const int32_t* classes, int32_t k_windows,
                             int64_t window, int64_t stride, const lsp_peak* peaks) {
  if (!grid || !(grid->f_min > 0.0) || !(grid->f_max > grid->f_min) || grid->n_f < 1)
    return err_arg("bad grid");
  if (n_obj < 0 || n_obj > INT32_MAX || total_nt < 0) return err_arg("bad n_obj or total_nt");
  if (n_obj == 0) return LSP_OK;
  if (!t || !y || !offsets || !peaks) return err_arg("NULL argument");
  if (!classes) return err_arg("classes is NULL");
  if (k_windows < 1 || k_windows > 64) return err_arg("k_windows must be 1..64");
  const int64_t chunk = (int64_t)kRefineThreads * 2 * kRefineK;
  if (window < 1 || window > chunk) return err_arg("window must be 1..2048");
  if (stride < 1) return err_arg("stride must be >= 1");
  return LSP_OK;
}

// The windowed refine and the full-grid fallback on a laid-out workspace
// (arguments already checked).
lsp_status refine_impl(const double* t, const float* y, const int64_t* offsets, int64_t n_obj, int64_t total_nt,
                       const lsp_grid* grid, int32_t norm, const int32_t* classes, int32_t k_windows,
                       int64_t window, int64_t stride, float stop_power, float fallback_power,
                       int32_t inconclusive_fallback, lsp_peak* peaks, int32_t* info, char* ws,
                       const RefineLayout& r, cudaStream_t s) {
  ObjInfo* obj = (ObjInfo*)(ws + r.off_obj);
  RecF32* rec = (RecF32*)(ws + r.off_rec);
  RefineState* state = (RefineState*)(ws + r.off_state);
  ChunkBest* best = (ChunkBest*)(ws + r.off_best);
  ChunkBest* full = (ChunkBest*)(ws + r.off_full);
  int32_t* win = (int32_t*)(ws + r.off_win);
  int32_t* list = (int32_t*)(ws + r.off_list);
  uint32_t* cnt = (uint32_t*)(ws + r.off_cnt);  // [0] list count, [1] items, [2] queue
  const double df = (grid->f_max - grid->f_min) / (double)grid->n_f;
  int n_sm = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  int bps = main_blocks_per_sm(0, 1, kRefineK, 2 * kRefineK, kRefineThreads, 0);
  if (bps < 1) bps = 1;

  LEARN_CUDA(launch_stats(t, y, false, offsets, n_obj, total_nt, 1, norm, obj, s), "refine prologue");
  LEARN_CUDA(launch_records(t, y, false, obj, n_obj, total_nt, grid->f_min, df, false, rec, s),
             "refine records");
  const unsigned g1 = (unsigned)((n_obj + 255) / 256);
  refine_init<<<g1, 256, 0, s>>>(n_obj, obj, state);
  MainLaunch ml;
  ml.prec = 0;
  ml.packed = 1;
  ml.k_reseed = kRefineK;
  ml.fpt = 2 * kRefineK;
  ml.threads = kRefineThreads;
  ml.top = 0;
  ml.rec = rec;
  ml.obj = obj;
  ml.order = list;
  ml.power_out = nullptr;
  ml.part = nullptr;
  ml.cand = nullptr;
  ml.queue = cnt + 2;
  ml.n_f = grid->n_f;
  ml.split = 1;
  for (int rr = 0; rr < k_windows; ++rr) {
    LEARN_CUDA(cudaMemsetAsync(cnt, 0, 16, s), "refine counters");
    refine_list<<<g1, 256, 0, s>>>(n_obj, rr, k_windows, classes, stride, window, grid->n_f, state, win,
                                    list, cnt);
    items_from_count<<<1, 1, 0, s>>>(cnt, 1u, cnt + 1);
    ml.best = best;
    ml.n_chunks = 1;
    ml.n_items = n_obj;  // upper bound; the kernel reads the count
    ml.n_items_dev = cnt + 1;
    ml.win_start = win;
    ml.win_len = (int32_t)window;
    ml.grid = (int)(n_sm * bps);
    LEARN_CUDA(launch_main(ml, s), "refine main kernel");
    refine_merge<<<g1, 256, 0, s>>>(n_obj, rr, k_windows, stop_power, best, state);
  }
  // full-grid fallback for the objects whose refined peak stayed weak
  LEARN_CUDA(cudaMemsetAsync(cnt, 0, 16, s), "fallback counters");
  fallback_list<<<g1, 256, 0, s>>>(n_obj, fallback_power, inconclusive_fallback, obj, state, list, cnt);
  items_from_count<<<1, 1, 0, s>>>(cnt, (uint32_t)r.n_chunks, cnt + 1);
  ml.best = full;
  ml.n_chunks = r.n_chunks;
  ml.n_items = n_obj * (int64_t)r.n_chunks;
  ml.n_items_dev = cnt + 1;
  ml.win_start = nullptr;
  ml.win_len = 0;
  ml.grid = (int)(n_sm * bps);
  LEARN_CUDA(launch_main(ml, s), "fallback main kernel");
  refine_finalize<<<g1, 256, 0, s>>>(n_obj, obj, state, fallback_power, inconclusive_fallback, full,
                                     r.n_chunks, grid->f_min, df, peaks, info);
  LEARN_CUDA(cudaGetLastError(), "refine finalize");
  return LSP_OK;
}

}  // namespace

extern "C" {

lsp_status lsp_refine_windows(const double* t, const float* y, const int64_t* offsets, int64_t n_obj,
                              int64_t total_nt, const lsp_grid* grid, int32_t norm, const int32_t* classes,
                              int32_t k_windows, int64_t window, int64_t stride, float stop_power,
                              float fallback_power, int32_t inconclusive_fallback, lsp_peak* peaks,
                              int32_t* info, void* workspace, size_t ws_bytes, lsp_stream_t stream) {
  lsp_status st = check_refine_args(t, y, offsets, n_obj, total_nt, grid, classes, k_windows, window, stride,
                                    peaks);
  if (st || n_obj == 0) return st;
  RefineLayout r;
  refine_layout(n_obj, total_nt, grid->n_f, &r);
  if (!workspace || ws_bytes < r.total || ((uintptr_t)workspace) % 256)
    return err_arg("refine workspace too small or misaligned");
  return refine_impl(t, y, offsets, n_obj, total_nt, grid, norm, classes, k_windows, window, stride, stop_power,
                     fallback_power, inconclusive_fallback, peaks, info, (char*)workspace, r,
                     (cudaStream_t)stream);
}

}  // extern "C"

// ============================================== the learned path in one call
namespace {

// The network runs on passes of at most kProposeRows objects, which bounds
// its scratch and keeps each GEMM's grid within its limits.
constexpr int64_t kProposeRows = (int64_t)1 << 20;

struct ProposeLayout {
  size_t off_feat, off_wt[8], off_act[2], off_logits, off_cls, off_refine, total;
  RefineLayout r;
};

void propose_layout(const Layers& L, int64_t n_obj, int64_t total_nt, int64_t n_f, int k_windows,
                    ProposeLayout* p) {
  size_t off = 0;
  auto take = [&](size_t b) {
    size_t at = off;
    off = align256(off + b);
    return at;
  };
  p->off_feat = take((size_t)n_obj * LSP_FEAT_DIM * sizeof(bf16));
  int maxw = 0;
  for (int l = 0; l + 1 < L.n; ++l) maxw = L.out[l] > maxw ? L.out[l] : maxw;
  const int64_t rows = n_obj < kProposeRows ? n_obj : kProposeRows;
  for (int l = 0; l < L.n; ++l) p->off_wt[l] = take((size_t)L.out[l] * ld8(L.in[l]) * sizeof(bf16));
  for (int i = 0; i < 2; ++i) p->off_act[i] = take((size_t)rows * ld8(maxw) * sizeof(bf16));
  p->off_logits = take((size_t)rows * L.out[L.n - 1] * sizeof(float));
  p->off_cls = take((size_t)n_obj * k_windows * sizeof(int32_t));
  refine_layout(n_obj, total_nt, n_f, &p->r);
  p->off_refine = take(p->r.total);
  p->total = off;
}

lsp_status check_proposer(const lsp_proposer* net, Layers* L) {
  if (!net) return err_arg("proposer is NULL");
  lsp_status st = make_layers(&net->dims, L);
  if (st) return st;
  if (net->dims.in_dim != LSP_FEAT_DIM) return err_arg("the proposer's in_dim must be LSP_FEAT_DIM");
  if (!net->params || !net->params_bf16) return err_arg("the proposer's parameters are NULL");
  if (net->k_windows < 1 || net->k_windows > 16 || net->k_windows > net->dims.n_classes)
    return err_arg("k_windows must be 1..16 and at most n_classes");
  if (!(net->lag_max > 0.0f)) return err_arg("lag_max must be > 0");
  if (net->norm != LSP_NORM_PSD && net->norm != LSP_NORM_STANDARD) return err_arg("bad norm");
  return LSP_OK;
}

}  // namespace

extern "C" {

lsp_status lsp_window_labels(const lsp_peak* peaks, int64_t n_obj, int64_t stride, int32_t n_classes,
                             int32_t* labels, lsp_stream_t stream) {
  if (n_obj < 0 || stride < 1 || n_classes < 1) return err_arg("bad n_obj, stride or n_classes");
  if (n_obj == 0) return LSP_OK;
  if (!peaks || !labels) return err_arg("NULL argument");
  labels_kernel<<<(unsigned)((n_obj + 255) / 256), 256, 0, (cudaStream_t)stream>>>(peaks, n_obj, stride,
                                                                                   n_classes, labels);
  LEARN_CUDA(cudaGetLastError(), "window labels");
  return LSP_OK;
}

lsp_status lsp_propose_refine_workspace_size(const lsp_proposer* net, int64_t n_obj, int64_t total_nt,
                                             const lsp_grid* grid, size_t* bytes) {
  if (!bytes || !grid || n_obj < 0 || total_nt < 0 || grid->n_f < 1) return err_arg("bad argument");
  Layers L;
  lsp_status st = check_proposer(net, &L);
  if (st) return st;
  ProposeLayout p;
  propose_layout(L, n_obj, total_nt, grid->n_f, net->k_windows, &p);
  *bytes = p.total;
  return LSP_OK;
}

lsp_status lsp_propose_refine(const lsp_proposer* net, const double* t, const float* y, const int64_t* offsets,
                              int64_t n_obj, int64_t total_nt, const lsp_grid* grid, lsp_peak* peaks,
                              int32_t* info, int32_t* classes_out, void* workspace, size_t ws_bytes,
                              lsp_stream_t stream) {
  Layers L;
  lsp_status st = check_proposer(net, &L);
  if (st) return st;
  // the classes pointer is checked once it exists (inside the workspace)
  int32_t dummy = 0;
  st = check_refine_args(t, y, offsets, n_obj, total_nt, grid, &dummy, net->k_windows, net->window, net->stride,
                         peaks);
  if (st || n_obj == 0) return st;
  ProposeLayout p;
  propose_layout(L, n_obj, total_nt, grid->n_f, net->k_windows, &p);
  if (!workspace || ws_bytes < p.total || ((uintptr_t)workspace) % 256)
    return err_arg("propose-refine workspace too small or misaligned");
  cudaStream_t s = (cudaStream_t)stream;
  char* ws = (char*)workspace;
  bf16* feat = (bf16*)(ws + p.off_feat);
  int32_t* cls = classes_out ? classes_out : (int32_t*)(ws + p.off_cls);
  // 1. features
  featurize_kernel<<<(unsigned)n_obj, kFeatThreads, 0, s>>>(t, y, offsets, total_nt, grid->f_min, grid->f_max,
                                                             net->lag_max, feat, nullptr);
  LEARN_CUDA(cudaGetLastError(), "featurize");
  // 2. logits (hidden activations alternate between two buffers) and
  // 3. the k best window classes per object, a pass of rows at a time
  MlpWs w;
  memset(&w, 0, sizeof w);
  for (int l = 0; l < L.n; ++l) w.wt[l] = (bf16*)(ws + p.off_wt[l]);
  for (int l = 0; l + 1 < L.n; ++l) w.act[l] = (bf16*)(ws + p.off_act[l & 1]);
  w.logits = (float*)(ws + p.off_logits);
  if ((st = prep_forward_weights(L, (const bf16*)net->params_bf16, w, s))) return st;
  for (int64_t r0 = 0; r0 < n_obj; r0 += kProposeRows) {
    const int64_t rows = n_obj - r0 < kProposeRows ? n_obj - r0 : kProposeRows;
    if ((st = mlp_forward_impl(L, net->params, feat + r0 * LSP_FEAT_DIM, rows, w, false, s))) return st;
    topk_kernel<<<(unsigned)((rows + 127) / 128), 128, 0, s>>>(w.logits, rows, L.out[L.n - 1], net->k_windows,
                                                                cls + r0 * net->k_windows);
    LEARN_CUDA(cudaGetLastError(), "top classes");
  }
  // 4. refine in rank order, full grid where the refined peak is weak
  return refine_impl(t, y, offsets, n_obj, total_nt, grid, net->norm, cls, net->k_windows, net->window,
                     net->stride, net->stop_power, net->fallback_power, net->inconclusive_fallback, peaks, info,
                     ws + p.off_refine, p.r, s);
}

}  // extern "C"
