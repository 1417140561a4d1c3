// lsp_launch.h -- host-side launchers of the library's kernels (internal).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "lsp_common.cuh"

struct lsp_peak;

namespace lsp {

// Opts a kernel in to `dyn` bytes of dynamic shared memory where its static
// and dynamic shared memory together pass the 48 KB available by default.
template <typename Kern>
inline cudaError_t allow_dyn_smem(Kern kern, size_t dyn) {
  cudaFuncAttributes a{};
  cudaError_t e = cudaFuncGetAttributes(&a, kern);
  if (e != cudaSuccess) return e;
  if (dyn + a.sharedSizeBytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
}

// Prologue, Section 2 (zero-mean magnitudes) and the per-observation phase
// data of the grid recurrences (rotation step, three-term coefficients).  y is float (y64 = false) or double.
// gls: weighted statistics / records of the generalized periodogram (dy
// NULL: unit weights).
cudaError_t launch_stats(const double* t, const void* y, bool y64, const int64_t* offsets,
                         int64_t n_obj, int64_t total_nt, int center, int norm, ObjInfo* obj,
                         cudaStream_t stream, bool gls = false, const void* dy = nullptr,
                         void* slices_ws = nullptr, uint32_t* ticket = nullptr);
// Scratch of the one-object statistics pass (slices_ws of launch_stats): with
// it, and a zeroed ticket word, one object without offsets is reduced by
// many CTAs; without it by one.
size_t stats_slices_bytes(int64_t total_nt);
cudaError_t launch_records(const double* t, const void* y, bool y64, const ObjInfo* obj,
                           int64_t n_obj, int64_t max_nt_single, double f_min, double df,
                           bool rec64, void* rec, cudaStream_t stream, bool gls = false,
                           const void* dy = nullptr);
// One object of at most kFusedMaxNt observations: statistics and records in
// one launch, which also clears the four work-counter words at `queue` (no
// memset, no ticket).  Every CTA redoes the object's FP64 statistics, about
// 3.5 clocks per observation on one SM at GB300's FP64 rate, which caps it.
constexpr int64_t kFusedMaxNt = 2048;
cudaError_t launch_single_prologue(const double* t, const void* y, bool y64, int64_t n, int center, int norm,
                                   double f_min, double df, bool rec64, ObjInfo* obj, void* rec, uint32_t* queue,
                                   cudaStream_t stream, bool gls = false, const void* dy = nullptr);
// The work-queue order: objects by N_t (counting sort), the longest and the
// shortest alternating.
cudaError_t launch_lpt_order(const ObjInfo* obj, int64_t n_obj, uint32_t* hist, int32_t* order,
                             cudaStream_t stream);

// Main kernel variants.
struct MainLaunch {
  int prec;      // 0 FP32, 1 FP64
  int packed;    // FP32 only
  int k_reseed;  // chain length K
  int fpt;       // frequencies per thread (packed: 2K; scalar: K)
  int gls = 0;   // generalized periodogram kernels
  int abl = 0;   // ablation kernel: trig + 3 * staging (lsp_config), 0 = production
  int threads;
  int grid;      // persistent CTAs
  int top;       // 1: top-k candidates
  const void* rec;
  const ObjInfo* obj;
  const int32_t* order;
  void* power_out;
  void* part;
  ChunkBest* best;
  ChunkCand* cand;
  uint32_t* queue;
  int64_t n_f;
  int32_t n_chunks;
  int32_t split;
  int64_t n_items;
  const uint32_t* n_items_dev = nullptr;  // device item count (overrides n_items)
  const int32_t* win_start = nullptr;     // per-object window origins (packed FP32 kernels)
  int32_t win_len = 0;
};
bool main_variant_exists(int prec, int packed, int k_reseed, int fpt, int gls = 0, int abl = 0);
cudaError_t launch_main(const MainLaunch& ml, cudaStream_t stream);
// CTAs of the main variant resident per SM (0 if the variant does not exist).
int main_blocks_per_sm(int prec, int packed, int k_reseed, int fpt, int threads, int top, int gls = 0,
                      int abl = 0);
size_t main_dyn_smem(int prec, int fpt, int threads, int top);

// Split-N_t combine (single object; gls: the generalized periodogram's six
// sums in stride-8 slots): sums the partial sums in a fixed order,
// evaluates the power, stores it (optional) and reduces chunk results; with
// peaks, no candidates and a zeroed ticket word it also writes the first
// maximum (no finalize launch needed).
constexpr int kCombineThreads = 256;
#ifndef LSP_COMBINE_PER_THREAD
#define LSP_COMBINE_PER_THREAD 1
#endif
constexpr int kCombinePerThread = LSP_COMBINE_PER_THREAD;
cudaError_t launch_combine(int prec, const void* part, int split, int64_t n_f, const ObjInfo* obj,
                           const void* rec, void* power_out, ChunkBest* best, ChunkCand* cand,
                           cudaStream_t stream, lsp_peak* peaks = nullptr, double f_min = 0.0,
                           double df = 0.0, uint32_t* ticket = nullptr, bool gls = false);

// Per-object peaks from the chunk results.
cudaError_t launch_finalize(const ObjInfo* obj, const ChunkBest* best, const ChunkCand* cand,
                            int64_t n_obj, int n_chunks, int top_k, double f_min, double df,
                            lsp_peak* peaks, cudaStream_t stream);

// First maximum of stored periodograms (no workspace: the peak records hold
// the reduction state).
cudaError_t launch_argmax_period(const void* power, bool p64, int64_t n_obj, int64_t n_f,
                                 double f_min, double df, lsp_peak* peaks, cudaStream_t stream);

// Autotuner error gate helpers.
cudaError_t launch_f32_to_f64(const float* a, double* b, int64_t n, cudaStream_t stream);
cudaError_t launch_max_abs_diff(const float* a, const double* b, int64_t n, double* out,
                                cudaStream_t stream);
// out[r] = max_i |a[r n + i] - b[r n + i]| for each of `rows` rows.
cudaError_t launch_row_max_abs_diff(const float* a, const double* b, int64_t rows, int64_t n, double* out,
                                    cudaStream_t stream);
// score[i] = max over the grid of |sum_j exp(2 pi i 2 f_k t_j)| / N for the
// observations t[begin[i] .. begin[i] + count[i]) (device arrays).
cudaError_t launch_window_score(const double* t, const int64_t* begin, const int64_t* count, int n_list,
                                double f_min, double df, int64_t n_f, float* score, cudaStream_t stream);

}  // namespace lsp
