// lsp_api.cu -- the C ABI of include/lsp.h: validation, workspace layout,
// launch sequence, plans (CUDA-graph replay, host entry point, autotuner).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <fstream>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/lsp.h"
#include "lsp_launch.h"

using namespace lsp;

static_assert(sizeof(lsp_peak) == 40, "lsp_peak layout");
static_assert(sizeof(RecF32) == 32 && sizeof(RecF64) == 48, "record layout");

namespace {

thread_local std::string g_err;

lsp_status fail(lsp_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

lsp_status cuda_fail(cudaError_t e, const char* what) {
  return fail(LSP_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define LSP_CUDA(call, what)                       \
  do {                                             \
    cudaError_t e__ = (call);                      \
    if (e__ != cudaSuccess) return cuda_fail(e__, what); \
  } while (0)

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

int current_sm_count() {
  static std::mutex mu;
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  std::lock_guard<std::mutex> lk(mu);
  if (cache[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
      cudaGetLastError();
      n = 152;
    }
    cache[dev] = n;
  }
  return cache[dev];
}

// Resolved configuration and workspace layout of one call.
struct Layout {
  int prec, packed, k, fpt, threads, split, top_k, top, norm, center, gls;
  int abl = 0;  // ablation kernel code (lsp_config trig + 3 * staging)
  int64_t n_obj, total_nt, n_f;
  double f_min, df;
  int32_t n_chunks, n_res_chunks;
  int64_t n_items;
  int grid;  // persistent CTAs
  size_t off_obj, off_rec, off_order, off_hist, off_queue, off_best, off_cand, off_part, off_stats, total;
};

constexpr int64_t kMaxNf = (int64_t)1 << 31;  // k0 + F must fit in 32 bits
constexpr int kMinObsPerSplit = 32;
constexpr int kMaxObsPerSplit = 8192;  // bounds each FP32 partial sum
constexpr int kMaxSplit = 256;
constexpr int kGateObjects = 8;  // objects the autotuner's error gate checks

lsp_status check_grid(const lsp_grid* g) {
  if (!g) return fail(LSP_E_ARG, "grid is NULL");
  if (!std::isfinite(g->f_min) || !std::isfinite(g->f_max))
    return fail(LSP_E_ARG, "grid limits must be finite");
  if (!(g->f_min > 0.0)) return fail(LSP_E_ARG, "f_min must be > 0 (Eq. 1 divides by 2w)");
  if (!(g->f_max > g->f_min)) return fail(LSP_E_ARG, "f_max must be > f_min");
  if (g->n_f < 1 || g->n_f > kMaxNf - 65536) return fail(LSP_E_ARG, "n_f must be in [1, 2^31 - 2^16]");
  return LSP_OK;
}

lsp_status resolve(int64_t n_obj, int64_t total_nt, const lsp_grid* g, const lsp_opts* opts_in,
                   const lsp_config* cfg, Layout* L, bool gls = false) {
  lsp_status st = check_grid(g);
  if (st) return st;
  if (n_obj < 0 || n_obj > INT32_MAX) return fail(LSP_E_ARG, "n_obj out of range");
  if (total_nt < 0) return fail(LSP_E_ARG, "total_nt must be >= 0");
  if (n_obj == 1 && total_nt > INT32_MAX) return fail(LSP_E_ARG, "n_t must be < 2^31");
  lsp_opts o = opts_in ? *opts_in : lsp_default_opts();
  if (o.precision != LSP_FP32 && o.precision != LSP_FP64) return fail(LSP_E_ARG, "bad precision");
  if (o.norm != LSP_NORM_PSD && o.norm != LSP_NORM_STANDARD) return fail(LSP_E_ARG, "bad norm");
  if (o.top_k < 1 || o.top_k > 3) return fail(LSP_E_ARG, "top_k must be 1..3");
  if (o.k_reseed < 0 || o.freqs_per_thread < 0 || o.block_threads < 0 || o.obs_split < 0)
    return fail(LSP_E_ARG, "negative option");

  Layout& l = *L;
  memset(&l, 0, sizeof l);
  l.prec = o.precision;
  l.norm = o.norm;
  l.center = o.center_y ? 1 : 0;
  l.top_k = o.top_k;
  l.top = o.top_k > 1;
  l.n_obj = n_obj;
  l.total_nt = total_nt;
  l.n_f = g->n_f;
  l.f_min = g->f_min;
  l.df = (g->f_max - g->f_min) / (double)g->n_f;
  l.gls = gls ? 1 : 0;

  int k, fpt, threads, packed, split_req, abl = 0;
  if (cfg) {
    k = cfg->k_reseed;
    fpt = cfg->freqs_per_thread;
    threads = cfg->block_threads;
    packed = cfg->packed;
    split_req = cfg->obs_split;
    if (cfg->trig < 0 || cfg->trig > 2 || cfg->staging < 0 || cfg->staging > 1)
      return fail(LSP_E_ARG, "trig must be 0, 1 or 2 and staging 0 or 1");
    abl = cfg->trig + 3 * cfg->staging;
  } else {
    // FP64 standard periodogram: chains of 16 (each seed is an FP64
    // sincospi; measured on GB300, the 1e5-observation object on 1e6 bins:
    // 1.31 s against 1.66 s at 8); the generalized FP64 kernel has K = 8
    k = o.k_reseed ? o.k_reseed : ((l.prec == LSP_FP64 && !gls) ? 16 : 8);
    if (l.prec == LSP_FP64) {
      fpt = o.freqs_per_thread ? o.freqs_per_thread : k;
      threads = o.block_threads ? o.block_threads : 128;
    } else {
      fpt = o.freqs_per_thread ? o.freqs_per_thread
                               : (main_variant_exists(0, 1, k, 2 * k) ? 2 * k : k);
      // measured on GB300: 128-thread CTAs for batches and for the generalized
      // kernels (six sums per frequency), 256 for one object
      threads = o.block_threads ? o.block_threads : ((n_obj > 1 || gls) ? 128 : 256);
    }
    packed = (l.prec == LSP_FP32 && fpt == 2 * k) ? 1 : 0;
    split_req = o.obs_split;
  }
  if (threads < 64 || threads > 256 || threads % 32)
    return fail(LSP_E_ARG, "block_threads must be a multiple of 32 in [64, 256]");
  if (!main_variant_exists(l.prec, packed, k, fpt, l.gls, abl))
    return fail(LSP_E_UNSUPPORTED,
                "no %skernel for precision %d with k_reseed=%d, freqs_per_thread=%d, packed=%d%s",
                gls ? "generalized " : "", l.prec, k, fpt, packed,
                abl ? " (the trig/staging ablation kernels are FP32, scalar, k_reseed=freqs_per_thread=16)" : "");
  l.abl = abl;
  l.k = k;
  l.fpt = fpt;
  l.threads = threads;
  l.packed = packed;

  const int64_t chunk = (int64_t)threads * fpt;
  l.n_chunks = (int32_t)((l.n_f + chunk - 1) / chunk);
  int split = 1;
  if (n_obj == 1) {
    if (split_req > 0) {
      split = split_req;
    } else {
      const int64_t target = (int64_t)current_sm_count() * 4;
      int64_t s = (target + l.n_chunks - 1) / l.n_chunks;
      int64_t s_min = (total_nt + kMaxObsPerSplit - 1) / kMaxObsPerSplit;
      if (s < s_min) s = s_min;
      int64_t s_max = total_nt / kMinObsPerSplit;
      if (s > s_max) s = s_max;
      split = (int)(s < 1 ? 1 : s);
    }
    if (split > kMaxSplit) split = kMaxSplit;
  }
  l.split = split;
  const int64_t cchunk = (int64_t)kCombineThreads * kCombinePerThread;
  l.n_res_chunks = split > 1 ? (int32_t)((l.n_f + cchunk - 1) / cchunk) : l.n_chunks;
  l.n_items = n_obj * (int64_t)l.n_chunks * split;

  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off = align_up(off + bytes);
    return at;
  };
  l.off_obj = take((size_t)n_obj * sizeof(ObjInfo));
  l.off_rec = take((size_t)total_nt * (l.prec ? sizeof(RecF64) : sizeof(RecF32)));
  l.off_order = take(n_obj > 1 ? (size_t)n_obj * sizeof(int32_t) : 0);
  l.off_hist = take(n_obj > 1 ? (LSP_HIST_BINS + 1) * sizeof(uint32_t) : 0);
  l.off_queue = take(16);
  l.off_best = take((size_t)n_obj * l.n_res_chunks * sizeof(ChunkBest));
  l.off_cand = take(l.top ? (size_t)n_obj * l.n_res_chunks * sizeof(ChunkCand) : 0);
  // partial sums: 4 per frequency, the generalized periodogram's 6 in slots of 8
  l.off_part = take(split > 1 ? (size_t)split * l.n_f * (gls ? 8 : 4) * (l.prec ? 8 : 4) : 0);
  l.off_stats = take(n_obj == 1 ? stats_slices_bytes(total_nt) : 0);
  l.total = off;

  int bps = main_blocks_per_sm(l.prec, l.packed, l.k, l.fpt, l.threads, l.top, l.gls, l.abl);
  if (bps <= 0) {
    cudaGetLastError();
    bps = 1;
  }
  int64_t grid = (int64_t)bps * current_sm_count();
  if (grid > l.n_items) grid = l.n_items;
  l.grid = (int)(grid < 1 ? 1 : grid);
  return LSP_OK;
}

// One object given without offsets and short enough for the fused prologue
// (statistics and records in one launch).
bool fused_prologue(const Layout& L, const int64_t* offsets) {
  return L.n_obj == 1 && !offsets && L.total_nt <= kFusedMaxNt;
}

// The launch sequence of one periodogram call (stream-ordered, no syncs).
lsp_status run(const Layout& L, const double* t, const void* y, const int64_t* offsets,
               void* power_out, lsp_peak* peaks, char* ws, cudaStream_t st,
               cudaEvent_t ev_main0 = nullptr, cudaEvent_t ev_main1 = nullptr,
               const void* dy = nullptr) {
  if (L.n_obj == 0) return LSP_OK;
  ObjInfo* obj = (ObjInfo*)(ws + L.off_obj);
  void* rec = ws + L.off_rec;
  int32_t* order = L.n_obj > 1 ? (int32_t*)(ws + L.off_order) : nullptr;
  uint32_t* hist = (uint32_t*)(ws + L.off_hist);
  uint32_t* queue = (uint32_t*)(ws + L.off_queue);
  ChunkBest* best = (ChunkBest*)(ws + L.off_best);
  ChunkCand* cand = L.top ? (ChunkCand*)(ws + L.off_cand) : nullptr;
  void* part = L.split > 1 ? (void*)(ws + L.off_part) : nullptr;
  const bool y64 = L.prec == LSP_FP64;

  // queue[0]: the main kernel's work counter; queue[1], queue[2]: last-CTA
  // tickets of the one-object statistics and combine kernels
  if (fused_prologue(L, offsets)) {  // one launch, which also clears the queue words
    LSP_CUDA(launch_single_prologue(t, y, y64, L.total_nt, L.center, L.norm, L.f_min, L.df, y64, obj, rec, queue,
                                    st, L.gls != 0, dy),
             "prologue");
  } else {
    LSP_CUDA(cudaMemsetAsync(queue, 0, 16, st), "queue reset");
    LSP_CUDA(launch_stats(t, y, y64, offsets, L.n_obj, L.total_nt, L.center, L.norm, obj, st, L.gls != 0,
                          dy, L.n_obj == 1 ? ws + L.off_stats : nullptr, queue + 1),
             "prologue (statistics)");
    LSP_CUDA(launch_records(t, y, y64, obj, L.n_obj, L.total_nt, L.f_min, L.df, y64, rec, st, L.gls != 0, dy),
             "prologue (records)");
  }
  if (order) LSP_CUDA(launch_lpt_order(obj, L.n_obj, hist, order, st), "work-queue order");
  MainLaunch ml;
  ml.prec = L.prec;
  ml.packed = L.packed;
  ml.abl = L.abl;
  ml.k_reseed = L.k;
  ml.fpt = L.fpt;
  ml.gls = L.gls;
  ml.threads = L.threads;
  ml.grid = L.grid;
  ml.top = L.top && L.split == 1;
  ml.rec = rec;
  ml.obj = obj;
  ml.order = order;
  ml.power_out = L.split == 1 ? power_out : nullptr;
  ml.part = part;
  ml.best = best;
  ml.cand = L.split == 1 ? cand : nullptr;
  ml.queue = queue;
  ml.n_f = L.n_f;
  ml.n_chunks = L.n_chunks;
  ml.split = L.split;
  ml.n_items = L.n_items;
  // External records become event-record nodes when captured into a graph.
  if (ev_main0) LSP_CUDA(cudaEventRecordWithFlags(ev_main0, st, cudaEventRecordExternal), "timing event");
  LSP_CUDA(launch_main(ml, st), "main kernel");
  if (ev_main1) LSP_CUDA(cudaEventRecordWithFlags(ev_main1, st, cudaEventRecordExternal), "timing event");
  // one object, first maximum: the combine kernel writes the peak itself
  const bool fused = L.split > 1 && !L.top && peaks;
  if (L.split > 1)
    LSP_CUDA(launch_combine(L.prec, part, L.split, L.n_f, obj, rec, power_out, best, cand, st,
                            fused ? peaks : nullptr, L.f_min, L.df, queue + 2, L.gls != 0),
             "split combine");
  if (peaks && !fused)
    LSP_CUDA(launch_finalize(obj, best, cand, L.n_obj, L.n_res_chunks, L.top_k, L.f_min, L.df,
                             peaks, st),
             "finalize");
  return LSP_OK;
}

lsp_status check_ws(const Layout& L, void* ws, size_t ws_bytes) {
  if (L.total && !ws) return fail(LSP_E_WORKSPACE, "workspace is NULL (need %zu bytes)", L.total);
  if (ws_bytes < L.total)
    return fail(LSP_E_WORKSPACE, "workspace has %zu bytes, need %zu", ws_bytes, L.total);
  if (((uintptr_t)ws) % kAlign) return fail(LSP_E_WORKSPACE, "workspace must be 256-byte aligned");
  return LSP_OK;
}

lsp_status check_io(int64_t n, const double* t, const void* y) {
  if (n > 0 && (!t || !y)) return fail(LSP_E_ARG, "t and y must not be NULL");
  return LSP_OK;
}

}  // namespace

namespace lsp {
// Lets other translation units of the library report through lsp_last_error.
void set_last_error(const char* msg) { g_err = msg ? msg : ""; }
}  // namespace lsp

// ======================================================================= C ABI
extern "C" {

const char* lsp_status_string(lsp_status s) {
  switch (s) {
    case LSP_OK: return "LSP_OK";
    case LSP_E_ARG: return "LSP_E_ARG: invalid argument";
    case LSP_E_CUDA: return "LSP_E_CUDA: CUDA runtime error";
    case LSP_E_NOMEM: return "LSP_E_NOMEM: device allocation failed";
    case LSP_E_WORKSPACE: return "LSP_E_WORKSPACE: workspace too small or misaligned";
    case LSP_E_NUMERIC: return "LSP_E_NUMERIC: numeric problem";
    case LSP_E_TIMEOUT: return "LSP_E_TIMEOUT: device wait timed out";
    case LSP_E_UNSUPPORTED: return "LSP_E_UNSUPPORTED: not implemented in this build";
  }
  return "unknown lsp_status";
}

const char* lsp_last_error(void) { return g_err.c_str(); }

int32_t lsp_version(void) { return 10000; }

lsp_opts lsp_default_opts(void) {
  lsp_opts o;
  memset(&o, 0, sizeof o);
  o.precision = LSP_FP32;
  o.norm = LSP_NORM_STANDARD;
  o.center_y = 1;
  o.top_k = 1;
  return o;
}

lsp_status lsp_grid_for_span(double f_min, double f_max, double t_span, lsp_grid* grid) {
  g_err.clear();
  if (!grid) return fail(LSP_E_ARG, "grid is NULL");
  if (!(t_span > 0.0) || !std::isfinite(t_span)) return fail(LSP_E_ARG, "t_span must be > 0");
  if (!(f_max > f_min)) return fail(LSP_E_ARG, "f_max must be > f_min");
  const double df = 0.1 / t_span;  // 0.2 pi / T_max rad per unit time, in cycles
  const double n = std::nearbyint((f_max - f_min) / df);
  if (n < 1.0 || n > (double)(kMaxNf - 65536)) return fail(LSP_E_ARG, "resulting n_f out of range");
  grid->f_min = f_min;
  grid->f_max = f_max;
  grid->n_f = (int64_t)n;
  return LSP_OK;
}

lsp_status lsp_workspace_size(int64_t n_obj, int64_t total_nt, const lsp_grid* grid,
                              const lsp_opts* opts, size_t* bytes) {
  if (!bytes) return fail(LSP_E_ARG, "bytes is NULL");
  Layout L;
  lsp_status st = resolve(n_obj, total_nt, grid, opts, nullptr, &L);
  if (st) return st;
  *bytes = L.total;
  return LSP_OK;
}

lsp_status lsp_periodogram(const double* t, const void* y, int64_t n_t, const lsp_grid* grid,
                           const lsp_opts* opts, void* power_out, lsp_peak* peaks, void* workspace,
                           size_t ws_bytes, lsp_stream_t stream) {
  g_err.clear();
  Layout L;
  lsp_status st = resolve(1, n_t, grid, opts, nullptr, &L);
  if (st) return st;
  if ((st = check_io(n_t, t, y))) return st;
  if ((st = check_ws(L, workspace, ws_bytes))) return st;
  return run(L, t, y, nullptr, power_out, peaks, (char*)workspace, (cudaStream_t)stream);
}

lsp_status lsp_batch(const double* t, const void* y, const int64_t* offsets, int64_t n_obj,
                     int64_t total_nt, const lsp_grid* grid, const lsp_opts* opts, void* power_out,
                     lsp_peak* peaks, void* workspace, size_t ws_bytes, lsp_stream_t stream) {
  g_err.clear();
  Layout L;
  lsp_status st = resolve(n_obj, total_nt, grid, opts, nullptr, &L);
  if (st) return st;
  if (n_obj == 0) return LSP_OK;
  if (!offsets) return fail(LSP_E_ARG, "offsets must not be NULL");
  if ((st = check_io(total_nt, t, y))) return st;
  if ((st = check_ws(L, workspace, ws_bytes))) return st;
  return run(L, t, y, offsets, power_out, peaks, (char*)workspace, (cudaStream_t)stream);
}

lsp_status lsp_workspace_size_gls(int64_t n_obj, int64_t total_nt, const lsp_grid* grid,
                                  const lsp_opts* opts, size_t* bytes) {
  if (!bytes) return fail(LSP_E_ARG, "bytes is NULL");
  Layout L;
  lsp_status st = resolve(n_obj, total_nt, grid, opts, nullptr, &L, true);
  if (st) return st;
  *bytes = L.total;
  return LSP_OK;
}

lsp_status lsp_batch_gls(const double* t, const void* y, const void* dy, const int64_t* offsets,
                         int64_t n_obj, int64_t total_nt, const lsp_grid* grid, const lsp_opts* opts,
                         void* power_out, lsp_peak* peaks, void* workspace, size_t ws_bytes,
                         lsp_stream_t stream) {
  g_err.clear();
  Layout L;
  lsp_status st = resolve(n_obj, total_nt, grid, opts, nullptr, &L, true);
  if (st) return st;
  if (n_obj == 0) return LSP_OK;
  if (!offsets) return fail(LSP_E_ARG, "offsets must not be NULL");
  if ((st = check_io(total_nt, t, y))) return st;
  if ((st = check_ws(L, workspace, ws_bytes))) return st;
  return run(L, t, y, offsets, power_out, peaks, (char*)workspace, (cudaStream_t)stream, nullptr, nullptr, dy);
}

lsp_status lsp_periodogram_gls(const double* t, const void* y, const void* dy, int64_t n_t,
                               const lsp_grid* grid, const lsp_opts* opts, void* power_out,
                               lsp_peak* peaks, void* workspace, size_t ws_bytes, lsp_stream_t stream) {
  g_err.clear();
  Layout L;
  lsp_status st = resolve(1, n_t, grid, opts, nullptr, &L, true);
  if (st) return st;
  if ((st = check_io(n_t, t, y))) return st;
  if ((st = check_ws(L, workspace, ws_bytes))) return st;
  return run(L, t, y, nullptr, power_out, peaks, (char*)workspace, (cudaStream_t)stream, nullptr, nullptr, dy);
}

lsp_status lsp_argmax_period(const void* power, int64_t n_obj, int64_t n_f, const lsp_grid* grid,
                             int32_t precision, lsp_peak* peaks, lsp_stream_t stream) {
  g_err.clear();
  lsp_status st = check_grid(grid);
  if (st) return st;
  if (n_f != grid->n_f) return fail(LSP_E_ARG, "n_f must equal grid->n_f");
  if (n_obj < 0) return fail(LSP_E_ARG, "n_obj must be >= 0");
  if (precision != LSP_FP32 && precision != LSP_FP64) return fail(LSP_E_ARG, "bad precision");
  if (n_obj == 0) return LSP_OK;
  if (!power || !peaks) return fail(LSP_E_ARG, "power and peaks must not be NULL");
  if (((uintptr_t)peaks) % 8) return fail(LSP_E_ARG, "peaks must be 8-byte aligned");
  const double df = (grid->f_max - grid->f_min) / (double)grid->n_f;
  LSP_CUDA(launch_argmax_period(power, precision == LSP_FP64, n_obj, n_f, grid->f_min, df, peaks,
                                (cudaStream_t)stream),
           "argmax");
  return LSP_OK;
}

}  // extern "C"

// ======================================================================= plans
struct lsp_plan {
  Layout L;
  lsp_grid grid;
  lsp_opts opts;
  lsp_config cfg;
  int64_t n_obj = 0, total_nt = 0;
  int device = 0;
  char* ws = nullptr;
  size_t ws_cap = 0;
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  const void* cap_args[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // timing probe (nullptr: off)
  // staging of the host entry point (allocated by its first call)
  double* d_t = nullptr;
  void* d_y = nullptr;
  int64_t* d_off = nullptr;
  lsp_peak* d_peaks = nullptr;
  void* d_power = nullptr;
  // grouped periodogram return of the host entry point
  int32_t host_parts = 0;  // 0: chosen from the periodogram's size
  int64_t* d_rel = nullptr;
  size_t d_rel_cap = 0;
  std::vector<int64_t> h_rel;
  cudaStream_t copy_stream = nullptr;
  std::vector<cudaEvent_t> part_ev;
  cudaEvent_t copy_done = nullptr;
  // input streaming: each group's observations are copied on in_stream
  cudaStream_t in_stream = nullptr;
  std::vector<cudaEvent_t> in_ev;
  cudaEvent_t start_ev = nullptr;
  // the last autotune's error gate: objects and the chosen configuration's errors
  std::vector<int64_t> gate_obj;
  std::vector<double> gate_err;
};

namespace {

lsp_config config_of(const Layout& L) {
  lsp_config c;
  memset(&c, 0, sizeof c);
  c.k_reseed = L.k;
  c.freqs_per_thread = L.fpt;
  c.block_threads = L.threads;
  c.obs_split = L.split;
  c.packed = L.packed;
  c.trig = L.abl % 3;
  c.staging = L.abl / 3;
  return c;
}

void drop_graph(lsp_plan* p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  p->exec = nullptr;
  p->graph = nullptr;
  for (auto& a : p->cap_args) a = nullptr;
}

lsp_status ensure_ws(lsp_plan* p, size_t bytes) {
  if (bytes <= p->ws_cap) return LSP_OK;
  drop_graph(p);  // a captured graph may reference the old workspace
  if (p->ws) {
    cudaDeviceSynchronize();
    cudaFree(p->ws);
  }
  p->ws = nullptr;
  p->ws_cap = 0;
  if (cudaMalloc(&p->ws, bytes ? bytes : kAlign) != cudaSuccess) {
    cudaGetLastError();
    return fail(LSP_E_NOMEM, "plan workspace of %zu bytes", bytes);
  }
  p->ws_cap = bytes;
  return LSP_OK;
}

lsp_status apply_config(lsp_plan* p, const lsp_config* c) {
  Layout L;
  lsp_status st = resolve(p->n_obj, p->total_nt, &p->grid, &p->opts, c, &L);
  if (st) return st;
  if ((st = ensure_ws(p, L.total))) return st;
  p->L = L;
  p->cfg = config_of(L);
  drop_graph(p);
  return LSP_OK;
}

// Times `reps` runs of the plan's current layout with events on `st`.
lsp_status time_runs(lsp_plan* p, const double* t, const void* y, const int64_t* off, int reps,
                     cudaStream_t st, float* ms) {
  cudaEvent_t a, b;
  LSP_CUDA(cudaEventCreate(&a), "event");
  LSP_CUDA(cudaEventCreate(&b), "event");
  lsp_status s = run(p->L, t, y, off, nullptr, nullptr, p->ws, st);  // warm-up
  if (!s) {
    cudaEventRecord(a, st);
    for (int i = 0; i < reps && !s; ++i) s = run(p->L, t, y, off, nullptr, nullptr, p->ws, st);
    cudaEventRecord(b, st);
    cudaError_t e = cudaEventSynchronize(b);
    if (e != cudaSuccess) s = cuda_fail(e, "autotune timing");
    else cudaEventElapsedTime(ms, a, b);
    *ms /= reps;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return s;
}

std::string tune_key(const lsp_plan* p) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  memset(&prop, 0, sizeof prop);
  cudaGetDeviceProperties(&prop, dev);
  auto cls = [](int64_t x) { int c = 0; while (x > 1) { x >>= 1; ++c; } return c; };
  char buf[512];
  snprintf(buf, sizeof buf, "%s|sm%d|p%d|n%d|k%d|obj%d|nt%d|nf%d", prop.name,
           prop.multiProcessorCount, p->opts.precision, p->opts.norm, p->opts.top_k,
           cls(p->n_obj), cls(p->n_obj ? p->total_nt / p->n_obj : 0), cls(p->grid.n_f));
  return buf;
}

bool cache_lookup(const char* path, const std::string& key, lsp_config* c) {
  std::ifstream f(path);
  if (!f) return false;
  std::string line;
  bool found = false;
  const std::string needle = "\"key\": \"" + key + "\"";
  while (std::getline(f, line)) {
    if (line.find(needle) == std::string::npos) continue;
    lsp_config t;
    memset(&t, 0, sizeof t);
    auto get = [&](const char* name, int32_t* v) {
      std::string k = std::string("\"") + name + "\": ";
      size_t at = line.find(k);
      if (at == std::string::npos) return false;
      return sscanf(line.c_str() + at + k.size(), "%d", v) == 1;
    };
    if (get("k_reseed", &t.k_reseed) && get("freqs_per_thread", &t.freqs_per_thread) &&
        get("block_threads", &t.block_threads) && get("obs_split", &t.obs_split) &&
        get("packed", &t.packed)) {
      get("trig", &t.trig);        // absent in older entries: 0
      get("staging", &t.staging);
      *c = t;
      found = true;
    }
  }
  return found;
}

void cache_store(const char* path, const std::string& key, const lsp_config& c, float ms, double err) {
  std::ofstream f(path, std::ios::app);
  if (!f) return;
  f << "{\"key\": \"" << key << "\", \"k_reseed\": " << c.k_reseed << ", \"freqs_per_thread\": "
    << c.freqs_per_thread << ", \"block_threads\": " << c.block_threads << ", \"obs_split\": "
    << c.obs_split << ", \"packed\": " << c.packed << ", \"trig\": " << c.trig << ", \"staging\": "
    << c.staging << ", \"ms\": " << ms << ", \"max_err\": " << err
    << "}\n";
}

// Number of object groups of the host entry point (power_bytes: the size of
// the periodogram it returns, 0 for peaks only).
int host_parts_for(const lsp_plan* p, size_t power_bytes) {
  int parts = p->host_parts;
  if (parts == 0) {
    const size_t in_bytes = (size_t)p->total_nt * (p->opts.precision == LSP_FP64 ? 16 : 12);
    parts = power_bytes >= ((size_t)256 << 20) ? 8 : in_bytes >= ((size_t)64 << 20) ? 4 : 1;
  }
  const int64_t most = p->n_obj / 2;  // every group a batch of >= 2 objects
  if (parts > most) parts = (int)most;
  return parts < 1 ? 1 : parts;
}

// Group boundaries first[0..parts] (objects).  With a periodogram to return,
// groups of (nearly) equal object counts: each group's rows leave while the
// next group computes, and the last group's copy is the exposed one.  Without
// one, the groups' observation counts grow four-fold (1 : 4 : 16 : ...): a
// group's inputs arrive while the previous group computes, so only the first,
// smallest group's copy is exposed.  Offsets are monotonic here; more than 16
// groups, or a boundary that would leave a group under two objects, fall back
// to equal counts.
void host_group_bounds(const lsp_plan* p, int parts, const int64_t* offsets, bool by_count,
                       std::vector<int64_t>& first) {
  const int64_t n = p->n_obj;
  first.assign((size_t)parts + 1, 0);
  for (int j = 0; j <= parts; ++j) first[(size_t)j] = n * j / parts;
  if (by_count || parts > 16) return;
  std::vector<int64_t> g((size_t)parts + 1, 0);
  const double nt = (double)(offsets[n] - offsets[0]);
  double w = 1.0, cum = 0.0, all = 0.0;
  for (int j = 0; j < parts; ++j, w *= 4.0) all += w;
  w = 1.0;
  g[(size_t)parts] = n;
  for (int j = 1; j < parts; ++j, w *= 4.0) {
    cum += w;
    const int64_t target = offsets[0] + (int64_t)(nt * (cum / all));
    g[(size_t)j] = std::lower_bound(offsets, offsets + n + 1, target) - offsets;
  }
  for (int j = 0; j < parts; ++j)
    if (g[(size_t)j + 1] - g[(size_t)j] < 2) return;
  first.swap(g);
}

// The host entry point in `parts` contiguous object groups (the overlap of
// transfers with computation of Section 3.5).  Each group's observations are
// copied on a second stream, and the group runs as a batch of its own on `s`
// once they have arrived, while the next group's copy proceeds; with a
// periodogram to return, a third stream copies each group's rows of the
// device power buffer to power_out while the next group computes.  An
// object's powers and peaks do not depend on the other objects of its batch,
// so the results equal those of one pass bit for bit.  The groups share the
// plan's workspace, which only kernels on `s` touch.
lsp_status execute_host_parts(lsp_plan* p, int parts, const double* t, const void* y, const int64_t* offsets,
                              void* power_out, bool want_peaks, cudaStream_t s) {
  const Layout& F = p->L;
  const size_t ysz = F.prec == LSP_FP64 ? 8 : 4;
  const size_t row = (size_t)F.n_f * ysz;
  std::vector<Layout> G((size_t)parts);
  std::vector<int64_t> first;
  host_group_bounds(p, parts, offsets, power_out != nullptr, first);
  size_t ws_need = 0;
  p->h_rel.assign((size_t)(p->n_obj + parts), 0);
  for (int j = 0; j < parts; ++j) {
    const int64_t a = first[(size_t)j], b = first[(size_t)j + 1];
    for (int64_t i = a; i <= b; ++i) p->h_rel[(size_t)(i + j)] = offsets[i] - offsets[a];
    lsp_status st = resolve(b - a, offsets[b] - offsets[a], &p->grid, &p->opts, &p->cfg, &G[(size_t)j]);
    if (st) return st;
    if (G[(size_t)j].total > ws_need) ws_need = G[(size_t)j].total;
  }
  lsp_status st = ensure_ws(p, ws_need);
  if (st) return st;
  const size_t rel_bytes = p->h_rel.size() * sizeof(int64_t);
  if (rel_bytes > p->d_rel_cap) {
    cudaFree(p->d_rel);
    p->d_rel = nullptr;
    p->d_rel_cap = 0;
    if (cudaMalloc(&p->d_rel, rel_bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(LSP_E_NOMEM, "group offsets of %zu bytes", rel_bytes);
    }
    p->d_rel_cap = rel_bytes;
  }
  if (!p->copy_stream)
    LSP_CUDA(cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking), "copy stream");
  if (!p->in_stream) LSP_CUDA(cudaStreamCreateWithFlags(&p->in_stream, cudaStreamNonBlocking), "input stream");
  if (!p->copy_done) LSP_CUDA(cudaEventCreateWithFlags(&p->copy_done, cudaEventDisableTiming), "event");
  if (!p->start_ev) LSP_CUDA(cudaEventCreateWithFlags(&p->start_ev, cudaEventDisableTiming), "event");
  while (p->part_ev.size() < (size_t)parts) {
    cudaEvent_t e;
    LSP_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
    p->part_ev.push_back(e);
  }
  while (p->in_ev.size() < (size_t)parts) {
    cudaEvent_t e;
    LSP_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
    p->in_ev.push_back(e);
  }
  LSP_CUDA(cudaMemcpyAsync(p->d_rel, p->h_rel.data(), rel_bytes, cudaMemcpyHostToDevice, s), "H2D group offsets");
  // the input copies come after the work enqueued on `s` before this call
  LSP_CUDA(cudaEventRecord(p->start_ev, s), "start event");
  LSP_CUDA(cudaStreamWaitEvent(p->in_stream, p->start_ev, 0), "input wait");
  // each group's copy, then its kernels: a copy from pageable memory holds the
  // calling thread while it stages, so enqueued in this order it still
  // overlaps the previous group's kernels
  for (int j = 0; j < parts; ++j) {
    const int64_t a = first[(size_t)j], b = first[(size_t)j + 1];
    const int64_t o = offsets[a], m = offsets[b] - offsets[a];
    if (m > 0) {
      LSP_CUDA(cudaMemcpyAsync(p->d_t + o, t + o, (size_t)m * sizeof(double), cudaMemcpyHostToDevice,
                               p->in_stream), "H2D t group");
      LSP_CUDA(cudaMemcpyAsync((char*)p->d_y + o * ysz, (const char*)y + o * ysz, (size_t)m * ysz,
                               cudaMemcpyHostToDevice, p->in_stream), "H2D y group");
    }
    LSP_CUDA(cudaEventRecord(p->in_ev[(size_t)j], p->in_stream), "input event");
    LSP_CUDA(cudaStreamWaitEvent(s, p->in_ev[(size_t)j], 0), "group wait");
    st = run(G[(size_t)j], p->d_t + o, (const char*)p->d_y + o * ysz, p->d_rel + a + j,
             power_out ? (char*)p->d_power + a * row : nullptr,
             want_peaks ? p->d_peaks + a * p->opts.top_k : nullptr, p->ws, s);
    if (st) return st;
    LSP_CUDA(cudaEventRecord(p->part_ev[(size_t)j], s), "group event");
  }
  if (power_out) {
    // the copies after every group's kernels: a copy into pageable memory
    // may hold the calling thread until it ends
    for (int j = 0; j < parts; ++j) {
      const int64_t a = first[(size_t)j], b = first[(size_t)j + 1];
      LSP_CUDA(cudaStreamWaitEvent(p->copy_stream, p->part_ev[(size_t)j], 0), "copy wait");
      LSP_CUDA(cudaMemcpyAsync((char*)power_out + a * row, (const char*)p->d_power + a * row, (b - a) * row,
                               cudaMemcpyDeviceToHost, p->copy_stream),
               "D2H power group");
    }
    LSP_CUDA(cudaEventRecord(p->copy_done, p->copy_stream), "copy event");
    LSP_CUDA(cudaStreamWaitEvent(s, p->copy_done, 0), "join copies");
  }
  // the input stream rejoins `s` (its last event is already waited on)
  return LSP_OK;
}

}  // namespace

extern "C" {

lsp_status lsp_plan_create(lsp_plan** plan, int64_t n_obj, int64_t total_nt, const lsp_grid* grid,
                           const lsp_opts* opts) {
  g_err.clear();
  if (!plan) return fail(LSP_E_ARG, "plan is NULL");
  *plan = nullptr;
  if (n_obj < 1) return fail(LSP_E_ARG, "a plan needs n_obj >= 1");
  Layout L;
  lsp_status st = resolve(n_obj, total_nt, grid, opts, nullptr, &L);
  if (st) return st;
  lsp_plan* p = new lsp_plan();
  p->L = L;
  p->grid = *grid;
  p->opts = opts ? *opts : lsp_default_opts();
  p->cfg = config_of(L);
  p->n_obj = n_obj;
  p->total_nt = total_nt;
  cudaGetDevice(&p->device);
  if ((st = ensure_ws(p, L.total))) {
    delete p;
    return st;
  }
  if (cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    lsp_plan_destroy(p);
    return fail(LSP_E_CUDA, "plan stream");
  }
  *plan = p;
  return LSP_OK;
}

void lsp_plan_destroy(lsp_plan* p) {
  if (!p) return;
  drop_graph(p);
  if (p->ev0) cudaEventDestroy(p->ev0);
  if (p->ev1) cudaEventDestroy(p->ev1);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  cudaFree(p->ws);
  cudaFree(p->d_t);
  cudaFree(p->d_y);
  cudaFree(p->d_off);
  cudaFree(p->d_peaks);
  cudaFree(p->d_power);
  cudaFree(p->d_rel);
  for (cudaEvent_t e : p->part_ev) cudaEventDestroy(e);
  for (cudaEvent_t e : p->in_ev) cudaEventDestroy(e);
  if (p->copy_done) cudaEventDestroy(p->copy_done);
  if (p->start_ev) cudaEventDestroy(p->start_ev);
  if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
  if (p->in_stream) cudaStreamDestroy(p->in_stream);
  delete p;
}

lsp_status lsp_plan_enable_timing(lsp_plan* p, int32_t enable) {
  g_err.clear();
  if (!p) return fail(LSP_E_ARG, "plan is NULL");
  drop_graph(p);
  if (p->ev0) cudaEventDestroy(p->ev0);
  if (p->ev1) cudaEventDestroy(p->ev1);
  p->ev0 = p->ev1 = nullptr;
  if (enable) {
    LSP_CUDA(cudaEventCreate(&p->ev0), "timing event");
    LSP_CUDA(cudaEventCreate(&p->ev1), "timing event");
  }
  return LSP_OK;
}

lsp_status lsp_plan_main_kernel_ms(lsp_plan* p, float* ms) {
  g_err.clear();
  if (!p || !ms) return fail(LSP_E_ARG, "NULL argument");
  if (!p->ev0) return fail(LSP_E_ARG, "timing is not enabled on this plan");
  LSP_CUDA(cudaEventSynchronize(p->ev1), "timing event");
  LSP_CUDA(cudaEventElapsedTime(ms, p->ev0, p->ev1), "timing event");
  return LSP_OK;
}

lsp_status lsp_plan_kernel_count(const lsp_plan* p, int32_t* count) {
  if (!p || !count) return fail(LSP_E_ARG, "NULL argument");
  const Layout& L = p->L;
  // statistics + records (one fused launch for a short single object) + main
  // (+ 3 for the LPT order) (+ combine) (+ finalize, which a split single
  // object with a first-maximum output folds into the combine); peaks
  // requested; plans of one object run without offsets
  const bool fused = L.split > 1 && !L.top;
  const bool one_prologue = L.n_obj == 1 && L.total_nt <= kFusedMaxNt;
  *count = (one_prologue ? 2 : 3) + (L.n_obj > 1 ? 3 : 0) + (L.split > 1 ? 1 : 0) + (fused ? 0 : 1);
  return LSP_OK;
}

lsp_status lsp_plan_gate_report(const lsp_plan* p, int64_t* objects, float* max_err, int32_t cap,
                                int32_t* n) {
  if (!p || !n || cap < 0 || (cap > 0 && (!objects || !max_err))) return fail(LSP_E_ARG, "bad argument");
  *n = (int32_t)p->gate_obj.size();
  for (int32_t i = 0; i < cap && i < *n; ++i) {
    objects[i] = p->gate_obj[(size_t)i];
    max_err[i] = i < (int32_t)p->gate_err.size() ? (float)p->gate_err[(size_t)i] : -1.0f;
  }
  return LSP_OK;
}

lsp_status lsp_plan_get_config(const lsp_plan* p, lsp_config* c) {
  if (!p || !c) return fail(LSP_E_ARG, "NULL argument");
  *c = p->cfg;
  return LSP_OK;
}

lsp_status lsp_plan_set_config(lsp_plan* p, const lsp_config* c) {
  g_err.clear();
  if (!p || !c) return fail(LSP_E_ARG, "NULL argument");
  return apply_config(p, c);
}

lsp_status lsp_plan_execute(lsp_plan* p, const double* t, const void* y, const int64_t* offsets,
                            void* power_out, lsp_peak* peaks, lsp_stream_t stream) {
  g_err.clear();
  if (!p) return fail(LSP_E_ARG, "plan is NULL");
  lsp_status st = check_io(p->total_nt, t, y);
  if (st) return st;
  if (p->n_obj > 1 && !offsets) return fail(LSP_E_ARG, "offsets must not be NULL");
  const void* args[5] = {t, y, offsets, power_out, peaks};
  bool same = p->exec != nullptr;
  for (int i = 0; i < 5 && same; ++i) same = args[i] == p->cap_args[i];
  if (!same) {
    drop_graph(p);
    LSP_CUDA(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    st = run(p->L, t, y, offsets, power_out, peaks, p->ws, p->cap_stream, p->ev0, p->ev1);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(p->cap_stream, &g);
    if (st) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    p->graph = g;
    e = cudaGraphInstantiate(&p->exec, g, 0);
    if (e != cudaSuccess) {
      drop_graph(p);
      return cuda_fail(e, "graph instantiate");
    }
    for (int i = 0; i < 5; ++i) p->cap_args[i] = args[i];
  }
  LSP_CUDA(cudaGraphLaunch(p->exec, (cudaStream_t)stream), "graph launch");
  return LSP_OK;
}

static lsp_status execute_host_impl(lsp_plan* p, const double* t, const void* y,
                                    const int64_t* offsets, void* power_out, lsp_peak* peaks,
                                    lsp_stream_t stream) {
  g_err.clear();
  if (!p) return fail(LSP_E_ARG, "plan is NULL");
  lsp_status st = check_io(p->total_nt, t, y);
  if (st) return st;
  if (p->n_obj > 1 && !offsets) return fail(LSP_E_ARG, "offsets must not be NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t ysz = p->opts.precision == LSP_FP64 ? 8 : 4;
  const size_t n_peaks = (size_t)p->n_obj * p->opts.top_k;
  const size_t pbytes = (size_t)p->n_obj * p->grid.n_f * ysz;
  auto alloc = [&](void** ptr, size_t bytes) -> lsp_status {
    if (*ptr) return LSP_OK;
    if (cudaMalloc(ptr, bytes ? bytes : 16) != cudaSuccess) {
      cudaGetLastError();
      return fail(LSP_E_NOMEM, "staging buffer of %zu bytes", bytes);
    }
    return LSP_OK;
  };
  if ((st = alloc((void**)&p->d_t, p->total_nt * sizeof(double)))) return st;
  if ((st = alloc(&p->d_y, p->total_nt * ysz))) return st;
  if ((st = alloc((void**)&p->d_off, (p->n_obj + 1) * sizeof(int64_t)))) return st;
  if ((st = alloc((void**)&p->d_peaks, n_peaks * sizeof(lsp_peak)))) return st;
  // A page-locked, device-addressable power_out is written by the kernels
  // directly (zero copy over the chip-to-chip link); otherwise stage it.
  void* power_direct = nullptr;
  if (power_out) {
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, power_out) == cudaSuccess && attr.type == cudaMemoryTypeHost &&
        attr.devicePointer)
      power_direct = attr.devicePointer;
    cudaGetLastError();
  }
  int parts = host_parts_for(p, power_out ? pbytes : 0);
  if (parts > 1) {
    // groups index t and y by the offsets: they need monotonic offsets inside
    // the inputs (others take the one-pass route, which flags the objects)
    bool ok = offsets[0] >= 0 && offsets[p->n_obj] <= p->total_nt;
    for (int64_t i = 0; ok && i < p->n_obj; ++i) ok = offsets[i] <= offsets[i + 1];
    if (!ok) parts = 1;
  }
  if (parts > 1) power_direct = nullptr;
  if (power_out && !power_direct && (st = alloc(&p->d_power, pbytes))) return st;
  if (parts > 1) {
    if ((st = execute_host_parts(p, parts, t, y, offsets, power_out, peaks != nullptr, s))) return st;
    if (peaks)
      LSP_CUDA(cudaMemcpyAsync(peaks, p->d_peaks, n_peaks * sizeof(lsp_peak), cudaMemcpyDeviceToHost, s),
               "D2H peaks");
    LSP_CUDA(cudaStreamSynchronize(s), "synchronize");
    return LSP_OK;
  }
  LSP_CUDA(cudaMemcpyAsync(p->d_t, t, p->total_nt * sizeof(double), cudaMemcpyHostToDevice, s), "H2D t");
  LSP_CUDA(cudaMemcpyAsync(p->d_y, y, p->total_nt * ysz, cudaMemcpyHostToDevice, s), "H2D y");
  const int64_t* d_off = nullptr;
  if (offsets) {
    LSP_CUDA(cudaMemcpyAsync(p->d_off, offsets, (p->n_obj + 1) * sizeof(int64_t),
                             cudaMemcpyHostToDevice, s), "H2D offsets");
    d_off = p->d_off;
  }
  st = lsp_plan_execute(p, p->d_t, p->d_y, d_off,
                        power_direct ? power_direct : (power_out ? p->d_power : nullptr),
                        peaks ? p->d_peaks : nullptr, stream);
  if (st) return st;
  if (peaks)
    LSP_CUDA(cudaMemcpyAsync(peaks, p->d_peaks, n_peaks * sizeof(lsp_peak), cudaMemcpyDeviceToHost, s),
             "D2H peaks");
  if (power_out && !power_direct)
    LSP_CUDA(cudaMemcpyAsync(power_out, p->d_power, pbytes, cudaMemcpyDeviceToHost, s), "D2H power");
  LSP_CUDA(cudaStreamSynchronize(s), "synchronize");
  return LSP_OK;
}

lsp_status lsp_plan_execute_host(lsp_plan* p, const double* t, const void* y,
                                 const int64_t* offsets, void* power_out, lsp_peak* peaks,
                                 lsp_stream_t stream) {
  const lsp_status st = execute_host_impl(p, t, y, offsets, power_out, peaks, stream);
  if (st != LSP_OK && p) {
    // copies enqueued before the failure may still read or write the caller's
    // host buffers: let them end before the error is reported
    cudaStreamSynchronize((cudaStream_t)stream);
    if (p->copy_stream) cudaStreamSynchronize(p->copy_stream);
    if (p->in_stream) cudaStreamSynchronize(p->in_stream);
    cudaGetLastError();
  }
  return st;
}

lsp_status lsp_plan_set_host_parts(lsp_plan* p, int32_t parts) {
  g_err.clear();
  if (!p) return fail(LSP_E_ARG, "plan is NULL");
  if (parts < 0) return fail(LSP_E_ARG, "parts must be >= 0");
  p->host_parts = parts;
  return LSP_OK;
}

lsp_status lsp_plan_get_host_parts(const lsp_plan* p, int64_t power_bytes, int32_t* parts) {
  if (!p || !parts) return fail(LSP_E_ARG, "NULL argument");
  if (power_bytes < 0) return fail(LSP_E_ARG, "power_bytes must be >= 0");
  *parts = host_parts_for(p, (size_t)power_bytes);
  return LSP_OK;
}

lsp_status lsp_plan_autotune(lsp_plan* p, const double* t, const void* y, const int64_t* offsets,
                             const char* cache_path, lsp_stream_t stream) {
  return lsp_plan_autotune_ex(p, t, y, offsets, cache_path, 0, nullptr, 0, nullptr, stream);
}

lsp_status lsp_plan_autotune_ex(lsp_plan* p, const double* t, const void* y, const int64_t* offsets,
                                const char* cache_path, int32_t flags, lsp_trial* trials,
                                int32_t max_trials, int32_t* n_trials, lsp_stream_t stream) {
  g_err.clear();
  if (n_trials) *n_trials = 0;
  if (!p) return fail(LSP_E_ARG, "plan is NULL");
  if (flags & ~LSP_TUNE_ABLATIONS) return fail(LSP_E_ARG, "unknown autotune flags 0x%x", (unsigned)flags);
  if (max_trials < 0 || (max_trials > 0 && !trials)) return fail(LSP_E_ARG, "trials must hold max_trials records");
  const bool ablations = (flags & LSP_TUNE_ABLATIONS) != 0;
  lsp_status st = check_io(p->total_nt, t, y);
  if (st) return st;
  if (p->n_obj > 1 && !offsets) return fail(LSP_E_ARG, "offsets must not be NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const std::string key = tune_key(p);
  lsp_config cached;
  p->gate_obj.clear();
  p->gate_err.clear();
  if (cache_path && !ablations && cache_lookup(cache_path, key, &cached)) {
    if (!apply_config(p, &cached)) return LSP_OK;
    g_err.clear();  // stale entry: tune again
  }

  // Candidates: reseed interval K, frequencies per thread, CTA size and (one
  // object) the N_t split.
  std::vector<lsp_config> cands;
  auto add = [&](int k, int fpt, int thr, int packed, int split, int abl = 0) {
    lsp_config c;
    memset(&c, 0, sizeof c);
    c.k_reseed = k;
    c.freqs_per_thread = fpt;
    c.block_threads = thr;
    c.packed = packed;
    c.obs_split = split;
    c.trig = abl % 3;
    c.staging = abl / 3;
    if (main_variant_exists(p->opts.precision, packed, k, fpt, 0, abl)) cands.push_back(c);
  };
  std::vector<int> splits = {0};
  if (p->n_obj == 1) {
    Layout L0;
    if ((st = resolve(1, p->total_nt, &p->grid, &p->opts, nullptr, &L0))) return st;
    for (int f : {2, 4}) {
      if (L0.split * f <= kMaxSplit && p->total_nt / (L0.split * f) >= kMinObsPerSplit)
        splits.push_back(L0.split * f);
      if (L0.split / f >= 1) splits.push_back(L0.split / f);
    }
  }
  for (int sp : splits) {
    if (p->opts.precision == LSP_FP64) {
      for (int k : {4, 8, 16})
        for (int thr : {128, 256}) add(k, k, thr, 0, sp);
    } else {
      // 64-thread CTAs: the same warps per SM at K = 16 with half the chunk,
      // so a ragged last chunk wastes less (measured: 1-2 % on N_f = 5e4)
      for (int k : {4, 8, 12, 16})
        for (int thr : {64, 128, 256}) add(k, 2 * k, thr, 1, sp);
      for (int k : {8, 16}) add(k, k, 256, 0, sp);
      if (ablations)
        for (int abl = 1; abl <= 5; ++abl)
          for (int thr : {128, 256}) add(16, 16, thr, 0, sp, abl);
    }
  }

  // Error gate (FP32): each candidate's periodograms of a few objects against
  // the FP64 path -- the first object, the one with the most observations
  // (the longest FP32 sums), the worst-conditioned one of a pool (the largest
  // R/N of the spectral window at twice the frequency, where Eq. 2's smaller
  // denominator (N - R)/2 is smallest relative to N) and objects spread over
  // the batch.  Objects with fewer than two observations or offsets outside
  // the inputs are left out.
  std::vector<int64_t> gobj, gbeg, gcnt;
  auto gate_add = [&](int64_t o, int64_t b0, int64_t n0) {
    for (int64_t x : gobj)
      if (x == o) return;
    if (gobj.size() < (size_t)kGateObjects) {
      gobj.push_back(o);
      gbeg.push_back(b0);
      gcnt.push_back(n0);
    }
  };
  const bool fp32 = p->opts.precision == LSP_FP32;
  if (fp32 && p->n_obj == 1) {
    if (p->total_nt >= 2) gate_add(0, 0, p->total_nt);
  } else if (fp32) {
    std::vector<int64_t> off((size_t)p->n_obj + 1);
    LSP_CUDA(cudaMemcpyAsync(off.data(), offsets, off.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, s),
             "offsets probe");
    LSP_CUDA(cudaStreamSynchronize(s), "offsets probe");
    auto count = [&](int64_t o) -> int64_t {
      const int64_t b0 = off[(size_t)o], e0 = off[(size_t)o + 1];
      return (b0 >= 0 && e0 >= b0 && e0 <= p->total_nt) ? e0 - b0 : -1;
    };
    const int64_t n = p->n_obj;
    int64_t longest = -1;
    for (int64_t o = 0; o < n; ++o)
      if (count(o) >= 2 && (longest < 0 || count(o) > count(longest))) longest = o;
    std::vector<int64_t> spread;
    for (int i = 0; i < 5; ++i) spread.push_back(n > 1 ? (n - 1) * i / 4 : 0);
    // conditioning pool: the shortest objects (three observations or more)
    // and objects spread by index
    std::vector<int64_t> pool;
    {
      std::vector<std::pair<int64_t, int64_t>> by_n;
      for (int64_t o = 0; o < n; ++o)
        if (count(o) >= 3) by_n.push_back({count(o), o});
      const size_t k = by_n.size() < 32 ? by_n.size() : 32;
      std::partial_sort(by_n.begin(), by_n.begin() + k, by_n.end());
      for (size_t i = 0; i < k; ++i) pool.push_back(by_n[i].second);
      for (int i = 0; i < 32 && n > 0; ++i) {
        const int64_t o = (n - 1) * i / 31;
        if (count(o) >= 3 && std::find(pool.begin(), pool.end(), o) == pool.end()) pool.push_back(o);
      }
    }
    int64_t worst = -1;
    if (!pool.empty()) {
      std::vector<int64_t> pb(pool.size()), pc(pool.size());
      for (size_t i = 0; i < pool.size(); ++i) {
        pb[i] = off[(size_t)pool[i]];
        pc[i] = count(pool[i]);
      }
      int64_t* d_pool = nullptr;
      float* d_score = nullptr;
      std::vector<float> score(pool.size());
      cudaError_t e = cudaMalloc(&d_pool, 2 * pool.size() * sizeof(int64_t));
      if (e == cudaSuccess) e = cudaMalloc(&d_score, pool.size() * sizeof(float));
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_pool, pb.data(), pb.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_pool + pool.size(), pc.data(), pc.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess)
        e = launch_window_score(t, d_pool, d_pool + pool.size(), (int)pool.size(), p->grid.f_min, p->L.df,
                                p->grid.n_f, d_score, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(score.data(), d_score, score.size() * sizeof(float), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      cudaFree(d_pool);
      cudaFree(d_score);
      if (e != cudaSuccess) return cuda_fail(e, "autotune conditioning score");
      for (size_t i = 0; i < pool.size(); ++i)
        if (worst < 0 || score[i] > score[(size_t)worst]) worst = (int64_t)i;
      worst = pool[(size_t)worst];
    }
    for (int64_t o : {(int64_t)0, longest, worst})
      if (o >= 0 && count(o) >= 2) gate_add(o, off[(size_t)o], count(o));
    for (int64_t o : spread)
      if (count(o) >= 2) gate_add(o, off[(size_t)o], count(o));
  }
  const bool gate = !gobj.empty();
  // a batch plan is gated as a batch of two or more objects (one object
  // alone would take the split single-object path)
  int64_t g_rows = (int64_t)gobj.size();
  if (gate && p->n_obj > 1 && g_rows == 1) {
    gbeg.push_back(gbeg[0]);
    gcnt.push_back(gcnt[0]);
    g_rows = 2;
  }
  int64_t g_total = 0;
  for (int64_t c : gcnt) g_total += c;
  double* ref = nullptr;   // FP64 periodograms of the gate objects
  double* y64 = nullptr;
  double* gt = nullptr;    // the gate objects' observations, back to back
  float* gy = nullptr;
  int64_t* goff = nullptr;
  float* pw = nullptr;
  double* d_err = nullptr;
  char* gws = nullptr;
  size_t gws_bytes = 0;
  lsp_opts o64 = p->opts;
  o64.precision = LSP_FP64;
  o64.k_reseed = o64.freqs_per_thread = o64.block_threads = o64.obs_split = 0;
  o64.top_k = 1;
  o64.norm = LSP_NORM_STANDARD;  // the gate compares P_n (1e-4 absolute)
  lsp_opts o1 = p->opts;
  o1.top_k = 1;
  o1.norm = LSP_NORM_STANDARD;
  auto cleanup = [&]() {
    cudaFree(ref);
    cudaFree(y64);
    cudaFree(gt);
    cudaFree(gy);
    cudaFree(goff);
    cudaFree(pw);
    cudaFree(d_err);
    cudaFree(gws);
  };
  const int64_t g_nobj = p->n_obj == 1 ? 1 : g_rows;
  if (gate) {
    Layout L64;
    if ((st = resolve(g_nobj, g_total, &p->grid, &o64, nullptr, &L64))) return st;
    gws_bytes = L64.total;
    for (const auto& c : cands) {  // room for every candidate's layout too
      Layout Lc;
      if (!resolve(g_nobj, g_total, &p->grid, &o1, &c, &Lc) && Lc.total > gws_bytes) gws_bytes = Lc.total;
    }
    g_err.clear();
    const size_t rows = (size_t)g_rows;
    if (cudaMalloc(&ref, rows * p->grid.n_f * sizeof(double)) || cudaMalloc(&y64, g_total * sizeof(double)) ||
        cudaMalloc(&gt, g_total * sizeof(double)) || cudaMalloc(&gy, g_total * sizeof(float)) ||
        cudaMalloc(&goff, (rows + 1) * sizeof(int64_t)) || cudaMalloc(&pw, rows * p->grid.n_f * sizeof(float)) ||
        cudaMalloc(&d_err, rows * sizeof(double)) || cudaMalloc(&gws, gws_bytes)) {
      cudaGetLastError();
      cleanup();
      return fail(LSP_E_NOMEM, "autotune scratch");
    }
    std::vector<int64_t> hoff(rows + 1, 0);
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; i < rows && e == cudaSuccess; ++i) {
      hoff[i + 1] = hoff[i] + gcnt[i];
      e = cudaMemcpyAsync(gt + hoff[i], t + gbeg[i], gcnt[i] * sizeof(double), cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(gy + hoff[i], (const float*)y + gbeg[i], gcnt[i] * sizeof(float),
                            cudaMemcpyDeviceToDevice, s);
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(goff, hoff.data(), hoff.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_f32_to_f64(gy, y64, g_total, s);
    // the host offsets must outlive the copy
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "autotune gate inputs"); }
    if ((st = run(L64, gt, y64, g_nobj > 1 ? goff : nullptr, ref, nullptr, gws, s))) { cleanup(); return st; }
  }
  std::vector<double> cur_err((size_t)g_rows), best_obj_err;

  float best_ms = 1e30f;
  double best_err = 0.0;
  lsp_config best = p->cfg;
  bool any = false;
  int32_t n_meas = 0;
  auto record = [&](const lsp_config& c, float ms, double err, bool passed, int64_t worst_obj) {
    if (n_meas < max_trials) {
      lsp_trial& tr = trials[n_meas];
      memset(&tr, 0, sizeof tr);
      tr.config = c;
      tr.ms = ms;
      tr.max_err = (float)err;
      tr.passed = passed ? 1 : 0;
      tr.worst_object = (int32_t)worst_obj;
    }
    ++n_meas;
    if (n_trials) *n_trials = n_meas;
  };
  for (const auto& c : cands) {
    Layout Lc;
    if (resolve(p->n_obj, p->total_nt, &p->grid, &p->opts, &c, &Lc)) { g_err.clear(); continue; }
    double err = 0.0;
    int64_t worst_obj = -1;
    if (gate) {
      // the candidate's own configuration (a single object keeps its split)
      Layout Lg;
      if (resolve(g_nobj, g_total, &p->grid, &o1, &c, &Lg)) { g_err.clear(); continue; }
      if ((st = run(Lg, gt, gy, g_nobj > 1 ? goff : nullptr, pw, nullptr, gws, s))) { cleanup(); return st; }
      cudaError_t e = launch_row_max_abs_diff(pw, ref, g_rows, p->grid.n_f, d_err, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(cur_err.data(), d_err, cur_err.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "autotune gate"); }
      for (size_t i = 0; i < gobj.size(); ++i)
        if (!(cur_err[i] <= err)) {  // NaN counts as the worst
          err = std::isnan(cur_err[i]) ? INFINITY : cur_err[i];
          worst_obj = gobj[i];
        }
      if (!(err <= 1e-4)) {
        record(c, -1.f, err, false, worst_obj);
        continue;
      }
    }
    if ((st = ensure_ws(p, Lc.total))) { cleanup(); return st; }
    Layout saved = p->L;
    p->L = Lc;
    float ms = 0.f;
    st = time_runs(p, t, y, offsets, 3, s, &ms);
    p->L = saved;
    if (st) { cleanup(); return st; }
    record(config_of(Lc), ms, err, true, worst_obj);
    if (ms < best_ms) {
      best_ms = ms;
      best = config_of(Lc);
      best_err = err;
      best_obj_err.assign(cur_err.begin(), cur_err.begin() + (gate ? (ptrdiff_t)gobj.size() : 0));
      any = true;
    }
  }
  cleanup();
  if (!any) return fail(LSP_E_NUMERIC, "no candidate configuration passed the error gate");
  if ((st = apply_config(p, &best))) return st;
  p->gate_obj = gobj;
  p->gate_err.assign(best_obj_err.begin(), best_obj_err.end());
  if (cache_path) cache_store(cache_path, key, best, best_ms, best_err);
  return LSP_OK;
}

}  // extern "C"
