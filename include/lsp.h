/*
 * lsp.h -- C ABI of the GB300 (sm_103a) Lomb-Scargle periodogram library.
 *
 * The library computes the direct O(N_t * N_f) Lomb-Scargle periodogram of
 * Gowanlock et al. (arXiv:2105.04006) for one light curve or for a ragged
 * batch of light curves, and the period given by each periodogram's maximum.
 *
 *   Section 2, Eq. 1:  tan(2 w tau) = sum_j sin(2 w t_j) / sum_j cos(2 w t_j)
 *   Section 2, Eq. 2:  P(f) = 1/2 ( [sum_j y_j cos w(t_j-tau)]^2 / sum_j cos^2 w(t_j-tau)
 *                                 + [sum_j y_j sin w(t_j-tau)]^2 / sum_j sin^2 w(t_j-tau) )
 *   with w = 2 pi f, y the zero-mean magnitudes (Section 2), and the
 *   half-open grid f_k = f_min + k (f_max - f_min)/N_f, k = 0..N_f-1 (Section 2).
 *
 * Conventions shared by every entry point:
 *   - Frequencies are in cycles per unit of t (e.g. cycles/day); the period
 *     of bin k is 1/f_k.  (The paper's grid is angular, w = 2 pi f.)
 *   - Unless stated otherwise, array arguments are DEVICE pointers owned by
 *     the caller; the library never frees them and never keeps them past
 *     the call (plans keep nothing either, except what lsp_plan_execute
 *     captured into a CUDA graph, see there).
 *   - An output array (power_out, peaks) may also be page-locked host memory
 *     that the GPU can address (cudaHostAlloc, cudaHostRegister, or a pinned
 *     torch tensor): the kernels then write the periodogram straight to the
 *     host while they compute -- the library's form of the paper's
 *     periodogram return (Section 3.5), without staging buffers.
 *   - Every compute entry point is asynchronous on `stream` (0 = the legacy
 *     default stream) and performs no device allocation: scratch memory is
 *     the caller's `workspace` (size from lsp_workspace_size) or a plan's.
 *   - Arguments are validated on the host before anything is launched; a
 *     failure returns a nonzero lsp_status, launches nothing, and leaves a
 *     message for lsp_last_error() (per calling thread).
 *   - Problems of one object (fewer than two observations, zero variance,
 *     NaN/Inf input) do not fail the call: that object gets power 0,
 *     idx -1 and a nonzero lsp_peak.flags.
 *   - Results are deterministic: two calls with the same inputs and options
 *     give bit-identical outputs.  Ties of the maximum go to the lowest
 *     frequency index (the first maximum, Section 3.3).
 */
#ifndef LSP_H
#define LSP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t (the CUDA runtime's stream handle); 0 = legacy default stream. */
typedef struct CUstream_st* lsp_stream_t;

typedef enum lsp_status {
  LSP_OK = 0,
  LSP_E_ARG = 1,         /* invalid argument; nothing was launched */
  LSP_E_CUDA = 2,        /* a CUDA runtime call failed (launch, copy, graph) */
  LSP_E_NOMEM = 3,       /* a plan could not allocate its device memory */
  LSP_E_WORKSPACE = 4,   /* the caller's workspace is smaller than required */
  LSP_E_NUMERIC = 5,     /* reserved: per-object problems go to lsp_peak.flags */
  LSP_E_TIMEOUT = 6,     /* a bounded device-side wait gave up */
  LSP_E_UNSUPPORTED = 7  /* a valid request this build does not implement */
} lsp_status;

typedef enum lsp_precision {
  LSP_FP32 = 0, /* trig sums in FP32; phases reduced in FP64 / fixed point (y, power: float) */
  LSP_FP64 = 1  /* everything in FP64 (y, power: double) */
} lsp_precision;

typedef enum lsp_norm {
  LSP_NORM_PSD = 0,      /* P of Eq. 2, in units of y^2 */
  LSP_NORM_STANDARD = 1  /* P_n = 2 P / sum_j (y_j - mean)^2, in [0, 1] */
} lsp_norm;

/* Per-object flags (lsp_peak.flags). */
#define LSP_FLAG_FEW_OBS 1     /* fewer than two observations */
#define LSP_FLAG_ZERO_VAR 2    /* the (centred) magnitudes are all zero */
#define LSP_FLAG_NONFINITE 4   /* a NaN or Inf in the object's t or y */
#define LSP_FLAG_BAD_OFFSETS 8 /* offsets[o+1] < offsets[o] or outside [0, total_nt] */

/* Half-open evenly spaced grid [f_min, f_max) of n_f frequencies (Section 2). */
typedef struct lsp_grid {
  double f_min; /* > 0 (Eq. 1 divides by 2w) */
  double f_max; /* > f_min */
  int64_t n_f;  /* >= 1 */
} lsp_grid;

/* Options.  Zero-initialise and set what you need, or use lsp_default_opts(). */
typedef struct lsp_opts {
  int32_t precision;     /* lsp_precision (default LSP_FP32) */
  int32_t norm;          /* lsp_norm (default LSP_NORM_STANDARD) */
  int32_t center_y;      /* nonzero: subtract each object's mean of y, in FP64 (default 1) */
  int32_t top_k;         /* peaks per object, 1..3 (default 1); 2..3 = largest local maxima */
  int32_t k_reseed;      /* frequencies between exact sin/cos reseeds; 0 = tuned default */
  int32_t freqs_per_thread; /* frequencies per thread (multiple of k_reseed); 0 = tuned default */
  int32_t block_threads; /* threads per CTA of the main kernel (64..256, /32); 0 = default */
  int32_t obs_split;     /* single object: N_t split over this many CTAs; 0 = auto */
} lsp_opts;

/* One peak.  For top_k = 1 it is the periodogram's first maximum. */
typedef struct lsp_peak {
  int64_t idx;    /* grid index, -1 if the object has none (flags != 0) */
  double power;   /* power at idx in the requested normalisation */
  double freq;    /* f_min + idx (f_max - f_min)/n_f */
  double period;  /* 1 / freq */
  int32_t flags;  /* LSP_FLAG_* of the object */
  int32_t reserved;
} lsp_peak; /* 40 bytes */

/* ---- status ------------------------------------------------------------ */

const char* lsp_status_string(lsp_status status);
/* Text of the last failure in the calling thread ("" if none). */
const char* lsp_last_error(void);
lsp_opts lsp_default_opts(void);
/* Library version, as major*10000 + minor*100 + patch. */
int32_t lsp_version(void);

/*
 * Grid-selection rule of Section 4.3: spacing df = 0.1 / t_span in cycles
 * per unit time (the paper's 0.2 pi / T_max in angular frequency; t_span is
 * the observing window, the largest one of a batch) and
 * n_f = round((f_max - f_min) / df).  Writes *grid = {f_min, f_max, n_f};
 * LSP_E_ARG for a non-positive span or an empty range.
 */
lsp_status lsp_grid_for_span(double f_min, double f_max, double t_span, lsp_grid* grid);

/* ---- one-shot entry points -------------------------------------------- */

/*
 * Bytes of device workspace that lsp_periodogram (n_obj = 1) or lsp_batch
 * need for this shape and options.  Writes *bytes; never launches anything.
 */
lsp_status lsp_workspace_size(int64_t n_obj, int64_t total_nt, const lsp_grid* grid,
                              const lsp_opts* opts, size_t* bytes);

/*
 * Single-object mode (Section 3.3).  t[n_t] (double) and y[n_t] (float for
 * LSP_FP32, double for LSP_FP64) hold one light curve, in any time order.
 * power_out (nullable) receives n_f powers of the precision's type -- the
 * paper's "return the periodogram or not" option; leaving it NULL keeps the
 * periodogram out of HBM entirely.  peaks (nullable) receives opts->top_k
 * lsp_peak entries.  workspace must hold lsp_workspace_size(1, n_t, ...)
 * bytes and be 256-byte aligned; the call may use all of it.
 */
lsp_status lsp_periodogram(const double* t, const void* y, int64_t n_t, const lsp_grid* grid,
                           const lsp_opts* opts, void* power_out, lsp_peak* peaks,
                           void* workspace, size_t ws_bytes, lsp_stream_t stream);

/*
 * Batch mode (Section 3.4) over a CSR layout: object o owns
 * t/y[offsets[o] .. offsets[o+1]), offsets has n_obj + 1 int64 entries with
 * offsets[0] = 0 and offsets[n_obj] = total_nt (device array; a violated
 * entry flags the objects it touches with LSP_FLAG_BAD_OFFSETS instead of
 * being read out of bounds).  All objects share one grid.  power_out
 * (nullable) is n_obj x n_f, row-major; peaks (nullable) is n_obj x top_k.
 * One launch sequence covers the whole batch: a prologue, a persistent
 * main kernel that pulls (object, frequency-chunk) items from a queue
 * ordered by decreasing N_t, and a finalize kernel.
 */
lsp_status lsp_batch(const double* t, const void* y, const int64_t* offsets, int64_t n_obj,
                     int64_t total_nt, const lsp_grid* grid, const lsp_opts* opts,
                     void* power_out, lsp_peak* peaks, void* workspace, size_t ws_bytes,
                     lsp_stream_t stream);

/*
 * lsp_batch without a caller workspace, for callers that cannot allocate
 * device memory (a real-time pipeline whose device-memory budget is fixed at
 * start-up, a plugin whose host framework has reserved the device memory for
 * its own pool, a C caller without a device allocator).  The paper has no
 * counterpart: this is a deployment convenience of this library.
 * Arguments and results are those of lsp_batch; the scratch memory is a
 * fixed device array of LSP_NOALLOC_SCRATCH_BYTES inside the library.  A
 * shape whose lsp_workspace_size exceeds it returns LSP_E_WORKSPACE,
 * launching nothing; an empty batch returns LSP_OK at once.  The call
 * allocates nothing itself.  The CUDA runtime reserves the array in a
 * device's memory when it loads the library's module there -- with lazy
 * module loading, at the first lsp_noalloc_prepare or lsp_batch_noalloc on
 * that device -- and keeps it until the process exits; a caller that must
 * not see that reservation later calls lsp_noalloc_prepare at start-up.  If
 * the device has no room for it the call returns LSP_E_NOMEM.  All calls
 * share the one array: calls that overlap on the GPU (different streams or
 * unordered host threads) race on it, so order them.  Each call clears what
 * must start at zero.  The array's address is looked up once per device,
 * with that device current, in the runtime's primary context: make the
 * first call outside any stream capture, and call lsp_noalloc_prepare again
 * after cudaDeviceReset or when another context is current.
 */
#define LSP_NOALLOC_SCRATCH_BYTES (32u << 20)
lsp_status lsp_batch_noalloc(const double* t, const void* y, const int64_t* offsets, int64_t n_obj,
                             int64_t total_nt, const lsp_grid* grid, const lsp_opts* opts,
                             void* power_out, lsp_peak* peaks, lsp_stream_t stream);
/* Reserves the scratch array of lsp_batch_noalloc on the current device (if
 * not yet done) and looks its address up afresh.  LSP_E_NOMEM if the device
 * has no room for it, LSP_E_CUDA for another runtime error. */
lsp_status lsp_noalloc_prepare(void);

/*
 * Generalized periodogram (Section 4.11: photometric errors, floating
 * mean).  The paper ports Astropy's implementation without giving a
 * formula; this library computes, at each grid frequency, the weighted
 * least-squares fit y ~ a cos(wt) + b sin(wt) + c with weights 1/dy^2 and
 * the power P = 1 - chi2_min(w) / chi2_0 (chi2_0 about the weighted mean) for
 * LSP_NORM_STANDARD, or (chi2_0 - chi2_min)/2 for LSP_NORM_PSD.  dy has y's
 * type and layout (NULL: unit weights).  Objects need at least three
 * observations; a non-positive or non-finite dy flags LSP_FLAG_NONFINITE.
 * Arguments otherwise as lsp_batch / lsp_periodogram; the workspace size
 * comes from lsp_workspace_size_gls.  A single object is split over its
 * observations as in lsp_periodogram (opts.obs_split; automatic: every
 * partial sum over at most 8192 observations, and enough items for all SMs),
 * the six weighted sums of the slices added in a fixed order.
 */
lsp_status lsp_workspace_size_gls(int64_t n_obj, int64_t total_nt, const lsp_grid* grid,
                                  const lsp_opts* opts, size_t* bytes);
lsp_status lsp_batch_gls(const double* t, const void* y, const void* dy, const int64_t* offsets,
                         int64_t n_obj, int64_t total_nt, const lsp_grid* grid, const lsp_opts* opts,
                         void* power_out, lsp_peak* peaks, void* workspace, size_t ws_bytes,
                         lsp_stream_t stream);
lsp_status lsp_periodogram_gls(const double* t, const void* y, const void* dy, int64_t n_t,
                               const lsp_grid* grid, const lsp_opts* opts, void* power_out,
                               lsp_peak* peaks, void* workspace, size_t ws_bytes, lsp_stream_t stream);

/*
 * Period of stored periodograms (Section 3.3's separate argmax step):
 * power is n_obj x n_f of type float (LSP_FP32) or double (LSP_FP64); each
 * row's first maximum is written to peaks[o] (idx, power, freq, period;
 * flags 0).  NaN entries are never selected.  No workspace is needed.
 */
lsp_status lsp_argmax_period(const void* power, int64_t n_obj, int64_t n_f, const lsp_grid* grid,
                             int32_t precision, lsp_peak* peaks, lsp_stream_t stream);

/* ---- plans: tuned, graph-captured repeats ------------------------------ */

typedef struct lsp_plan lsp_plan;

/*
 * The launch configuration a plan uses (see lsp_plan_autotune).  trig and
 * staging select the ablation kernels of the paper's own comparisons
 * (Section 3.6 and Table 3: observations staged in shared memory or read
 * from global memory; Section 4.12 and Table 6: fast or accurate sin/cos) and
 * are 0 in every configuration the library picks by itself:
 *   trig     0: reseeded recurrence (default);
 *            1: every pair's (cos, sin) from the SFU intrinsic of its exact phase;
 *            2: every pair's (cos, sin) from the accurate sincospif;
 *   staging  0: observation tiles in shared memory (default);
 *            1: every thread reads each observation record from global memory.
 * The ablation kernels (trig or staging non-zero) are FP32, scalar
 * (packed 0), k_reseed = freqs_per_thread = 16, standard periodogram only;
 * other combinations return LSP_E_UNSUPPORTED.
 */
typedef struct lsp_config {
  int32_t k_reseed;
  int32_t freqs_per_thread;
  int32_t block_threads;
  int32_t obs_split;
  int32_t packed;      /* 1: packed f32x2 arithmetic across two reseed chains */
  int32_t trig;
  int32_t staging;
  int32_t reserved;
} lsp_config;

/*
 * A plan owns a workspace (and staging buffers for the host entry point,
 * allocated by its first call) for one shape: n_obj objects (1 = single-
 * object mode) with total_nt observations on `grid`.  lsp_plan_execute
 * never allocates.
 */
lsp_status lsp_plan_create(lsp_plan** plan, int64_t n_obj, int64_t total_nt, const lsp_grid* grid,
                           const lsp_opts* opts);

/*
 * Run the plan on device inputs (offsets may be NULL when n_obj == 1).
 * The launch sequence is captured into a CUDA graph on the first call and
 * replayed afterwards while the pointer arguments stay the same (a change
 * re-captures).  Do not make the first call inside another stream capture.
 */
lsp_status lsp_plan_execute(lsp_plan* plan, const double* t, const void* y, const int64_t* offsets,
                            void* power_out, lsp_peak* peaks, lsp_stream_t stream);

/*
 * End-to-end variant on HOST buffers: copies t, y, offsets to the device,
 * runs the plan, copies the peaks back, and synchronises `stream` before
 * returning.  The periodogram (when power_out is not NULL) is written by the
 * kernels directly into power_out if it is page-locked host memory, and
 * otherwise computed into a device buffer and copied back.  Pinned host
 * memory gives the fastest copies.  The first call allocates the plan's
 * device staging buffers (later calls reuse them).  On an error the call
 * still waits for the copies it had enqueued, so the host buffers are free
 * to reuse once it returns.
 */
lsp_status lsp_plan_execute_host(lsp_plan* plan, const double* t, const void* y,
                                 const int64_t* offsets, void* power_out, lsp_peak* peaks,
                                 lsp_stream_t stream);

/*
 * How lsp_plan_execute_host runs a batch in object groups (the overlap of
 * host transfers with computation, Section 3.5).  parts = 1: one pass, as
 * described above.  parts >= 2: the objects are cut into `parts` contiguous
 * groups, each run as a batch of its own once its observations have been
 * copied in on a second stream, so that the next group's copy overlaps this
 * group's kernels.  With power_out the groups have (nearly) equal object
 * counts and run into their rows of a device buffer, and a third stream
 * copies each group's rows to power_out while the following groups compute
 * (the copies always come from the device buffer, also for page-locked
 * power_out).  Without power_out the groups' observation counts grow
 * four-fold (1 : 4 : 16 : ...), so that only the first, smallest group's
 * input copy is exposed (more than 16 groups, or boundaries that would leave
 * a group with fewer than two objects, fall back to equal counts).  Powers
 * and peaks equal those of one pass bit for bit.  parts = 0 (the default): 8
 * groups for periodograms of at least 256 MiB, else 4 for inputs (t and y)
 * of at least 64 MiB, else one pass.  The count is clamped to n_obj / 2
 * (every group has two objects or more; a one-object plan always runs in one
 * pass).  Offsets that are not monotonic inside [0, total_nt] take the
 * one-pass route (which flags the objects they touch).
 * Errors: LSP_E_ARG for a NULL plan or parts < 0.
 */
lsp_status lsp_plan_set_host_parts(lsp_plan* plan, int32_t parts);

/*
 * The group count lsp_plan_execute_host uses for a call that returns
 * power_bytes bytes of periodogram (n_obj * n_f * 4 for FP32 plans, * 8 for
 * FP64; 0 for a call that returns peaks only), after the default rule and
 * the clamp above.  Host only.
 */
lsp_status lsp_plan_get_host_parts(const lsp_plan* plan, int64_t power_bytes, int32_t* parts);

/*
 * Measure the candidate launch configurations on these inputs, keep the
 * fastest one whose powers stay within the FP32 error gate, and use it from
 * now on.  The gate compares each candidate's P_n with the FP64 path's,
 * 1e-4 absolute at every grid frequency, on up to eight objects of the
 * inputs: the first, the one with the most observations, the worst-
 * conditioned of a pool (the largest R/N over the grid, R = |sum_j
 * exp(4 pi i f t_j)|: where R approaches N, Eq. 2's smaller denominator
 * (N - R)/2 is small and FP32 sums lose relative accuracy; the pool is the
 * 32 shortest objects with three or more observations and 32 spread over
 * the batch) and five spread over the batch.  Objects with fewer than two
 * observations or offsets outside the inputs are left out; without any, the
 * gate is skipped.  A single-object plan is gated on its object with each
 * candidate's own split.  Synchronises `stream`.  When cache_path is not
 * NULL the choice is read from / appended to that JSON-lines file, keyed by
 * device, shape class and options.
 */
lsp_status lsp_plan_autotune(lsp_plan* plan, const double* t, const void* y, const int64_t* offsets,
                             const char* cache_path, lsp_stream_t stream);

/* One candidate measured by lsp_plan_autotune_ex. */
typedef struct lsp_trial {
  lsp_config config;
  float ms;          /* time of one execution (mean of 3 graph replays), ms; -1 if not timed */
  float max_err;     /* max |P_n - P_n(FP64)| over the gate's objects (0 for FP64 plans) */
  int32_t passed;    /* 1: within the error gate, so eligible (failed candidates are not timed) */
  int32_t worst_object; /* the gate object (batch index) with that error; -1 without a gate */
} lsp_trial;

#define LSP_TUNE_ABLATIONS 1  /* also measure the trig/staging ablation kernels (lsp_config) */

/*
 * lsp_plan_autotune with a record of what it measured.  flags: 0 or
 * LSP_TUNE_ABLATIONS (the ablation kernels join the candidates; they win only
 * where they are faster).  trials (host array, nullable) receives the first
 * max_trials of the measured candidates in the order measured and
 * *n_trials (nullable) their number.  With LSP_TUNE_ABLATIONS the cache is
 * not consulted (every candidate is measured); the choice is still appended
 * to it.  lsp_plan_autotune(...) is lsp_plan_autotune_ex(..., 0, NULL, 0,
 * NULL, stream).
 */
lsp_status lsp_plan_autotune_ex(lsp_plan* plan, const double* t, const void* y, const int64_t* offsets,
                                const char* cache_path, int32_t flags, lsp_trial* trials,
                                int32_t max_trials, int32_t* n_trials, lsp_stream_t stream);

/*
 * The last lsp_plan_autotune(_ex) error gate: its objects (batch indices,
 * into objects) and, for the configuration it chose, each object's
 * max |P_n - P_n(FP64)| (into max_err), at most cap of each; *n = the number
 * of gate objects (0 after a cache hit or for FP64 plans).  Host only.
 */
lsp_status lsp_plan_gate_report(const lsp_plan* plan, int64_t* objects, float* max_err, int32_t cap,
                                int32_t* n);

/*
 * Timing probe.  While enabled, each execution of the plan also records two
 * CUDA events on its stream, around the main (trig-sum) kernel, inside the
 * captured graph.  lsp_plan_main_kernel_ms waits for the last execution's
 * second event and returns the main kernel's duration in milliseconds.
 * Enabling or disabling re-captures the graph on the next execution.  A host
 * call that returns the periodogram in object groups (lsp_plan_set_host_parts)
 * runs outside the graph and records no events: the probe keeps describing
 * the last graph execution.
 */
lsp_status lsp_plan_enable_timing(lsp_plan* plan, int32_t enable);
lsp_status lsp_plan_main_kernel_ms(lsp_plan* plan, float* ms);
/* Number of the library's kernels one execution of the plan launches when
 * peaks are requested (a memset, not a kernel, clears the work counters). */
lsp_status lsp_plan_kernel_count(const lsp_plan* plan, int32_t* count);

lsp_status lsp_plan_get_config(const lsp_plan* plan, lsp_config* config);
lsp_status lsp_plan_set_config(lsp_plan* plan, const lsp_config* config);
void lsp_plan_destroy(lsp_plan* plan);

/* ---- learned proposal stage ------------------------------------------------
 * Not in the paper: a small MLP proposes, per light curve, the grid windows
 * most likely to hold the periodogram's maximum; the direct method refines
 * only those windows and falls back to the full grid when the refined peak
 * is weak.  The network trains on light curves and periodograms that the
 * direct method itself produces (lsp_batch labels).
 *
 * Parameters are one flat FP32 vector in the order W1, b1, W2, b2, ..., with
 * W_l row-major of shape (fan_in, fan_out), plus its bfloat16 copy (same
 * layout; the GEMMs read the weights from the copy and the biases from the
 * FP32 vector).  bfloat16 arrays are passed as uint16_t.
 */
#define LSP_FEAT_DIM 512
#define LSP_REFINE_FALLBACK 256 /* bit of lsp_refine_windows' info word */

typedef struct lsp_mlp_dims {
  int32_t in_dim;    /* LSP_FEAT_DIM for lsp_featurize inputs */
  int32_t hidden;    /* width of each hidden layer */
  int32_t n_hidden;  /* hidden layers, 1..6 (Linear + ReLU each) */
  int32_t n_classes; /* output logits: one per refinement window */
} lsp_mlp_dims;

/* Length of the flat parameter vector. */
lsp_status lsp_mlp_param_count(const lsp_mlp_dims* dims, int64_t* count);
/* Scratch bytes of lsp_mlp_forward / lsp_mlp_loss_grad for a batch. */
lsp_status lsp_mlp_workspace_size(const lsp_mlp_dims* dims, int64_t batch, size_t* bytes);

/*
 * 512 features per light curve (CSR batch as in lsp_batch; y float):
 * with z the standardised magnitudes and all pairs i < j with
 * |t_j - t_i| < lag_max, features 0..255 are the short-lag periodogram
 * sum_pairs z_i z_j cos(2 pi f_c dt) / (pairs + 1) at the 256 coarse bin
 * centres f_c of [f_min, f_max), and features 256..511 are log(1 + pairs)
 * in 256 equal lag bins of [0, lag_max).  feat_bf16 (n_obj x 512) is
 * required, feat_f32 optional.  Objects with fewer than two observations or
 * zero variance get zeros.
 */
lsp_status lsp_featurize(const double* t, const float* y, const int64_t* offsets, int64_t n_obj,
                         int64_t total_nt, const lsp_grid* grid, float lag_max, uint16_t* feat_bf16,
                         float* feat_f32, lsp_stream_t stream);

/* Logits (batch x n_classes, FP32) of the MLP on bfloat16 inputs x (batch x in_dim);
 * batch <= LSP_MLP_MAX_BATCH rows per call.  The products run on the tcgen05
 * tensor cores with operands loaded by TMA: when in_dim is a multiple of 8,
 * x_bf16 must be 16-byte aligned (LSP_E_ARG otherwise; any row of a
 * contiguous allocation is); other widths are copied to a padded pitch in the
 * workspace first. */
#define LSP_MLP_MAX_BATCH 4194240
lsp_status lsp_mlp_forward(const lsp_mlp_dims* dims, const float* params, const uint16_t* params_bf16,
                           const uint16_t* x_bf16, int64_t batch, float* logits, void* workspace,
                           size_t ws_bytes, lsp_stream_t stream);

/*
 * Mean softmax cross-entropy of the batch against labels (class indices)
 * into *loss (device float) and its gradient into grad (flat FP32, the
 * parameters' layout).  Hidden activations and back-propagated
 * pre-activation gradients are stored in bfloat16; products accumulate in
 * FP32 on the tensor cores (the weight gradient's sum over the batch is split
 * over several CTAs and added in a fixed order, so results are
 * deterministic).  x_bf16 as for lsp_mlp_forward.
 */
lsp_status lsp_mlp_loss_grad(const lsp_mlp_dims* dims, const float* params, const uint16_t* params_bf16,
                             const uint16_t* x_bf16, const int32_t* labels, int64_t batch, float* loss,
                             float* grad, void* workspace, size_t ws_bytes, lsp_stream_t stream);

/* One AdamW step (decoupled weight decay; step counts from 1) on the FP32
 * parameters; refreshes the bfloat16 copy. */
lsp_status lsp_mlp_adamw(int64_t n, float* params, uint16_t* params_bf16, const float* grad, float* m,
                         float* v, int64_t step, float lr, float beta1, float beta2, float eps,
                         float weight_decay, lsp_stream_t stream);

/* Number of tensor-core GEMM tiles of lsp_mlp_forward / lsp_mlp_loss_grad /
 * lsp_propose_refine on the current device whose bounded device-side waits
 * (about one second each) gave up since the last call, and reset it to 0.
 * Such a tile writes NaN over its outputs instead of hanging.  Synchronous
 * (reads device memory). */
lsp_status lsp_mlp_gemm_timeouts(uint32_t* count);

/* Self-test of those bounded waits: one GEMM tile whose first operand slice
 * is deliberately never loaded, so the tile's wait for it runs out after
 * about one second.  Synchronizes the stream, then reports the timeout count
 * of that launch (1 expected) and how many of its 128 x 16 outputs are NaN
 * (2048 expected); the device stays usable.  workspace: device memory of at
 * least LSP_MLP_WAIT_TEST_BYTES, 256-byte aligned, overwritten. */
#define LSP_MLP_WAIT_TEST_BYTES 65536
lsp_status lsp_mlp_gemm_wait_test(void* workspace, size_t ws_bytes, uint32_t* timeouts, int32_t* nan_outputs,
                                  lsp_stream_t stream);

/* FP32 -> bfloat16 (round to nearest even). */
lsp_status lsp_to_bf16(const float* a, uint16_t* b, int64_t n, lsp_stream_t stream);

/* The k (<= 16) largest logits' classes per row, largest first, ties to the lower class. */
lsp_status lsp_top_classes(const float* logits, int64_t rows, int32_t n_classes, int32_t k,
                           int32_t* classes, lsp_stream_t stream);

lsp_status lsp_refine_workspace_size(int64_t n_obj, int64_t total_nt, const lsp_grid* grid,
                                     size_t* bytes);

/*
 * Refine proposed windows, then fall back.  classes (n_obj x k_windows,
 * best first) name windows: class c covers bins
 * [c*stride + stride/2 - window/2, +window) moved inside the grid
 * (window <= 2048).  Windows are evaluated in rank order with the FP32 direct
 * method; an object stops once its best refined power reaches stop_power.
 * Objects whose best refined power is below fallback_power get the full
 * grid, and so do, when inconclusive_fallback is nonzero, objects that
 * evaluated all k_windows windows without reaching stop_power (for short
 * light curves a noise peak in a wrong window can exceed fallback_power).
 * peaks[o] is the result (first maximum of what was evaluated);
 * info[o] (nullable) = windows evaluated | LSP_REFINE_FALLBACK if the full
 * grid was used.  norm is an lsp_norm; thresholds are in that normalisation.
 */
lsp_status lsp_refine_windows(const double* t, const float* y, const int64_t* offsets, int64_t n_obj,
                              int64_t total_nt, const lsp_grid* grid, int32_t norm,
                              const int32_t* classes, int32_t k_windows, int64_t window,
                              int64_t stride, float stop_power, float fallback_power,
                              int32_t inconclusive_fallback, lsp_peak* peaks, int32_t* info,
                              void* workspace, size_t ws_bytes, lsp_stream_t stream);

/*
 * The learned path in one call: the 512 features of every light curve
 * (lsp_featurize), the network's logits (lsp_mlp_forward), each object's
 * k_windows best window classes (lsp_top_classes) and the ranked refine
 * with its full-grid fallback (lsp_refine_windows), launched on `stream`
 * with no host synchronisation.  The results equal those of the four calls
 * made in that order, bit for bit.  Not in the paper: the proposal network
 * and its windows are this library's learned stage (see above).
 *
 * The network is described by an lsp_proposer; its parameter arrays are the
 * caller's device memory and are only read.  t, y, offsets, n_obj, total_nt
 * and grid are as in lsp_batch (y float).  peaks (n_obj records) and info
 * (n_obj words, nullable) are as in lsp_refine_windows; classes_out
 * (nullable, n_obj x k_windows int32) receives the proposed classes, best
 * first.  workspace must hold lsp_propose_refine_workspace_size bytes and be
 * 256-byte aligned; it holds the features, the hidden activations, the
 * logits, the classes and the refine's state.
 * Errors: LSP_E_ARG for a bad proposer (in_dim not LSP_FEAT_DIM, k_windows
 * outside 1..16 or above n_classes, lag_max <= 0, NULL parameters), bad
 * window or stride, NULL arrays, or a small or misaligned workspace;
 * LSP_E_CUDA if a launch fails.
 */
typedef struct lsp_proposer {
  lsp_mlp_dims dims;             /* in_dim = LSP_FEAT_DIM; n_classes = window classes of the grid */
  const float* params;           /* device: FP32 flat parameters (layout of lsp_mlp_forward) */
  const uint16_t* params_bf16;   /* device: their bfloat16 copy */
  int64_t window;                /* bins per refinement window, 1..2048 */
  int64_t stride;                /* bins between window classes (class c centred on c*stride + stride/2) */
  float lag_max;                 /* the featurizer's lag limit, in units of t */
  int32_t k_windows;             /* proposals per object, 1..16 and at most n_classes */
  float stop_power;              /* an object stops once its best refined power reaches this */
  float fallback_power;          /* full grid when the best refined power is below this */
  int32_t inconclusive_fallback; /* nonzero: full grid also when no window reached stop_power */
  int32_t norm;                  /* lsp_norm of the thresholds and of the returned powers */
} lsp_proposer; /* 72 bytes */

lsp_status lsp_propose_refine_workspace_size(const lsp_proposer* net, int64_t n_obj, int64_t total_nt,
                                             const lsp_grid* grid, size_t* bytes);
lsp_status lsp_propose_refine(const lsp_proposer* net, const double* t, const float* y, const int64_t* offsets,
                              int64_t n_obj, int64_t total_nt, const lsp_grid* grid, lsp_peak* peaks,
                              int32_t* info, int32_t* classes_out, void* workspace, size_t ws_bytes,
                              lsp_stream_t stream);

/*
 * Training labels of the learned stage: labels[o] = the window class of
 * peaks[o].idx, i.e. idx / stride clamped to [0, n_classes - 1] (0 for an
 * object without a peak).  peaks are device records from lsp_batch
 * (top_k = 1).  Errors: LSP_E_ARG for stride < 1, n_classes < 1 or NULL arrays.
 */
lsp_status lsp_window_labels(const lsp_peak* peaks, int64_t n_obj, int64_t stride, int32_t n_classes,
                             int32_t* labels, lsp_stream_t stream);

/*
 * Calibration probe of the FMA pipes (no counterpart in the paper): runs
 * register-only kernels of independent FMA chains (scalar FP32, packed
 * f32x2, FP64) on the current device, 64 warps per SM, and writes the
 * sustained rate of each in FMA lane-operations per second for the whole
 * device (a packed FMA counts two).  These are the ceilings the trig-sum
 * kernels' FP32 and FP64 fractions are read against.  Takes a few tens of
 * milliseconds, synchronizes `stream`, and allocates and frees a small
 * device buffer (one float per probe thread).  Outputs are host pointers,
 * each nullable.  Errors: LSP_E_CUDA (message in lsp_last_error).
 */
lsp_status lsp_probe_fma_rates(double* f32_per_s, double* f32x2_per_s, double* f64_per_s,
                               lsp_stream_t stream);

/*
 * Accuracy probe of the FP64 path's sin/cos of a fixed-point phase (no
 * counterpart in the paper): the library evaluates (cos, sin)(2 pi phi) for
 * a 64-bit phase phi = frac in units of 2^-64 cycle from a 256-entry table of
 * e^{2 pi i j / 256} and a short Taylor series of the remaining angle
 * (< 2 pi / 256), rotated together.  The probe draws n phases on the device
 * (the table points and their neighbours, then splitmix64 of seed + i),
 * evaluates each both that way and with CUDA's sincospi, and writes the
 * largest absolute difference of either component to *max_abs_err (host
 * pointer).  Synchronises `stream`; allocates and frees one device word.
 * Errors: LSP_E_ARG for n < 1 or a NULL output, LSP_E_CUDA.
 */
lsp_status lsp_probe_sincos_fixed64(int64_t n, uint64_t seed, double* max_abs_err, lsp_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* LSP_H */
