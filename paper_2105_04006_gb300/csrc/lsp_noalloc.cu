// lsp_noalloc.cu -- lsp_batch_noalloc: the batch periodogram with its scratch
// memory in a fixed device array of the library, for callers that cannot
// allocate device memory.
//
// Who needs it: code that must not call cudaMalloc (or any allocator) on its
// path -- e.g. a real-time alert pipeline with a fixed device-memory budget
// set at start-up, a plugin whose host framework already reserved nearly
// all device memory for its own pool, or a C caller with no device-memory
// manager of its own.  Such callers still own their inputs and outputs; only
// the workspace comes from here.
//
// Limits and sharing:
//   - The scratch array holds LSP_NOALLOC_SCRATCH_BYTES (32 MiB).  A shape
//     whose lsp_workspace_size exceeds it is rejected with LSP_E_WORKSPACE
//     before anything is launched.
//   - When the array is reserved: the CUDA runtime places it in device
//     memory when it loads this file's module on a device.  With lazy module
//     loading (the default of recent CUDA releases) that happens at the
//     first address lookup on that device, i.e. in lsp_noalloc_prepare or the
//     first lsp_batch_noalloc there.  A caller whose device memory fills up
//     later should call lsp_noalloc_prepare at start-up.  The reservation
//     lasts until the process exits.
//   - All calls share the one array and it keeps the last call's contents.
//     The launch sequence clears what must start at zero (the queue counter
//     and the work-order histogram) and overwrites the rest.  Calls that
//     overlap on the GPU (on different streams, or from different host
//     threads without ordering between them) race on the array: order them,
//     e.g. issue them on one stream.
//   - The address is looked up with cudaGetSymbolAddress, with the device
//     current, and cached per device.  It belongs to the runtime's primary
//     context of that device: after cudaDeviceReset, or with another context
//     current, call lsp_noalloc_prepare again, which looks the address up
//     afresh.  Make the first call on a device outside any stream capture.
#include <cstdio>
#include <mutex>

#include "../../include/lsp.h"

namespace lsp {
void set_last_error(const char* msg);
}

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[LSP_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device; `refresh`
// repeats the lookup even when an address is cached.
lsp_status scratch_address(void** out, bool refresh) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    char msg[160];
    snprintf(msg, sizeof msg, "lsp_batch_noalloc: no usable current device (%s)",
             e != cudaSuccess ? cudaGetErrorString(e) : "device index out of range");
    lsp::set_last_error(msg);
    return LSP_E_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (refresh || !g_scratch_ptr[dev]) {
    g_scratch_ptr[dev] = nullptr;
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      char msg[256];
      if (e == cudaErrorMemoryAllocation) {
        snprintf(msg, sizeof msg,
                 "lsp_batch_noalloc: the device has no room for the library's %u-byte scratch array "
                 "(reserved when its module loads; call lsp_noalloc_prepare at start-up)",
                 (unsigned)LSP_NOALLOC_SCRATCH_BYTES);
        lsp::set_last_error(msg);
        return LSP_E_NOMEM;
      }
      snprintf(msg, sizeof msg, "lsp_batch_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      lsp::set_last_error(msg);
      return LSP_E_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return LSP_OK;
}

}  // namespace

extern "C" lsp_status lsp_noalloc_prepare(void) {
  void* p = nullptr;
  return scratch_address(&p, true);
}

extern "C" lsp_status lsp_batch_noalloc(const double* t, const void* y, const int64_t* offsets,
                                        int64_t n_obj, int64_t total_nt, const lsp_grid* grid,
                                        const lsp_opts* opts, void* power_out, lsp_peak* peaks,
                                        lsp_stream_t stream) {
  size_t need = 0;
  lsp_status st = lsp_workspace_size(n_obj, total_nt, grid, opts, &need);
  if (st != LSP_OK) return st;
  if (n_obj == 0) return LSP_OK;  // nothing to do: no lookup, no module load
  if (need > (size_t)LSP_NOALLOC_SCRATCH_BYTES) {
    char msg[200];
    snprintf(msg, sizeof msg,
             "lsp_batch_noalloc: this shape needs %zu bytes of scratch, the static array holds %zu "
             "(use lsp_batch with a caller workspace)",
             need, (size_t)LSP_NOALLOC_SCRATCH_BYTES);
    lsp::set_last_error(msg);
    return LSP_E_WORKSPACE;
  }
  void* ws = nullptr;
  if ((st = scratch_address(&ws, false)) != LSP_OK) return st;
  return lsp_batch(t, y, offsets, n_obj, total_nt, grid, opts, power_out, peaks, ws,
                   (size_t)LSP_NOALLOC_SCRATCH_BYTES, stream);
}
