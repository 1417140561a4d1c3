// lsp_main_f64.cu -- instantiations of the FP64 trig-sum kernel.
#include "lsp_launch.h"
#include "lsp_main_impl.cuh"

namespace lsp {

namespace {
template <typename Fn>
bool dispatch_f64(int k, int gls, Fn&& fn) {
  if (gls) {
    switch (k) {
      case 4: fn(main_f64_gls<4>); return true;
      case 8: fn(main_f64_gls<8>); return true;
    }
    return false;
  }
  switch (k) {
    case 4: fn(main_scalar<double, RecF64, 4>); return true;
    case 8: fn(main_scalar<double, RecF64, 8>); return true;
    case 16: fn(main_scalar<double, RecF64, 16>); return true;
  }
  return false;
}
}  // namespace

bool main_variant_exists_f64(int k, int fpt, int gls) {
  if (fpt != k) return false;
  return dispatch_f64(k, gls, [](auto) {});
}

int main_blocks_per_sm_f64(int k, int fpt, int threads, int top, int gls) {
  int nb = 0;
  size_t dyn = main_dyn_smem(1, fpt, threads, top);
  dispatch_f64(k, gls, [&](auto kern) {
    if (allow_dyn_smem(kern, dyn) != cudaSuccess || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, dyn) != cudaSuccess)
      nb = 0;
  });
  return nb;
}

cudaError_t launch_main_f64(const MainLaunch& ml, cudaStream_t stream) {
  MainParams<RecF64, double> p;
  p.rec = (const RecF64*)ml.rec;
  p.obj = ml.obj;
  p.order = ml.order;
  p.power_out = (double*)ml.power_out;
  p.part = (double*)ml.part;
  p.best = ml.best;
  p.cand = ml.cand;
  p.queue = ml.queue;
  p.n_f = ml.n_f;
  p.n_chunks = ml.n_chunks;
  p.split = ml.split;
  p.n_items = ml.n_items;
  p.n_items_dev = ml.n_items_dev;
  p.win_start = ml.win_start;
  p.win_len = ml.win_len;
  cudaError_t err = cudaErrorInvalidValue;
  size_t dyn = main_dyn_smem(1, ml.fpt, ml.threads, ml.top);
  dispatch_f64(ml.k_reseed, ml.gls, [&](auto kern) {
    err = allow_dyn_smem(kern, dyn);
    if (err != cudaSuccess) return;
    kern<<<ml.grid, ml.threads, dyn, stream>>>(p);
    err = cudaGetLastError();
  });
  return err;
}

}  // namespace lsp
