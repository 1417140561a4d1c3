// lsp_main_f32.cu -- instantiations of the FP32 trig-sum kernels.
#include "lsp_launch.h"
#include "lsp_main_impl.cuh"

namespace lsp {

namespace {
template <typename Kern, typename P>
cudaError_t launch_kernel(Kern kern, const MainLaunch& ml, const P& p, cudaStream_t stream) {
  size_t dyn = main_dyn_smem(ml.prec, ml.fpt, ml.threads, ml.top);
  cudaError_t e = allow_dyn_smem(kern, dyn);
  if (e != cudaSuccess) return e;
  kern<<<ml.grid, ml.threads, dyn, stream>>>(p);
  return cudaGetLastError();
}

template <typename Kern>
int occupancy(Kern kern, int threads, size_t dyn) {
  int nb = 0;
  if (allow_dyn_smem(kern, dyn) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, dyn) != cudaSuccess) return 0;
  return nb;
}

// abl: ablation code trig + 3 * staging (0: the production kernels); the
// ablation kernels are scalar, K = 16, standard periodogram only.
template <typename Fn>
bool dispatch_f32(int packed, int k, int gls, int abl, int threads, Fn&& fn) {
  if (abl) {
    if (packed || gls || k != 16) return false;
    switch (abl) {
      case 1: fn(main_scalar<float, RecF32, 16, 1, false>); return true;
      case 2: fn(main_scalar<float, RecF32, 16, 2, false>); return true;
      case 3: fn(main_scalar<float, RecF32, 16, 0, true>); return true;
      case 4: fn(main_scalar<float, RecF32, 16, 1, true>); return true;
      case 5: fn(main_scalar<float, RecF32, 16, 2, true>); return true;
    }
    return false;
  }
  if (gls) {
    if (!packed) return false;
    switch (k) {
      case 4: fn(main_f32_packed_gls<4>); return true;
      case 8: fn(main_f32_packed_gls<8>); return true;
    }
    return false;
  }
  if (packed) {
    // 64- and 128-thread CTAs of K = 8 and 12: instantiations whose launch
    // bounds ask for 16 and 12 warps per SM (128 and 168 registers); left
    // to itself the compiler took 128 to 193 registers for these kernels and
    // ran 7-13 % slower per pair
    if (threads == 64 || threads == 128) {
      switch (k * 1000 + threads) {
        case 8064: fn(main_f32_packed_floor<8, 64, 8>); return true;
        case 8128: fn(main_f32_packed_floor<8, 128, 4>); return true;
        case 12064: fn(main_f32_packed_floor<12, 64, 6>); return true;
        case 12128: fn(main_f32_packed_floor<12, 128, 3>); return true;
      }
    }
    switch (k) {
      case 4: fn(main_f32_packed<4>); return true;
      case 8: fn(main_f32_packed<8>); return true;
      case 12: fn(main_f32_packed<12>); return true;
      case 16: fn(main_f32_packed<16>); return true;
    }
  } else {
    switch (k) {
      case 8: fn(main_scalar<float, RecF32, 8>); return true;
      case 16: fn(main_scalar<float, RecF32, 16>); return true;
    }
  }
  return false;
}
}  // namespace

bool main_variant_exists_f32(int packed, int k, int fpt, int gls, int abl) {
  if (fpt != (packed ? 2 * k : k)) return false;
  return dispatch_f32(packed, k, gls, abl, 256, [](auto) {});
}

int main_blocks_per_sm_f32(int packed, int k, int fpt, int threads, int top, int gls, int abl) {
  int nb = 0;
  size_t dyn = main_dyn_smem(0, fpt, threads, top);
  dispatch_f32(packed, k, gls, abl, threads, [&](auto kern) { nb = occupancy(kern, threads, dyn); });
  return nb;
}

cudaError_t launch_main_f32(const MainLaunch& ml, cudaStream_t stream) {
  MainParams<RecF32, float> p;
  p.rec = (const RecF32*)ml.rec;
  p.obj = ml.obj;
  p.order = ml.order;
  p.power_out = (float*)ml.power_out;
  p.part = (float*)ml.part;
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
  dispatch_f32(ml.packed, ml.k_reseed, ml.gls, ml.abl, ml.threads, [&](auto kern) { err = launch_kernel(kern, ml, p, stream); });
  return err;
}

}  // namespace lsp
