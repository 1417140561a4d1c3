// lsp_main_impl.cuh -- the trig-sum kernels (internal).
//
// What they compute: for every object o and grid frequency k the single-scan
// sums of Section 2 (the refactoring the paper ports from SciPy, Listing 1):
//   XC = sum_j y_j cos phi_jk,  XS = sum_j y_j sin phi_jk,
//   CC = sum_j cos^2 phi_jk,    CS = sum_j cos phi_jk sin phi_jk,
// with phi_jk = 2 pi f_k (t_j - t0); sum sin^2 = N - CC.  The epilogue turns
// them into Eq. 2's power (lsp_power) and reduces each chunk of frequencies
// to its maximum, so the periodogram reaches HBM only on request.
//
// How (the GB300 design; the paper's one-thread-per-frequency kernel with a
// library sincos per pair is prior art):
//   - a CTA owns a chunk of blockDim.x * F consecutive frequencies of one
//     object; each thread owns F consecutive frequencies of it;
//   - observations are staged through shared memory in tiles and read by
//     all threads at once (broadcast), so every (t, y) load is shared by the
//     CTA's blockDim.x * F frequencies;
//   - sin/cos come from a rotation recurrence across the uniform grid,
//     (c, s) <- (c cr - s sr, s cr + c sr) with (cr, sr) = e^{2 pi i df t'},
//     reseeded from the exact fixed-point phase every K frequencies (the
//     paper, Section 4.5, rejects the recurrence as serial; here it runs
//     along a thread's own frequencies while threads, CTAs and objects run
//     in parallel);
//   - the FP32 kernel packs two reseed chains into f32x2 lanes, so one
//     instruction advances two frequencies;
//   - CTAs are persistent and pull (object, chunk, split) items from a queue
//     ordered by decreasing N_t.
#pragma once

#include <type_traits>

#include "lsp_common.cuh"

namespace lsp {

template <int F>
__device__ __forceinline__ void store_row(float* row, int64_t k0, const float (&pv)[F], int64_t n_f) {
  if (k0 + F <= n_f && ((reinterpret_cast<uintptr_t>(row + k0) & 15) == 0)) {
    float4* d = reinterpret_cast<float4*>(row + k0);
#pragma unroll
    for (int q = 0; q < F / 4; ++q)
      __stcs(d + q, make_float4(pv[4 * q], pv[4 * q + 1], pv[4 * q + 2], pv[4 * q + 3]));
  } else {
#pragma unroll
    for (int m = 0; m < F; ++m)
      if (k0 + m < n_f) row[k0 + m] = pv[m];
  }
}

template <int F>
__device__ __forceinline__ void store_row(double* row, int64_t k0, const double (&pv)[F], int64_t n_f) {
  if (k0 + F <= n_f && ((reinterpret_cast<uintptr_t>(row + k0) & 15) == 0)) {
    double2* d = reinterpret_cast<double2*>(row + k0);
#pragma unroll
    for (int q = 0; q < F / 2; ++q) __stcs(d + q, make_double2(pv[2 * q], pv[2 * q + 1]));
  } else {
#pragma unroll
    for (int m = 0; m < F; ++m)
      if (k0 + m < n_f) row[k0 + m] = pv[m];
  }
}

__device__ __forceinline__ void store_part(float* part, int64_t idx, float a, float b, float c, float d) {
  reinterpret_cast<float4*>(part)[idx] = make_float4(a, b, c, d);
}
__device__ __forceinline__ void store_part(double* part, int64_t idx, double a, double b, double c,
                                           double d) {
  double2* p2 = reinterpret_cast<double2*>(part) + 2 * idx;
  p2[0] = make_double2(a, b);
  p2[1] = make_double2(c, d);
}

// Item decoding shared by the kernels.
struct Item {
  int64_t o;
  int chunk;
  int s;
};
template <typename P>
__device__ __forceinline__ Item decode_item(const P& p, int64_t item) {
  Item it;
  it.s = (int)(item % p.split);
  const int64_t oc = item / p.split;
  it.chunk = (int)(oc % p.n_chunks);
  const int64_t orank = oc / p.n_chunks;
  it.o = p.order ? (int64_t)p.order[orank] : orank;
  return it;
}

// ------------------------------------------------------------------------
// FP32, two reseed chains of K frequencies per thread in packed f32x2 lanes:
// lane 0 covers k0 .. k0+K-1, lane 1 covers k0+K .. k0+2K-1.
//
// The shared-memory tile holds the 32-byte records as they are.  Each
// observation costs every thread two SFU seeds (one per chain) and 2K-1
// packed recurrence steps.  (Measured alternatives that did not pay on
// GB300: issuing the next observation's seeds one step ahead, integer
// bit-building of the seed angle instead of I2F, and deriving the second
// chain's seed from the first by a K-step rotation.)

__device__ __forceinline__ f2_t f2_of(uint32_t lo, uint32_t hi) {
  f2_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "r"(lo), "r"(hi));
  return r;
}

__device__ __forceinline__ void seed_pair(const uint4 w2, uint32_t k0, uint32_t k1, f2_t& c2, f2_t& s2) {
  float c0, s0, c1, s1;
  seed_sincos_f32(phase_hi32(w2.x, w2.y, w2.z, k0), c0, s0);
  seed_sincos_f32(phase_hi32(w2.x, w2.y, w2.z, k1), c1, s1);
  c2 = f2_pack(c0, c1);
  s2 = f2_pack(s0, s1);
}

// K steps of the two packed reseed chains at one observation: accumulate the
// four sums at the current (cos, sin), then rotate by one grid step.
template <int K>
__device__ __forceinline__ void recurrence_steps(f2_t (&xc)[K], f2_t (&xs)[K], f2_t (&cc)[K], f2_t (&cs)[K],
                                                 f2_t c2, f2_t s2, f2_t y2, f2_t cr2, f2_t sr2, f2_t nsr2) {
#pragma unroll
  for (int m = 0; m < K; ++m) {
    xc[m] = f2_fma(y2, c2, xc[m]);
    xs[m] = f2_fma(y2, s2, xs[m]);
    cc[m] = f2_fma(c2, c2, cc[m]);
    cs[m] = f2_fma(c2, s2, cs[m]);
    if (m + 1 < K) {
      const f2_t tc = f2_mul(c2, cr2);
      const f2_t tsr = f2_mul(s2, cr2);
      const f2_t cn = f2_fma(s2, nsr2, tc);
      s2 = f2_fma(c2, sr2, tsr);
      c2 = cn;
    }
  }
}

template <int K>
__global__ void __launch_bounds__(256) main_f32_packed(MainParams<RecF32, float> p) {
  constexpr int F = 2 * K;
  __shared__ uint4 s_obs[2 * LSP_TILE_OBS];
  __shared__ unsigned long long red[32];
  __shared__ uint32_t s_item;
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  float* s_pw = reinterpret_cast<float*>(dyn_smem);
  const int tid = threadIdx.x;
  const uint32_t n_items = p.n_items_dev ? *p.n_items_dev : (uint32_t)p.n_items;
  const uint32_t split = (uint32_t)p.split, n_chunks = (uint32_t)p.n_chunks;

  for (;;) {
    if (tid == 0) s_item = atomicAdd(p.queue, 1u);
    __syncthreads();
    const uint32_t item = s_item;
    __syncthreads();
    if (item >= n_items) break;
    const uint32_t is = item % split;
    const uint32_t oc = item / split;
    const uint32_t chunk = oc % n_chunks;
    const uint32_t orank = oc / n_chunks;
    const int64_t o = p.order ? (int64_t)p.order[orank] : (int64_t)orank;
    const ObjInfo oi = p.obj[o];
    const int64_t kc0 = p.win_start ? (int64_t)p.win_start[o] : (int64_t)chunk * blockDim.x * F;
    // bins of this item lie in [kc0, kend): the grid, or the object's window
    const int64_t kend = p.win_start ? (kc0 + p.win_len < p.n_f ? kc0 + p.win_len : p.n_f) : p.n_f;
    const uint32_t k0 = (uint32_t)(kc0 + (int64_t)tid * F);
    const uint32_t k1 = k0 + K;
    const int64_t ob = oi.begin + (int64_t)oi.n * is / split;
    int64_t oe = oi.begin + (int64_t)oi.n * (is + 1) / split;
    if (oi.flags) oe = ob;  // flagged objects: zero power

    f2_t xc[K], xs[K], cc[K], cs[K];
#pragma unroll
    for (int m = 0; m < K; ++m) xc[m] = xs[m] = cc[m] = cs[m] = 0ull;

    for (int64_t ts = ob; ts < oe; ts += LSP_TILE_OBS) {
      const int nt = (int)((oe - ts) < LSP_TILE_OBS ? (oe - ts) : LSP_TILE_OBS);
      const uint4* src = reinterpret_cast<const uint4*>(p.rec + ts);
      for (int i = tid; i < 2 * nt; i += blockDim.x) s_obs[i] = __ldg(src + i);
      __syncthreads();
      for (int j = 0; j < nt; ++j) {
        const uint4 r0 = s_obs[2 * j];
        const uint4 r1 = s_obs[2 * j + 1];
        f2_t c2, s2;
        seed_pair(make_uint4(r0.w, r1.x, r1.y, 0u), k0, k1, c2, s2);
        const uint32_t nsr = r0.z ^ 0x80000000u;
        recurrence_steps<K>(xc, xs, cc, cs, c2, s2, f2_of(r0.x, r0.x), f2_of(r0.y, r0.y),
                            f2_of(r0.z, r0.z), f2_of(nsr, nsr));
      }
      __syncthreads();
    }

    if (split == 1) {
      float pv[F];
      const float nf = (float)oi.n, scale = oi.norm_scale_f;
      uint32_t bad = 0u;
#pragma unroll
      for (int m = 0; m < K; ++m) {
        float a0, a1, b0, b1, c0, c1, d0, d1;
        f2_unpack(xc[m], a0, a1);
        f2_unpack(xs[m], b0, b1);
        f2_unpack(cc[m], c0, c1);
        f2_unpack(cs[m], d0, d1);
        bool ill0, ill1;
        pv[m] = scale * lsp_power_f32(a0, b0, c0, d0, nf, ill0);
        pv[K + m] = scale * lsp_power_f32(a1, b1, c1, d1, nf, ill1);
        if (ill0 && (int64_t)k0 + m < kend) bad |= 1u << m;
        if (ill1 && (int64_t)k1 + m < kend) bad |= 1u << (K + m);
      }
      if (oi.flags) bad = 0u;
      fix_ill_conditioned<F>(pv, bad, k0, p.rec, oi.begin, oi.n, oi.norm_scale);
      if (p.power_out) store_row<F>(p.power_out + o * p.n_f, (int64_t)k0, pv, kend);
      const int64_t res = o * (int64_t)n_chunks + chunk;
      chunk_results_f32<F>(pv, k0, kc0, kend, p.best + res, p.cand ? p.cand + res : nullptr, s_pw, red);
    } else {
      float* part = p.part + (int64_t)is * p.n_f * 4;
#pragma unroll
      for (int m = 0; m < K; ++m) {
        float a0, a1, b0, b1, c0, c1, d0, d1;
        f2_unpack(xc[m], a0, a1);
        f2_unpack(xs[m], b0, b1);
        f2_unpack(cc[m], c0, c1);
        f2_unpack(cs[m], d0, d1);
        if ((int64_t)k0 + m < p.n_f) store_part(part, (int64_t)k0 + m, a0, b0, c0, d0);
        if ((int64_t)k1 + m < p.n_f) store_part(part, (int64_t)k1 + m, a1, b1, c1, d1);
      }
    }
  }
}

// ------------------------------------------------------------------------
// Generalized periodogram (Section 4.11), FP32, two packed reseed chains:
// the same tiling and seeding as main_f32_packed with six weighted sums per
// frequency (11 FP32 operations per pair instead of 8).  Records carry
// u = w (y - ybar_w) in the y word and w in the spare word.
template <int K>
__global__ void __launch_bounds__(256) main_f32_packed_gls(MainParams<RecF32, float> p) {
  constexpr int F = 2 * K;
  __shared__ uint4 s_obs[2 * LSP_TILE_OBS];
  __shared__ unsigned long long red[32];
  __shared__ uint32_t s_item;
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  float* s_pw = reinterpret_cast<float*>(dyn_smem);
  const int tid = threadIdx.x;
  const uint32_t n_items = p.n_items_dev ? *p.n_items_dev : (uint32_t)p.n_items;
  const uint32_t n_chunks = (uint32_t)p.n_chunks;

  for (;;) {
    if (tid == 0) s_item = atomicAdd(p.queue, 1u);
    __syncthreads();
    const uint32_t item = s_item;
    __syncthreads();
    if (item >= n_items) break;
    const uint32_t chunk = item % n_chunks;
    const uint32_t orank = item / n_chunks;
    const int64_t o = p.order ? (int64_t)p.order[orank] : (int64_t)orank;
    const ObjInfo oi = p.obj[o];
    const int64_t kc0 = (int64_t)chunk * blockDim.x * F;
    const uint32_t k0 = (uint32_t)(kc0 + (int64_t)tid * F);
    const uint32_t k1 = k0 + K;
    const int64_t ob = oi.begin;
    const int64_t oe = oi.flags ? ob : oi.begin + oi.n;

    f2_t xc[K], xs[K], cw[K], sw[K], cc[K], cs[K];
#pragma unroll
    for (int m = 0; m < K; ++m) xc[m] = xs[m] = cw[m] = sw[m] = cc[m] = cs[m] = 0ull;

    for (int64_t ts = ob; ts < oe; ts += LSP_TILE_OBS) {
      const int nt = (int)((oe - ts) < LSP_TILE_OBS ? (oe - ts) : LSP_TILE_OBS);
      const uint4* src = reinterpret_cast<const uint4*>(p.rec + ts);
      for (int i = tid; i < 2 * nt; i += blockDim.x) s_obs[i] = __ldg(src + i);
      __syncthreads();
      for (int j = 0; j < nt; ++j) {
        const uint4 r0 = s_obs[2 * j];
        const uint4 r1 = s_obs[2 * j + 1];
        f2_t c2, s2;
        seed_pair(make_uint4(r0.w, r1.x, r1.y, 0u), k0, k1, c2, s2);
        const f2_t u2 = f2_of(r0.x, r0.x), w2 = f2_of(r1.w, r1.w);
        const f2_t cr2 = f2_of(r0.y, r0.y), sr2 = f2_of(r0.z, r0.z);
        const uint32_t nsr = r0.z ^ 0x80000000u;
        const f2_t nsr2 = f2_of(nsr, nsr);
#pragma unroll
        for (int m = 0; m < K; ++m) {
          xc[m] = f2_fma(u2, c2, xc[m]);
          xs[m] = f2_fma(u2, s2, xs[m]);
          cw[m] = f2_fma(w2, c2, cw[m]);
          sw[m] = f2_fma(w2, s2, sw[m]);
          const f2_t wc = f2_mul(w2, c2);
          cc[m] = f2_fma(wc, c2, cc[m]);
          cs[m] = f2_fma(wc, s2, cs[m]);
          if (m + 1 < K) {
            const f2_t tc = f2_mul(c2, cr2);
            const f2_t tsr = f2_mul(s2, cr2);
            const f2_t cn = f2_fma(s2, nsr2, tc);
            s2 = f2_fma(c2, sr2, tsr);
            c2 = cn;
          }
        }
      }
      __syncthreads();
    }

    float pv[F];
    const float scale = oi.norm_scale_f, wsum = oi.wsum_f, yy = (float)oi.sum_y2;
    uint32_t bad = 0u;
#pragma unroll
    for (int m = 0; m < K; ++m) {
      float v[2][6];
      f2_unpack(xc[m], v[0][0], v[1][0]);
      f2_unpack(xs[m], v[0][1], v[1][1]);
      f2_unpack(cw[m], v[0][2], v[1][2]);
      f2_unpack(sw[m], v[0][3], v[1][3]);
      f2_unpack(cc[m], v[0][4], v[1][4]);
      f2_unpack(cs[m], v[0][5], v[1][5]);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        bool ill;
        const float pw = gls_power<float>(v[h][0], v[h][1], v[h][2], v[h][3], v[h][4], v[h][5], wsum, yy,
                                          EpsRel<float>::v, ill);
        const int idx = h * K + m;
        pv[idx] = scale * pw;
        if (ill && (int64_t)k0 + idx < p.n_f) bad |= 1u << idx;
      }
    }
    if (oi.flags) bad = 0u;
    fix_ill_conditioned_gls<F>(pv, bad, k0, p.rec, oi);
    if (p.power_out) store_row<F>(p.power_out + o * p.n_f, (int64_t)k0, pv, p.n_f);
    const int64_t res = o * (int64_t)n_chunks + chunk;
    chunk_results_f32<F>(pv, k0, kc0, p.n_f, p.best + res, p.cand ? p.cand + res : nullptr, s_pw, red);
  }
}

// Generalized periodogram, FP64 scalar chains (one chain of K per thread).
template <int K>
__global__ void __launch_bounds__(256) main_f64_gls(MainParams<RecF64, double> p) {
  constexpr int F = K;
  __shared__ uint4 s_rec[3 * LSP_TILE_OBS];
  __shared__ double red_p[32];
  __shared__ int64_t red_k[32];
  __shared__ uint32_t s_item;
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  double* s_pw = reinterpret_cast<double*>(dyn_smem);
  const int tid = threadIdx.x;
  const RecF64* srec = reinterpret_cast<const RecF64*>(s_rec);
  for (;;) {
    if (tid == 0) s_item = atomicAdd(p.queue, 1u);
    __syncthreads();
    const int64_t item = s_item;
    __syncthreads();
    if (item >= p.n_items) break;
    const int chunk = (int)(item % p.n_chunks);
    const int64_t orank = item / p.n_chunks;
    const int64_t o = p.order ? (int64_t)p.order[orank] : orank;
    const ObjInfo oi = p.obj[o];
    const int64_t kc0 = (int64_t)chunk * blockDim.x * F;
    const uint32_t k0 = (uint32_t)(kc0 + (int64_t)tid * F);
    const int64_t ob = oi.begin;
    const int64_t oe = oi.flags ? ob : oi.begin + oi.n;
    double xc[K], xs[K], cw[K], sw[K], cc[K], cs[K];
#pragma unroll
    for (int m = 0; m < K; ++m) xc[m] = xs[m] = cw[m] = sw[m] = cc[m] = cs[m] = 0.0;
    for (int64_t ts = ob; ts < oe; ts += LSP_TILE_OBS) {
      const int nt = (int)((oe - ts) < LSP_TILE_OBS ? (oe - ts) : LSP_TILE_OBS);
      const uint4* src = reinterpret_cast<const uint4*>(p.rec + ts);
      for (int i = tid; i < 3 * nt; i += blockDim.x) s_rec[i] = __ldg(src + i);
      __syncthreads();
      for (int j = 0; j < nt; ++j) {
        const RecF64 r = srec[j];
        double c, s;
        seed_sincos_f64(r.a + (uint64_t)k0 * r.b, c, s);
        const double u = r.y, w = __longlong_as_double((long long)r.pad), cr = r.cr, sr = r.sr;
#pragma unroll
        for (int m = 0; m < K; ++m) {
          xc[m] = fma(u, c, xc[m]);
          xs[m] = fma(u, s, xs[m]);
          cw[m] = fma(w, c, cw[m]);
          sw[m] = fma(w, s, sw[m]);
          const double wc = w * c;
          cc[m] = fma(wc, c, cc[m]);
          cs[m] = fma(wc, s, cs[m]);
          if (m + 1 < K) {
            const double cn = fma(-s, sr, c * cr);
            s = fma(c, sr, s * cr);
            c = cn;
          }
        }
      }
      __syncthreads();
    }
    double pv[F];
#pragma unroll
    for (int m = 0; m < K; ++m) {
      bool ill;
      pv[m] = oi.norm_scale * gls_power<double>(xc[m], xs[m], cw[m], sw[m], cc[m], cs[m], oi.wsum, oi.sum_y2,
                                                EpsRel<double>::v, ill);
    }
    if (p.power_out) store_row<F>(p.power_out + o * p.n_f, (int64_t)k0, pv, p.n_f);
    const int64_t res = o * p.n_chunks + chunk;
    chunk_results<double, F>(pv, (int64_t)k0, kc0, p.n_f, p.best + res, p.cand ? p.cand + res : nullptr, s_pw,
                             red_p, red_k);
  }
}

// ------------------------------------------------------------------------
// Scalar kernel: one reseed chain of K frequencies per thread.  Real = float
// (FP32 records, SFU seeds) or double (FP64 records, FP64 sincospi seeds).
template <typename Real, typename Rec, int K>
__global__ void __launch_bounds__(256) main_scalar(MainParams<Rec, Real> p) {
  constexpr int F = K;
  constexpr int RW = sizeof(Rec) / 16;
  __shared__ uint4 s_rec[RW * LSP_TILE_OBS];
  __shared__ double red_p[32];
  __shared__ int64_t red_k[32];
  __shared__ uint32_t s_item;
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  Real* s_pw = reinterpret_cast<Real*>(dyn_smem);
  const int tid = threadIdx.x;
  const Rec* srec = reinterpret_cast<const Rec*>(s_rec);

  for (;;) {
    if (tid == 0) s_item = atomicAdd(p.queue, 1u);
    __syncthreads();
    const int64_t item = s_item;
    __syncthreads();
    if (item >= p.n_items) break;
    const Item it = decode_item(p, item);
    const ObjInfo oi = p.obj[it.o];
    const int64_t kc0 = (int64_t)it.chunk * blockDim.x * F;
    const uint32_t k0 = (uint32_t)(kc0 + (int64_t)tid * F);
    int64_t ob = oi.begin + (int64_t)oi.n * it.s / p.split;
    int64_t oe = oi.begin + (int64_t)oi.n * (it.s + 1) / p.split;
    if (oi.flags) oe = ob;

    Real xc[K], xs[K], cc[K], cs[K];
#pragma unroll
    for (int m = 0; m < K; ++m) xc[m] = xs[m] = cc[m] = cs[m] = Real(0);

    for (int64_t ts = ob; ts < oe; ts += LSP_TILE_OBS) {
      const int nt = (int)((oe - ts) < LSP_TILE_OBS ? (oe - ts) : LSP_TILE_OBS);
      const uint4* src = reinterpret_cast<const uint4*>(p.rec + ts);
      for (int i = tid; i < RW * nt; i += blockDim.x) s_rec[i] = __ldg(src + i);
      __syncthreads();
      for (int j = 0; j < nt; ++j) {
        const Rec r = srec[j];
        Real c, s;
        if constexpr (std::is_same<Real, float>::value) {
          seed_sincos_f32(phase_hi32(r.a_hi, r.b_hi, r.b_lo, k0), c, s);
        } else {
          seed_sincos_f64(r.a + (uint64_t)k0 * r.b, c, s);
        }
        const Real y = r.y, cr = r.cr, sr = r.sr;
#pragma unroll
        for (int m = 0; m < K; ++m) {
          xc[m] = fma(y, c, xc[m]);
          xs[m] = fma(y, s, xs[m]);
          cc[m] = fma(c, c, cc[m]);
          cs[m] = fma(c, s, cs[m]);
          if (m + 1 < K) {
            const Real cn = fma(-s, sr, c * cr);
            s = fma(c, sr, s * cr);
            c = cn;
          }
        }
      }
      __syncthreads();
    }

    if (p.split == 1) {
      Real pv[F];
      const int64_t res = it.o * p.n_chunks + it.chunk;
      if constexpr (std::is_same<Real, float>::value) {
        const float nf = (float)oi.n, scale = oi.norm_scale_f;
        uint32_t bad = 0u;
#pragma unroll
        for (int m = 0; m < K; ++m) {
          bool ill;
          pv[m] = scale * lsp_power_f32(xc[m], xs[m], cc[m], cs[m], nf, ill);
          if (ill && (int64_t)k0 + m < p.n_f) bad |= 1u << m;
        }
        if (oi.flags) bad = 0u;
        fix_ill_conditioned<F>(pv, bad, k0, p.rec, oi.begin, oi.n, oi.norm_scale);
        if (p.power_out) store_row<F>(p.power_out + it.o * p.n_f, (int64_t)k0, pv, p.n_f);
        chunk_results_f32<F>(pv, k0, kc0, p.n_f, p.best + res, p.cand ? p.cand + res : nullptr,
                             reinterpret_cast<float*>(s_pw), reinterpret_cast<unsigned long long*>(red_p));
      } else {
        const Real nf = (Real)oi.n, scale = (Real)oi.norm_scale;
#pragma unroll
        for (int m = 0; m < K; ++m)
          pv[m] = scale * lsp_power<Real>(xc[m], xs[m], cc[m], cs[m], nf, EpsRel<Real>::v);
        if (p.power_out) store_row<F>(p.power_out + it.o * p.n_f, (int64_t)k0, pv, p.n_f);
        chunk_results<Real, F>(pv, (int64_t)k0, kc0, p.n_f, p.best + res,
                               p.cand ? p.cand + res : nullptr, s_pw, red_p, red_k);
      }
    } else {
      Real* part = p.part + (int64_t)it.s * p.n_f * 4;
#pragma unroll
      for (int m = 0; m < K; ++m)
        if ((int64_t)k0 + m < p.n_f) store_part(part, (int64_t)k0 + m, xc[m], xs[m], cc[m], cs[m]);
    }
  }
}

}  // namespace lsp
