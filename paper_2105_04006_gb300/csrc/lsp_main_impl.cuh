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
//   - sin/cos come from a recurrence across the uniform grid, reseeded from
//     the exact fixed-point phase every K frequencies (the paper, Section
//     4.5, rejects the recurrence as serial; here it runs along a thread's
//     own frequencies while threads, CTAs and objects run in parallel).
//     One rotation by (cr, sr) = e^{2 pi i df t'} gives the second value,
//     then a three-term recurrence of one FMA per component gives the rest
//     (chain3 below): 6 FP32 operations per pair instead of the rotation's 8;
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

// The six generalized sums of one frequency in a stride-8 slot (two 16-byte
// words for FP32, three for FP64; the last two entries stay unused).
__device__ __forceinline__ void store_part_gls(float* part, int64_t idx, float a, float b, float c, float d,
                                               float e, float f) {
  reinterpret_cast<float4*>(part)[2 * idx] = make_float4(a, b, c, d);
  reinterpret_cast<float2*>(part)[4 * idx + 2] = make_float2(e, f);
}
__device__ __forceinline__ void store_part_gls(double* part, int64_t idx, double a, double b, double c,
                                               double d, double e, double f) {
  double2* p2 = reinterpret_cast<double2*>(part) + 4 * idx;
  p2[0] = make_double2(a, b);
  p2[1] = make_double2(c, d);
  p2[2] = make_double2(e, f);
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
// Each tile of observations is staged as expanded 64-byte entries (ObsF2
// below).  Each observation costs every thread two SFU seeds (one per
// chain), one packed rotation and K-2 packed three-term steps (chain3).  (Measured alternatives
// that did not pay on GB300: issuing the next observation's seeds one step
// ahead, integer bit-building of the seed angle instead of I2F, deriving the
// second chain's seed from the first by a K-step rotation, unrolling the
// observation loop by two, and unpacked scalar rotations.)

__device__ __forceinline__ f2_t f2_of(uint32_t lo, uint32_t hi) {
  f2_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "r"(lo), "r"(hi));
  return r;
}

// ------------------------------------------------------- three-term chains
// Element-wise helpers for the three chain types: packed f32x2 pairs, float
// and double.  neg_ flips the sign bit; dbl_ doubles by adding one to the
// exponent field (exact for normal numbers; a zero or subnormal input, which
// a rounded cos or sin of a grid step essentially never is, becomes a number
// of magnitude <= 2^-125 (FP32) or 2^-1021 (FP64) instead, a negligible
// coefficient error).
__device__ __forceinline__ f2_t mul_(f2_t a, f2_t b) { return f2_mul(a, b); }
__device__ __forceinline__ f2_t fma_(f2_t a, f2_t b, f2_t c) { return f2_fma(a, b, c); }
__device__ __forceinline__ f2_t neg_(f2_t a) { return a ^ 0x8000000080000000ull; }
__device__ __forceinline__ f2_t dbl_(f2_t a) { return a + 0x0080000000800000ull; }
__device__ __forceinline__ float mul_(float a, float b) { return a * b; }
__device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float neg_(float a) { return __uint_as_float(__float_as_uint(a) ^ 0x80000000u); }
__device__ __forceinline__ float dbl_(float a) { return __uint_as_float(__float_as_uint(a) + 0x00800000u); }
__device__ __forceinline__ double mul_(double a, double b) { return a * b; }
__device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ double neg_(double a) {
  return __longlong_as_double(__double_as_longlong(a) ^ (long long)0x8000000000000000ull);
}
__device__ __forceinline__ double dbl_(double a) {
  return __longlong_as_double(__double_as_longlong(a) + (1ll << 52));
}
// |sin| > |cos| from the bit patterns (IEEE magnitudes order like integers).
__device__ __forceinline__ bool sin_dominates(uint32_t cr_bits, uint32_t sr_bits) {
  return (sr_bits & 0x7fffffffu) > (cr_bits & 0x7fffffffu);
}
__device__ __forceinline__ bool sin_dominates(double cr, double sr) {
  return (__double_as_longlong(sr) & 0x7fffffffffffffffll) > (__double_as_longlong(cr) & 0x7fffffffffffffffll);
}

// One reseed chain at one observation: the K values e_m = e_0 e^{i m theta},
// m = 0 .. K-1, theta = 2 pi df t', (cr, sr) = (cos theta, sin theta).
// body(m, neg, c, s) receives (c, s) = sigma_m e_m, sigma_m = -1 when neg.
//
// e_1 = e_0 (cr + i sr) by one rotation (4 operations); the rest by one of
// two three-term recurrences at 2 operations per step, chosen per
// observation so that its error amplification stays <= sqrt 2:
//   Chebyshev  e_{m+1} = 2 cos(theta) e_m - e_{m-1}   where |sin| > |cos|;
//              a rounding error propagates as sin((n+1) theta) / sin theta
//              and the coefficient's rounding moves theta by <= ulp cot(theta);
//   leapfrog   e_{m+1} = e_{m-1} + 2 i sin(theta) e_m  elsewhere; its roots
//              e^{i theta} and -e^{-i theta} stay 2 |cos theta| apart and
//              the coefficient's rounding moves theta by <= ulp tan(theta).
// The Chebyshev chain stores x_m = sigma_m e_m with sigma = + + - - + + ...,
// which turns its subtraction into an FMA addend of + x_{m-1}:
// x_{m+1} = (sigma_{m+1} sigma_m) 2 cr x_m + x_{m-1}, the product sign
// alternating + - + - with m.  The choice is the same for every thread of a
// CTA (one observation at a time), so the branch never diverges.
template <int K, bool CHEB, typename T, typename Body>
__device__ __forceinline__ void chain3_mode(T c, T s, T cr, T sr, T nsr, T coef, T ncoef, Body&& body) {
  body(0, false, c, s);
  if constexpr (K > 1) {
    const T c1 = fma_(s, nsr, mul_(c, cr));
    const T s1 = fma_(c, sr, mul_(s, cr));
    body(1, false, c1, s1);
    T cp = c, sp = s;
    c = c1;
    s = s1;
#pragma unroll
    for (int m = 1; m + 1 < K; ++m) {
      T cn, sn;
      if constexpr (CHEB) {
        const T cm = (m & 1) ? ncoef : coef;
        cn = fma_(cm, c, cp);
        sn = fma_(cm, s, sp);
      } else {
        cn = fma_(ncoef, s, cp);
        sn = fma_(coef, c, sp);
      }
      cp = c;
      sp = s;
      c = cn;
      s = sn;
      body(m + 1, CHEB && ((m + 1) & 2) != 0, c, s);
    }
  }
}

// chain3_mode with the coefficients formed here and the form chosen at run
// time: coef = 2 cr (Chebyshev, cheb true) or 2 sr (leapfrog).
template <int K, typename T, typename Body>
__device__ __forceinline__ void chain3(T c, T s, T cr, T sr, bool cheb, Body&& body) {
  if (cheb) {
    const T a = dbl_(cr);
    chain3_mode<K, true>(c, s, cr, sr, neg_(sr), a, neg_(a), body);
  } else {
    const T b = dbl_(sr);
    chain3_mode<K, false>(c, s, cr, sr, neg_(sr), b, neg_(b), body);
  }
}

// ------------------------------------------------ expanded observation tile
// The packed kernels stage each tile of observations into shared memory as
// ObsF2 entries that hold every operand of the inner loop already paired for
// f32x2 (negated where a negation is needed), with the tile's Chebyshev observations first
// and its leapfrog observations after them (a stable partition by index,
// so the summation order is fixed).  The inner loops then issue no packing,
// sign or mode instructions and no per-observation branch.
struct __align__(16) ObsF2 {
  f2_t y;             // {y, y}  (GLS: u = w (y - ybar_w))
  f2_t cr, sr, nsr;   // cos, sin and -sin of the grid step angle theta
  f2_t coef, ncoef;   // +-2 cos theta (Chebyshev) or +-2 sin theta (leapfrog)
  uint32_t a_hi, b_hi, b_lo, kb_hi;  // phase words and the high word of K b
};
struct __align__(16) ObsF2W {
  ObsF2 e;            // e.y = {v, v} with v = u / sqrt(w) = sqrt(w) (y - ybar_w)
  f2_t w, nu, nw;     // {r, r} with r = sqrt(w), w = 1 / dy^2; {-v, -v}; {-r, -r} (generalized periodogram)
};

__device__ __forceinline__ f2_t f2_dup(uint32_t v) { return f2_of(v, v); }

__device__ __forceinline__ void expand_obs(const uint4 r0, const uint4 r1, bool cheb, uint32_t K, ObsF2& e) {
  const uint32_t sign = 0x80000000u;
  const uint32_t cf = cheb ? r0.y + 0x00800000u : r0.z + 0x00800000u;  // 2 cr or 2 sr (exponent + 1)
  e.y = f2_dup(r0.x);
  e.cr = f2_dup(r0.y);
  e.sr = f2_dup(r0.z);
  e.nsr = f2_dup(r0.z ^ sign);
  e.coef = f2_dup(cf);
  e.ncoef = f2_dup(cf ^ sign);
  e.a_hi = r0.w;
  e.b_hi = r1.x;
  e.b_lo = r1.y;
  e.kb_hi = K * r1.x + __umulhi(K, r1.y);  // high word of K b (mod 2^64)
}
// The generalized kernel runs its chains on sqrt(w) (cos, sin): the rotation
// and the three-term steps are linear in the seeds, so scaled seeds give
// scaled values c' = r c, s' = r s (r = sqrt(w)), and the six weighted sums
// take one operation each: w c^2 = c'^2, w c s = c' s', w c = r c',
// u c = (u / r) c' (and the same for s).
__device__ __forceinline__ void expand_obs(const uint4 r0, const uint4 r1, bool cheb, uint32_t K, ObsF2W& e) {
  expand_obs(r0, r1, cheb, K, e.e);
  const float r = sqrtf(__uint_as_float(r1.w));
  const uint32_t v = __float_as_uint(__fdiv_rn(__uint_as_float(r0.x), r));
  e.e.y = f2_dup(v);
  e.w = f2_dup(__float_as_uint(r));
  e.nu = f2_dup(v ^ 0x80000000u);
  e.nw = f2_dup(__float_as_uint(r) ^ 0x80000000u);
}

// Stage records [0, nt) of src (32-byte RecF32, nt <= LSP_TILE_OBS) into
// ent; returns the number of Chebyshev entries.  blockDim.x is a multiple of
// 32, so each warp's 32 consecutive records form one ballot slice.
template <typename Ent>
__device__ __forceinline__ int stage_tile(const uint4* __restrict__ src, int nt, uint32_t K, Ent* ent,
                                          uint32_t* s_bal) {
  const int tid = threadIdx.x, lane = tid & 31;
  for (int i = tid; i < LSP_TILE_OBS; i += blockDim.x) {
    bool cheb = false;
    if (i < nt) {
      const uint4 r0 = __ldg(src + 2 * i);
      cheb = sin_dominates(r0.y, r0.z);
    }
    const uint32_t bal = __ballot_sync(0xffffffffu, cheb);
    if (lane == 0) s_bal[i >> 5] = bal;
  }
  __syncthreads();
  int n_cheb = 0;
#pragma unroll
  for (int q = 0; q < LSP_TILE_OBS / 32; ++q) n_cheb += __popc(s_bal[q]);
  for (int i = tid; i < nt; i += blockDim.x) {
    const uint4 r0 = __ldg(src + 2 * i), r1 = __ldg(src + 2 * i + 1);
    const int sl = i >> 5;
    int before = 0;
    for (int q = 0; q < sl; ++q) before += __popc(s_bal[q]);
    const uint32_t b = s_bal[sl];
    before += __popc(b & ((1u << lane) - 1u));
    const bool cheb = (b >> lane) & 1u;
    expand_obs(r0, r1, cheb, K, ent[cheb ? before : n_cheb + (i - before)]);
  }
  __syncthreads();
  return n_cheb;
}

// Loop over staged observation entries [j0, j1).  kRolled keeps it rolled:
// the chains of up to 12 frequencies run measurably faster per pair that way
// (unrolled, their register count rose past the occupancy the launch bounds
// ask for); the 16-frequency chains gain from the compiler's unrolling.
template <bool kRolled, typename Fn>
__device__ __forceinline__ void obs_loop(int j0, int j1, Fn&& fn) {
  if constexpr (kRolled) {
#pragma unroll 1
    for (int j = j0; j < j1; ++j) fn(j);
  } else {
    for (int j = j0; j < j1; ++j) fn(j);
  }
}

// Seeds of the two packed chains: bins k0 and k0 + K.
__device__ __forceinline__ void seed_pair_kb(const ObsF2& e, uint32_t k0, f2_t& c2, f2_t& s2) {
  float c0, s0, c1, s1;
  const uint32_t ph0 = phase_hi32(e.a_hi, e.b_hi, e.b_lo, k0);
  seed_sincos_f32(ph0, c0, s0);
  seed_sincos_f32(ph0 + e.kb_hi, c1, s1);  // error <= 2^-31 cycle from the dropped carries
  c2 = f2_pack(c0, c1);
  s2 = f2_pack(s0, s1);
}

template <int K>
__device__ __forceinline__ void main_f32_packed_body(const MainParams<RecF32, float>& p) {
  constexpr int F = 2 * K;
  __shared__ ObsF2 s_ent[LSP_TILE_OBS];
  __shared__ uint32_t s_bal[LSP_TILE_OBS / 32];
  __shared__ unsigned long long red[32];
  __shared__ uint32_t s_item;
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  float* s_pw = reinterpret_cast<float*>(dyn_smem);
  const int tid = threadIdx.x;
  const uint32_t n_items = p.n_items_dev ? *p.n_items_dev : (uint32_t)p.n_items;
  const uint32_t split = (uint32_t)p.split, n_chunks = (uint32_t)p.n_chunks;

  // A CTA's first item is its own index; later ones come from the queue
  // counter, offset by the grid, thread 0 taking the next item's ticket one
  // item ahead so that the atomic's round trip overlaps the current item.
  // (Prefetching from the first item on let the CTAs that start first claim
  // two items each while later ones found the queue empty: a one-wave
  // launch, one object split over its observations, ran up to 1.7x longer.)
  uint32_t ticket = blockIdx.x;
  for (;;) {
    if (tid == 0) s_item = ticket;
    __syncthreads();
    const uint32_t item = s_item;
    __syncthreads();
    if (item >= n_items) break;
    if (tid == 0) ticket = gridDim.x + atomicAdd(p.queue, 1u);
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
      const int n_ch = stage_tile(reinterpret_cast<const uint4*>(p.rec + ts), nt, (uint32_t)K, s_ent, s_bal);
      // The Chebyshev values carry sigma_m; rather than alternate y and -y (a
      // measured 10 % loss of FMA throughput), the y-weighted sums of the
      // sigma_m = -1 frequencies are negated around the Chebyshev run, which
      // is exact: the sums come out bit-identical.
      auto obs = [&](const ObsF2& e, auto cheb_tag) {
        f2_t c2, s2;
        seed_pair_kb(e, k0, c2, s2);
        const f2_t y2 = e.y;
        chain3_mode<K, decltype(cheb_tag)::value>(c2, s2, e.cr, e.sr, e.nsr, e.coef, e.ncoef,
                                                  [&](int m, bool, f2_t c, f2_t s) {
                                                    xc[m] = f2_fma(y2, c, xc[m]);
                                                    xs[m] = f2_fma(y2, s, xs[m]);
                                                    cc[m] = f2_fma(c, c, cc[m]);
                                                    cs[m] = f2_fma(c, s, cs[m]);
                                                  });
      };
      auto flip = [&]() {
#pragma unroll
        for (int m = 0; m < K; ++m)
          if (m & 2) {
            xc[m] = neg_(xc[m]);
            xs[m] = neg_(xs[m]);
          }
      };
      // threads whose bins all lie past the end of the grid (the ragged last
      // chunk) only help stage tiles; a warp of them leaves its FMA pipe to
      // the other CTAs on the SM
      if ((int64_t)k0 < kend) {
        if (n_ch > 0) {
          flip();
          obs_loop<(K <= 12)>(0, n_ch, [&](int j) { obs(s_ent[j], std::true_type{}); });
          flip();
        }
        obs_loop<(K <= 12)>(n_ch, nt, [&](int j) { obs(s_ent[j], std::false_type{}); });
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
      // the 16-frequency chains keep the staged epilogue: with the register
      // one their main loop compiled slower (one large object: 22.9 against
      // 21.7 ms), more than the epilogue saves
      if constexpr (K >= 16)
        chunk_results_f32_staged<F>(pv, k0, kc0, kend, p.best + res, p.cand ? p.cand + res : nullptr, s_pw, red);
      else
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

// The standard kernel with the default launch bounds, and with launch bounds
// that ask for MINB resident CTAs of MAXT threads (a register floor).
template <int K>
__global__ void __launch_bounds__(256) main_f32_packed(MainParams<RecF32, float> p) {
  main_f32_packed_body<K>(p);
}
template <int K, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) main_f32_packed_floor(MainParams<RecF32, float> p) {
  main_f32_packed_body<K>(p);
}

// ------------------------------------------------------------------------
// Generalized periodogram (Section 4.11), FP32, two packed reseed chains:
// the same tiling and seeding as main_f32_packed with six weighted sums per
// frequency (11 FP32 operations per pair instead of 8 in the rotation form;
// the kernel spends 8: two for the three-term step and one per sum, its
// chains carrying sqrt(w) (cos, sin)).  Records carry u = w (y - ybar_w) in
// the y word and w in the spare word.
template <int K>
__global__ void __launch_bounds__(256) main_f32_packed_gls(MainParams<RecF32, float> p) {
  constexpr int F = 2 * K;
  __shared__ ObsF2W s_ent[LSP_TILE_OBS];
  __shared__ uint32_t s_bal[LSP_TILE_OBS / 32];
  __shared__ unsigned long long red[32];
  __shared__ uint32_t s_item;
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  float* s_pw = reinterpret_cast<float*>(dyn_smem);
  const int tid = threadIdx.x;
  const uint32_t n_items = p.n_items_dev ? *p.n_items_dev : (uint32_t)p.n_items;
  const uint32_t split = (uint32_t)p.split, n_chunks = (uint32_t)p.n_chunks;

  uint32_t ticket = blockIdx.x;  // first item static, then one ticket ahead (see main_f32_packed_body)
  for (;;) {
    if (tid == 0) s_item = ticket;
    __syncthreads();
    const uint32_t item = s_item;
    __syncthreads();
    if (item >= n_items) break;
    if (tid == 0) ticket = gridDim.x + atomicAdd(p.queue, 1u);
    const uint32_t is = item % split;
    const uint32_t oc = item / split;
    const uint32_t chunk = oc % n_chunks;
    const uint32_t orank = oc / n_chunks;
    const int64_t o = p.order ? (int64_t)p.order[orank] : (int64_t)orank;
    const ObjInfo oi = p.obj[o];
    const int64_t kc0 = (int64_t)chunk * blockDim.x * F;
    const uint32_t k0 = (uint32_t)(kc0 + (int64_t)tid * F);
    const int64_t ob = oi.begin + (int64_t)oi.n * is / split;
    int64_t oe = oi.begin + (int64_t)oi.n * (is + 1) / split;
    if (oi.flags) oe = ob;  // flagged objects: zero power

    f2_t xc[K], xs[K], cw[K], sw[K], cc[K], cs[K];
#pragma unroll
    for (int m = 0; m < K; ++m) xc[m] = xs[m] = cw[m] = sw[m] = cc[m] = cs[m] = 0ull;

    for (int64_t ts = ob; ts < oe; ts += LSP_TILE_OBS) {
      const int nt = (int)((oe - ts) < LSP_TILE_OBS ? (oe - ts) : LSP_TILE_OBS);
      const int n_ch = stage_tile(reinterpret_cast<const uint4*>(p.rec + ts), nt, (uint32_t)K, s_ent, s_bal);
      auto obs = [&](const ObsF2W& ew, auto cheb_tag) {
        const ObsF2& e = ew.e;
        f2_t c2, s2;
        seed_pair_kb(e, k0, c2, s2);
        const f2_t v2 = e.y, nv2 = ew.nu, r2 = ew.w, nr2 = ew.nw;
        c2 = f2_mul(r2, c2);  // chains of sqrt(w) (cos, sin)
        s2 = f2_mul(r2, s2);
        chain3_mode<K, decltype(cheb_tag)::value>(c2, s2, e.cr, e.sr, e.nsr, e.coef, e.ncoef,
                                                  [&](int m, bool neg, f2_t c, f2_t s) {
                                                    const f2_t vv = neg ? nv2 : v2, rr = neg ? nr2 : r2;
                                                    xc[m] = f2_fma(vv, c, xc[m]);
                                                    xs[m] = f2_fma(vv, s, xs[m]);
                                                    cw[m] = f2_fma(rr, c, cw[m]);
                                                    sw[m] = f2_fma(rr, s, sw[m]);
                                                    cc[m] = f2_fma(c, c, cc[m]);
                                                    cs[m] = f2_fma(c, s, cs[m]);
                                                  });
      };
      // (the accumulator flip of main_f32_packed costs this kernel registers
      // and occupancy: here the weights alternate sign instead)
      if ((int64_t)k0 < p.n_f) {  // bins past the grid end: staging only
        for (int j = 0; j < n_ch; ++j) obs(s_ent[j], std::true_type{});
        for (int j = n_ch; j < nt; ++j) obs(s_ent[j], std::false_type{});
      }
      __syncthreads();
    }

    if (split > 1) {  // one slice of a single object: partial sums for the combine
      float* part = p.part + (int64_t)is * p.n_f * 8;
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
          const int64_t k = (int64_t)k0 + h * K + m;
          if (k < p.n_f) store_part_gls(part, k, v[h][0], v[h][1], v[h][2], v[h][3], v[h][4], v[h][5]);
        }
      }
      continue;
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
    chunk_results_f32_staged<F>(pv, k0, kc0, p.n_f, p.best + res, p.cand ? p.cand + res : nullptr, s_pw, red);
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
    const Item it = decode_item(p, item);
    const int64_t o = it.o;
    const int chunk = it.chunk;
    const ObjInfo oi = p.obj[o];
    const int64_t kc0 = (int64_t)chunk * blockDim.x * F;
    const uint32_t k0 = (uint32_t)(kc0 + (int64_t)tid * F);
    const int64_t ob = oi.begin + (int64_t)oi.n * it.s / p.split;
    int64_t oe = oi.begin + (int64_t)oi.n * (it.s + 1) / p.split;
    if (oi.flags) oe = ob;  // flagged objects: zero power
    double xc[K], xs[K], cw[K], sw[K], cc[K], cs[K];
#pragma unroll
    for (int m = 0; m < K; ++m) xc[m] = xs[m] = cw[m] = sw[m] = cc[m] = cs[m] = 0.0;
    for (int64_t ts = ob; ts < oe; ts += LSP_TILE_OBS) {
      const int nt = (int)((oe - ts) < LSP_TILE_OBS ? (oe - ts) : LSP_TILE_OBS);
      const uint4* src = reinterpret_cast<const uint4*>(p.rec + ts);
      for (int i = tid; i < 3 * nt; i += blockDim.x) s_rec[i] = __ldg(src + i);
      __syncthreads();
      // chains of sqrt(w) (cos, sin), as in main_f32_packed_gls: the staged
      // record holds v = u / sqrt(w) in the y word and sqrt(w) in the spare word
      for (int i = tid; i < nt; i += blockDim.x) {
        RecF64* q = reinterpret_cast<RecF64*>(s_rec) + i;
        const double r = sqrt(__longlong_as_double((long long)q->pad));
        q->y = q->y / r;
        q->pad = (uint64_t)__double_as_longlong(r);
      }
      __syncthreads();
      const int nt_c = (int64_t)k0 < p.n_f ? nt : 0;  // bins past the grid end: staging only
      for (int j = 0; j < nt_c; ++j) {
        const RecF64 r = srec[j];
        double c, s;
        seed_sincos_f64(r.a + (uint64_t)k0 * r.b, c, s);
        const double v = r.y, rw = __longlong_as_double((long long)r.pad), nv = neg_(v), nrw = neg_(rw);
        c *= rw;
        s *= rw;
        chain3<K>(c, s, r.cr, r.sr, sin_dominates(r.cr, r.sr), [&](int m, bool neg, double cm, double sm) {
          const double vv = neg ? nv : v, rr = neg ? nrw : rw;
          xc[m] = fma(vv, cm, xc[m]);
          xs[m] = fma(vv, sm, xs[m]);
          cw[m] = fma(rr, cm, cw[m]);
          sw[m] = fma(rr, sm, sw[m]);
          cc[m] = fma(cm, cm, cc[m]);
          cs[m] = fma(cm, sm, cs[m]);
        });
      }
      __syncthreads();
    }
    if (p.split > 1) {  // one slice of a single object: partial sums for the combine
      double* part = p.part + (int64_t)it.s * p.n_f * 8;
#pragma unroll
      for (int m = 0; m < K; ++m)
        if ((int64_t)k0 + m < p.n_f)
          store_part_gls(part, (int64_t)k0 + m, xc[m], xs[m], cw[m], sw[m], cc[m], cs[m]);
      continue;
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

// (cos, sin) of a 32-bit fixed-point phase with CUDA's accurate FP32
// sincospif: the argument (int)ph * 2^-31 half-cycles is exact up to the
// integer-to-float rounding (<= 2^-25 half-cycle).
__device__ __forceinline__ void sincos_accurate_f32(uint32_t ph, float& c, float& s) {
  sincospif(__int2float_rn((int)ph) * 4.656612873077393e-10f, &s, &c);  // 2^-31
}

// One 32-byte record read straight from global memory (every thread of the
// CTA reads the same record: an L1 broadcast).
__device__ __forceinline__ RecF32 load_rec_global(const RecF32* rec) {
  const uint4* q = reinterpret_cast<const uint4*>(rec);
  const uint4 a = __ldg(q), b = __ldg(q + 1);
  RecF32 r;
  r.y = __uint_as_float(a.x);
  r.cr = __uint_as_float(a.y);
  r.sr = __uint_as_float(a.z);
  r.a_hi = a.w;
  r.b_hi = b.x;
  r.b_lo = b.y;
  r.a_lo = b.z;
  r.pad = b.w;
  return r;
}

// ------------------------------------------------------------------------
// Scalar kernel: one reseed chain of K frequencies per thread.  Real = float
// (FP32 records, SFU seeds) or double (FP64 records, FP64 sincospi seeds).
//
// Ablations (FP32 only; the paper's Section 3.6 / Table 3 and Section 4.12 /
// Table 6 choices, selectable through lsp_config): TRIG = 1 evaluates every
// pair's (cos, sin) with the SFU intrinsic from the exact phase, TRIG = 2
// with the accurate sincospif, instead of the reseeded recurrence (TRIG = 0);
// GLOBAL = true reads each observation record from global memory in every
// thread instead of staging tiles in shared memory.
template <typename Real, typename Rec, int K, int TRIG = 0, bool GLOBAL = false>
__global__ void __launch_bounds__(256) main_scalar(MainParams<Rec, Real> p) {
  constexpr int F = K;
  constexpr int RW = sizeof(Rec) / 16;
  __shared__ uint4 s_rec[GLOBAL ? 1 : RW * LSP_TILE_OBS];
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

    auto one_obs = [&](const Rec& r) {
      if constexpr (TRIG == 0) {
        Real c, s;
        if constexpr (std::is_same<Real, float>::value) {
          seed_sincos_f32(phase_hi32(r.a_hi, r.b_hi, r.b_lo, k0), c, s);
        } else {
          seed_sincos_f64(r.a + (uint64_t)k0 * r.b, c, s);
        }
        const Real y = r.y, ny = neg_(y);
        bool cheb;
        if constexpr (std::is_same<Real, float>::value)
          cheb = sin_dominates(__float_as_uint(r.cr), __float_as_uint(r.sr));
        else
          cheb = sin_dominates(r.cr, r.sr);
        chain3<K>(c, s, (Real)r.cr, (Real)r.sr, cheb, [&](int m, bool neg, Real cm, Real sm) {
          const Real yy = neg ? ny : y;
          xc[m] = fma(yy, cm, xc[m]);
          xs[m] = fma(yy, sm, xs[m]);
          cc[m] = fma(cm, cm, cc[m]);
          cs[m] = fma(cm, sm, cs[m]);
        });
      } else {
        const float y = r.y;
#pragma unroll
        for (int m = 0; m < K; ++m) {
          const uint32_t ph = phase_hi32(r.a_hi, r.b_hi, r.b_lo, k0 + (uint32_t)m);
          float c, s;
          if constexpr (TRIG == 1)
            seed_sincos_f32(ph, c, s);
          else
            sincos_accurate_f32(ph, c, s);
          xc[m] = fmaf(y, c, xc[m]);
          xs[m] = fmaf(y, s, xs[m]);
          cc[m] = fmaf(c, c, cc[m]);
          cs[m] = fmaf(c, s, cs[m]);
        }
      }
    };
    if constexpr (GLOBAL) {
      const int64_t oe_c = (int64_t)k0 < p.n_f ? oe : ob;  // bins past the grid end: nothing to do
      for (int64_t j = ob; j < oe_c; ++j) one_obs(load_rec_global(p.rec + j));
    } else {
      for (int64_t ts = ob; ts < oe; ts += LSP_TILE_OBS) {
        const int nt = (int)((oe - ts) < LSP_TILE_OBS ? (oe - ts) : LSP_TILE_OBS);
        const uint4* src = reinterpret_cast<const uint4*>(p.rec + ts);
        for (int i = tid; i < RW * nt; i += blockDim.x) s_rec[i] = __ldg(src + i);
        __syncthreads();
        const int nt_c = (int64_t)k0 < p.n_f ? nt : 0;  // bins past the grid end: staging only
        for (int j = 0; j < nt_c; ++j) one_obs(srec[j]);
        __syncthreads();
      }
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
