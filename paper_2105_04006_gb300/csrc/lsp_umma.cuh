// lsp_umma.cuh -- bfloat16 GEMM on the fifth-generation tensor cores
// (tcgen05.mma, accumulator in tensor memory, operands staged by TMA), used by
// the proposal network's forward and backward passes.
//
//   C[M, N] = A[M, K] * B[N, K]^T        (A, B bfloat16, both K-contiguous)
//
// One CTA of 128 threads computes a 128 x n_tile tile (n_tile a multiple of
// 16, at most 256) over a range of K:
//   * warp 0, lane 0 -- TMA producer: 64-wide K slices of A (128 rows) and B
//     (n_tile rows) into a 2-stage ring of shared-memory buffers in the
//     128-byte-swizzled K-major layout, one mbarrier per stage ("full");
//   * warp 1, lane 0 -- issues tcgen05.mma (M 128, N n_tile, K 16, four per
//     slice) into an FP32 accumulator of n_tile tensor-memory columns, and
//     releases each stage with tcgen05.commit onto its "empty" mbarrier;
//   * warp 2 allocates and frees the tensor memory;
//   * all four warps then read the accumulator back with tcgen05.ld (warp w
//     owns tile rows 32w..32w+31, one row per thread), add the bias, apply
//     ReLU, and stage the FP32 tile in the idle ring, 128 columns at a time;
//     the stores to global memory then run along rows, 8 columns per lane
//     with 16-byte writes (or, for the transposed copy, down columns), so
//     that each warp writes contiguous bytes: multiplication by a ReLU mask,
//     FP32 and/or bfloat16 outputs, and an optional transposed bfloat16 copy
//     (the operand layout the weight-gradient GEMM reads).
// Two CTAs share an SM (99 KiB of shared memory and 256 TMEM columns each),
// so one CTA's epilogue overlaps the other's loads and MMAs.
// Rows and columns outside the matrices are zero-filled by TMA, so any M, N,
// K work; the operands need 16-byte-aligned bases and row pitches.
//
// Every wait is bounded (about a second of global time).  A CTA that gives up
// waits, again bounded, for its own copies in flight, writes NaN over its
// output tile, frees its tensor memory and counts itself in g_umma_timeouts.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cstdint>

namespace umma {

typedef __nv_bfloat16 bf16;

constexpr int BM = 128;      // tile rows (tcgen05 M)
constexpr int BK = 64;       // K slice per stage: 64 bfloat16 = one 128-byte swizzle row
constexpr int STAGES = 2;    // two CTAs share an SM: one's epilogue overlaps the other's loads
constexpr int MAX_BN = 256;  // tcgen05 N limit for M = 128
constexpr int THREADS = 128;
constexpr int TMEM_COLS = 256;
constexpr int A_STAGE = BM * BK * 2;      // 16 KiB
constexpr int B_STAGE = MAX_BN * BK * 2;  // 32 KiB
constexpr int SMEM_BYTES = 1024 /* alignment slack */ + STAGES * (A_STAGE + B_STAGE) + 128 /* mbarriers */;
constexpr int EPI_COLS = 128;  // accumulator columns staged at a time (FP32, in the idle ring)
constexpr unsigned long long kWaitNs = 1000000000ull;

struct Args {
  int M, N, K;
  int n_tile;        // columns per CTA: multiple of 16, <= 256
  int kb_per_split;  // K slices per blockIdx.z
  const float* bias; // [N] or NULL
  int relu;
  const bf16* mask;  // [M][ldm]: output kept where mask > 0, or NULL
  int64_t ldm;
  float* C32;        // [M][ldc32] (+ blockIdx.z * split_stride), or NULL
  int64_t ldc32, split_stride;
  bf16* C16;         // [M][ldc16] or NULL
  int64_t ldc16;
  bf16* C16T;        // [N][ldt] (transposed) or NULL
  int64_t ldt;
  int withhold_first_load;  // wait test only: the first K slice is never loaded, so its waits run out
};

__device__ unsigned int g_umma_timeouts;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase of parity `parity` to complete.  Gives up (false) after
// kWaitNs, or early once *abort is set when abort is given.
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, const volatile int* abort) {
  const uint64_t t0 = global_ns();
  for (uint32_t i = 1;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63u) == 0) {
      if (abort && *abort) return false;
      if (global_ns() - t0 > kWaitNs) return false;
    }
  }
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// 2-D tiled TMA load: box at (x = K element, y = row) into shared memory,
// completing `bytes` on the mbarrier.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand in the 128-byte swizzle
// layout (rows of 128 bytes, groups of 8 rows 1024 bytes apart).
__device__ __forceinline__ uint64_t sw128_kmajor_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4)  // start address
         | ((uint64_t)1 << 16)               // leading-dimension offset (unused by this layout)
         | ((uint64_t)(1024 >> 4) << 32)     // stride between 8-row groups
         | ((uint64_t)1 << 46)               // descriptor version of this architecture
         | ((uint64_t)2 << 61);              // 128-byte swizzle
}

// Instruction descriptor: kind::f16 with bfloat16 A and B, FP32 accumulator,
// both operands K-major, M = 128, N = n.
__device__ __forceinline__ uint32_t idesc_bf16_f32(int n) {
  return (1u << 4)                        // accumulator FP32
         | (1u << 7)                      // A bfloat16
         | (1u << 10)                     // B bfloat16
         | ((uint32_t)(n >> 3) << 17)     // N / 8
         | ((uint32_t)(BM >> 4) << 24);   // M / 16
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrive on `bar` once every tcgen05.mma this thread issued so far has completed.
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's accumulator row.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__global__ void __launch_bounds__(THREADS, 2)
    gemm_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b, Args g) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // 1024-byte-aligned ring (the swizzle pattern is a function of the address)
  const uint32_t raw = smem_addr(smem_raw);
  const uint32_t ring = (raw + 1023u) & ~1023u;
  const uint32_t a_ring = ring, b_ring = ring + STAGES * A_STAGE;
  const uint32_t full0 = ring + STAGES * (A_STAGE + B_STAGE);
  const uint32_t empty0 = full0 + 8 * STAGES, done = full0 + 16 * STAGES;

  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * g.n_tile;
  const int kb_total = (g.K + BK - 1) / BK;
  const int kb0 = blockIdx.z * g.kb_per_split;
  const int kb1 = min(kb_total, kb0 + g.kb_per_split);
  const int nkb = kb1 - kb0;  // >= 1: the host sizes the split so

  if (tid == 0) {
    s_abort = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  volatile int* abort_flag = &s_abort;

  if (warp == 0 && lane == 0) {
    // ---- producer
    const uint32_t stage_bytes = (uint32_t)(A_STAGE + g.n_tile * BK * 2);
    int issued = 0;
    for (int i = 0; i < nkb; ++i) {
      const int s = i % STAGES;
      if (i >= STAGES && !mbar_wait(empty0 + 8 * s, (uint32_t)((i / STAGES) - 1) & 1u, abort_flag)) {
        *abort_flag = 1;
        break;
      }
      mbar_expect_tx(full0 + 8 * s, stage_bytes);
      if (!(i == 0 && g.withhold_first_load)) {
        tma_load_2d(a_ring + s * A_STAGE, &map_a, (kb0 + i) * BK, m0, full0 + 8 * s);
        tma_load_2d(b_ring + s * B_STAGE, &map_b, (kb0 + i) * BK, n0, full0 + 8 * s);
      }
      issued = i + 1;
    }
    // no copy may still be landing when the CTA exits: wait (bounded) for
    // every stage's last load
    for (int i = issued > STAGES ? issued - STAGES : 0; i < issued; ++i) {
      if (i == 0 && g.withhold_first_load) continue;  // nothing in flight
      if (!mbar_wait(full0 + 8 * (i % STAGES), (uint32_t)(i / STAGES) & 1u, nullptr)) *abort_flag = 1;
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    const uint32_t idesc = idesc_bf16_f32(g.n_tile);
    for (int i = 0; i < nkb; ++i) {
      const int s = i % STAGES;
      if (!mbar_wait(full0 + 8 * s, (uint32_t)(i / STAGES) & 1u, abort_flag)) {
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      const uint32_t a = a_ring + s * A_STAGE, b = b_ring + s * B_STAGE;
#pragma unroll
      for (int k = 0; k < BK / 16; ++k)  // 16 bfloat16 = 32 bytes along the swizzled row
        umma_bf16(tmem, sw128_kmajor_desc(a + 32 * k), sw128_kmajor_desc(b + 32 * k), idesc,
                  (i | k) != 0 ? 1u : 0u);
      umma_commit(empty0 + 8 * s);
    }
    umma_commit(done);  // after the last MMA (at once if none was issued)
  }
  __syncwarp();
  __syncthreads();

  // ---- epilogue: accumulator -> registers (bias, ReLU) -> FP32 tile staged
  // in the idle ring -> coalesced stores (mask, FP32 / bfloat16 / transposed)
  bool ok = mbar_wait(done, 0u, nullptr);
  tc_fence_after();
  ok = __syncthreads_and(ok && !*abort_flag) != 0;
  if (!ok && tid == 0) atomicAdd(&g_umma_timeouts, 1u);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  float* stile = reinterpret_cast<float*>(smem_raw + (ring - raw));
  const uint32_t t_row = tmem + ((uint32_t)(warp * 32) << 16);
  const bool use_mask = g.mask && ok;
  float* c32 = g.C32 ? g.C32 + (int64_t)blockIdx.z * g.split_stride : nullptr;
  const int n_valid = min(g.n_tile, g.N - n0);
  // 16-byte vector access where pitch and base allow (column offsets are multiples of 8)
  const bool vec_c16 = g.C16 && g.ldc16 % 8 == 0 && ((uintptr_t)g.C16) % 16 == 0;
  const bool vec_c32 = c32 && g.ldc32 % 4 == 0 && ((uintptr_t)c32) % 16 == 0;
  const bool vec_mask = g.mask && g.ldm % 8 == 0 && ((uintptr_t)g.mask) % 16 == 0;
  for (int h0 = 0; h0 < n_valid; h0 += EPI_COLS) {
    const int hw = min(EPI_COLS, g.n_tile - h0);  // a multiple of 16
    const int sp = hw + 4;                         // staged row pitch (floats): conflict-free float4 rows
    for (int c0 = 0; c0 < hw; c0 += 16) {
      float v[16];
      if (ok) {
        tmem_ld16(t_row + (uint32_t)(h0 + c0), v);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = n0 + h0 + c0 + j;
          if (g.bias && n < g.N) v[j] += g.bias[n];
          if (g.relu) v[j] = fmaxf(v[j], 0.0f);
        }
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = __int_as_float(0x7fc00000);  // NaN marks a tile that gave up
      }
      float4* dst = reinterpret_cast<float4*>(stile + tid * sp + c0);
#pragma unroll
      for (int q = 0; q < 4; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
    __syncthreads();
    const int cols = min(hw, n_valid - h0);
    if (c32 || g.C16) {
      // 8 columns per lane, 16 lanes per row (EPI_COLS = 128): two rows per
      // warp and eight per CTA at a time, 16-byte stores where aligned
      const int r_sub = lane >> 4, c = (lane & 15) * 8;
      const int cnt = min(8, cols - c);
      if (cnt > 0) {
        for (int r = warp * 2 + r_sub; r < BM; r += THREADS / 16) {
          const int m = m0 + r;
          if (m >= g.M) break;
          const float4* src = reinterpret_cast<const float4*>(stile + r * sp + c);
          const float4 lo = src[0], hi = src[1];
          float x[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
          const int n = n0 + h0 + c;
          if (use_mask) {
            const bf16* mk = g.mask + (int64_t)m * g.ldm + n;
            if (cnt == 8 && vec_mask) {
              const uint4 u = *reinterpret_cast<const uint4*>(mk);
              const bf16* hv = reinterpret_cast<const bf16*>(&u);
#pragma unroll
              for (int j = 0; j < 8; ++j)
                if (!(__bfloat162float(hv[j]) > 0.0f)) x[j] = 0.0f;
            } else {
              for (int j = 0; j < cnt; ++j)
                if (!(__bfloat162float(mk[j]) > 0.0f)) x[j] = 0.0f;
            }
          }
          if (c32) {
            float* d = c32 + (int64_t)m * g.ldc32 + n;
            if (cnt == 8 && vec_c32) {
              reinterpret_cast<float4*>(d)[0] = make_float4(x[0], x[1], x[2], x[3]);
              reinterpret_cast<float4*>(d)[1] = make_float4(x[4], x[5], x[6], x[7]);
            } else {
              for (int j = 0; j < cnt; ++j) d[j] = x[j];
            }
          }
          if (g.C16) {
            bf16* d = g.C16 + (int64_t)m * g.ldc16 + n;
            if (cnt == 8 && vec_c16) {
              uint4 u;
              __nv_bfloat162* hv = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
              for (int j = 0; j < 4; ++j) hv[j] = __floats2bfloat162_rn(x[2 * j], x[2 * j + 1]);
              *reinterpret_cast<uint4*>(d) = u;
            } else {
              for (int j = 0; j < cnt; ++j) d[j] = __float2bfloat16_rn(x[j]);
            }
          }
        }
      }
    }
    if (g.C16T) {
      for (int c = warp; c < cols; c += THREADS / 32) {  // one column per warp, lanes down it
        const int n = n0 + h0 + c;
#pragma unroll
        for (int r = lane; r < BM; r += 32) {
          const int m = m0 + r;
          if (m >= g.M) break;
          float x = stile[r * sp + c];
          if (use_mask && !(__bfloat162float(g.mask[(int64_t)m * g.ldm + n]) > 0.0f)) x = 0.0f;
          g.C16T[(int64_t)n * g.ldt + m] = __float2bfloat16_rn(x);
        }
      }
    }
    __syncthreads();  // the staged half is consumed before the next overwrites it
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

}  // namespace umma
