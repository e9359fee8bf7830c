// Device helpers for the S_N kernels: mbarrier and TMA wrappers (inline PTX for
// sm_103a), bounded waits, storage conversions, warp/block reductions and the
// deterministic QoI finalize that closes every stage launch.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#include "rt_internal.h"

namespace rtk {

// ------------------------------------------------------------------ storage
template <typename T> struct Store;
template <> struct Store<float> {
  static __device__ __forceinline__ float load(const float* p) { return *p; }
  static __device__ __forceinline__ float from_smem(const float v) { return v; }
  static __device__ __forceinline__ float round(float v) { return v; }
  static __device__ __forceinline__ float round_sr(float v, uint32_t) { return v; }
  static __device__ __forceinline__ float2 round_sr2(float2 v, uint32_t) { return v; }
  static __device__ __forceinline__ void store(float* p, float v) { *p = v; }
};
template <> struct Store<__nv_bfloat16> {
  static __device__ __forceinline__ float load(const __nv_bfloat16* p) { return __bfloat162float(*p); }
  static __device__ __forceinline__ float from_smem(const __nv_bfloat16 v) { return __bfloat162float(v); }
  // round-to-nearest-even to bf16 and back
  static __device__ __forceinline__ float round(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
  // stochastic rounding to bf16 and back, with 16 random bits r: the magnitude
  // is rounded up with probability (dropped low 16 bits) / 2^16, so the stored
  // value is unbiased; exactly representable values are kept
  static __device__ __forceinline__ float round_sr(float v, uint32_t r) {
    return __uint_as_float((__float_as_uint(v) + (r & 0xffffu)) & 0xffff0000u);
  }
  // the pair (a, b) with the 32 random bits r: low half for a, high half for b
  static __device__ __forceinline__ float2 round_sr2(float2 v, uint32_t r) {
    return make_float2(__uint_as_float((__float_as_uint(v.x) + (r & 0xffffu)) & 0xffff0000u),
                       __uint_as_float((__float_as_uint(v.y) + (r >> 16)) & 0xffff0000u));
  }
  static __device__ __forceinline__ void store(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
};

// ------------------------------------------------------------------ random bits for BF16 stores
// BF16 keeps 8 significant bits. Rounding every stored state to nearest drops
// any per-step change smaller than half a unit in the last place; with small
// time steps (a triangle mesh takes dt from its smallest cells, so most cells
// change by a small fraction per step) the state then stops moving where it
// varies slowly and particles are lost. The stage kernels therefore round BF16
// stores stochastically (Store::round_sr) with 16 random bits per element.
// The bits are a counter-based hash of (cell, ordinate, step, stage), so a run
// is reproducible, independent of the launch configuration (tiles, ordinates
// per lane, batching), and different from step to step:
//   salt  = mix(4 step + stage + c)                  once per launch
//   gkey  = g * K1 ^ salt                             per group g = k / 4 of
//                                                     four ordinates
//   h     = mix(cell * K2 + gkey)                     per cell and group
//   h2    = xorshift-multiply of h
// ordinate 4g + e takes the low (e even) or high (e odd) half of h (e < 2) or
// h2 (e >= 2). mix is Wellons' "lowbias32" 32-bit integer mixer; K1, K2 odd
// constants (cell * K2 is a bijection of the 32-bit cell index, so no index
// wraps: cells are below 2^31). One mixer call serves four elements.
__device__ __forceinline__ uint32_t sr_mix(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}
// salt of one stage launch: step counter and stage (Euler, Heun 1, Heun 2)
__device__ __forceinline__ uint32_t sr_salt(int64_t step, int stage) {
  return sr_mix((uint32_t)step * 4u + (uint32_t)stage + 0x2545f491u);
}
// key of the ordinate group g (ordinates 4g .. 4g+3) in one launch
__device__ __forceinline__ uint32_t sr_gkey(int g, uint32_t salt) { return ((uint32_t)g * 0x85ebca77u) ^ salt; }
// 64 random bits of the group's four elements in one cell: .x for ordinates
// 4g, 4g+1 (low, high half), .y for 4g+2, 4g+3
__device__ __forceinline__ uint2 sr_bits4(uint32_t cell, uint32_t gkey) {
  const uint32_t h = sr_mix(cell * 0x9e3779b1u + gkey);
  uint32_t h2 = (h ^ (h >> 15)) * 0x2c1b3c6du;
  h2 ^= h2 >> 13;
  return make_uint2(h, h2);
}
// the 32 random bits of the pair (4g + 2p, 4g + 2p + 1), p = 0 or 1
__device__ __forceinline__ uint32_t sr_pair(uint2 b, int p) { return p ? b.y : b.x; }
// the 16 random bits (low half) of ordinate 4g + e
__device__ __forceinline__ uint32_t sr_elem(uint2 b, int e) {
  const uint32_t w = (e & 2) ? b.y : b.x;
  return (e & 1) ? (w >> 16) : w;
}

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make the initialised barriers visible to the async (TMA) proxy.
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Order this thread's earlier generic-proxy shared-memory accesses (and those
// made visible to it by a barrier) before later async-proxy (TMA) writes.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of `bar` to complete, for at most `limit` SM clock
// cycles. Returns false if the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int64_t limit) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (clock64() - t0 > limit) return false;
  }
}

// 3-D tiled TMA load of one box into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                            int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

// The tensor maps live in global memory (written before the launch); make
// them visible to the tensormap proxy before the first TMA use.
__device__ __forceinline__ void fence_tensormap_acquire(const CUtensorMap* map) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(map))
               : "memory");
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ------------------------------------------------------------------ math
// minmod(a, b): 0 unless a and b have the same sign, else the one of smaller magnitude.
__device__ __forceinline__ float minmod(float a, float b) {
  const float m = fminf(fabsf(a), fabsf(b));
  return (a * b > 0.f) ? copysignf(m, a) : 0.f;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum V per-lane values over the 32 lanes of a warp with log2(V) + 5 - log2(V)
// butterfly steps; afterwards lane l holds the total of value index
// (l >> (5 - log2 V)). Fixed order: deterministic.
template <int V>
__device__ __forceinline__ float multi_warp_sum(float (&v)[V], int lane) {
  static_assert(V == 1 || V == 2 || V == 4 || V == 8, "V must be 1, 2, 4 or 8");
  if constexpr (V == 1) {
    return warp_sum(v[0]);
  } else {
    // step with offset 16: keep half of the values, send the other half
    constexpr int H = V / 2;
    float a[H];
    const bool hi = (lane & 16) != 0;
#pragma unroll
    for (int i = 0; i < H; ++i) {
      const float keep = hi ? v[H + i] : v[i];
      const float send = hi ? v[i] : v[H + i];
      a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    if constexpr (H == 1) {
      float s = a[0];
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      return s;
    } else {
      constexpr int Q = H / 2;
      float b[Q];
      const bool hi8 = (lane & 8) != 0;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const float keep = hi8 ? a[Q + i] : a[i];
        const float send = hi8 ? a[i] : a[Q + i];
        b[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
      }
      if constexpr (Q == 1) {
        float s = b[0];
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        return s;
      } else {
        const bool hi4 = (lane & 4) != 0;
        float s = (hi4 ? b[1] : b[0]) + __shfl_xor_sync(0xffffffffu, hi4 ? b[0] : b[1], 4);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        return s;
      }
    }
  }
}

// Lane that holds the total of value index u after multi_warp_sum<V>.
template <int V>
__device__ __forceinline__ constexpr int multi_sum_lane(int u) {
  return u * (32 / V);
}

// ------------------------------------------------------------------ QoI finalize
// Block-wide FP64 reduction of `acc` (nq values per thread, nq <= NQ) into
// red[0..nq) in shared memory, in a fixed order. Must be called by all threads.
template <int NT>
__device__ __forceinline__ void block_reduce_q(const double (&acc)[NQ], int nq, double* red /*[NT/32][NQ]*/) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    if (q < nq) {
      const double s = warp_sum_d(acc[q]);
      if (lane == 0) red[warp * NQ + q] = s;
    }
  }
  __syncthreads();
  if (threadIdx.x < nq) {
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += red[w * NQ + threadIdx.x];
    red[threadIdx.x] = s;    // row 0 reused for the result (read above by this thread only)
  }
  __syncthreads();
}

// Write this work item's QoI partial (red[0..nq)), and if it is the last item of
// its instance in this launch, reduce all partials in item order and apply the
// time-integration update of `stage`. Must be called by all threads.
template <int NT>
__device__ void finalize_item(const InstDesc& d, const WorkItem& it, const double* red, int stage,
                              double* scratch /*[NT/32][NQ]*/) {
  __shared__ uint32_t s_last;
  const int nq = d.n_regions + 2;
  if (threadIdx.x < NQ) d.partials[(size_t)it.item * NQ + threadIdx.x] = (threadIdx.x < nq) ? red[threadIdx.x] : 0.0;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t t = atomicAdd(&d.st->ticket, 1u);
    s_last = (t == static_cast<uint32_t>(it.count - 1)) ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // fixed-order reduction over the count partial rows
  double acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
  for (int i = threadIdx.x; i < it.count; i += NT) {
    const double* row = d.partials + (size_t)i * NQ;
#pragma unroll
    for (int q = 0; q < NQ; ++q)
      if (q < nq) acc[q] += __ldcg(row + q);
  }
  block_reduce_q<NT>(acc, nq, scratch);
  if (threadIdx.x == 0) {
    InstState* st = d.st;
    double S[NQ];
    // map compact order (regions..., mass, outflow) to the NQ layout
#pragma unroll
    for (int q = 0; q < NQ; ++q) S[q] = 0.0;
    for (int r = 0; r < d.n_regions; ++r) S[r] = scratch[r];
    S[kQMass] = scratch[d.n_regions];
    S[kQOut] = scratch[d.n_regions + 1];
    const double dt = d.dt_d;
    if (stage == STAGE_EULER) {
      for (int q = 0; q < NQ; ++q) st->I[q] += dt * st->S_cur[q];
      for (int q = 0; q < NQ; ++q) st->S_cur[q] = S[q];
      st->step += 1;
      st->parity ^= 1;
    } else if (stage == STAGE_HEUN1) {
      for (int q = 0; q < NQ; ++q) st->I[q] += 0.5 * dt * st->S_cur[q];
      for (int q = 0; q < NQ; ++q) st->S_mid[q] = S[q];
    } else if (stage == STAGE_HEUN2) {
      for (int q = 0; q < NQ; ++q) st->I[q] += 0.5 * dt * st->S_mid[q];
      for (int q = 0; q < NQ; ++q) st->S_cur[q] = S[q];
      st->step += 1;
    } else {  // STAGE_INIT
      for (int q = 0; q < NQ; ++q) st->S_cur[q] = S[q];
    }
    bool finite = isfinite(S[kQMass]) && isfinite(S[kQOut]);
    for (int r = 0; r < d.n_regions; ++r) finite = finite && isfinite(S[r]);
    if (!finite && st->status == DEV_OK) st->status = DEV_NONFINITE;
    st->ticket = 0u;
    __threadfence();
  }
}

}  // namespace rtk
