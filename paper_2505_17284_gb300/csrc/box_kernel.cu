// Outflow through the boundaries of axis-aligned QoI boxes (the lattice's
// QoI-1 and QoI-2 of Sec. 3.1, through the squares S_l): for a face f of the
// boundary of box b, with n_f the normal pointing out of the box and l_f its
// length, the box loses l_f sum_k w_k max(omega_k . n_f, 0) psi_hat_k,f, where
// psi_hat is the scheme's upwind trace (Sec. 4.2): for an ordinate leaving the
// box the upwind cell is the inside one, so the trace is its value at first
// order and its MUSCL-minmod reconstruction toward the face at second order.
//
// One launch per time step, after the step's last stage (and one on the
// initial state). It reads three cells per face (inside, outside, and the
// inside cell's other neighbour along the normal), only in the blocks of
// ordinates that hold leaving ones, and applies the time
// integration with the scheme's weights: Euler adds dt S(psi^n); Heun adds
// dt/2 (S(psi^n) + S(psi^(1))), and since stage 2 leaves psi^(1) in buffer 1
// next to psi^(n+1) in buffer 0, the Heun launch evaluates both states.
// S(psi^n) is carried from the previous launch. Partial sums are FP64 per
// work item, reduced by the last item of the instance in item order
// (deterministic).
#include "device_common.cuh"

namespace rtk {

namespace {

constexpr int kBoxThreads = 256;
constexpr int kBoxTasksPerWarp = kBoxTasksPerItem / (kBoxThreads / 32);
static_assert(kBoxTasksPerWarp * (kBoxThreads / 32) == kBoxTasksPerItem && kBoxTasksPerWarp % 2 == 0,
              "whole pairs of tasks per warp");

// Four consecutive stored values (16-byte aligned for FP32, 8-byte for BF16) as floats.
template <typename T> __device__ __forceinline__ void load4(const T* p, float (&v)[4]);
template <> __device__ __forceinline__ void load4<float>(const float* p, float (&v)[4]) {
  const float4 x = *reinterpret_cast<const float4*>(p);
  v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
}
template <> __device__ __forceinline__ void load4<__nv_bfloat16>(const __nv_bfloat16* p, float (&v)[4]) {
  const uint2 x = *reinterpret_cast<const uint2*>(p);
  v[0] = __uint_as_float(x.x << 16); v[1] = __uint_as_float(x.x & 0xffff0000u);
  v[2] = __uint_as_float(x.y << 16); v[3] = __uint_as_float(x.y & 0xffff0000u);
}

// stage: STAGE_EULER or STAGE_INIT (the current state, buffer `parity`) or
// STAGE_HEUN2 (after a Heun step: psi^(1) in buffer 1, psi^(n+1) in buffer 0).
// A task is one face and one block of 128 ordinates holding at least one
// ordinate that leaves through it: record {inside cell, outside cell, the
// inside cell's other neighbour along the normal, box | side << 8 | block << 12}.
// Lane l takes ordinates 128 block + 4 l .. +3; a warp runs its tasks two at a
// time with every load of the pair in flight, and keeps FP32 sums per state
// and box in each lane until the end.
template <typename T>
__global__ void __launch_bounds__(kBoxThreads, 2)
    box_outflow_kernel(const InstDesc* __restrict__ descs, const WorkItem* __restrict__ items, int stage) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const WorkItem it = items[blockIdx.x];
  const InstDesc& d = descs[it.inst];
  InstState* st = d.st;
  // Prologue, independent of the stage before: the warp's task records (lane j
  // holds task j). With a programmatic launch it overlaps the end of that
  // stage; griddepcontrol.wait then waits for the stage grid to complete and
  // its writes to be visible (without a programmatic dependency it returns at once).
  int4 rec = make_int4(0, 0, 0, -1);
  if (lane < kBoxTasksPerWarp) {
    const int t = it.a + warp + lane * (kBoxThreads / 32);
    if (t < it.a + it.b) rec = d.box_tasks[t];
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");
  // skip when the step before was masked (a finished or failed instance of a
  // batch): it ran iff the step counter advanced since the last update
  if (stage != STAGE_INIT && st->step == st->box_step) return;
  const bool heun = stage == STAGE_HEUN2;
  const T* psiA = reinterpret_cast<const T*>(d.psi[heun ? 1 : st->parity]);   // state 0
  const T* psiB = reinterpret_cast<const T*>(d.psi[0]);                        // state 1 (Heun)
  const int Mpad = d.Mpad;
  const bool second = d.order == 2;
  const float lx = (float)d.dx_d, ly = (float)d.dy_d;

  float acc[2][kMaxBox];
#pragma unroll
  for (int e = 0; e < 2; ++e)
#pragma unroll
    for (int b = 0; b < kMaxBox; ++b) acc[e][b] = 0.f;
#pragma unroll
  for (int r = 0; r < kBoxTasksPerWarp; r += 2) {
    int4 tk[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      tk[j].x = __shfl_sync(0xffffffffu, rec.x, r + j);
      tk[j].y = __shfl_sync(0xffffffffu, rec.y, r + j);
      tk[j].z = __shfl_sync(0xffffffffu, rec.z, r + j);
      tk[j].w = __shfl_sync(0xffffffffu, rec.w, r + j);
    }
    float on[2][4], wl[2][4], c[2][2][4], o[2][2][4], g[2][2][4];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int side = (tk[j].w >> 8) & 3;
      const int k = ((tk[j].w >> 12) << 7) + 4 * lane;
      // a task slot past the item's end, or (M_pad not a multiple of 128) a lane
      // past the last ordinate, reads nothing
      const bool live = tk[j].w >= 0 && k < Mpad;
      const float* dir = (side < 2) ? d.xi : d.eta;
      const float sg = (side & 1) ? 1.f : -1.f;
      const float l = (side < 2) ? ly : lx;
      float4 dv = make_float4(0.f, 0.f, 0.f, 0.f), wv = dv;
      if (live) {
        dv = *reinterpret_cast<const float4*>(dir + k);
        wv = *reinterpret_cast<const float4*>(d.w + k);
      }
      const float dd[4] = {dv.x, dv.y, dv.z, dv.w}, ww[4] = {wv.x, wv.y, wv.z, wv.w};
      bool any = false;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        on[j][v] = sg * dd[v];                       // omega_k . n_f
        wl[j][v] = on[j][v] > 0.f ? l * ww[v] * on[j][v] : 0.f;
        any = any || on[j][v] > 0.f;
      }
#pragma unroll
      for (int e = 0; e < 2; ++e)
#pragma unroll
        for (int v = 0; v < 4; ++v) c[j][e][v] = o[j][e][v] = g[j][e][v] = 0.f;
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        if (!any || (e == 1 && !heun)) continue;
        const T* ps = e ? psiB : psiA;
        load4<T>(ps + (size_t)tk[j].x * Mpad + k, c[j][e]);
        if (second) {
          load4<T>(ps + (size_t)tk[j].y * Mpad + k, o[j][e]);
          load4<T>(ps + (size_t)tk[j].z * Mpad + k, g[j][e]);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int box = tk[j].w & 0xff;
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        float sum = 0.f;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          float tr = c[j][e][v];
          if (second) {
            // slope toward the face: minmod(outside - inside, inside - far)
            const float a = o[j][e][v] - c[j][e][v], bb = c[j][e][v] - g[j][e][v];
            const float mm = (a * bb > 0.f) ? (fabsf(a) < fabsf(bb) ? a : bb) : 0.f;
            tr = fmaf(0.5f, mm, c[j][e][v]);
          }
          sum = fmaf(wl[j][v], tr, sum);
        }
#pragma unroll
        for (int b = 0; b < kMaxBox; ++b)
          if (b == box) acc[e][b] += sum;
      }
    }
  }

  // block reduction in a fixed order: lanes (FP64 from here), then warps
  constexpr int NB = 2 * kMaxBox;
  __shared__ double red[kBoxThreads / 32][NB];
  __shared__ double tot[NB];
  __shared__ uint32_t s_last;
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const double v = warp_sum_d((double)acc[q / kMaxBox][q % kMaxBox]);
    if (lane == 0) red[warp][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < NB) {
    double v = 0.0;
    for (int w = 0; w < kBoxThreads / 32; ++w) v += red[w][threadIdx.x];
    d.box_partials[(size_t)it.item * NB + threadIdx.x] = v;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t t = atomicAdd(&st->box_ticket, 1u);
    s_last = (t == static_cast<uint32_t>(it.count - 1)) ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // all threads: item i goes to thread i mod kBoxThreads, then the fixed-order
  // block reduction
  double part[NB];
#pragma unroll
  for (int q = 0; q < NB; ++q) part[q] = 0.0;
  for (int i = threadIdx.x; i < it.count; i += kBoxThreads) {
#pragma unroll
    for (int q = 0; q < NB; ++q) part[q] += __ldcg(d.box_partials + (size_t)i * NB + q);
  }
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const double v = warp_sum_d(part[q]);
    if (lane == 0) red[warp][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < NB) {
    double v = 0.0;
    for (int w = 0; w < kBoxThreads / 32; ++w) v += red[w][threadIdx.x];
    tot[threadIdx.x] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double dt = d.dt_d;
    for (int b = 0; b < kMaxBox; ++b) {
      const bool on = b < d.n_boxes;
      const double S0 = on ? tot[b] : 0.0, S1 = on ? tot[kMaxBox + b] : 0.0;
      if (stage == STAGE_EULER) {
        st->B_I[b] += dt * st->B_cur[b];
        st->B_cur[b] = S0;
      } else if (stage == STAGE_HEUN2) {
        st->B_I[b] += 0.5 * dt * (st->B_cur[b] + S0);
        st->B_cur[b] = S1;
      } else {  // STAGE_INIT
        st->B_cur[b] = S0;
      }
    }
    st->box_step = st->step;
    st->box_ticket = 0u;
    __threadfence();
  }
}

}  // namespace

cudaError_t launch_box_outflow(const InstDesc* d_desc, const WorkItem* d_items, int n_items, int stage,
                               int storage, cudaStream_t stream) {
  if (n_items <= 0) return cudaSuccess;
  // programmatic dependent launch: the CTAs may start (and run the prologue)
  // while the stage before finishes; the kernel waits for it before reading
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)n_items);
  cfg.blockDim = dim3(kBoxThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (storage == 1) return cudaLaunchKernelEx(&cfg, box_outflow_kernel<__nv_bfloat16>, d_desc, d_items, stage);
  return cudaLaunchKernelEx(&cfg, box_outflow_kernel<float>, d_desc, d_items, stage);
}

}  // namespace rtk
