// Outflow through the boundaries of axis-aligned QoI boxes (the lattice's
// QoI-1 and QoI-2 of Sec. 3.1, through the squares S_l): for a face f of the
// boundary of box b, with n_f the normal pointing out of the box and l_f its
// length, the box gains l_f sum_k w_k max(omega_k . n_f, 0) psi_hat_k,f, where
// psi_hat is the scheme's upwind trace (Sec. 4.2): for an ordinate leaving the
// box the upwind cell is the inside one, so the trace is its value at first
// order and its MUSCL-minmod reconstruction toward the face at second order.
//
// The kernel runs after every stage on the state that stage wrote (and once on
// the initial state), reads three cells per face (inside, outside, and the
// inside cell's other neighbour along the normal), and closes with the same
// time-integration update as the other QoIs: Euler adds dt S(psi^n), Heun
// dt/2 (S(psi^n) + S(psi^(1))). Partial sums are FP64 per work item, reduced
// by the last item of the instance in item order (deterministic).
#include "device_common.cuh"

namespace rtk {

namespace {

constexpr int kBoxThreads = 256;

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

template <typename T>
__global__ void __launch_bounds__(kBoxThreads, 4)
    box_outflow_kernel(const InstDesc* __restrict__ descs, const WorkItem* __restrict__ items, int stage) {
  const WorkItem it = items[blockIdx.x];
  const InstDesc& d = descs[it.inst];
  InstState* st = d.st;
  // skip when the stage before was masked (a finished or failed instance of a
  // batch): Heun stage 1 ran iff the stage kernel's own test passes (it does
  // not change the step); Euler and Heun stage 2 ran iff the step advanced
  if (stage == STAGE_HEUN1) {
    if (st->step >= d.n_steps || st->status != DEV_OK) return;
  } else if (stage != STAGE_INIT) {
    if (st->step == st->box_step) return;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // the stage's output: Heun stage 1 writes buffer 1; every other stage leaves the
  // current state in the buffer named by the parity (Heun keeps it at 0)
  const int buf = (stage == STAGE_HEUN1) ? 1 : st->parity;
  const T* __restrict__ psi = reinterpret_cast<const T*>(d.psi[buf]);
  const int Mpad = d.Mpad;
  const bool second = d.order == 2;
  const float lx = (float)d.dx_d, ly = (float)d.dy_d;

  double acc[kMaxBox];
#pragma unroll
  for (int b = 0; b < kMaxBox; ++b) acc[b] = 0.0;
  // one face per warp at a time; each lane takes 4 consecutive ordinates per
  // pass (one 16-byte load for FP32, 8 bytes for BF16), and loads a cell only
  // for ordinates that leave the box
  for (int f = it.a + warp; f < it.a + it.b; f += kBoxThreads / 32) {
    const int4 fc = d.box_faces[f];
    const int box = fc.w & 0xff, side = fc.w >> 8;
    const T* pin = psi + (size_t)fc.x * Mpad;
    const T* pout = psi + (size_t)fc.y * Mpad;
    const T* pfar = psi + (size_t)fc.z * Mpad;
    const float* dir = (side < 2) ? d.xi : d.eta;
    const float sgn = (side & 1) ? 1.f : -1.f;
    float s = 0.f;
#pragma unroll 4
    for (int k0 = 4 * lane; k0 < Mpad; k0 += 128) {
      const float4 dv = *reinterpret_cast<const float4*>(dir + k0);
      const float4 wv = *reinterpret_cast<const float4*>(d.w + k0);
      const float on[4] = {sgn * dv.x, sgn * dv.y, sgn * dv.z, sgn * dv.w};   // omega_k . n_f
      const float wk[4] = {wv.x, wv.y, wv.z, wv.w};
      if (on[0] > 0.f || on[1] > 0.f || on[2] > 0.f || on[3] > 0.f) {
        float c[4], o[4], g[4];
        load4<T>(pin + k0, c);
        if (second) {
          load4<T>(pout + k0, o);
          load4<T>(pfar + k0, g);
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          float tr = c[v];
          if (second) {
            // slope toward the face: minmod(outside - inside, inside - far)
            const float a = o[v] - c[v], bb = c[v] - g[v];
            const float mm = (a * bb > 0.f) ? (fabsf(a) < fabsf(bb) ? a : bb) : 0.f;
            tr = fmaf(0.5f, mm, c[v]);
          }
          s = fmaf(on[v] > 0.f ? wk[v] * on[v] : 0.f, tr, s);
        }
      }
    }
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
    const double face = (double)s * (double)((side < 2) ? ly : lx);
#pragma unroll
    for (int b = 0; b < kMaxBox; ++b)
      if (b == box) acc[b] += face;
  }

  // block reduction in a fixed order
  __shared__ double red[kBoxThreads / 32][kMaxBox];
  __shared__ double tot[kMaxBox];
  __shared__ uint32_t s_last;
  // (every lane of a warp holds the warp's sums after the shuffles)
  if (lane == 0) {
#pragma unroll
    for (int b = 0; b < kMaxBox; ++b) red[warp][b] = acc[b];
  }
  __syncthreads();
  if (threadIdx.x < kMaxBox) {
    double v = 0.0;
    for (int w = 0; w < kBoxThreads / 32; ++w) v += red[w][threadIdx.x];
    d.box_partials[(size_t)it.item * kMaxBox + threadIdx.x] = v;
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
#pragma unroll
  for (int b = 0; b < kMaxBox; ++b) acc[b] = 0.0;
  for (int i = threadIdx.x; i < it.count; i += kBoxThreads) {
#pragma unroll
    for (int b = 0; b < kMaxBox; ++b) acc[b] += __ldcg(d.box_partials + (size_t)i * kMaxBox + b);
  }
#pragma unroll
  for (int b = 0; b < kMaxBox; ++b) {
    const double v = warp_sum_d(acc[b]);
    if (lane == 0) red[warp][b] = v;
  }
  __syncthreads();
  if (threadIdx.x < kMaxBox) {
    double v = 0.0;
    for (int w = 0; w < kBoxThreads / 32; ++w) v += red[w][threadIdx.x];
    tot[threadIdx.x] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double dt = d.dt_d;
    for (int b = 0; b < kMaxBox; ++b) {
      const double S = (b < d.n_boxes) ? tot[b] : 0.0;
      if (stage == STAGE_EULER) {
        st->B_I[b] += dt * st->B_cur[b];
        st->B_cur[b] = S;
      } else if (stage == STAGE_HEUN1) {
        st->B_I[b] += 0.5 * dt * st->B_cur[b];
        st->B_mid[b] = S;
      } else if (stage == STAGE_HEUN2) {
        st->B_I[b] += 0.5 * dt * st->B_mid[b];
        st->B_cur[b] = S;
      } else {  // STAGE_INIT
        st->B_cur[b] = S;
      }
    }
    if (stage != STAGE_HEUN1) st->box_step = st->step;
    st->box_ticket = 0u;
    __threadfence();
  }
}

}  // namespace

cudaError_t launch_box_outflow(const InstDesc* d_desc, const WorkItem* d_items, int n_items, int stage,
                               int storage, cudaStream_t stream) {
  if (n_items <= 0) return cudaSuccess;
  if (storage == 1)
    box_outflow_kernel<__nv_bfloat16><<<n_items, kBoxThreads, 0, stream>>>(d_desc, d_items, stage);
  else
    box_outflow_kernel<float><<<n_items, kBoxThreads, 0, stream>>>(d_desc, d_items, stage);
  return cudaGetLastError();
}

}  // namespace rtk
