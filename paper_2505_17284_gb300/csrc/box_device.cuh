// Outflow through the boundaries of axis-aligned QoI boxes (the lattice's
// QoI-1 and QoI-2 of Sec. 3.1, through the squares S_l): for a face f of the
// boundary of box b, with n_f the normal pointing out of the box and l_f its
// length, the box loses l_f sum_k w_k max(omega_k . n_f, 0) psi_hat_k,f, where
// psi_hat is the scheme's upwind trace (Sec. 4.2): for an ordinate leaving the
// box the upwind cell is the inside one, so the trace is its value at first
// order and its MUSCL-minmod reconstruction toward the face at second order.
//
// Face records {inside cell, outside cell, the inside cell's other neighbour
// along the normal, box | side << 8} come from the host; every cell named
// there lies inside the domain.
#pragma once
#include "device_common.cuh"

namespace rtk {

// Four consecutive stored values (16-byte aligned for FP32, 8-byte for BF16) as floats.
template <typename T> __device__ __forceinline__ void box_load4(const T* p, float (&v)[4]);
template <> __device__ __forceinline__ void box_load4<float>(const float* p, float (&v)[4]) {
  const float4 x = *reinterpret_cast<const float4*>(p);
  v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
}
template <> __device__ __forceinline__ void box_load4<__nv_bfloat16>(const __nv_bfloat16* p, float (&v)[4]) {
  const uint2 x = *reinterpret_cast<const uint2*>(p);
  v[0] = __uint_as_float(x.x << 16); v[1] = __uint_as_float(x.x & 0xffff0000u);
  v[2] = __uint_as_float(x.y << 16); v[3] = __uint_as_float(x.y & 0xffff0000u);
}

// Outflow of faces it.a .. it.a+it.b-1 for the state psi ([cell][Mpad]), summed
// per box into out[0..kMaxBox) in FP64 (identical in every thread on return).
// One face per warp at a time; each lane takes 4 consecutive ordinates per pass
// and loads a cell only for ordinates that leave the box. red: shared scratch
// of NT/32 * kMaxBox doubles. Must be called by all NT threads.
template <int NT, typename T>
__device__ __forceinline__ void box_face_sums(const InstDesc& d, const WorkItem& it, const T* __restrict__ psi,
                                              double* red, double (&out)[kMaxBox]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int Mpad = d.Mpad;
  const bool second = d.order == 2;
  const float lx = (float)d.dx_d, ly = (float)d.dy_d;
  double acc[kMaxBox];
#pragma unroll
  for (int b = 0; b < kMaxBox; ++b) acc[b] = 0.0;
  for (int f = it.a + warp; f < it.a + it.b; f += NT / 32) {
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
        float c[4], o[4] = {0.f, 0.f, 0.f, 0.f}, g[4] = {0.f, 0.f, 0.f, 0.f};
        box_load4<T>(pin + k0, c);
        if (second) {
          box_load4<T>(pout + k0, o);
          box_load4<T>(pfar + k0, g);
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
  // every lane of a warp holds the warp's sums; combine the warps in order
  if (lane == 0) {
#pragma unroll
    for (int b = 0; b < kMaxBox; ++b) red[warp * kMaxBox + b] = acc[b];
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < kMaxBox; ++b) {
    double v = 0.0;
    for (int w = 0; w < NT / 32; ++w) v += red[w * kMaxBox + b];
    out[b] = v;
  }
  __syncthreads();
}

}  // namespace rtk
