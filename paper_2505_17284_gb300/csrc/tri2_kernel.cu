// Second-order finite volumes on triangle meshes (Sec. 4.2, the paper's own
// scheme): the trace on edge e of cell i is R_i = psi_i + L_i g_i . r_ie at the
// edge midpoint (r_ie = x_e - x_i, x_i the centroid), with the Green-Gauss
// gradient g_i = (1/A_i) sum_e l_e n_e (psi_i + psi_e)/2 and the Venkatakrishnan
// limiter L_i = min_e L_ie (Eq. V_limiter: Delta = (1/2) g_i . r_ie, beta from
// the max / min of psi over the cell and its neighbours, epsilon = A_i^3).
// Boundary edges see the ghost value psi^- (the side's inflow value for
// entering ordinates, 0 otherwise) in the gradient and the max / min, and carry
// first-order fluxes.
//
// Two kernels per stage, both persistent over 64-cell chunks like the
// first-order stage kernel (chunk metadata staged in shared memory by bulk
// copies, one warp per cell, lanes over ordinates; 3 CTAs per SM, so the
// 3-per-SM persistent grid is resident at once):
//   tri_grad_kernel    reads psi of a cell and its three neighbours and writes
//                      the limited gradient L g (two FP32 rows per cell);
//   tri_stage2_kernel  reads psi and L g of a cell and its neighbours, takes
//                      the upwind reconstructed trace on each edge (the
//                      neighbour's R at the shared midpoint, r_je = r_ie - d_ij
//                      with d_ij = x_j - x_i) and writes the stage output, phi
//                      and the FP64 QoI partials as the first-order kernel does.
#include <cuda_bf16.h>

#include "device_common.cuh"

namespace rtk {

namespace {

constexpr int kT2Threads = 256;
constexpr int kT2Warps = kT2Threads / 32;
constexpr int kT2Chunk = 64;
constexpr uint32_t kT2MetaBytes = 16u + 32u + 48u;   // per cell: neighbours, geometry, second-order geometry

template <typename T, int VEC>
struct alignas(sizeof(T) * VEC) Vec2T {
  T v[VEC];
};

template <typename T, int VEC>
__device__ __forceinline__ void ld_vec(const T* p, float (&out)[VEC]) {
  const Vec2T<T, VEC> x = *reinterpret_cast<const Vec2T<T, VEC>*>(p);
#pragma unroll
  for (int l = 0; l < VEC; ++l) out[l] = Store<T>::from_smem(x.v[l]);
}

template <typename T, int VEC>
__device__ __forceinline__ void st_vec(T* p, const float (&in)[VEC]) {
  Vec2T<T, VEC> x;
#pragma unroll
  for (int l = 0; l < VEC; ++l) {
    if constexpr (sizeof(T) == 4) {
      x.v[l] = in[l];
    } else {
      x.v[l] = __float2bfloat16_rn(in[l]);
    }
  }
  *reinterpret_cast<Vec2T<T, VEC>*>(p) = x;
}

__device__ __forceinline__ void t2_bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// psi^- of boundary side s for an ordinate: the side's inflow value if the
// ordinate enters through it (outward normals x- (-1,0), x+ (1,0), y- (0,-1),
// y+ (0,1)), else 0
__device__ __forceinline__ float ghost_value(const InstDesc& d, int s, float xi, float eta) {
  const float on = (s == 0) ? -xi : (s == 1) ? xi : (s == 2) ? -eta : eta;
  return on < 0.f ? d.ghost[s] : 0.f;
}

// Venkatakrishnan value of one edge (Eq. V_limiter with the 1/Delta factor
// cancelled): 1 for Delta = 0 (and for a vanishing denominator)
__device__ __forceinline__ float venkat(float delta, float bmax, float bmin, float eps2) {
  if (delta == 0.f) return 1.f;
  const float b = delta > 0.f ? bmax : bmin;
  const float num = b * b + eps2 + 2.f * delta * b;
  const float den = b * b + 2.f * delta * delta + b * delta + eps2;
  return den > 0.f ? num / den : 1.f;
}

// Chunk metadata in shared memory, double-buffered.
struct T2Meta {
  int4 nbr[2][kT2Chunk];
  float4 geo[2][2 * kT2Chunk];
  float4 geo2[2][3 * kT2Chunk];
  uint64_t bar[2];
};

__device__ __forceinline__ void t2_stage_meta(const InstDesc& d, T2Meta& m, int k, int b, int n_cells) {
  const int c0 = k * kT2Chunk;
  const int cells = min(kT2Chunk, n_cells - c0);
  mbar_arrive_expect_tx(&m.bar[b], (uint32_t)cells * kT2MetaBytes);
  t2_bulk_load(m.nbr[b], d.tri_nbr + c0, (uint32_t)cells * 16u, &m.bar[b]);
  t2_bulk_load(m.geo[b], d.tri_geo + 2 * (size_t)c0, (uint32_t)cells * 32u, &m.bar[b]);
  t2_bulk_load(m.geo2[b], d.tri_geo2 + 3 * (size_t)c0, (uint32_t)cells * 48u, &m.bar[b]);
}

// -------------------------------------------------------------------- gradient
template <int VEC, typename T>
__global__ void __launch_bounds__(kT2Threads, 3)
    tri_grad_kernel(const InstDesc* __restrict__ descs, const WorkItem* __restrict__ items, int stage) {
  __shared__ __align__(16) T2Meta meta;
  const WorkItem it = items[blockIdx.x];
  const InstDesc& d = descs[it.inst];
  InstState* st = d.st;
  if (st->step >= d.n_steps || st->status != DEV_OK) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int in_buf = (stage == STAGE_EULER) ? st->parity : (stage == STAGE_HEUN1 ? 0 : 1);
  const T* __restrict__ psi = reinterpret_cast<const T*>(d.psi[in_buf]);
  float* __restrict__ lg = d.tri_lg;
  const int Mpad = d.Mpad;
  const int nv = Mpad / (32 * VEC);
  const int n_cells = (int)d.n_cells;
  const int n_chunks = (n_cells + kT2Chunk - 1) / kT2Chunk;
  const int G = it.b;
  const int64_t limit = d.wait_limit;
  if (threadIdx.x == 0) {
    mbar_init(&meta.bar[0], 1);
    mbar_init(&meta.bar[1], 1);
    fence_barrier_init();
    if (it.a < n_chunks) t2_stage_meta(d, meta, it.a, 0, n_cells);
    if (it.a + G < n_chunks) t2_stage_meta(d, meta, it.a + G, 1, n_cells);
  }
  __syncthreads();
  bool ok = true;
  int i = 0;
  for (int k = it.a; k < n_chunks; k += G, ++i) {
    const int b = i & 1;
    const bool mok = mbar_wait_bounded(&meta.bar[b], (uint32_t)((i >> 1) & 1), limit);
    if (__syncthreads_or(!mok)) {
      ok = false;
      break;
    }
    const int c0 = k * kT2Chunk;
    const int c_end = min(n_cells, c0 + kT2Chunk);
    for (int cell = c0 + warp; cell < c_end; cell += kT2Warps) {
      const int li = cell - c0;
      const int4 nb = meta.nbr[b][li];
      const float4 g0 = meta.geo[b][2 * li], g1 = meta.geo[b][2 * li + 1];
      const float4 h0 = meta.geo2[b][3 * li], h1 = meta.geo2[b][3 * li + 1];
      const float ax[3] = {g0.x, g0.z, g1.x}, ay[3] = {g0.y, g0.w, g1.y};
      const float rx[3] = {h0.x, h0.z, h1.x}, ry[3] = {h0.y, h0.w, h1.y};
      const float eps2 = g1.w;
      const int nbr[3] = {nb.x, nb.y, nb.z};
      for (int v = 0; v < nv; ++v) {
        const int kk = (v * 32 + lane) * VEC;
        float c[VEC], nv3[3][VEC];
        ld_vec<T, VEC>(psi + (size_t)cell * Mpad + kk, c);
#pragma unroll
        for (int e = 0; e < 3; ++e)
          if (nbr[e] >= 0) ld_vec<T, VEC>(psi + (size_t)nbr[e] * Mpad + kk, nv3[e]);
        float xi[VEC], eta[VEC];
        ld_vec<float, VEC>(d.xi + kk, xi);
        ld_vec<float, VEC>(d.eta + kk, eta);
        float ox[VEC], oy[VEC];
#pragma unroll
        for (int l = 0; l < VEC; ++l) {
          float nbv[3];
#pragma unroll
          for (int e = 0; e < 3; ++e) nbv[e] = (nbr[e] >= 0) ? nv3[e][l] : ghost_value(d, -1 - nbr[e], xi[l], eta[l]);
          float gx = 0.f, gy = 0.f;
#pragma unroll
          for (int e = 0; e < 3; ++e) {
            const float avg = 0.5f * (c[l] + nbv[e]);
            gx = fmaf(ax[e], avg, gx);
            gy = fmaf(ay[e], avg, gy);
          }
          const float pmax = fmaxf(fmaxf(c[l], nbv[0]), fmaxf(nbv[1], nbv[2]));
          const float pmin = fminf(fminf(c[l], nbv[0]), fminf(nbv[1], nbv[2]));
          const float bmax = pmax - c[l], bmin = pmin - c[l];
          float L = INFINITY;
#pragma unroll
          for (int e = 0; e < 3; ++e) L = fminf(L, venkat(0.5f * (gx * rx[e] + gy * ry[e]), bmax, bmin, eps2));
          ox[l] = L * gx;
          oy[l] = L * gy;
        }
        st_vec<float, VEC>(lg + (size_t)cell * 2 * Mpad + kk, ox);
        st_vec<float, VEC>(lg + (size_t)cell * 2 * Mpad + Mpad + kk, oy);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0 && k + 2 * G < n_chunks) t2_stage_meta(d, meta, k + 2 * G, b, n_cells);
  }
  if (!ok && threadIdx.x == 0) {
    for (int j = i; j < i + 2; ++j) {
      const int kj = it.a + j * G;
      if (kj < n_chunks) mbar_wait_bounded(&meta.bar[j & 1], (uint32_t)((j >> 1) & 1), limit);
    }
    atomicCAS(&st->status, DEV_OK, DEV_TIMEOUT);
    st->timeout_where = ((int64_t)blockIdx.x << 32) | (int64_t)i;
  }
}

// -------------------------------------------------------------------- stage
template <int VEC, int STAGE, typename T>
__global__ void __launch_bounds__(kT2Threads, 3)
    tri_stage2_kernel(const InstDesc* __restrict__ descs, const WorkItem* __restrict__ items) {
  __shared__ __align__(16) T2Meta meta;
  __shared__ double red[(kT2Warps + 1) * NQ];
  __shared__ float wacc[kT2Warps][NQ];
  __shared__ double wdacc[kT2Warps][NQ];
  const WorkItem it = items[blockIdx.x];
  const InstDesc& d = descs[it.inst];
  InstState* st = d.st;
  if (st->step >= d.n_steps || st->status != DEV_OK) return;

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int parity = (STAGE == STAGE_EULER) ? st->parity : 0;
  [[maybe_unused]] const uint32_t salt = sr_salt(st->step, STAGE);   // BF16 stochastic rounding
  const int in_buf = (STAGE == STAGE_EULER) ? parity : (STAGE == STAGE_HEUN1 ? 0 : 1);
  const int out_buf = (STAGE == STAGE_EULER) ? (1 - parity) : (STAGE == STAGE_HEUN1 ? 1 : 0);
  const T* __restrict__ psi_in = reinterpret_cast<const T*>(d.psi[in_buf]);
  const T* __restrict__ psi_base = reinterpret_cast<const T*>(d.psi[0]);
  T* __restrict__ psi_out = reinterpret_cast<T*>(d.psi[out_buf]);
  const float* __restrict__ lg = d.tri_lg;
  const float* __restrict__ phi_in = d.phi[in_buf];
  float* __restrict__ phi_out = d.phi[out_buf];
  const int Mpad = d.Mpad;
  const int nv = Mpad / (32 * VEC);
  const float dt = d.dt;
  const int nreg = d.n_regions, nq = nreg + 2;
  const int n_cells = (int)d.n_cells;
  const int n_chunks = (n_cells + kT2Chunk - 1) / kT2Chunk;
  const int G = it.b;
  const int64_t limit = d.wait_limit;

  if (lane < NQ) {
    wacc[warp][lane] = 0.f;
    wdacc[warp][lane] = 0.0;
  }
  if (threadIdx.x == 0) {
    mbar_init(&meta.bar[0], 1);
    mbar_init(&meta.bar[1], 1);
    fence_barrier_init();
    if (it.a < n_chunks) t2_stage_meta(d, meta, it.a, 0, n_cells);
    if (it.a + G < n_chunks) t2_stage_meta(d, meta, it.a + G, 1, n_cells);
  }
  __syncthreads();
  bool ok = true;
  int ncell = 0;
  int i = 0;
  for (int k = it.a; k < n_chunks; k += G, ++i) {
    const int b = i & 1;
    const bool mok = mbar_wait_bounded(&meta.bar[b], (uint32_t)((i >> 1) & 1), limit);
    if (__syncthreads_or(!mok)) {
      ok = false;
      break;
    }
    const int c0 = k * kT2Chunk;
    const int c_end = min(n_cells, c0 + kT2Chunk);
    for (int cell = c0 + warp; cell < c_end; cell += kT2Warps) {
      const int li = cell - c0;
      const int4 nb = meta.nbr[b][li];
      const float4 g0 = meta.geo[b][2 * li], g1 = meta.geo[b][2 * li + 1];
      const float4 h0 = meta.geo2[b][3 * li], h1 = meta.geo2[b][3 * li + 1], h2 = meta.geo2[b][3 * li + 2];
      const float ax[3] = {g0.x, g0.z, g1.x}, ay[3] = {g0.y, g0.w, g1.y};
      const float rx[3] = {h0.x, h0.z, h1.x}, ry[3] = {h0.y, h0.w, h1.y};
      // r_je = r_ie - d_ij: the neighbour's centroid-to-midpoint vector of the shared edge
      const float sx[3] = {rx[0] - h1.z, rx[1] - h2.x, rx[2] - h2.z};
      const float sy[3] = {ry[0] - h1.w, ry[1] - h2.y, ry[2] - h2.w};
      const int nbr[3] = {nb.x, nb.y, nb.z};
      const int m = nb.w & 255, reg = (nb.w >> 8) & 255;
      const float area = g1.z;
      const float sig_t = d.sig_t[m];
      const float phin = phi_in[cell];
      const float src = d.sig_s2pi[m] * phin + d.q_src[m];
      const bool has_bnd = (nbr[0] < 0) | (nbr[1] < 0) | (nbr[2] < 0);
      float gh[3];
#pragma unroll
      for (int e = 0; e < 3; ++e) gh[e] = (nbr[e] < 0) ? d.ghost[-1 - nbr[e]] : 0.f;

      float phi_part = 0.f, bpart = 0.f;
      for (int v = 0; v < nv; ++v) {
        const int kk = (v * 32 + lane) * VEC;
        float c[VEC], cx[VEC], cy[VEC], base[VEC];
        float nbv[3][VEC], nx[3][VEC], ny[3][VEC];
        ld_vec<T, VEC>(psi_in + (size_t)cell * Mpad + kk, c);
        ld_vec<float, VEC>(lg + (size_t)cell * 2 * Mpad + kk, cx);
        ld_vec<float, VEC>(lg + (size_t)cell * 2 * Mpad + Mpad + kk, cy);
#pragma unroll
        for (int e = 0; e < 3; ++e) {
          if (nbr[e] >= 0) {
            ld_vec<T, VEC>(psi_in + (size_t)nbr[e] * Mpad + kk, nbv[e]);
            ld_vec<float, VEC>(lg + (size_t)nbr[e] * 2 * Mpad + kk, nx[e]);
            ld_vec<float, VEC>(lg + (size_t)nbr[e] * 2 * Mpad + Mpad + kk, ny[e]);
          } else {
#pragma unroll
            for (int l = 0; l < VEC; ++l) nbv[e][l] = nx[e][l] = ny[e][l] = 0.f;
          }
        }
        if constexpr (STAGE == STAGE_HEUN2) ld_vec<T, VEC>(psi_base + (size_t)cell * Mpad + kk, base);
        float xi[VEC], eta[VEC], w[VEC], out[VEC];
        ld_vec<float, VEC>(d.xi + kk, xi);
        ld_vec<float, VEC>(d.eta + kk, eta);
        ld_vec<float, VEC>(d.w + kk, w);
        // BF16 rounding bits of the lane's ordinates kk .. kk+VEC-1 (one group of four)
        [[maybe_unused]] uint2 rb4;
        if constexpr (sizeof(T) == 2) rb4 = sr_bits4((uint32_t)cell, sr_gkey(kk >> 2, salt));
#pragma unroll
        for (int l = 0; l < VEC; ++l) {
          float div = 0.f;
#pragma unroll
          for (int e = 0; e < 3; ++e) {
            const float on = xi[l] * ax[e] + eta[l] * ay[e];
            float tr;
            if (nbr[e] < 0) {
              tr = (on > 0.f) ? c[l] : gh[e];   // first order on the boundary
            } else if (on > 0.f) {
              tr = fmaf(cx[l], rx[e], fmaf(cy[l], ry[e], c[l]));
            } else {
              tr = fmaf(nx[e][l], sx[e], fmaf(ny[e][l], sy[e], nbv[e][l]));
            }
            div = fmaf(on, tr, div);
          }
          const float F = -div - sig_t * c[l] + src;
          float o;
          if constexpr (STAGE == STAGE_HEUN2) {
            o = 0.5f * (base[l] + c[l] + dt * F);
          } else {
            o = c[l] + dt * F;
          }
          if constexpr (sizeof(T) == 2) {
            const int ko = kk + l;
            o = Store<T>::round_sr(o, sr_elem(rb4, ko & 3));
          }
          out[l] = o;
          phi_part += w[l] * o;
          if (has_bnd) {
#pragma unroll
            for (int e = 0; e < 3; ++e) {
              if (nbr[e] < 0) {
                const float on = xi[l] * ax[e] + eta[l] * ay[e];
                bpart += w[l] * on * ((on > 0.f) ? o : gh[e]);
              }
            }
          }
        }
        st_vec<T, VEC>(psi_out + (size_t)cell * Mpad + kk, out);
      }
      const float ph = warp_sum(phi_part);
      float bsum = 0.f;
      if (has_bnd) bsum = warp_sum(bpart);
      if (lane == 0) {
        phi_out[cell] = ph;
        wacc[warp][reg] += d.sig_a_f[m] * area * ph;
        wacc[warp][nreg] += area * ph;
        wacc[warp][nreg + 1] += bsum * area;
      }
      if ((++ncell & 31) == 0) {
        __syncwarp();
        if (lane < nq) {
          wdacc[warp][lane] += (double)wacc[warp][lane];
          wacc[warp][lane] = 0.f;
        }
        __syncwarp();
      }
    }
    __syncthreads();
    if (threadIdx.x == 0 && k + 2 * G < n_chunks) t2_stage_meta(d, meta, k + 2 * G, b, n_cells);
  }
  if (!ok && threadIdx.x == 0) {
    for (int j = i; j < i + 2; ++j) {
      const int kj = it.a + j * G;
      if (kj < n_chunks) mbar_wait_bounded(&meta.bar[j & 1], (uint32_t)((j >> 1) & 1), limit);
    }
    atomicCAS(&st->status, DEV_OK, DEV_TIMEOUT);
    st->timeout_where = ((int64_t)blockIdx.x << 32) | (int64_t)i;
  }
  __syncwarp();
  if (lane < nq) wdacc[warp][lane] += (double)wacc[warp][lane];
  __syncthreads();
  if (threadIdx.x < nq) {
    double s = 0.0;
    for (int w2 = 0; w2 < kT2Warps; ++w2) s += wdacc[w2][threadIdx.x];
    red[threadIdx.x] = s;
  }
  __syncthreads();
  finalize_item<kT2Threads>(d, it, red, STAGE, red + NQ);
}

}  // namespace

cudaError_t launch_tri2_stage(const InstDesc* d_desc, const WorkItem* d_items, int n_items, int stage, int storage,
                              int vec, int grad_vec, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  // the gradient pass takes 4 ordinates per lane where the quadrature allows
  // (fewer, wider loads); the stage pass at most 2 (its registers)
#define RTK_T2(V, ST, TT)                                                                       \
  if (vec == V && stage == ST) {                                                                \
    if (grad_vec == 4) tri_grad_kernel<4, TT><<<n_items, kT2Threads, 0, s>>>(d_desc, d_items, ST); \
    else tri_grad_kernel<V, TT><<<n_items, kT2Threads, 0, s>>>(d_desc, d_items, ST);            \
    cudaError_t e = cudaGetLastError();                                                         \
    if (e != cudaSuccess) return e;                                                             \
    tri_stage2_kernel<V, ST, TT><<<n_items, kT2Threads, 0, s>>>(d_desc, d_items);               \
    return cudaGetLastError();                                                                  \
  }
#define RTK_T2_ALL(TT)                                                                          \
  RTK_T2(1, STAGE_EULER, TT) RTK_T2(1, STAGE_HEUN1, TT) RTK_T2(1, STAGE_HEUN2, TT)              \
  RTK_T2(2, STAGE_EULER, TT) RTK_T2(2, STAGE_HEUN1, TT) RTK_T2(2, STAGE_HEUN2, TT)
  if (storage == 0) { RTK_T2_ALL(float) } else { RTK_T2_ALL(__nv_bfloat16) }
#undef RTK_T2_ALL
#undef RTK_T2
  return cudaErrorInvalidValue;
}

}  // namespace rtk
