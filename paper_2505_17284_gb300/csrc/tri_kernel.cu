// Triangle-mesh stage kernel (first-order upwind, Sec. 4.2 on triangles) and
// the cell-range kernels shared by both mesh kinds: initial phi/QoIs of a state
// and the FP64 <-> storage conversions.
//
// Stage kernel: one warp per cell, lanes over ordinates (VEC consecutive
// ordinates per lane per access, so a row of M_pad values is read with 16-byte
// vector loads). For each ordinate k the three edges of cell i contribute
// (omega_k . n_e) l_e / A_i * psi_hat with psi_hat = psi_i if omega_k . n_e > 0 else
// the neighbour's psi (or psi^- of the boundary side) (Eq. upwind1stOrder);
// F = -sum_e(...) - sigma_t psi + sigma_s/(2 pi) phi + Q (Eq. sn_2d_eqn_fv).
// The warp sums w_k out_k over all ordinates to phi_out of the cell directly.
// Cells are ordered by grid row, so the neighbours one row up/down (2n cells
// away) stay in L2 while a band of rows is processed.
#include <cuda_bf16.h>

#include "device_common.cuh"

namespace rtk {

constexpr int kTriThreads = 256;
constexpr int kTriWarps = kTriThreads / 32;

template <typename T, int VEC>
struct alignas(sizeof(T) * VEC) VecT {
  T v[VEC];
};

template <typename T, int VEC>
__device__ __forceinline__ void load_vec(const T* p, float (&out)[VEC]) {
  const VecT<T, VEC> x = *reinterpret_cast<const VecT<T, VEC>*>(p);
#pragma unroll
  for (int l = 0; l < VEC; ++l) out[l] = Store<T>::from_smem(x.v[l]);
}

template <typename T, int VEC>
__device__ __forceinline__ void store_vec(T* p, const float (&in)[VEC]) {
  VecT<T, VEC> x;
#pragma unroll
  for (int l = 0; l < VEC; ++l) {
    if constexpr (sizeof(T) == 4) {
      x.v[l] = in[l];
    } else {
      x.v[l] = __float2bfloat16_rn(in[l]);
    }
  }
  *reinterpret_cast<VecT<T, VEC>*>(p) = x;
}

// Per-lane QoI accumulation: lane (n & 31) keeps the n-th cell of its warp;
// every 32 cells all lanes add their kept cell (fixed order, FP32 per lane),
// so the region switch costs one pass per 32 cells.
struct LaneQoI {
  float fa[kMaxReg];
  float fm;
  float keep_va, keep_vm;
  int keep_reg;
  __device__ void init() {
#pragma unroll
    for (int g = 0; g < kMaxReg; ++g) fa[g] = 0.f;
    fm = 0.f;
    keep_va = keep_vm = 0.f;
    keep_reg = -1;
  }
  __device__ void flush() {
#pragma unroll
    for (int g = 0; g < kMaxReg; ++g)
      if (g == keep_reg) fa[g] += keep_va;
    fm += keep_vm;
    keep_va = keep_vm = 0.f;
    keep_reg = -1;
  }
};

// Persistent stage kernel: work item g of G processes the 64-cell chunks
// g, g + G, g + 2G, ... in increasing order, so all SMs sweep the mesh together
// and the rows of the neighbouring grid row (2n cells away on the split grid)
// are still in L2 when they are gathered. The neighbour lists and edge
// geometry of a chunk (contiguous arrays) are staged in shared memory by two
// TMA bulk copies, double-buffered one chunk ahead, so a warp starts a cell
// with its metadata at hand and goes straight to the row loads. Warp w takes
// cells w, w + 8, ... of a chunk (neighbours one cell apart are fetched by
// adjacent warps at the same time, L1), and loads the rows of two ordinate
// blocks before computing either. QoI terms are summed per warp in shared
// memory (FP32 over 32 cells, then FP64).
constexpr int kTriChunk = 64;

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

template <int VEC, int STAGE, typename T>
__global__ void __launch_bounds__(kTriThreads, 3)
    tri_stage_kernel(const InstDesc* __restrict__ descs, const WorkItem* __restrict__ items) {
  __shared__ double red[(kTriWarps + 1) * NQ];
  __shared__ float wacc[kTriWarps][NQ];
  __shared__ double wdacc[kTriWarps][NQ];
  __shared__ __align__(16) int4 s_nbr[2][kTriChunk];
  __shared__ __align__(16) float4 s_geo[2][2 * kTriChunk];
  __shared__ __align__(8) uint64_t s_bar[2];
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
  const float* __restrict__ phi_in = d.phi[in_buf];
  float* __restrict__ phi_out = d.phi[out_buf];
  const int Mpad = d.Mpad;
  const int nv = Mpad / (32 * VEC);
  const float dt = d.dt;
  const int nreg = d.n_regions, nq = nreg + 2;
  const int n_cells = (int)d.n_cells;
  const int n_chunks = (n_cells + kTriChunk - 1) / kTriChunk;
  const int G = it.b;
  const int64_t limit = d.wait_limit;

  // metadata of chunk k into buffer b (thread 0)
  auto stage_meta = [&](int k, int b) {
    const int c0 = k * kTriChunk;
    const int cells = min(kTriChunk, n_cells - c0);
    mbar_arrive_expect_tx(&s_bar[b], (uint32_t)cells * 48u);
    bulk_load(s_nbr[b], d.tri_nbr + c0, (uint32_t)cells * 16u, &s_bar[b]);
    bulk_load(s_geo[b], d.tri_geo + 2 * (size_t)c0, (uint32_t)cells * 32u, &s_bar[b]);
  };
  if (lane < NQ) {
    wacc[warp][lane] = 0.f;
    wdacc[warp][lane] = 0.0;
  }
  if (threadIdx.x == 0) {
    mbar_init(&s_bar[0], 1);
    mbar_init(&s_bar[1], 1);
    fence_barrier_init();
    if (it.a < n_chunks) stage_meta(it.a, 0);
    if (it.a + G < n_chunks) stage_meta(it.a + G, 1);
  }
  __syncthreads();
  bool ok = true;
  int ncell = 0;
  int i = 0;   // chunks done by this CTA
  for (int k = it.a; k < n_chunks; k += G, ++i) {
    const int b = i & 1;
    const bool mok = mbar_wait_bounded(&s_bar[b], (uint32_t)((i >> 1) & 1), limit);
    if (__syncthreads_or(!mok)) {   // the chunk's metadata never arrived: every warp stops here
      ok = false;
      break;
    }
    const int c0 = k * kTriChunk;
    const int c_end = min(n_cells, c0 + kTriChunk);
    for (int cell = c0 + warp; cell < c_end; cell += kTriWarps) {
      const int li = cell - c0;
      const int4 nb = s_nbr[b][li];
      const float4 g0 = s_geo[b][2 * li], g1 = s_geo[b][2 * li + 1];
      const float ax[3] = {g0.x, g0.z, g1.x};
      const float ay[3] = {g0.y, g0.w, g1.y};
      const int nbr[3] = {nb.x, nb.y, nb.z};
      const int m = nb.w & 255, reg = (nb.w >> 8) & 255;
      const float area = g1.z;
      const float sig_t = d.sig_t[m];
      const float phin = phi_in[cell];
      const bool has_bnd = (nbr[0] < 0) | (nbr[1] < 0) | (nbr[2] < 0);
      float gh[3];
#pragma unroll
      for (int e = 0; e < 3; ++e) gh[e] = (nbr[e] < 0) ? d.ghost[-1 - nbr[e]] : 0.f;

      float phi_part = 0.f, bpart = 0.f;
      for (int v0 = 0; v0 < nv; v0 += 2) {
        // the rows of two ordinate blocks are loaded before either is computed
        float c2[2][VEC], nbv2[2][3][VEC], base2[2][VEC];
        const bool two = v0 + 1 < nv;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (h == 1 && !two) break;
          const int kk = ((v0 + h) * 32 + lane) * VEC;
          load_vec<T, VEC>(psi_in + (size_t)cell * Mpad + kk, c2[h]);
#pragma unroll
          for (int e = 0; e < 3; ++e) {
            if (nbr[e] >= 0) {
              load_vec<T, VEC>(psi_in + (size_t)nbr[e] * Mpad + kk, nbv2[h][e]);
            } else {
#pragma unroll
              for (int l = 0; l < VEC; ++l) nbv2[h][e][l] = gh[e];
            }
          }
          if constexpr (STAGE == STAGE_HEUN2) load_vec<T, VEC>(psi_base + (size_t)cell * Mpad + kk, base2[h]);
        }
        const float src = d.sig_s2pi[m] * phin + d.q_src[m];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (h == 1 && !two) break;
          const int kk = ((v0 + h) * 32 + lane) * VEC;
          float xi[VEC], eta[VEC], w[VEC], out[VEC];
          load_vec<float, VEC>(d.xi + kk, xi);
          load_vec<float, VEC>(d.eta + kk, eta);
          load_vec<float, VEC>(d.w + kk, w);
          // BF16 rounding bits of the lane's ordinates kk .. kk+VEC-1 (one group of four)
          [[maybe_unused]] uint2 rb4;
          if constexpr (sizeof(T) == 2) rb4 = sr_bits4((uint32_t)cell, sr_gkey(kk >> 2, salt));
#pragma unroll
          for (int l = 0; l < VEC; ++l) {
            const float c = c2[h][l];
            float div = 0.f;
#pragma unroll
            for (int e = 0; e < 3; ++e) {
              const float on = xi[l] * ax[e] + eta[l] * ay[e];
              div += on * ((on > 0.f) ? c : nbv2[h][e][l]);
            }
            const float F = -div - sig_t * c + src;
            float o;
            if constexpr (STAGE == STAGE_HEUN2) {
              o = 0.5f * (base2[h][l] + c + dt * F);
            } else {
              o = c + dt * F;
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
          store_vec<T, VEC>(psi_out + (size_t)cell * Mpad + kk, out);
        }
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
    // every warp is done with buffer b: it takes the chunk two ahead
    __syncthreads();
    if (threadIdx.x == 0 && k + 2 * G < n_chunks) stage_meta(k + 2 * G, b);
  }
  if (!ok && threadIdx.x == 0) {
    // drain: the metadata copies issued and not consumed (chunks i and i + 1)
    for (int j = i; j < i + 2; ++j) {
      const int kj = it.a + j * G;
      if (kj < n_chunks) mbar_wait_bounded(&s_bar[j & 1], (uint32_t)((j >> 1) & 1), limit);
    }
    atomicCAS(&st->status, DEV_OK, DEV_TIMEOUT);
    st->timeout_where = ((int64_t)blockIdx.x << 32) | (int64_t)i;
  }
  __syncwarp();
  if (lane < nq) wdacc[warp][lane] += (double)wacc[warp][lane];
  __syncthreads();
  if (threadIdx.x < nq) {
    double s = 0.0;
    for (int w2 = 0; w2 < kTriWarps; ++w2) s += wdacc[w2][threadIdx.x];
    red[threadIdx.x] = s;
  }
  __syncthreads();
  finalize_item<kTriThreads>(d, it, red, STAGE, red + NQ);
}

template <int VEC, int STAGE, typename T>
static cudaError_t tri_launch_one(const InstDesc* d_desc, const WorkItem* d_items, int n_items, cudaStream_t s) {
  tri_stage_kernel<VEC, STAGE, T><<<n_items, kTriThreads, 0, s>>>(d_desc, d_items);
  return cudaGetLastError();
}

cudaError_t launch_tri_stage(const InstDesc* d_desc, const WorkItem* d_items, int n_items, int stage, int storage,
                             int vec, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
#define RTK_T(V, ST, TT) \
  if (vec == V && stage == ST) return tri_launch_one<V, ST, TT>(d_desc, d_items, n_items, s);
#define RTK_T_ALL(TT)                                                                         \
  RTK_T(1, STAGE_EULER, TT) RTK_T(1, STAGE_HEUN1, TT) RTK_T(1, STAGE_HEUN2, TT)               \
  RTK_T(2, STAGE_EULER, TT) RTK_T(2, STAGE_HEUN1, TT) RTK_T(2, STAGE_HEUN2, TT)               \
  RTK_T(4, STAGE_EULER, TT) RTK_T(4, STAGE_HEUN1, TT) RTK_T(4, STAGE_HEUN2, TT)
  if (storage == 0) { RTK_T_ALL(float) } else { RTK_T_ALL(__nv_bfloat16) }
#undef RTK_T_ALL
#undef RTK_T
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// phi and QoI integrands of the current state (after create / set_psi): one warp
// per cell; finalizes with STAGE_INIT (sets the current integrands, no time step).
template <int VEC, typename T>
__global__ void __launch_bounds__(kTriThreads)
    init_kernel(const InstDesc* __restrict__ descs, const WorkItem* __restrict__ items) {
  __shared__ double red[(kTriWarps + 1) * NQ];
  const WorkItem it = items[blockIdx.x];
  const InstDesc& d = descs[it.inst];
  InstState* st = d.st;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int buf = st->parity;
  const T* __restrict__ psi = reinterpret_cast<const T*>(d.psi[buf]);
  float* __restrict__ phi = d.phi[buf];
  const int Mpad = d.Mpad, nv = Mpad / (32 * VEC);
  const bool tri = d.kind == KIND_TRI;

  LaneQoI qa;
  qa.init();
  float bacc = 0.f;
  int ncell = 0;
  for (int cell = it.a + warp; cell < it.a + it.b; cell += kTriWarps, ++ncell) {
    // boundary faces of this cell: (n*l) per face and the side's inflow value
    float fx[4] = {0.f, 0.f, 0.f, 0.f}, fy[4] = {0.f, 0.f, 0.f, 0.f}, gh[4] = {0.f, 0.f, 0.f, 0.f};
    int nf = 0;
    int m, reg;
    float area;
    if (tri) {
      const int4 nb = d.tri_nbr[cell];
      const float4 g0 = d.tri_geo[2 * (size_t)cell];
      const float4 g1 = d.tri_geo[2 * (size_t)cell + 1];
      const float ax[3] = {g0.x, g0.z, g1.x}, ay[3] = {g0.y, g0.w, g1.y};
      const int nbr[3] = {nb.x, nb.y, nb.z};
      area = g1.z;
      m = nb.w & 255;
      reg = (nb.w >> 8) & 255;
      for (int e = 0; e < 3; ++e)
        if (nbr[e] < 0) {
          fx[nf] = ax[e] * area;
          fy[nf] = ay[e] * area;
          gh[nf] = d.ghost[-1 - nbr[e]];
          ++nf;
        }
    } else {
      const int i = cell % d.nx, j = cell / d.nx;
      area = (float)d.area_d;
      m = d.mat[cell];
      reg = d.region[cell];
      const float ly = (float)d.dy_d, lx = (float)d.dx_d;
      // boundary faces (a periodic axis has none)
      if (!d.periodic_x && i == 0) { fx[nf] = -ly; fy[nf] = 0.f; gh[nf] = d.ghost[0]; ++nf; }
      if (!d.periodic_x && i == d.nx - 1) { fx[nf] = ly; fy[nf] = 0.f; gh[nf] = d.ghost[1]; ++nf; }
      if (!d.periodic_y && j == 0) { fx[nf] = 0.f; fy[nf] = -lx; gh[nf] = d.ghost[2]; ++nf; }
      if (!d.periodic_y && j == d.ny - 1) { fx[nf] = 0.f; fy[nf] = lx; gh[nf] = d.ghost[3]; ++nf; }
    }
    float ph_part = 0.f, bpart = 0.f;
    for (int v = 0; v < nv; ++v) {
      const int k = (v * 32 + lane) * VEC;
      float c[VEC], xi[VEC], eta[VEC], w[VEC];
      load_vec<T, VEC>(psi + (size_t)cell * Mpad + k, c);
      load_vec<float, VEC>(d.xi + k, xi);
      load_vec<float, VEC>(d.eta + k, eta);
      load_vec<float, VEC>(d.w + k, w);
#pragma unroll
      for (int l = 0; l < VEC; ++l) {
        ph_part += w[l] * c[l];
        for (int f = 0; f < nf; ++f) {
          const float on = xi[l] * fx[f] + eta[l] * fy[f];
          bpart += w[l] * on * ((on > 0.f) ? c[l] : gh[f]);
        }
      }
    }
    const float ph = warp_sum(ph_part);
    if (lane == 0) phi[cell] = ph;
    bacc += bpart;
    if (lane == (ncell & 31)) {
      qa.keep_va = d.sig_a_f[m] * area * ph;
      qa.keep_vm = area * ph;
      qa.keep_reg = reg;
    }
    if ((ncell & 31) == 31) qa.flush();
  }
  qa.flush();
  const int nreg = d.n_regions;
  double acc[NQ];
#pragma unroll
  for (int g = 0; g < NQ; ++g) acc[g] = 0.0;
#pragma unroll
  for (int g = 0; g < kMaxReg; ++g)
    if (g < nreg) acc[g] = (double)qa.fa[g];
#pragma unroll
  for (int g = 0; g < kMaxReg + 1; ++g)
    if (g == nreg) acc[g] = (double)qa.fm;
#pragma unroll
  for (int g = 0; g < kMaxReg + 2; ++g)
    if (g == nreg + 1) acc[g] = (double)bacc;
  block_reduce_q<kTriThreads>(acc, nreg + 2, red);
  finalize_item<kTriThreads>(d, it, red, STAGE_INIT, red + NQ);
}

cudaError_t launch_init(const InstDesc* d_desc, const WorkItem* d_items, int n_items, int vec, int storage,
                        cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
#define RTK_I(V, TT) \
  if (vec == V) { init_kernel<V, TT><<<n_items, kTriThreads, 0, s>>>(d_desc, d_items); return cudaGetLastError(); }
  if (storage == 0) { RTK_I(1, float) RTK_I(2, float) RTK_I(4, float) }
  else { RTK_I(1, __nv_bfloat16) RTK_I(2, __nv_bfloat16) RTK_I(4, __nv_bfloat16) }
#undef RTK_I
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Storage conversions between the caller's FP64 [cell][M] and the device
// layout [cell][Mpad] of T (round to nearest even for bf16; padding zeroed).
template <typename T>
__global__ void convert_in_kernel(const double* __restrict__ src, T* __restrict__ dst, int64_t n_cells, int M,
                                  int Mpad, const int32_t* __restrict__ inv) {
  const int64_t n = n_cells * Mpad;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = i / Mpad;
    const int slot = (int)(i - cell * Mpad);
    const int k = inv ? inv[slot] : (slot < M ? slot : -1);
    const float v = (k >= 0) ? (float)src[cell * M + k] : 0.f;
    Store<T>::store(dst + i, v);
  }
}

template <typename T>
__global__ void convert_out_kernel(const T* __restrict__ src, double* __restrict__ dst, int64_t n_cells, int M,
                                   int Mpad, const int32_t* __restrict__ kmap) {
  const int64_t n = n_cells * M;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = i / M;
    const int k = (int)(i - cell * M);
    dst[i] = (double)Store<T>::load(src + cell * Mpad + (kmap ? kmap[k] : k));
  }
}

cudaError_t launch_convert_in(const double* src, void* dst, int64_t n_cells, int M, int Mpad, int storage,
                              const int32_t* inv, cudaStream_t s) {
  const int64_t n = n_cells * Mpad;
  const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  if (n == 0) return cudaSuccess;
  if (storage == 0)
    convert_in_kernel<float><<<blocks, 256, 0, s>>>(src, (float*)dst, n_cells, M, Mpad, inv);
  else
    convert_in_kernel<__nv_bfloat16><<<blocks, 256, 0, s>>>(src, (__nv_bfloat16*)dst, n_cells, M, Mpad, inv);
  return cudaGetLastError();
}

cudaError_t launch_convert_out(const void* src, double* dst, int64_t n_cells, int M, int Mpad, int storage,
                               const int32_t* kmap, cudaStream_t s) {
  const int64_t n = n_cells * M;
  const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  if (n == 0) return cudaSuccess;
  if (storage == 0)
    convert_out_kernel<float><<<blocks, 256, 0, s>>>((const float*)src, dst, n_cells, M, Mpad, kmap);
  else
    convert_out_kernel<__nv_bfloat16><<<blocks, 256, 0, s>>>((const __nv_bfloat16*)src, dst, n_cells, M, Mpad, kmap);
  return cudaGetLastError();
}

}  // namespace rtk
