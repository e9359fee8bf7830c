// Cartesian stage kernel of the explicit S_N step (Sec. 4.2-4.3).
//
// Work split. One CTA (8 warps) owns a strip of TX = 8R cells in x by a segment
// of `ly` rows in y and loops over the ordinate chunks of C = 32V ordinates
// (lane l holds ordinates l*V .. l*V+V-1 of the chunk, read as one vector from
// shared memory). Warp w owns the run of R consecutive cells w*R .. w*R+R-1.
// For each chunk the CTA walks its rows in +y: every row of (TX + 2H) cells x C
// ordinates (H = halo = order) arrives by one TMA box load into a ring of shared
// memory slots guarded by mbarriers; a row stays resident until it has been
// completed (H rows after its arrival), then its slot takes the next load.
//
// Fluxes. Each face value is computed once (Eq. upwind1stOrder with R =
// psi +/- slope/2, minmod slopes per dimension):
//   x: the lane reads its run in upwind order (addresses step by the sign d of
//      xi), so face m (outgoing face of the m-th cell along the flow) is
//      u_m + h_m minmod(u_{m+1} - u_m, u_m - u_{m-1}) and the divergence of cell
//      m is |xi|/dx (F_m - F_{m-1});
//   y: a register window over the rows gives the face j+1/2 once per row, from
//      the upwind cell (j if eta > 0, j+1 if eta < 0), and the divergence of row j
//      is eta/dy (G_{j+1/2} - G_{j-1/2}).
// minmod(a, b) is the median of (a, b, 0). h = 1/2 except on domain boundary
// faces, which are first order (h = 0). Cells outside the domain hold the side's
// ghost value psi^- (Sec. 4.2); only CTAs touching the boundary take that path.
//
// Update. With a = 1 - dt sigma_t and b = dt (sigma_s/(2 pi) phi + Q) per cell:
//   Euler / Heun stage 1: out = a psi + b - dt (div_x + div_y)
//   Heun stage 2:         out = (psi^n + a psi1 + b - dt (div_x + div_y)) / 2
// (Eq. sn_2d_eqn_fv and Sec. 4.3). phi_out = sum_k w_k out_k is accumulated per
// cell in shared memory chunk after chunk (fixed order). The epilogue writes
// phi_out and FP64 QoI partials (absorption per region, mass, boundary outflow)
// of the output state; the last CTA of the instance reduces them in order and
// applies the time-integration weights.
#pragma once
#include <cuda_bf16.h>

#include <atomic>
#include <type_traits>

#include "device_common.cuh"

namespace rtk {

constexpr int kCartThreads = 256;
constexpr int kCartWarps = kCartThreads / 32;

template <int ORDER, int R, int V, int STAGE, typename T>
struct CartCfg {
  static constexpr int H = ORDER;                 // halo cells in x and rows in y
  static constexpr int TX = kCartWarps * R;       // cells per strip
  static constexpr int C = 32 * V;                // ordinates per chunk
  static constexpr int NS = (STAGE == STAGE_HEUN2) ? 5 : 6;   // ring slots
  static constexpr int halo_bytes = (TX + 2 * H) * C * (int)sizeof(T);
  static constexpr int base_bytes = (STAGE == STAGE_HEUN2) ? TX * C * (int)sizeof(T) : 0;
  static constexpr int slot_bytes = (halo_bytes + base_bytes + 127) / 128 * 128;
  static constexpr int ring_bytes = NS * slot_bytes;
  static constexpr int NL = R + 2 * H - 1;        // values read per row: m = -H .. R+H-2
};

__host__ __device__ inline size_t cart_tile_bytes(int tx, int ly) {
  // a [ly][tx], b [ly][tx], phi_acc [ly][tx] (float)
  return ((size_t)ly * tx * 12 + 127) / 128 * 128;
}

// barriers (128) + FP64 reduction rows ((warps + 1) x NQ) + alignment slack
constexpr size_t kCartRedBytes = (kCartWarps + 1) * NQ * 8;
constexpr size_t kCartFixedBytes = 128 + kCartRedBytes + 128;

template <int ORDER, int R, int V, int STAGE, typename T>
size_t cart_smem_for(int ly) {
  using L = CartCfg<ORDER, R, V, STAGE, T>;
  return L::ring_bytes + cart_tile_bytes(L::TX, ly) + kCartFixedBytes;
}

// Index of cell or row g on a periodic axis of n cells (g may lie a few cells
// outside 0..n-1).
__device__ __forceinline__ int wrap_index(int g, int n) { return ((g % n) + n) % n; }

// minmod(a, b) = median(a, b, 0): 0 unless a and b share a sign, else the one of
// smaller magnitude.
__device__ __forceinline__ float minmod_med(float a, float b) {
  const float lo = fminf(a, b), hi = fmaxf(a, b);
  return fmaxf(lo, fminf(hi, 0.f));
}

template <typename T, int V>
__device__ __forceinline__ void lds_vec(const T* p, float (&out)[V]) {
  if constexpr (sizeof(T) == 4) {
    if constexpr (V == 4) {
      const float4 x = *reinterpret_cast<const float4*>(p);
      out[0] = x.x; out[1] = x.y; out[2] = x.z; out[3] = x.w;
    } else if constexpr (V == 2) {
      const float2 x = *reinterpret_cast<const float2*>(p);
      out[0] = x.x; out[1] = x.y;
    } else {
      out[0] = *reinterpret_cast<const float*>(p);
    }
  } else {
    if constexpr (V == 4) {
      const uint2 x = *reinterpret_cast<const uint2*>(p);
      const float2 fa = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&x.x));
      const float2 fb = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&x.y));
      out[0] = fa.x; out[1] = fa.y; out[2] = fb.x; out[3] = fb.y;
    } else if constexpr (V == 2) {
      const float2 fa = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
      out[0] = fa.x; out[1] = fa.y;
    } else {
      out[0] = __bfloat162float(*p);
    }
  }
}

template <typename T, int V>
__device__ __forceinline__ void stg_vec(T* p, const float (&in)[V]) {
  if constexpr (sizeof(T) == 4) {
    if constexpr (V == 4) {
      *reinterpret_cast<float4*>(p) = make_float4(in[0], in[1], in[2], in[3]);
    } else if constexpr (V == 2) {
      *reinterpret_cast<float2*>(p) = make_float2(in[0], in[1]);
    } else {
      *reinterpret_cast<float*>(p) = in[0];
    }
  } else {
    if constexpr (V == 4) {
      __nv_bfloat162 a = __floats2bfloat162_rn(in[0], in[1]);
      __nv_bfloat162 b = __floats2bfloat162_rn(in[2], in[3]);
      uint2 x;
      x.x = *reinterpret_cast<uint32_t*>(&a);
      x.y = *reinterpret_cast<uint32_t*>(&b);
      *reinterpret_cast<uint2*>(p) = x;
    } else if constexpr (V == 2) {
      *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(in[0], in[1]);
    } else {
      *p = __float2bfloat16_rn(in[0]);
    }
  }
}

// ---- paired FP32 helpers (two values per instruction on sm_100 and later)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);   // a - b, rounded once
}
__device__ __forceinline__ float2 minmod2(float2 a, float2 b) {
  return make_float2(minmod_med(a.x, b.x), minmod_med(a.y, b.y));
}
__device__ __forceinline__ float2 relu2(float2 a) { return make_float2(fmaxf(a.x, 0.f), fmaxf(a.y, 0.f)); }
// minmod(a, b) = min(max(a, b), max(a, 0), max(b, 0)), the last two given: for
// a <= b this is a when 0 <= a, 0 when a < 0 <= b and b when b < 0, i.e. the
// median of (a, b, 0). A difference feeds two faces, so its max(., 0) is shared.
__device__ __forceinline__ float fmin3f(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ float2 minmod2r(float2 a, float2 b, float2 ra, float2 rb) {
  return make_float2(fmin3f(fmaxf(a.x, b.x), ra.x, rb.x), fmin3f(fmaxf(a.y, b.y), ra.y, rb.y));
}

template <typename T, int V>
__device__ __forceinline__ void lds_vec2(const T* p, float2 (&out)[V / 2]) {
  static_assert(V == 2 || V == 4, "pairs need V = 2 or 4");
  if constexpr (sizeof(T) == 4) {
    if constexpr (V == 4) {
      const float4 x = *reinterpret_cast<const float4*>(p);
      out[0] = make_float2(x.x, x.y);
      out[1] = make_float2(x.z, x.w);
    } else {
      out[0] = *reinterpret_cast<const float2*>(p);
    }
  } else {
    if constexpr (V == 4) {
      const uint2 x = *reinterpret_cast<const uint2*>(p);
      out[0] = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&x.x));
      out[1] = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&x.y));
    } else {
      out[0] = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
    }
  }
}

template <typename T, int V>
__device__ __forceinline__ void stg_vec2(T* p, const float2 (&in)[V / 2]) {
  if constexpr (sizeof(T) == 4) {
    if constexpr (V == 4) {
      *reinterpret_cast<float4*>(p) = make_float4(in[0].x, in[0].y, in[1].x, in[1].y);
    } else {
      *reinterpret_cast<float2*>(p) = in[0];
    }
  } else {
    if constexpr (V == 4) {
      __nv_bfloat162 a = __floats2bfloat162_rn(in[0].x, in[0].y);
      __nv_bfloat162 b = __floats2bfloat162_rn(in[1].x, in[1].y);
      uint2 x;
      x.x = *reinterpret_cast<uint32_t*>(&a);
      x.y = *reinterpret_cast<uint32_t*>(&b);
      *reinterpret_cast<uint2*>(p) = x;
    } else {
      *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(in[0].x, in[0].y);
    }
  }
}

// Epilogue shared by the tile functions: write phi_out of the tile and reduce the
// FP64 QoI partials of the output state (absorption per region, mass, boundary
// outflow), then close the launch for this work item.
template <int TX, int STAGE>
__device__ __forceinline__ void cart_epilogue(const InstDesc& d, const WorkItem& it, float* __restrict__ phi_out,
                                              const float* tile_acc, double* red, int x0, int ya, int nrows,
                                              float bacc) {
  const int tid = threadIdx.x;
  const int nx = d.nx;
  const int nreg = d.n_regions;
  float fa[kMaxReg];
#pragma unroll
  for (int g = 0; g < kMaxReg; ++g) fa[g] = 0.f;
  float fm = 0.f;
  for (int i = tid; i < nrows * TX; i += kCartThreads) {
    const int r = i / TX, xl = i - r * TX;
    const int gx = x0 + xl;
    if (gx >= nx) continue;
    const size_t cell = (size_t)(ya + r) * nx + gx;
    const float ph = tile_acc[i];
    phi_out[cell] = ph;
    const int reg = d.region[cell];
    const float va = d.sig_a_f[d.mat[cell]] * ph;
#pragma unroll
    for (int g = 0; g < kMaxReg; ++g)
      if (g == reg) fa[g] += va;
    fm += ph;
  }
  double acc[NQ];
#pragma unroll
  for (int g = 0; g < NQ; ++g) acc[g] = 0.0;
#pragma unroll
  for (int g = 0; g < kMaxReg; ++g)
    if (g < nreg) acc[g] = (double)fa[g] * d.area_d;
#pragma unroll
  for (int g = 0; g < kMaxReg + 1; ++g)
    if (g == nreg) acc[g] = (double)fm * d.area_d;
#pragma unroll
  for (int g = 0; g < kMaxReg + 2; ++g)
    if (g == nreg + 1) acc[g] = (double)bacc;
  block_reduce_q<kCartThreads>(acc, nreg + 2, red);
  finalize_item<kCartThreads>(d, it, red, STAGE, red + NQ);
}

template <int ORDER, int R, int V, int STAGE, typename T, bool XB>
__device__ __forceinline__ void cart_tile(const InstDesc& d, const WorkItem& it, InstState* st, uint8_t* smem,
                                          const bool YB) {
  using L = CartCfg<ORDER, R, V, STAGE, T>;
  constexpr int H = L::H, TX = L::TX, C = L::C, NS = L::NS, NL = L::NL;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  const int parity = (STAGE == STAGE_EULER) ? st->parity : 0;
  [[maybe_unused]] const uint32_t salt = sr_salt(st->step, STAGE);   // BF16 stochastic rounding
  const int in_buf = (STAGE == STAGE_EULER) ? parity : (STAGE == STAGE_HEUN1 ? 0 : 1);
  const int out_buf = (STAGE == STAGE_EULER) ? (1 - parity) : (STAGE == STAGE_HEUN1 ? 1 : 0);
  const float* __restrict__ phi_in = d.phi[in_buf];
  float* __restrict__ phi_out = d.phi[out_buf];
  T* __restrict__ psi_out = reinterpret_cast<T*>(d.psi[out_buf]);
  const CUtensorMap* map_halo = &d.tm_psi_halo[in_buf];
  const CUtensorMap* map_base = &d.tm_psi_center;

  const int nx = d.nx, ny = d.ny, Mpad = d.Mpad;
  const int x0 = it.a * TX;
  const int ya = it.b * d.ly;
  const int yb = min(ny, ya + d.ly);
  const int nrows = yb - ya;
  const int Lc = nrows + 2 * H;     // rows pulled per chunk: ya-H .. yb+H-1
  const int total = d.n_chunks * Lc;

  uint8_t* ring = smem;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::ring_bytes);
  float* tile_a = reinterpret_cast<float*>(smem + L::ring_bytes + 128);
  float* tile_b = tile_a + d.ly * TX;
  float* tile_acc = tile_b + d.ly * TX;
  double* red = reinterpret_cast<double*>(smem + L::ring_bytes + 128 + cart_tile_bytes(TX, d.ly));
  const int64_t limit = d.wait_limit;

  auto issue = [&](int q) {
    const int slot = q % NS;
    const int c = q / Lc;
    const int p = ya - H + (q - c * Lc);
    uint8_t* dst = ring + slot * L::slot_bytes;
    // rows outside the domain: the wrapped row on a periodic axis, else none (ghost values)
    const bool wrapped = (p < 0 || p >= ny) && d.periodic_y;   // interior rows read no flag
    const bool halo = (p >= 0 && p < ny) || wrapped;
    const int pl = wrapped ? wrap_index(p, ny) : p;
    const bool base = (STAGE == STAGE_HEUN2) && (p - H >= ya);
    const uint32_t bytes = (halo ? L::halo_bytes : 0) + (base ? L::base_bytes : 0);
    if ((int64_t)q == d.drop_load) return;   // test hook: this slot never completes
    if (bytes == 0) {
      mbar_arrive(&bars[slot]);
      return;
    }
    mbar_arrive_expect_tx(&bars[slot], bytes);
    if (halo) tma_load_3d(dst, map_halo, &bars[slot], c * C, x0 - H, pl);
    if (base) tma_load_3d(dst + L::halo_bytes, map_base, &bars[slot], c * C, x0, p - H);
  };

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
    fence_barrier_init();
    fence_tensormap_acquire(map_halo);
    prefetch_tensormap(map_halo);
    if (STAGE == STAGE_HEUN2) {
      fence_tensormap_acquire(map_base);
      prefetch_tensormap(map_base);
    }
  }
  __syncthreads();
  if (tid == 0) {
    for (int q = 0; q < min(NS, total); ++q) issue(q);
  }
  // per-cell constants of the tile: a = 1 - dt sigma_t, b = dt (sigma_s/(2 pi) phi + Q)
  const float dt = d.dt;
  for (int i = tid; i < nrows * TX; i += kCartThreads) {
    const int r = i / TX, xl = i - r * TX;
    const int gx = x0 + xl;
    float a = 1.f, b = 0.f;
    if (gx < nx) {
      const size_t cell = (size_t)(ya + r) * nx + gx;
      const int m = d.mat[cell];
      a = 1.f - dt * d.sig_t[m];
      b = dt * (d.sig_s2pi[m] * phi_in[cell] + d.q_src[m]);
    }
    tile_a[i] = a;
    tile_b[i] = b;
    tile_acc[i] = 0.f;
  }
  __syncthreads();

  float bacc = 0.f;   // boundary outflow terms of this thread (FP32; FP64 from the block reduction on)
  const float ly_f = (float)d.dy_d, lx_f = (float)d.dx_d;
  const int xl0 = warp * R;   // first cell of this thread's run (tile-local)
  static_assert(NS >= H + 2, "the ring must hold the resident rows plus one load in flight");

  int q = 0;
  int issued = min(NS, total);
  for (int c = 0; c < d.n_chunks; ++c) {
    const int k0 = c * C + lane * V;
    [[maybe_unused]] const uint32_t gkey = sr_gkey(k0 >> 2, salt);   // BF16 rounding: the lane's group of 4
    float w[V], ax[V], ay[V], eneg[V];
    float xsum = 0.f;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const float xiv = d.xi[k0 + v], etav = d.eta[k0 + v];
      w[v] = d.w[k0 + v];
      xsum += xiv;
      ax[v] = dt * fabsf(xiv) * d.inv_dx;
      ay[v] = dt * etav * d.inv_dy;
      eneg[v] = (etav < 0.f) ? 1.f : 0.f;
    }
    const int dxs = (xsum >= 0.f) ? 1 : -1;    // lane's flow direction in x (uniform over its V ordinates)
    const int s0 = (dxs > 0) ? xl0 : xl0 + R - 1;
    // register window over rows (carried between pulls): c1 = row p-1, c2 = row p-2,
    // dprev = c_{p-2} - c_{p-3}, gprev = face value below the row being completed
    float c1[R][V], c2[R][V], dprev[R][V], gprev[R][V];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int v = 0; v < V; ++v) c1[r][v] = c2[r][v] = dprev[r][v] = gprev[r][v] = 0.f;

    for (int p = ya - H; p < yb + H; ++p, ++q) {
      const int slot = q % NS;
      const uint32_t par = (uint32_t)((q / NS) & 1);
      const bool ok = mbar_wait_bounded(&bars[slot], par, limit);
      const T* srow = reinterpret_cast<const T*>(ring + slot * L::slot_bytes);
      // ---- the new row p: own cells, in upwind order
      float c0[R][V];
      if (YB && !d.periodic_y && (p < 0 || p >= ny)) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const float etav = d.eta[k0 + v];
          const float gv = (p < 0) ? ((etav > 0.f) ? d.ghost[2] : 0.f) : ((etav < 0.f) ? d.ghost[3] : 0.f);
#pragma unroll
          for (int r = 0; r < R; ++r) c0[r][v] = gv;
        }
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) lds_vec<T, V>(srow + (s0 + dxs * r + H) * C + lane * V, c0[r]);
        if constexpr (XB) {
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const int g = x0 + s0 + dxs * r;
            if (g >= nx) {   // ragged tile: cells beyond the domain (never stored)
#pragma unroll
              for (int v = 0; v < V; ++v) c0[r][v] = 0.f;
            }
          }
        }
      }
      // ---- y face f + 1/2 with f = p - H, from the upwind cell of the face
      const int f = p - H;
      const bool do_face = (f >= ya - 1);
      float g[R][V];
      if constexpr (ORDER == 2) {
        float hmul = 0.5f;
        if (YB && !d.periodic_y) hmul = (f == -1 || f == ny - 1) ? 0.f : 0.5f;
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
          for (int v = 0; v < V; ++v) {
            const float db = c1[r][v] - c2[r][v];        // c_{f+1} - c_f
            const float dcv = c0[r][v] - c1[r][v];       // c_{f+2} - c_{f+1}
            const float qv = (eneg[v] != 0.f) ? dcv : dprev[r][v];
            const float gf = fmaf(eneg[v], db, c2[r][v]);
            const float hv = (eneg[v] != 0.f) ? -hmul : hmul;
            g[r][v] = do_face ? fmaf(hv, minmod_med(db, qv), gf) : gf;
            dprev[r][v] = db;
          }
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
          for (int v = 0; v < V; ++v) g[r][v] = fmaf(eneg[v], c0[r][v] - c1[r][v], c1[r][v]);
      }
      // ---- completion of row j = p - H (its slot, entry q - H, is still resident)
      const int j = p - H;
      if (j >= ya) {
        const T* jrow = reinterpret_cast<const T*>(ring + ((q - H) % NS) * L::slot_bytes);
        const T* sbase = reinterpret_cast<const T*>(ring + slot * L::slot_bytes + L::halo_bytes);
        const int rr = j - ya;
        float u[NL][V];
#pragma unroll
        for (int m = 0; m < NL; ++m) {
          const int pos = s0 + dxs * (m - H);   // tile-local cell of upwind index m - H
          lds_vec<T, V>(jrow + (pos + H) * C + lane * V, u[m]);
          if constexpr (XB) {
            const int gpos = x0 + pos;
            if (gpos < 0 || gpos >= nx) {
              if (d.periodic_x) {
                // periodic: the wrapped cell of the same row, from the input state
                lds_vec<T, V>(reinterpret_cast<const T*>(d.psi[in_buf]) + ((size_t)j * nx + wrap_index(gpos, nx)) * Mpad + k0,
                              u[m]);
              } else {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                  const float xiv = d.xi[k0 + v];
                  u[m][v] = (gpos < 0) ? ((xiv > 0.f) ? d.ghost[0] : 0.f) : ((xiv < 0.f) ? d.ghost[1] : 0.f);
                }
              }
            }
          }
        }
        // faces m = -1 .. R-1 along x (outgoing face of upwind cell m); first order on domain faces
        float F[R + 1][V];
#pragma unroll
        for (int m = -1; m < R; ++m) {
          float h = (ORDER == 2) ? 0.5f : 0.f;
          if constexpr (XB) {
            const int ga = x0 + s0 + dxs * m, gb = ga + dxs;
            if (!d.periodic_x && !((ga >= 0 && ga < nx) && (gb >= 0 && gb < nx))) h = 0.f;
          }
#pragma unroll
          for (int v = 0; v < V; ++v) {
            const float um = u[m + H][v];
            if constexpr (ORDER == 2) {
              const float dn = u[m + H + 1][v] - um, up = um - u[m + H - 1][v];
              F[m + 1][v] = fmaf(h, minmod_med(dn, up), um);
            } else {
              F[m + 1][v] = um;
            }
          }
        }
        float contrib[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int xl = s0 + dxs * r;
          const int gx = x0 + xl;
          const float ta = tile_a[rr * TX + xl], tb = tile_b[rr * TX + xl];
          float bse[V];
          if constexpr (STAGE == STAGE_HEUN2) lds_vec<T, V>(sbase + xl * C + lane * V, bse);
          const float(&cj)[V] = (ORDER == 2) ? c2[r] : c1[r];
          float out[V];
          float pw = 0.f;
#pragma unroll
          for (int v = 0; v < V; ++v) {
            const float dxv = ax[v] * (F[r + 1][v] - F[r][v]);
            const float div = fmaf(ay[v], g[r][v] - gprev[r][v], dxv);
            float t = fmaf(ta, cj[v], tb) - div;
            if constexpr (STAGE == STAGE_HEUN2) t = 0.5f * (bse[v] + t);
            if constexpr (sizeof(T) == 2)
              t = Store<T>::round_sr(t, sr_elem(sr_bits4((uint32_t)(j * nx + gx), gkey), (k0 + v) & 3));
            out[v] = t;
            pw = fmaf(w[v], t, pw);
          }
          contrib[r] = 0.f;
          if (!XB || gx < nx) {
            stg_vec<T, V>(psi_out + ((size_t)j * nx + gx) * Mpad + k0, out);
            contrib[r] = pw;
            if (XB || YB) {
              // boundary outflow of the output state (first-order traces)
#pragma unroll
              for (int v = 0; v < V; ++v) {
                const float o = out[v], xiv = d.xi[k0 + v], etav = d.eta[k0 + v];
                if (XB && !d.periodic_x && gx == 0) bacc += ly_f * (w[v] * -xiv * (xiv < 0.f ? o : (xiv > 0.f ? d.ghost[0] : 0.f)));
                if (XB && !d.periodic_x && gx == nx - 1) bacc += ly_f * (w[v] * xiv * (xiv > 0.f ? o : (xiv < 0.f ? d.ghost[1] : 0.f)));
                if (YB && !d.periodic_y && j == 0) bacc += lx_f * (w[v] * -etav * (etav < 0.f ? o : (etav > 0.f ? d.ghost[2] : 0.f)));
                if (YB && !d.periodic_y && j == ny - 1) bacc += lx_f * (w[v] * etav * (etav > 0.f ? o : (etav < 0.f ? d.ghost[3] : 0.f)));
              }
            }
          }
        }
        // phi partials in physical cell order, summed over the 32 lanes
        float phys[R];
#pragma unroll
        for (int r = 0; r < R; ++r) phys[r] = (dxs > 0) ? contrib[r] : contrib[R - 1 - r];
        const float sphi = multi_warp_sum<R>(phys, lane);
        if ((lane & (32 / R - 1)) == 0) tile_acc[rr * TX + xl0 + lane / (32 / R)] += sphi;
      }
      // every read of entry q - H (and of this row) is done, or a wait ran out
      if (__syncthreads_or(!ok)) {
        if (tid == 0) {
          for (int qq = q; qq < issued; ++qq) {
            if ((int64_t)qq == d.drop_load) continue;
            mbar_wait_bounded(&bars[qq % NS], (uint32_t)((qq / NS) & 1), limit);
          }
          atomicCAS(&st->status, DEV_OK, DEV_TIMEOUT);
          st->timeout_where = ((int64_t)blockIdx.x << 32) | (int64_t)q;
        }
        return;
      }
      // entry q - H is consumed: its slot takes entry q - H + NS
      if (tid == 0 && q >= H && issued < total) {
        fence_proxy_async_smem();
        issue(issued);
        ++issued;
      }
      // shift the window
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int v = 0; v < V; ++v) {
          gprev[r][v] = g[r][v];
          c2[r][v] = c1[r][v];
          c1[r][v] = c0[r][v];
        }
    }
  }
  __syncthreads();

  cart_epilogue<TX, STAGE>(d, it, phi_out, tile_acc, red, x0, ya, nrows, bacc);
}

// One row pull of the chunk-uniform tile: pull e (chunk c, row i of the chunk)
// into ring slot `slot`, completing full[slot]. Only tiles that touch the y
// sides of the domain (YB) pull rows outside it: the wrapped row on a periodic
// axis, else nothing (the ghost values are set in registers); interior tiles
// skip those tests, since the issuing thread is on the ring's critical path.
template <typename L, bool YB>
struct UniPull {
  const InstDesc* d;
  uint8_t* ring;
  uint64_t* full;
  int* slot_pull;   // [NS] last pull issued into each slot (read by the drain)
  const CUtensorMap* map_halo;
  const CUtensorMap* map_base;
  int x0, ya, yb;

  __device__ __forceinline__ void issue(int e, int c, int i, int slot) const {
    constexpr int H = L::H, C = L::C;
    const int dy = d->cdir_y[c];
    const int p = ((dy > 0) ? ya : yb - 1) + dy * (i - H);
    uint8_t* dst = ring + slot * L::slot_bytes;
    bool halo = true;
    int pl = p;
    if constexpr (YB) {
      if (p < 0 || p >= d->ny) {
        halo = d->periodic_y != 0;
        if (halo) pl = wrap_index(p, d->ny);
      }
    }
    const bool base = L::base_bytes > 0 && (i >= H + 1);   // Heun stage 2: psi^n of the row completed here
    const uint32_t bytes = (halo ? L::halo_bytes : 0) + (base ? L::base_bytes : 0);
    slot_pull[slot] = e;
    if ((int64_t)e == d->drop_load) return;   // test hook: that pull never completes
    if (bytes == 0) {
      mbar_arrive(&full[slot]);
      return;
    }
    mbar_arrive_expect_tx(&full[slot], bytes);
    if (halo) tma_load_3d(dst, map_halo, &full[slot], c * C, x0 - H, pl);
    if (base) tma_load_3d(dst + L::halo_bytes, map_base, &full[slot], c * C, x0, p - dy);
  }
};

// Chunk-uniform variant. When every chunk of C ordinates has one sign of xi and
// one of eta (the product quadrature's quadrants are contiguous, so its chunks
// are), the whole CTA shares the flow direction of a chunk. Each chunk then
// walks its rows along the flow in y (upwind row first): the face between two
// consecutive rows comes from the row already seen, so a row is completed one
// row after it arrives, and the window carries only the previous row, its
// difference to the row before, and the face value below it.
//
// Pipeline. Pull q of the tile (all chunks in order) lands in ring slot q mod NS
// and completes full[slot]. Pull q - 1 is needed until every warp has finished
// pull q; after the CTA barrier that closes row q, thread 0 issues pull
// q - 1 + NS into its slot. (Releasing slots per warp with shared-memory
// atomics or mbarrier arrivals, so that warps run apart, measured slower on
// sm_103a than this one barrier per row.) The waits are bounded; the barrier
// also carries a failed wait, so all warps stop together, drain the loads in
// flight and report the timeout.
// Register window of one row of the chunk-uniform tile, per lane: the row's
// values c, their difference to the row before along the flow d, and the face
// value g between the row before and this row.
template <int R, int V2>
struct UniRow {
  float2 c[R][V2], d[R][V2], g[R][V2];
};

template <int ORDER, int R, int V, int STAGE, typename T, bool XB, bool YB>
__device__ __forceinline__ void cart_tile_uni(const InstDesc& d, const WorkItem& it, InstState* st,
                                              uint8_t* smem) {
  using L = CartCfg<ORDER, R, V, STAGE, T>;
  constexpr int H = L::H, TX = L::TX, C = L::C, NS = L::NS, NL = L::NL;
  constexpr int V2 = V / 2;   // ordinate pairs per lane: arithmetic runs on float pairs
  static_assert(NS >= 3, "the ring must hold two resident rows plus one load in flight");
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  const int parity = (STAGE == STAGE_EULER) ? st->parity : 0;
  [[maybe_unused]] const uint32_t salt = sr_salt(st->step, STAGE);   // BF16 stochastic rounding
  const int in_buf = (STAGE == STAGE_EULER) ? parity : (STAGE == STAGE_HEUN1 ? 0 : 1);
  const int out_buf = (STAGE == STAGE_EULER) ? (1 - parity) : (STAGE == STAGE_HEUN1 ? 1 : 0);
  const float* __restrict__ phi_in = d.phi[in_buf];
  float* __restrict__ phi_out = d.phi[out_buf];
  T* __restrict__ psi_out = reinterpret_cast<T*>(d.psi[out_buf]);
  const CUtensorMap* map_halo = &d.tm_psi_halo[in_buf];
  const CUtensorMap* map_base = &d.tm_psi_center;

  const int nx = d.nx, ny = d.ny, Mpad = d.Mpad;
  const int x0 = it.a * TX;
  const int ya = it.b * d.ly;
  const int yb = min(ny, ya + d.ly);
  const int nrows = yb - ya;
  const int Lc = nrows + H + 1;     // rows pulled per chunk, in flow order: H before the tile, 1 after
  const int total = d.n_chunks * Lc;

  uint8_t* ring = smem;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::ring_bytes);
  int* slot_pull = reinterpret_cast<int*>(full + NS);   // [NS]
  float2* tile_ab = reinterpret_cast<float2*>(smem + L::ring_bytes + 128);   // (a, b) per cell
  float* tile_acc = reinterpret_cast<float*>(tile_ab + d.ly * TX);
  double* red = reinterpret_cast<double*>(smem + L::ring_bytes + 128 + cart_tile_bytes(TX, d.ly));
  const int64_t limit = d.wait_limit;
  static_assert(NS * (8 + 4) <= 128, "ring control block must fit its 128 bytes");
  const UniPull<L, YB> pull{&d, ring, full, slot_pull, map_halo, map_base, x0, ya, yb};

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      slot_pull[s] = -1;
    }
    fence_barrier_init();
    fence_tensormap_acquire(map_halo);
    prefetch_tensormap(map_halo);
    if (STAGE == STAGE_HEUN2) {
      fence_tensormap_acquire(map_base);
      prefetch_tensormap(map_base);
    }
  }
  __syncthreads();
  if (tid == 0) {
    for (int e = 0, c = 0, i = 0; e < min(NS, total); ++e) {
      pull.issue(e, c, i, e);
      if (++i == Lc) { i = 0; ++c; }
    }
  }
  const float dt = d.dt;
  for (int i = tid; i < nrows * TX; i += kCartThreads) {
    const int r = i / TX, xl = i - r * TX;
    const int gx = x0 + xl;
    float a = 1.f, b = 0.f;
    if (gx < nx) {
      const size_t cell = (size_t)(ya + r) * nx + gx;
      const int m = d.mat[cell];
      a = 1.f - dt * d.sig_t[m];
      b = dt * (d.sig_s2pi[m] * phi_in[cell] + d.q_src[m]);
    }
    tile_ab[i] = make_float2(a, b);
    tile_acc[i] = 0.f;
  }
  __syncthreads();

  float bacc = 0.f;
  const float ly_f = (float)d.dy_d, lx_f = (float)d.dx_d;
  const int xl0 = warp * R;
  bool ok = true;
  int q = 0;           // global pull index
  int slot = 0;        // ring slot of pull q
  uint32_t ph = 0;     // phase parity of full[slot] for pull q
  int pslot = NS - 1;  // ring slot of pull q - 1
  // chunk and row of pull q - 1 + NS, issued after row q (advanced once per pull from q = 1)
  int nc = 0, ni = NS;
  while (ni >= Lc) { ni -= Lc; ++nc; }

  for (int c = 0; c < d.n_chunks && ok; ++c) {
    auto chunk = [&](auto dir) {
      constexpr int DXS = decltype(dir)::value;   // sign of xi in this chunk
      const int k0 = c * C + lane * V;
      [[maybe_unused]] const uint32_t gkey = sr_gkey(k0 >> 2, salt);   // BF16 rounding: the lane's group of 4
      const int dys = d.cdir_y[c];
      const int s0 = (DXS > 0) ? xl0 : xl0 + R - 1;   // this warp's first cell along the flow
      float2 w2[V2], ax2[V2], ay2[V2];
#pragma unroll
      for (int v = 0; v < V2; ++v) {
        w2[v] = make_float2(d.w[k0 + 2 * v], d.w[k0 + 2 * v + 1]);
        ax2[v] = make_float2(dt * fabsf(d.xi[k0 + 2 * v]) * d.inv_dx, dt * fabsf(d.xi[k0 + 2 * v + 1]) * d.inv_dx);
        ay2[v] = make_float2(dt * fabsf(d.eta[k0 + 2 * v]) * d.inv_dy, dt * fabsf(d.eta[k0 + 2 * v + 1]) * d.inv_dy);
      }
      // psi^- of the rows before the tile in flow order (entering through that side)
      const float gy_up = (dys > 0) ? d.ghost[2] : d.ghost[3];
      const int start = (dys > 0) ? ya : yb - 1;
      // lane's element of cell position s0 within a slot, in bytes
      const int lofs = ((s0 + H) * C + lane * V) * (int)sizeof(T);
      constexpr int PSTEP = DXS * C * (int)sizeof(T);   // next cell along the flow
      // output row pointer (row `start`, cell s0) and its step per completed row
      T* op = psi_out + ((size_t)start * nx + (x0 + s0)) * Mpad + k0;
      const ptrdiff_t ostep = (ptrdiff_t)dys * nx * Mpad;
      const ptrdiff_t mstep = (ptrdiff_t)DXS * Mpad;
      const float2* tab = tile_ab + (start - ya) * TX + s0;
      const int tstep = dys * TX;
      float* tacc = tile_acc + (start - ya) * TX + xl0 + lane / (32 / R);
      int jrow = start;    // row completed next
      int p = start - dys * H;

      // Row i of the chunk (row p of the grid) into window X; Y holds the row
      // before it, which is completed here. The two windows swap roles from row
      // to row, so no register is copied.
      auto row = [&](const int i, UniRow<R, V2>& X, const UniRow<R, V2>& Y) -> bool {
        const bool wok = mbar_wait_bounded(&full[slot], ph, limit);
        const uint8_t* cur = ring + slot * L::slot_bytes + lofs;
        bool p_in = true;
        if constexpr (YB) p_in = d.periodic_y || (p >= 0 && p < ny);
        if (YB && !p_in) {
          const float gv = (i < H) ? gy_up : 0.f;   // after the tile only the first-order face sees it
#pragma unroll
          for (int r = 0; r < R; ++r)
#pragma unroll
            for (int v = 0; v < V2; ++v) X.c[r][v] = make_float2(gv, gv);
        } else {
#pragma unroll
          for (int r = 0; r < R; ++r) lds_vec2<T, V>(reinterpret_cast<const T*>(cur + r * PSTEP), X.c[r]);
        }
        // face between the previous row (upwind) and row p
        if constexpr (ORDER == 2) {
          bool second = true;
          if constexpr (YB) {
            const int pp = p - dys;
            if (!d.periodic_y && (pp >= 0 && pp < ny) != p_in) second = false;   // domain boundary face: first order
          }
#pragma unroll
          for (int r = 0; r < R; ++r)
#pragma unroll
            for (int v = 0; v < V2; ++v) {
              X.d[r][v] = sub2(X.c[r][v], Y.c[r][v]);
              const float2 ext = __ffma2_rn(make_float2(0.5f, 0.5f),
                                            minmod2r(X.d[r][v], Y.d[r][v], relu2(X.d[r][v]), relu2(Y.d[r][v])), Y.c[r][v]);
              X.g[r][v] = (!YB || second) ? ext : Y.c[r][v];
            }
        } else {
#pragma unroll
          for (int r = 0; r < R; ++r)
#pragma unroll
            for (int v = 0; v < V2; ++v) X.g[r][v] = Y.c[r][v];
        }
        // completion of the previous row (its slot, pull q - 1, is still resident)
        if (i >= H + 1) {
          const uint8_t* prv = ring + pslot * L::slot_bytes + lofs;
          float2 u[NL][V2];
#pragma unroll
          for (int m = 0; m < NL; ++m) {
            if (m >= H && m < H + R) {
              // the warp's own cells of the previous row are still in the window (loaded one row ago)
#pragma unroll
              for (int v = 0; v < V2; ++v) u[m][v] = Y.c[m - H][v];
            } else {
              lds_vec2<T, V>(reinterpret_cast<const T*>(prv + (m - H) * PSTEP), u[m]);
            }
            if constexpr (XB) {
              const int gpos = x0 + s0 + DXS * (m - H);
              if (gpos < 0 || gpos >= nx) {
                if (d.periodic_x) {
                  // periodic: the wrapped cell of the same row, from the input state
                  lds_vec2<T, V>(reinterpret_cast<const T*>(d.psi[in_buf]) + ((size_t)jrow * nx + wrap_index(gpos, nx)) * Mpad + k0,
                                 u[m]);
                } else {
                  // entering ordinates see psi^- of the side, leaving ones nothing (only
                  // first-order faces read it)
                  const float gside = (gpos < 0) ? d.ghost[0] : d.ghost[1];
                  const bool enter = (gpos < 0) == (DXS > 0);
#pragma unroll
                  for (int v = 0; v < V2; ++v) u[m][v] = enter ? make_float2(gside, gside) : make_float2(0.f, 0.f);
                }
              }
            }
          }
          // faces m = -1 .. R-1 along x (outgoing face of upwind cell m); first order on domain faces
          float2 F[R + 1][V2];
          if constexpr (ORDER == 2) {
            float2 D[NL][V2], RD[NL][V2];   // D[m] = u[m] - u[m-1], RD = max(D, 0)
#pragma unroll
            for (int m = 1; m < NL; ++m)
#pragma unroll
              for (int v = 0; v < V2; ++v) {
                D[m][v] = sub2(u[m][v], u[m - 1][v]);
                RD[m][v] = relu2(D[m][v]);
              }
#pragma unroll
            for (int m = -1; m < R; ++m) {
              bool second = true;
              if constexpr (XB) {
                const int ga = x0 + s0 + DXS * m, gb = ga + DXS;
                if (!d.periodic_x && !((ga >= 0 && ga < nx) && (gb >= 0 && gb < nx))) second = false;
              }
#pragma unroll
              for (int v = 0; v < V2; ++v)
                F[m + 1][v] = second ? __ffma2_rn(make_float2(0.5f, 0.5f),
                                                  minmod2r(D[m + H + 1][v], D[m + H][v], RD[m + H + 1][v], RD[m + H][v]),
                                                  u[m + H][v])
                                     : u[m + H][v];
            }
          } else {
#pragma unroll
            for (int m = -1; m < R; ++m)
#pragma unroll
              for (int v = 0; v < V2; ++v) F[m + 1][v] = u[m + H][v];
          }
          float contrib[R];
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const float2 ab = tab[DXS * r];
            const float2 ta2 = make_float2(ab.x, ab.x), tb2 = make_float2(ab.y, ab.y);
            [[maybe_unused]] float2 bse[V2];
            if constexpr (STAGE == STAGE_HEUN2)
              lds_vec2<T, V>(reinterpret_cast<const T*>(cur - H * C * (int)sizeof(T) + L::halo_bytes + r * PSTEP), bse);
            float2 out[V2];
            float2 pw2 = make_float2(0.f, 0.f);
            [[maybe_unused]] uint2 rb4;
            if constexpr (sizeof(T) == 2) rb4 = sr_bits4((uint32_t)(jrow * nx + (x0 + s0 + DXS * r)), gkey);
#pragma unroll
            for (int v = 0; v < V2; ++v) {
              const float2 div = __ffma2_rn(ax2[v], sub2(F[r + 1][v], F[r][v]), __fmul2_rn(ay2[v], sub2(X.g[r][v], Y.g[r][v])));
              float2 t = sub2(__ffma2_rn(ta2, Y.c[r][v], tb2), div);
              if constexpr (STAGE == STAGE_HEUN2) t = __fmul2_rn(make_float2(0.5f, 0.5f), __fadd2_rn(bse[v], t));
              if constexpr (sizeof(T) == 2) t = Store<T>::round_sr2(t, ((k0 + 2 * v) & 2) ? rb4.y : rb4.x);
              out[v] = t;
              pw2 = __ffma2_rn(w2[v], t, pw2);
            }
            contrib[r] = 0.f;
            const int gx = x0 + s0 + DXS * r;
            if (!XB || gx < nx) {
              stg_vec2<T, V>(op + r * mstep, out);
              contrib[r] = pw2.x + pw2.y;
              if (XB || YB) {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                  const float o = (v & 1) ? out[v / 2].y : out[v / 2].x;
                  const float wv = (v & 1) ? w2[v / 2].y : w2[v / 2].x;
                  const float xiv = d.xi[k0 + v], etav = d.eta[k0 + v];
                  if (XB && !d.periodic_x && gx == 0) bacc += ly_f * (wv * -xiv * (xiv < 0.f ? o : (xiv > 0.f ? d.ghost[0] : 0.f)));
                  if (XB && !d.periodic_x && gx == nx - 1) bacc += ly_f * (wv * xiv * (xiv > 0.f ? o : (xiv < 0.f ? d.ghost[1] : 0.f)));
                  if (YB && !d.periodic_y && jrow == 0) bacc += lx_f * (wv * -etav * (etav < 0.f ? o : (etav > 0.f ? d.ghost[2] : 0.f)));
                  if (YB && !d.periodic_y && jrow == ny - 1) bacc += lx_f * (wv * etav * (etav > 0.f ? o : (etav < 0.f ? d.ghost[3] : 0.f)));
                }
              }
            }
          }
          float phys[R];
#pragma unroll
          for (int r = 0; r < R; ++r) phys[r] = (DXS > 0) ? contrib[r] : contrib[R - 1 - r];
          const float sphi = multi_warp_sum<R>(phys, lane);
          if ((lane & (32 / R - 1)) == 0) *tacc += sphi;
          op += ostep;
          tab += tstep;
          tacc += tstep;
          jrow += dys;
        }
        if (__syncthreads_or(!wok)) return false;   // a wait ran out somewhere: every warp stops here
        if (tid == 0 && q >= 1 && q - 1 + NS < total) {
          fence_proxy_async_smem();
          pull.issue(q - 1 + NS, nc, ni, pslot);
        }
        if (q >= 1 && ++ni == Lc) { ni = 0; ++nc; }
        pslot = slot;
        if (++slot == NS) { slot = 0; ph ^= 1u; }
        ++q;
        p += dys;
        return true;
      };

      UniRow<R, V2> A, B;
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int v = 0; v < V2; ++v) B.c[r][v] = B.d[r][v] = B.g[r][v] = make_float2(0.f, 0.f);
      for (int i = 0; i < Lc; i += 2) {
        if (!row(i, A, B)) { ok = false; break; }
        if (i + 1 < Lc && !row(i + 1, B, A)) { ok = false; break; }
      }
    };
    if (d.cdir_x[c] > 0) chunk(std::integral_constant<int, 1>{});
    else chunk(std::integral_constant<int, -1>{});
  }
  __syncthreads();
  if (!ok) {
    if (tid == 0) {
      // drain: the last pull issued into each slot may still be in flight
      for (int s = 0; s < NS; ++s) {
        const int e = slot_pull[s];
        if (e < 0 || (int64_t)e == d.drop_load) continue;
        mbar_wait_bounded(&full[s], (uint32_t)((e / NS) & 1), limit);
      }
      atomicCAS(&st->status, DEV_OK, DEV_TIMEOUT);
      st->timeout_where = ((int64_t)blockIdx.x << 32) | (int64_t)q;
    }
    return;
  }
  cart_epilogue<TX, STAGE>(d, it, phi_out, tile_acc, red, x0, ya, nrows, bacc);
}

template <int ORDER, int R, int V, int STAGE, typename T, bool XB, bool YB>
__device__ __noinline__ void cart_tile_uni_edge(const InstDesc* dp, const WorkItem it, InstState* st, uint8_t* smem) {
  cart_tile_uni<ORDER, R, V, STAGE, T, XB, YB>(*dp, it, st, smem);
}

template <int ORDER, int R, int V, int STAGE, typename T, bool UNI>
__global__ void __launch_bounds__(kCartThreads, (R * V >= 8 ? 2 : 3))
    cart_stage_kernel(const InstDesc* __restrict__ descs, const WorkItem* __restrict__ items) {
  using L = CartCfg<ORDER, R, V, STAGE, T>;
  const WorkItem it = items[blockIdx.x];
  const InstDesc& d = descs[it.inst];
  InstState* st = d.st;
  // finished or failed instances are masked
  if (st->step >= d.n_steps || st->status != DEV_OK) return;
  extern __shared__ __align__(128) uint8_t smem_raw[];
  // TMA destinations want 128-byte alignment; the launch adds 128 bytes of slack
  uint8_t* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  const int x0 = it.a * L::TX;
  const int ya = it.b * d.ly;
  const bool xb = (x0 - L::H < 0) || (x0 + L::TX + L::H > d.nx);
  const bool yb = (ya - L::H < 0) || (ya + d.ly + L::H > d.ny);
  if constexpr (UNI) {
    // tiles on the domain boundary run out of line, so that their extra state
    // (ghost values, wrapped rows and cells) does not raise the register
    // pressure of the interior tiles
    if (xb) {
      if (yb) cart_tile_uni_edge<ORDER, R, V, STAGE, T, true, true>(&d, it, st, smem);
      else cart_tile_uni_edge<ORDER, R, V, STAGE, T, true, false>(&d, it, st, smem);
    } else {
      if (yb) cart_tile_uni_edge<ORDER, R, V, STAGE, T, false, true>(&d, it, st, smem);
      else cart_tile_uni<ORDER, R, V, STAGE, T, false, false>(d, it, st, smem);
    }
  } else {
    if (xb) cart_tile<ORDER, R, V, STAGE, T, true>(d, it, st, smem, yb);
    else cart_tile<ORDER, R, V, STAGE, T, false>(d, it, st, smem, yb);
  }
}

template <int ORDER, int R, int V, int STAGE, typename T, bool UNI>
static cudaError_t prepare_one(int ly_max) {
  // Raise the dynamic shared-memory limit of this kernel variant. The attribute
  // belongs to the current device, so the limit already raised is kept per
  // device (atomics: callers on several host threads may race here; setting
  // the attribute twice is harmless).
  constexpr int kDev = 64;
  static std::atomic<size_t> s_limit[kDev];
  const size_t smem = cart_smem_for<ORDER, R, V, STAGE, T>(ly_max);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const bool tracked = dev >= 0 && dev < kDev;
  if (tracked && smem <= s_limit[dev].load(std::memory_order_acquire)) return cudaSuccess;
  e = cudaFuncSetAttribute(cart_stage_kernel<ORDER, R, V, STAGE, T, UNI>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (tracked) {
    size_t cur = s_limit[dev].load(std::memory_order_relaxed);
    while (cur < smem && !s_limit[dev].compare_exchange_weak(cur, smem, std::memory_order_release)) {
    }
  }
  return cudaSuccess;
}

template <int ORDER, int R, int V, int STAGE, typename T, bool UNI>
static cudaError_t launch_one(const InstDesc* d_desc, const WorkItem* d_items, int n_items, int ly_max,
                              cudaStream_t stream) {
  cudaError_t e = prepare_one<ORDER, R, V, STAGE, T, UNI>(ly_max);
  if (e != cudaSuccess) return e;
  cart_stage_kernel<ORDER, R, V, STAGE, T, UNI>
      <<<n_items, kCartThreads, cart_smem_for<ORDER, R, V, STAGE, T>(ly_max), stream>>>(d_desc, d_items);
  return cudaGetLastError();
}

// Instantiation units: per storage type T and direction family U, the variants
// order {1, 2} x (run length R, ordinates per lane V) x stage, with (R, V) in
// {(2, 1), (2, 2), (2, 4)} for U = false and {(2, 2), (2, 4), (4, 2)} for U = true.
#define RTK_CART_STAGES(X, O, RR, VV, U, TT) \
  X(O, RR, VV, STAGE_EULER, U, TT) X(O, RR, VV, STAGE_HEUN1, U, TT) X(O, RR, VV, STAGE_HEUN2, U, TT)
#define RTK_CART_DEFINE_UNIT(NAME, TT, U, ...)                                                              \
  cudaError_t cart_prepare_##NAME(int stage, int order, int run, int vec, int ly_max) {                      \
    RTK_CART_UNIT_LIST(RTK_CART_P_, TT, U)                                                                  \
    return cudaErrorInvalidValue;                                                                           \
  }                                                                                                         \
  cudaError_t cart_launch_##NAME(const InstDesc* d_desc, const WorkItem* d_items, int n_items, int stage,   \
                                 int order, int run, int vec, int ly_max, cudaStream_t stream) {            \
    RTK_CART_UNIT_LIST(RTK_CART_L_, TT, U)                                                                  \
    return cudaErrorInvalidValue;                                                                           \
  }
#define RTK_CART_P_(O, RR, VV, ST, U, TT) \
  if (order == O && run == RR && vec == VV && stage == ST) return prepare_one<O, RR, VV, ST, TT, U>(ly_max);
#define RTK_CART_L_(O, RR, VV, ST, U, TT)                                  \
  if (order == O && run == RR && vec == VV && stage == ST)                 \
    return launch_one<O, RR, VV, ST, TT, U>(d_desc, d_items, n_items, ly_max, stream);

}  // namespace rtk
