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
    const bool halo = (p >= 0 && p < ny);
    const bool base = (STAGE == STAGE_HEUN2) && (p - H >= ya);
    const uint32_t bytes = (halo ? L::halo_bytes : 0) + (base ? L::base_bytes : 0);
    if ((int64_t)q == d.drop_load) return;   // test hook: this slot never completes
    if (bytes == 0) {
      mbar_arrive(&bars[slot]);
      return;
    }
    mbar_arrive_expect_tx(&bars[slot], bytes);
    if (halo) tma_load_3d(dst, map_halo, &bars[slot], c * C, x0 - H, p);
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
      if (YB && (p < 0 || p >= ny)) {
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
        if (YB) hmul = (f == -1 || f == ny - 1) ? 0.f : 0.5f;
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
#pragma unroll
              for (int v = 0; v < V; ++v) {
                const float xiv = d.xi[k0 + v];
                u[m][v] = (gpos < 0) ? ((xiv > 0.f) ? d.ghost[0] : 0.f) : ((xiv < 0.f) ? d.ghost[1] : 0.f);
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
            if (!((ga >= 0 && ga < nx) && (gb >= 0 && gb < nx))) h = 0.f;
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
            t = Store<T>::round(t);
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
                if (XB && gx == 0) bacc += ly_f * (w[v] * -xiv * (xiv < 0.f ? o : (xiv > 0.f ? d.ghost[0] : 0.f)));
                if (XB && gx == nx - 1) bacc += ly_f * (w[v] * xiv * (xiv > 0.f ? o : (xiv < 0.f ? d.ghost[1] : 0.f)));
                if (YB && j == 0) bacc += lx_f * (w[v] * -etav * (etav < 0.f ? o : (etav > 0.f ? d.ghost[2] : 0.f)));
                if (YB && j == ny - 1) bacc += lx_f * (w[v] * etav * (etav > 0.f ? o : (etav < 0.f ? d.ghost[3] : 0.f)));
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

// Chunk-uniform variant. When every chunk of C ordinates has one sign of xi and
// one of eta (the product quadrature's quadrants are contiguous, so its chunks
// are), the whole CTA shares the flow direction of a chunk. Each chunk then
// walks its rows along the flow in y (upwind row first): the face between two
// consecutive rows comes from the row already seen, so a row is completed one
// row after it arrives, and the window carries only the previous row, its
// difference to the row before, and the face value below it.
template <int ORDER, int R, int V, int STAGE, typename T, bool XB>
__device__ __forceinline__ void cart_tile_uni(const InstDesc& d, const WorkItem& it, InstState* st,
                                              uint8_t* smem, const bool YB) {
  using L = CartCfg<ORDER, R, V, STAGE, T>;
  constexpr int H = L::H, TX = L::TX, C = L::C, NS = L::NS, NL = L::NL;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  const int parity = (STAGE == STAGE_EULER) ? st->parity : 0;
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
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::ring_bytes);
  float* tile_a = reinterpret_cast<float*>(smem + L::ring_bytes + 128);
  float* tile_b = tile_a + d.ly * TX;
  float* tile_acc = tile_b + d.ly * TX;
  double* red = reinterpret_cast<double*>(smem + L::ring_bytes + 128 + cart_tile_bytes(TX, d.ly));
  const int64_t limit = d.wait_limit;

  // row of pull i of chunk c: the tile rows in flow order, with H rows before and one after
  auto pull_row = [&](int c, int i) {
    const int dy = d.cdir_y[c];
    return ((dy > 0) ? ya : yb - 1) + dy * (i - H);
  };
  auto issue = [&](int q) {
    const int slot = q % NS;
    const int c = q / Lc;
    const int i = q - c * Lc;
    const int p = pull_row(c, i);
    uint8_t* dst = ring + slot * L::slot_bytes;
    const bool halo = (p >= 0 && p < ny);
    const bool base = (STAGE == STAGE_HEUN2) && (i >= H + 1);   // the row completed at this pull
    const uint32_t bytes = (halo ? L::halo_bytes : 0) + (base ? L::base_bytes : 0);
    if ((int64_t)q == d.drop_load) return;   // test hook: this slot never completes
    if (bytes == 0) {
      mbar_arrive(&bars[slot]);
      return;
    }
    mbar_arrive_expect_tx(&bars[slot], bytes);
    if (halo) tma_load_3d(dst, map_halo, &bars[slot], c * C, x0 - H, p);
    if (base) tma_load_3d(dst + L::halo_bytes, map_base, &bars[slot], c * C, x0, p - d.cdir_y[c]);
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

  float bacc = 0.f;
  const float ly_f = (float)d.dy_d, lx_f = (float)d.dx_d;
  const int xl0 = warp * R;
  static_assert(NS >= 3, "the ring must hold two resident rows plus one load in flight");

  int q = 0;
  int issued = min(NS, total);
  for (int c = 0; c < d.n_chunks; ++c) {
    const int k0 = c * C + lane * V;
    const int dxs = d.cdir_x[c], dys = d.cdir_y[c];     // uniform over the CTA
    const int s0 = (dxs > 0) ? xl0 : xl0 + R - 1;
    float w[V], ax[V], ay[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      w[v] = d.w[k0 + v];
      ax[v] = dt * fabsf(d.xi[k0 + v]) * d.inv_dx;
      ay[v] = dt * fabsf(d.eta[k0 + v]) * d.inv_dy;
    }
    // psi^- of the rows before the tile in flow order (entering through that side)
    const float gy_up = (dys > 0) ? d.ghost[2] : d.ghost[3];
    const int start = (dys > 0) ? ya : yb - 1;
    float cm1[R][V], dprev[R][V], gprev[R][V];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int v = 0; v < V; ++v) cm1[r][v] = dprev[r][v] = gprev[r][v] = 0.f;

    for (int i = 0; i < Lc; ++i, ++q) {
      const int p = start + dys * (i - H);
      const int slot = q % NS;
      const uint32_t par = (uint32_t)((q / NS) & 1);
      const bool ok = mbar_wait_bounded(&bars[slot], par, limit);
      const T* srow = reinterpret_cast<const T*>(ring + slot * L::slot_bytes);
      float c0[R][V];
      const bool p_in = (p >= 0 && p < ny);
      if (YB && !p_in) {
        const float gv = (i < H) ? gy_up : 0.f;   // after the tile only the first-order face sees it
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
          for (int v = 0; v < V; ++v) c0[r][v] = gv;
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) lds_vec<T, V>(srow + (s0 + dxs * r + H) * C + lane * V, c0[r]);
      }
      // face between the previous row (upwind) and row p
      float g[R][V];
      if constexpr (ORDER == 2) {
        float h = 0.5f;
        if (YB) {
          const int pp = p - dys;
          const bool in_prev = (pp >= 0 && pp < ny);
          if (in_prev != p_in) h = 0.f;   // domain boundary face: first order
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
          for (int v = 0; v < V; ++v) {
            const float dn = c0[r][v] - cm1[r][v];
            g[r][v] = fmaf(h, minmod_med(dn, dprev[r][v]), cm1[r][v]);
            dprev[r][v] = dn;
          }
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
          for (int v = 0; v < V; ++v) g[r][v] = cm1[r][v];
      }
      // completion of the previous row j (its slot, entry q - 1, is still resident)
      if (i >= H + 1) {
        const int j = p - dys;
        const int rr = j - ya;
        const T* jrow = reinterpret_cast<const T*>(ring + ((q - 1) % NS) * L::slot_bytes);
        const T* sbase = reinterpret_cast<const T*>(ring + slot * L::slot_bytes + L::halo_bytes);
        float u[NL][V];
#pragma unroll
        for (int m = 0; m < NL; ++m) {
          const int pos = s0 + dxs * (m - H);
          lds_vec<T, V>(jrow + (pos + H) * C + lane * V, u[m]);
          if constexpr (XB) {
            const int gpos = x0 + pos;
            if (gpos < 0 || gpos >= nx) {
#pragma unroll
              for (int v = 0; v < V; ++v) {
                const float xiv = d.xi[k0 + v];
                u[m][v] = (gpos < 0) ? ((xiv > 0.f) ? d.ghost[0] : 0.f) : ((xiv < 0.f) ? d.ghost[1] : 0.f);
              }
            }
          }
        }
        float F[R + 1][V];
#pragma unroll
        for (int m = -1; m < R; ++m) {
          float hx = (ORDER == 2) ? 0.5f : 0.f;
          if constexpr (XB) {
            const int ga = x0 + s0 + dxs * m, gb = ga + dxs;
            if (!((ga >= 0 && ga < nx) && (gb >= 0 && gb < nx))) hx = 0.f;
          }
#pragma unroll
          for (int v = 0; v < V; ++v) {
            const float um = u[m + H][v];
            if constexpr (ORDER == 2) {
              F[m + 1][v] = fmaf(hx, minmod_med(u[m + H + 1][v] - um, um - u[m + H - 1][v]), um);
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
          float out[V];
          float pw = 0.f;
#pragma unroll
          for (int v = 0; v < V; ++v) {
            const float div = fmaf(ax[v], F[r + 1][v] - F[r][v], ay[v] * (g[r][v] - gprev[r][v]));
            float t = fmaf(ta, cm1[r][v], tb) - div;
            if constexpr (STAGE == STAGE_HEUN2) t = 0.5f * (bse[v] + t);
            t = Store<T>::round(t);
            out[v] = t;
            pw = fmaf(w[v], t, pw);
          }
          contrib[r] = 0.f;
          if (!XB || gx < nx) {
            stg_vec<T, V>(psi_out + ((size_t)j * nx + gx) * Mpad + k0, out);
            contrib[r] = pw;
            if (XB || YB) {
#pragma unroll
              for (int v = 0; v < V; ++v) {
                const float o = out[v], xiv = d.xi[k0 + v], etav = d.eta[k0 + v];
                if (XB && gx == 0) bacc += ly_f * (w[v] * -xiv * (xiv < 0.f ? o : (xiv > 0.f ? d.ghost[0] : 0.f)));
                if (XB && gx == nx - 1) bacc += ly_f * (w[v] * xiv * (xiv > 0.f ? o : (xiv < 0.f ? d.ghost[1] : 0.f)));
                if (YB && j == 0) bacc += lx_f * (w[v] * -etav * (etav < 0.f ? o : (etav > 0.f ? d.ghost[2] : 0.f)));
                if (YB && j == ny - 1) bacc += lx_f * (w[v] * etav * (etav > 0.f ? o : (etav < 0.f ? d.ghost[3] : 0.f)));
              }
            }
          }
        }
        float phys[R];
#pragma unroll
        for (int r = 0; r < R; ++r) phys[r] = (dxs > 0) ? contrib[r] : contrib[R - 1 - r];
        const float sphi = multi_warp_sum<R>(phys, lane);
        if ((lane & (32 / R - 1)) == 0) tile_acc[rr * TX + xl0 + lane / (32 / R)] += sphi;
      }
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
      // entry q - 1 is consumed: its slot takes entry q - 1 + NS
      if (tid == 0 && q >= 1 && issued < total) {
        fence_proxy_async_smem();
        issue(issued);
        ++issued;
      }
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int v = 0; v < V; ++v) {
          gprev[r][v] = g[r][v];
          cm1[r][v] = c0[r][v];
        }
    }
  }
  __syncthreads();
  cart_epilogue<TX, STAGE>(d, it, phi_out, tile_acc, red, x0, ya, nrows, bacc);
}

template <int ORDER, int R, int V, int STAGE, typename T, bool UNI>
__global__ void __launch_bounds__(kCartThreads, 2)
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
    if (xb) cart_tile_uni<ORDER, R, V, STAGE, T, true>(d, it, st, smem, yb);
    else cart_tile_uni<ORDER, R, V, STAGE, T, false>(d, it, st, smem, yb);
  } else {
    if (xb) cart_tile<ORDER, R, V, STAGE, T, true>(d, it, st, smem, yb);
    else cart_tile<ORDER, R, V, STAGE, T, false>(d, it, st, smem, yb);
  }
}

template <int ORDER, int R, int V, int STAGE, typename T, bool UNI>
static cudaError_t prepare_one(int ly_max) {
  // raise the dynamic shared-memory limit of this kernel variant (idempotent)
  static size_t s_limit = 0;
  const size_t smem = cart_smem_for<ORDER, R, V, STAGE, T>(ly_max);
  if (smem > s_limit) {
    cudaError_t e = cudaFuncSetAttribute(cart_stage_kernel<ORDER, R, V, STAGE, T, UNI>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    s_limit = smem;
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
// order {1, 2} x run length 2 x ordinates per lane V (U = false: V = 1, 2, 4;
// U = true: V = 2, 4) x stage.
#define RTK_CART_STAGES(X, O, VV, U, TT) X(O, VV, STAGE_EULER, U, TT) X(O, VV, STAGE_HEUN1, U, TT) X(O, VV, STAGE_HEUN2, U, TT)
#define RTK_CART_DEFINE_UNIT(NAME, TT, U, ...)                                                              \
  cudaError_t cart_prepare_##NAME(int stage, int order, int vec, int ly_max) {                               \
    RTK_CART_UNIT_LIST(RTK_CART_P_, TT, U)                                                                  \
    return cudaErrorInvalidValue;                                                                           \
  }                                                                                                         \
  cudaError_t cart_launch_##NAME(const InstDesc* d_desc, const WorkItem* d_items, int n_items, int stage,   \
                                 int order, int vec, int ly_max, cudaStream_t stream) {                     \
    RTK_CART_UNIT_LIST(RTK_CART_L_, TT, U)                                                                  \
    return cudaErrorInvalidValue;                                                                           \
  }
#define RTK_CART_P_(O, VV, ST, U, TT) \
  if (order == O && vec == VV && stage == ST) return prepare_one<O, 2, VV, ST, TT, U>(ly_max);
#define RTK_CART_L_(O, VV, ST, U, TT) \
  if (order == O && vec == VV && stage == ST) return launch_one<O, 2, VV, ST, TT, U>(d_desc, d_items, n_items, ly_max, stream);

}  // namespace rtk
