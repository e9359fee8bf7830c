// Cartesian stage kernel of the explicit S_N step (Sec. 4.2-4.3).
//
// One CTA owns a tile of TX cells in x (a strip) by `ly` rows in y (a segment)
// and loops over the ordinate chunks of 32 ordinates (lane = ordinate). For
// each chunk it walks the tile's rows in +y: every row (TX + 2H cells x 32
// ordinates, H = halo = order) arrives by one TMA box load into a ring of
// NS shared-memory slots guarded by mbarriers. When row p arrives each thread
//   - pulls its cells' values of row p into a register window in y,
//   - evaluates the x part of the upwind flux divergence of row p from the
//     shared row (MUSCL-minmod or first order, boundary faces first order),
// then the slot is released and the row p - H is completed from registers:
//   F = -(div_x + div_y) - sigma_t psi + sigma_s/(2 pi) phi + Q   (Eq. sn_2d_eqn_fv)
//   Euler / Heun stage 1: out = psi + dt F;  Heun stage 2: out = (psi^n + psi1 + dt F)/2
// and stored with coalesced 128-byte rows. phi_out = sum_k w_k out_k is
// accumulated per cell in shared memory, chunk after chunk (fixed order, no
// atomics). The epilogue writes phi_out and the FP64 QoI partials (absorption
// per region, mass, boundary outflow) of the output state; the last CTA of the
// instance reduces them and applies the time-integration weights.
//
// Upwind coordinates: for an ordinate with direction sign d along an axis the
// stencil is u2 = psi_{i-2d}, u1 = psi_{i-d}, c = psi_i, d1 = psi_{i+d}; the
// outgoing face carries c + minmod(d1 - c, c - u1)/2 and the incoming face
// u1 + minmod(c - u1, u1 - u2)/2, so div = |v|/h (F_out - F_in). Cells beyond
// the domain hold the ghost value psi^- of that side (Sec. 4.2); faces on the
// boundary are first order.
#include <cuda_bf16.h>

#include "device_common.cuh"

namespace rtk {

constexpr int kCartThreads = 256;
constexpr int kCartWarps = kCartThreads / 32;
constexpr int kSlots = 6;

template <int H, int TX, int STAGE, typename T>
struct CartLayout {
  static constexpr int halo_bytes = (TX + 2 * H) * kChunk * (int)sizeof(T);
  static constexpr int base_bytes = (STAGE == STAGE_HEUN2) ? TX * kChunk * (int)sizeof(T) : 0;
  static constexpr int slot_bytes = ((halo_bytes + base_bytes) + 127) / 128 * 128;
  static constexpr int ring_bytes = kSlots * slot_bytes;
};

__host__ __device__ inline size_t cart_tile_bytes(int tx, int ly) {
  // phi_in [ly][tx] float, phi_acc [ly][tx] float, mat [ly][tx] uint8 (padded)
  return (size_t)ly * tx * 8 + (((size_t)ly * tx + 127) / 128 * 128);
}

// barriers (128) + FP64 reduction rows ((warps + 1) x NQ) + material table + alignment slack
constexpr size_t kCartRedBytes = (kCartWarps + 1) * NQ * 8;
constexpr size_t kCartFixedBytes = 128 + kCartRedBytes + 3 * kMaxMat * 4 + 128;

template <int ORDER, int TX, int STAGE, typename T>
__global__ void __launch_bounds__(kCartThreads)
    cart_stage_kernel(const InstDesc* __restrict__ descs, const WorkItem* __restrict__ items) {
  constexpr int H = ORDER;
  constexpr int CPW = TX / kCartWarps;   // cells per warp in a row
  constexpr int WIN = 2 * H + 1;         // y window: rows j-H .. j+H
  using L = CartLayout<H, TX, STAGE, T>;
  static_assert(CPW == 4 || CPW == 8, "TX must be 32 or 64");

  const WorkItem it = items[blockIdx.x];
  const InstDesc& d = descs[it.inst];
  InstState* st = d.st;
  // finished or failed instances are masked
  if (st->step >= d.n_steps || st->status != DEV_OK) return;

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
  const int Lc = nrows + 2 * H;                 // pulled rows per chunk: ya-H .. yb+H-1
  const int total = d.n_chunks * Lc;

  extern __shared__ __align__(128) uint8_t smem_raw[];
  // TMA destinations want 128-byte alignment; the launch adds 128 bytes of slack
  uint8_t* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  uint8_t* ring = smem;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::ring_bytes);            // kSlots + 1
  float* tile_phi = reinterpret_cast<float*>(smem + L::ring_bytes + 128);         // [ly][TX]
  float* tile_acc = tile_phi + d.ly * TX;                                           // [ly][TX]
  uint8_t* tile_mat = reinterpret_cast<uint8_t*>(tile_acc + d.ly * TX);            // [ly][TX]
  double* red = reinterpret_cast<double*>(smem + L::ring_bytes + 128 + cart_tile_bytes(TX, d.ly));
  float* mtab = reinterpret_cast<float*>(red + (kCartWarps + 1) * NQ);              // sig_t, sig_s2pi, q

  const int64_t limit = d.wait_limit;

  // ---- producer: issue the loads of sequence entry q into slot q % kSlots
  auto issue = [&](int q) {
    const int slot = q % kSlots;
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
    if (halo) tma_load_3d(dst, map_halo, &bars[slot], c * kChunk, x0 - H, p);
    if (base) tma_load_3d(dst + L::halo_bytes, map_base, &bars[slot], c * kChunk, x0, p - H);
  };

  if (tid == 0) {
    for (int s = 0; s < kSlots; ++s) mbar_init(&bars[s], 1);
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
    for (int q = 0; q < min(kSlots, total); ++q) issue(q);
  }
  // ---- tile constants: phi of the stage input, material ids, material table
  for (int i = tid; i < nrows * TX; i += kCartThreads) {
    const int r = i / TX, xl = i - r * TX;
    const int gx = x0 + xl;
    const size_t cell = (size_t)(ya + r) * nx + gx;
    const bool in = gx < nx;
    tile_phi[i] = in ? phi_in[cell] : 0.f;
    tile_mat[i] = in ? d.mat[cell] : 0;
    tile_acc[i] = 0.f;
  }
  if (tid < kMaxMat) {
    mtab[tid] = d.sig_t[tid];
    mtab[kMaxMat + tid] = d.sig_s2pi[tid];
    mtab[2 * kMaxMat + tid] = d.q_src[tid];
  }
  __syncthreads();

  const float dt = d.dt;
  double bacc = 0.0;   // boundary outflow of the output state (this thread's terms)

  int q = 0;          // next sequence entry to consume
  int issued = min(kSlots, total);
  for (int c = 0; c < d.n_chunks; ++c) {
    const int k = c * kChunk + lane;
    const float xi = d.xi[k], eta = d.eta[k], wk = d.w[k];
    const int dxs = (xi > 0.f) ? 1 : -1;
    const int dys = (eta > 0.f) ? 1 : -1;
    const float ax = fabsf(xi) * d.inv_dx, ay = fabsf(eta) * d.inv_dy;
    // psi^- of each side for this ordinate: the inflow value if it enters there, else 0
    const float g_xlo = (xi > 0.f) ? d.ghost[0] : 0.f;
    const float g_xhi = (xi < 0.f) ? d.ghost[1] : 0.f;
    const float g_ylo = (eta > 0.f) ? d.ghost[2] : 0.f;
    const float g_yhi = (eta < 0.f) ? d.ghost[3] : 0.f;
    const float gx_up = (dxs > 0) ? g_xlo : g_xhi;   // ghost on the upwind side in x
    const float gy_up = (dys > 0) ? g_ylo : g_yhi;

    float win[CPW][WIN];     // psi at rows j-H..j+H for each cell of this thread
    float dxw[CPW][H + 1];   // x divergence at rows j..j+H
#pragma unroll
    for (int u = 0; u < CPW; ++u) {
#pragma unroll
      for (int r = 0; r < WIN; ++r) win[u][r] = 0.f;
#pragma unroll
      for (int r = 0; r <= H; ++r) dxw[u][r] = 0.f;
    }

    for (int p = ya - H; p < yb + H; ++p, ++q) {
      const int slot = q % kSlots;
      const uint32_t par = (uint32_t)((q / kSlots) & 1);
      const uint8_t* sl = ring + slot * L::slot_bytes;
      const T* srow = reinterpret_cast<const T*>(sl);
      const T* sbase = reinterpret_cast<const T*>(sl + L::halo_bytes);
      const bool ok = mbar_wait_bounded(&bars[slot], par, limit);
      const bool p_in = (p >= 0 && p < ny);
      const bool p_tile = (p >= ya && p < yb);
      float vnew[CPW], dnew[CPW], bse[CPW];
#pragma unroll
      for (int u = 0; u < CPW; ++u) {
        const int xl = warp + kCartWarps * u;
        const int xs = xl + H;
        const int gx = x0 + xl;
        float cv = p_in ? Store<T>::from_smem(srow[xs * kChunk + lane]) : (p < 0 ? g_ylo : g_yhi);
        vnew[u] = cv;
        float dv = 0.f;
        if (p_tile) {
          const float u1 = Store<T>::from_smem(srow[(xs - dxs) * kChunk + lane]);
          const bool in_bnd = (gx - dxs < 0) || (gx - dxs >= nx);
          const bool out_bnd = (gx + dxs < 0) || (gx + dxs >= nx);
          if constexpr (ORDER == 1) {
            const float f_in = in_bnd ? gx_up : u1;
            dv = ax * (cv - f_in);
          } else {
            const float u2 = Store<T>::from_smem(srow[(xs - 2 * dxs) * kChunk + lane]);
            const float d1 = Store<T>::from_smem(srow[(xs + dxs) * kChunk + lane]);
            const bool u2_out = (gx - 2 * dxs < 0) || (gx - 2 * dxs >= nx);
            const float u1v = in_bnd ? gx_up : u1;
            const float u2v = (in_bnd || u2_out) ? gx_up : u2;
            const float f_in = in_bnd ? gx_up : u1 + 0.5f * minmod(cv - u1, u1 - u2v);
            const float f_out = out_bnd ? cv : cv + 0.5f * minmod(d1 - cv, cv - u1v);
            dv = ax * (f_out - f_in);
          }
        }
        dnew[u] = dv;
        bse[u] = 0.f;
        if constexpr (STAGE == STAGE_HEUN2) {
          if (p - H >= ya) bse[u] = Store<T>::from_smem(sbase[xl * kChunk + lane]);
        }
      }
      // all reads of the slot are done (or the wait ran out)
      if (__syncthreads_or(!ok)) {
        if (tid == 0) {
          // wait (bounded) for loads still in flight into this CTA's slots
          for (int qq = q; qq < issued; ++qq) {
            if ((int64_t)qq == d.drop_load) continue;
            mbar_wait_bounded(&bars[qq % kSlots], (uint32_t)((qq / kSlots) & 1), limit);
          }
          atomicCAS(&st->status, DEV_OK, DEV_TIMEOUT);
          st->timeout_where = ((int64_t)blockIdx.x << 32) | (int64_t)q;
        }
        return;
      }
      if (tid == 0 && issued < total) {
        fence_proxy_async_smem();
        issue(issued);
        ++issued;
      }
      // shift the windows
#pragma unroll
      for (int u = 0; u < CPW; ++u) {
#pragma unroll
        for (int r = 0; r < WIN - 1; ++r) win[u][r] = win[u][r + 1];
        win[u][WIN - 1] = vnew[u];
#pragma unroll
        for (int r = 0; r < H; ++r) dxw[u][r] = dxw[u][r + 1];
        dxw[u][H] = dnew[u];
      }
      const int j = p - H;
      if (j < ya) continue;
      // ---- complete row j
      const bool yin_bnd = (j - dys < 0) || (j - dys >= ny);
      const bool yout_bnd = (j + dys < 0) || (j + dys >= ny);
      const bool yu2_out = (j - 2 * dys < 0) || (j - 2 * dys >= ny);
      const int r = j - ya;
      float contrib[CPW];
#pragma unroll
      for (int u = 0; u < CPW; ++u) {
        const int xl = warp + kCartWarps * u;
        const int gx = x0 + xl;
        const float cv = win[u][H];
        float dy;
        if constexpr (ORDER == 1) {
          const float u1 = (dys > 0) ? win[u][0] : win[u][2];
          const float f_in = yin_bnd ? gy_up : u1;
          dy = ay * (cv - f_in);
        } else {
          const float u1 = (dys > 0) ? win[u][1] : win[u][3];
          const float u2 = (dys > 0) ? win[u][0] : win[u][4];
          const float d1 = (dys > 0) ? win[u][3] : win[u][1];
          const float u1v = yin_bnd ? gy_up : u1;
          const float u2v = (yin_bnd || yu2_out) ? gy_up : u2;
          const float f_in = yin_bnd ? gy_up : u1 + 0.5f * minmod(cv - u1, u1 - u2v);
          const float f_out = yout_bnd ? cv : cv + 0.5f * minmod(d1 - cv, cv - u1v);
          dy = ay * (f_out - f_in);
        }
        const int ti = r * TX + xl;
        const int m = tile_mat[ti];
        const float F = -(dxw[u][0] + dy) - mtab[m] * cv + mtab[kMaxMat + m] * tile_phi[ti] + mtab[2 * kMaxMat + m];
        float outv;
        if constexpr (STAGE == STAGE_HEUN2) {
          outv = 0.5f * (bse[u] + cv + dt * F);
        } else {
          outv = cv + dt * F;
        }
        outv = Store<T>::round(outv);
        contrib[u] = 0.f;
        if (gx < nx) {
          Store<T>::store(psi_out + ((size_t)j * nx + gx) * Mpad + k, outv);
          contrib[u] = wk * outv;
          // boundary outflow of the output state: first-order traces
          if (gx == 0) bacc += (double)(d.dy_d * (double)(wk * -xi * (xi < 0.f ? outv : g_xlo)));
          if (gx == nx - 1) bacc += (double)(d.dy_d * (double)(wk * xi * (xi > 0.f ? outv : g_xhi)));
          if (j == 0) bacc += (double)(d.dx_d * (double)(wk * -eta * (eta < 0.f ? outv : g_ylo)));
          if (j == ny - 1) bacc += (double)(d.dx_d * (double)(wk * eta * (eta > 0.f ? outv : g_yhi)));
        }
      }
      const float s = multi_warp_sum<CPW>(contrib, lane);
      if ((lane & (32 / CPW - 1)) == 0) {
        const int u = lane / (32 / CPW);
        tile_acc[r * TX + warp + kCartWarps * u] += s;
      }
    }
  }
  __syncthreads();

  // ---- epilogue: phi_out and FP64 QoI partials of the output state
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
    const float va = (float)d.sig_a[tile_mat[i]] * ph;
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
  // compact layout for the reduction: regions, mass, outflow
#pragma unroll
  for (int g = 0; g < kMaxReg + 1; ++g)
    if (g == nreg) acc[g] = (double)fm * d.area_d;
#pragma unroll
  for (int g = 0; g < kMaxReg + 2; ++g)
    if (g == nreg + 1) acc[g] = bacc;
  block_reduce_q<kCartThreads>(acc, nreg + 2, red);
  finalize_item<kCartThreads>(d, it, red, STAGE, red + NQ);
}

template <int H, int TX, int STAGE, typename T>
static size_t smem_for(int ly) {
  using L = CartLayout<H, TX, STAGE, T>;
  return L::ring_bytes + cart_tile_bytes(TX, ly) + kCartFixedBytes;
}

template <int H, int TX, int STAGE, typename T>
static cudaError_t prepare_one(int ly_max) {
  // raise the dynamic shared-memory limit of this kernel variant (idempotent)
  static size_t s_limit = 0;
  const size_t smem = smem_for<H, TX, STAGE, T>(ly_max);
  if (smem > s_limit) {
    cudaError_t e = cudaFuncSetAttribute(cart_stage_kernel<H, TX, STAGE, T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    s_limit = smem;
  }
  return cudaSuccess;
}

template <int H, int TX, int STAGE, typename T>
static cudaError_t launch_one(const InstDesc* d_desc, const WorkItem* d_items, int n_items, int ly_max,
                              cudaStream_t stream) {
  cudaError_t e = prepare_one<H, TX, STAGE, T>(ly_max);
  if (e != cudaSuccess) return e;
  cart_stage_kernel<H, TX, STAGE, T><<<n_items, kCartThreads, smem_for<H, TX, STAGE, T>(ly_max), stream>>>(
      d_desc, d_items);
  return cudaGetLastError();
}

#define RTK_CART_VARIANTS(X, TT)                                                             \
  X(1, 32, STAGE_EULER, TT) X(1, 32, STAGE_HEUN1, TT) X(1, 32, STAGE_HEUN2, TT)              \
  X(2, 32, STAGE_EULER, TT) X(2, 32, STAGE_HEUN1, TT) X(2, 32, STAGE_HEUN2, TT)              \
  X(1, 64, STAGE_EULER, TT) X(1, 64, STAGE_HEUN1, TT) X(1, 64, STAGE_HEUN2, TT)              \
  X(2, 64, STAGE_EULER, TT) X(2, 64, STAGE_HEUN1, TT) X(2, 64, STAGE_HEUN2, TT)

cudaError_t prepare_cart_stage(int stage, int order, int storage, int tx, int ly_max) {
#define RTK_P(H, TXV, ST, TT) \
  if (order == H && tx == TXV && stage == ST) return prepare_one<H, TXV, ST, TT>(ly_max);
  if (storage == 0) { RTK_CART_VARIANTS(RTK_P, float) } else { RTK_CART_VARIANTS(RTK_P, __nv_bfloat16) }
#undef RTK_P
  return cudaErrorInvalidValue;
}

cudaError_t launch_cart_stage(const InstDesc* d_desc, const WorkItem* d_items, int n_items, int stage, int order,
                              int storage, int tx, int ly_max, cudaStream_t stream) {
  if (n_items <= 0) return cudaSuccess;
#define RTK_L(H, TXV, ST, TT) \
  if (order == H && tx == TXV && stage == ST) return launch_one<H, TXV, ST, TT>(d_desc, d_items, n_items, ly_max, stream);
  if (storage == 0) { RTK_CART_VARIANTS(RTK_L, float) } else { RTK_CART_VARIANTS(RTK_L, __nv_bfloat16) }
#undef RTK_L
  return cudaErrorInvalidValue;
}

size_t cart_smem_bytes(int order, int storage, int tx, int ly, int stage) {
#define RTK_SM(H, TXV, ST, TT) \
  if (order == H && tx == TXV && stage == ST) return smem_for<H, TXV, ST, TT>(ly);
  if (storage == 0) { RTK_CART_VARIANTS(RTK_SM, float) } else { RTK_CART_VARIANTS(RTK_SM, __nv_bfloat16) }
#undef RTK_SM
  return 0;
}

}  // namespace rtk
