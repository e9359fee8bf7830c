// Staged first-order stage kernel on triangle meshes (Sec. 4.2 on triangles,
// Eq. upwind1stOrder and Eq. sn_2d_eqn_fv; Euler or either Heun stage).
//
// The arithmetic per cell and ordinate is that of tri_stage_kernel: for each
// edge e of cell i, (omega_k . n_e) l_e / A_i times the upwind trace (psi_i when
// the ordinate leaves through e, else the neighbour's psi or the side's psi^-),
// F = -sum_e(...) - sigma_t psi + sigma_s/(2 pi) phi + Q, then the Euler or
// Heun update, phi_out = sum_k w_k out_k and the FP64 QoI partials.
//
// What differs is how the rows arrive. Cells are stored in the Morton order of
// their centroids, so a chunk of 64 consecutive cells is a compact patch whose
// edges lead to about 33 other cells (at most 43 on the jittered split
// meshes): its halo, listed per chunk on the host. For each block of W = 32 VEC
// ordinates, the CTA issues a bulk copy (cp.async.bulk) of the block's segment
// of every row the chunk needs, its own 64 rows, its halo rows and, in Heun
// stage 2, the 64 rows of psi^n, into shared memory, completing on one mbarrier;
// the whole CTA then computes the block from shared memory. Each row is read
// from L2/DRAM about 1.5 times per chunk instead of 4 (a cell's own row plus
// three gathers by its neighbours), and a whole block's rows, about 25 KB, are
// in flight at once. Blocks are double-buffered: the copies of block j + 2 are
// issued as soon as block j is done. The chunk metadata (neighbour ids, edge
// geometry, neighbour slots in the staged rows, the halo list) arrives by bulk
// copies three chunks ahead.
//
// Persistent: CTA g of G takes chunks g, g + G, ... (two CTAs of 8 warps per
// SM); warp w owns cells w, w + 8, ..., w + 56 of a chunk and keeps their phi
// and outflow partial sums in registers across the blocks. Every warp issues
// the copies of its share of the next rows. Every wait is
// bounded; a wait that runs out stops the whole CTA at the next barrier,
// drains the copies in flight and reports RT_ETIMEOUT.
#include <cuda_bf16.h>

#include "device_common.cuh"

namespace rtk {

namespace {

constexpr int kStgThreads = 256;
constexpr int kStgWarps = kStgThreads / 32;
constexpr int kStgChunk = kTriStgChunk;   // cells per chunk (32)
constexpr int kStgCellsPerWarp = kStgChunk / kStgWarps;
constexpr int kStgMeta = 4;   // metadata buffers: chunks i .. i+3
constexpr int kStgTab = 12;   // cell table entries: (n.l/A) x and y per edge, sigma_t, source, psi^- per edge,
                              // neighbour slots, boundary flag

__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

template <typename T, int VEC>
__device__ __forceinline__ void ld_row(const T* p, float (&out)[VEC]) {
  if constexpr (sizeof(T) == 4) {
    if constexpr (VEC == 4) {
      const float4 x = *reinterpret_cast<const float4*>(p);
      out[0] = x.x; out[1] = x.y; out[2] = x.z; out[3] = x.w;
    } else if constexpr (VEC == 2) {
      const float2 x = *reinterpret_cast<const float2*>(p);
      out[0] = x.x; out[1] = x.y;
    } else {
      out[0] = *reinterpret_cast<const float*>(p);
    }
  } else {
    if constexpr (VEC == 4) {
      const uint2 x = *reinterpret_cast<const uint2*>(p);
      out[0] = __uint_as_float(x.x << 16); out[1] = __uint_as_float(x.x & 0xffff0000u);
      out[2] = __uint_as_float(x.y << 16); out[3] = __uint_as_float(x.y & 0xffff0000u);
    } else if constexpr (VEC == 2) {
      const uint32_t x = *reinterpret_cast<const uint32_t*>(p);
      out[0] = __uint_as_float(x << 16); out[1] = __uint_as_float(x & 0xffff0000u);
    } else {
      out[0] = __bfloat162float(*p);
    }
  }
}

template <typename T, int VEC>
__device__ __forceinline__ void st_row(T* p, const float (&in)[VEC]) {
  if constexpr (sizeof(T) == 4) {
    if constexpr (VEC == 4) {
      *reinterpret_cast<float4*>(p) = make_float4(in[0], in[1], in[2], in[3]);
    } else if constexpr (VEC == 2) {
      *reinterpret_cast<float2*>(p) = make_float2(in[0], in[1]);
    } else {
      *reinterpret_cast<float*>(p) = in[0];
    }
  } else {
    if constexpr (VEC == 4) {
      __nv_bfloat162 a = __floats2bfloat162_rn(in[0], in[1]);
      __nv_bfloat162 b = __floats2bfloat162_rn(in[2], in[3]);
      uint2 x;
      x.x = *reinterpret_cast<uint32_t*>(&a);
      x.y = *reinterpret_cast<uint32_t*>(&b);
      *reinterpret_cast<uint2*>(p) = x;
    } else if constexpr (VEC == 2) {
      *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(in[0], in[1]);
    } else {
      *p = __float2bfloat16_rn(in[0]);
    }
  }
}

}  // namespace

// Shared-memory layout of the staged kernel: two row buffers of `rows` rows of
// W values (64 own rows, hmax halo rows, and in Heun stage 2 64 rows of psi^n),
// then kStgMeta metadata buffers (neighbour records, edge geometry, neighbour
// slots, halo ids), then the mbarriers and counters.
struct StgLayout {
  size_t row_bytes, rows, buf_bytes, meta_bytes, total;
  int hmax;
};

__host__ __device__ inline StgLayout stg_layout(int vec, int es, int hmax, bool base) {
  StgLayout L;
  L.hmax = hmax;
  L.row_bytes = (size_t)32 * vec * es;
  L.rows = (size_t)kStgChunk + hmax + (base ? kStgChunk : 0);
  L.buf_bytes = (L.rows * L.row_bytes + 127) / 128 * 128;
  L.meta_bytes = ((size_t)kStgChunk * 16 + 2 * kStgChunk * 16 + kStgChunk * 4 + (size_t)hmax * 4 + 127) / 128 * 128;
  L.total = 2 * L.buf_bytes + kStgMeta * L.meta_bytes + kStgChunk * kStgTab * 4 + 128 + 128;   // + cell table,
                                                                                            // control, slack
  return L;
}

template <int VEC, int STAGE, typename T>
__global__ void __launch_bounds__(kStgThreads, 2)
    tri_staged_kernel(const InstDesc* __restrict__ descs, const WorkItem* __restrict__ items) {
  __shared__ double red[(kStgWarps + 1) * NQ];
  __shared__ float wacc[kStgWarps][NQ];
  __shared__ double wdacc[kStgWarps][NQ];
  extern __shared__ __align__(128) uint8_t stg_raw[];
  const WorkItem it = items[blockIdx.x];
  const InstDesc& d = descs[it.inst];
  InstState* st = d.st;
  if (st->step >= d.n_steps || st->status != DEV_OK) return;

  constexpr int W = 32 * VEC;
  constexpr bool kBase = STAGE == STAGE_HEUN2;
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
  const int nb = Mpad / W;
  const float dt = d.dt;
  const int nreg = d.n_regions, nq = nreg + 2;
  const int n_cells = (int)d.n_cells;
  const int n_chunks = (n_cells + kStgChunk - 1) / kStgChunk;
  const int G = it.b;
  const int64_t limit = d.wait_limit;
  const StgLayout L = stg_layout(VEC, (int)sizeof(T), d.tri_hmax, kBase);
  const int base_row = kStgChunk + L.hmax;

  uint8_t* smem = stg_raw + ((128u - (smem_u32(stg_raw) & 127u)) & 127u);
  uint8_t* rowbuf[2] = {smem, smem + L.buf_bytes};
  uint8_t* meta0 = smem + 2 * L.buf_bytes;
  float* tab = reinterpret_cast<float*>(meta0 + kStgMeta * L.meta_bytes);   // [kStgChunk][kStgTab]
  uint64_t* row_bar = reinterpret_cast<uint64_t*>(tab + kStgChunk * kStgTab);
  uint64_t* meta_bar = row_bar + 2;                            // [kStgMeta]
  int* ctl = reinterpret_cast<int*>(meta_bar + kStgMeta);
  int* s_hcount = ctl;                  // [kStgMeta] halo rows of the chunk in each metadata buffer
  int* s_meta_last = ctl + kStgMeta;    // [kStgMeta] last chunk ordinal issued into each, -1 none
  int* s_row_last = ctl + 2 * kStgMeta; // [2] last (chunk, block) pair issued into each row buffer

  auto metabuf = [&](int mb) { return meta0 + (size_t)mb * L.meta_bytes; };
  auto meta_nbr = [&](int mb) { return reinterpret_cast<const int4*>(metabuf(mb)); };
  auto meta_geo = [&](int mb) { return reinterpret_cast<const float4*>(metabuf(mb) + kStgChunk * 16); };
  auto meta_lidx = [&](int mb) { return reinterpret_cast<const uint32_t*>(metabuf(mb) + 3 * kStgChunk * 16); };
  auto meta_halo = [&](int mb) {
    return reinterpret_cast<const int32_t*>(metabuf(mb) + 3 * kStgChunk * 16 + kStgChunk * 4);
  };
  const int n_my = (it.a < n_chunks) ? (n_chunks - 1 - it.a) / G + 1 : 0;
  const int J = n_my * nb;

  // metadata of chunk ordinal i into buffer i % kStgMeta (thread 0)
  auto issue_meta = [&](int i) {
    const int mb = i % kStgMeta;
    const int k = it.a + i * G;
    const int c0 = k * kStgChunk;
    const int cells = min(kStgChunk, n_cells - c0);
    const int2 oc = d.tri_halo_oc[k];
    const int hpad = (oc.y + 3) & ~3;
    s_hcount[mb] = oc.y;
    s_meta_last[mb] = i;
    uint8_t* m = metabuf(mb);
    mbar_arrive_expect_tx(&meta_bar[mb], (uint32_t)(cells * 48 + kStgChunk * 4 + hpad * 4));
    bulk_copy(m, d.tri_nbr + c0, (uint32_t)cells * 16u, &meta_bar[mb]);
    bulk_copy(m + kStgChunk * 16, d.tri_geo + 2 * (size_t)c0, (uint32_t)cells * 32u, &meta_bar[mb]);
    bulk_copy(m + 3 * kStgChunk * 16, d.tri_lidx + (size_t)k * kStgChunk, kStgChunk * 4u, &meta_bar[mb]);
    if (hpad > 0) bulk_copy(m + 3 * kStgChunk * 16 + kStgChunk * 4, d.tri_halo + oc.x, (uint32_t)hpad * 4u, &meta_bar[mb]);
  };
  // rows of pair j = (chunk ordinal i, block b) into row buffer j & 1, by every
  // warp: warp w takes a contiguous share of the rows and arrives on the buffer's
  // mbarrier (one arrival per warp) with its bytes before issuing its copies, so
  // the phase cannot complete before every warp's copies have landed. The
  // chunk's metadata must have arrived. Returns false if waiting for it ran out.
  auto issue_rows = [&](int j) -> bool {
    const int i = j / nb, b = j - i * nb, mb = i % kStgMeta, rb = j & 1;
    const bool mok = mbar_wait_bounded(&meta_bar[mb], (uint32_t)((i / kStgMeta) & 1), limit);
    if (!__all_sync(0xffffffffu, mok)) return false;
    const int k = it.a + i * G;
    const int c0 = k * kStgChunk;
    const int cells = min(kStgChunk, n_cells - c0);
    const int H = s_hcount[mb];
    const int n_rows = cells + H + (kBase ? cells : 0);
    const int per = (n_rows + kStgWarps - 1) / kStgWarps;   // at most 32 (n_rows <= 256)
    const int r0 = warp * per, r1 = min(n_rows, r0 + per);
    const uint32_t rbytes = (uint32_t)L.row_bytes;
    if (threadIdx.x == 0) s_row_last[rb] = j;
    if (lane == 0) mbar_arrive_expect_tx(&row_bar[rb], (uint32_t)max(0, r1 - r0) * rbytes);
    __syncwarp();
    const int r = r0 + lane;
    if (r < r1) {
      const int32_t* halo = meta_halo(mb);
      int cell, slot;
      const T* src = psi_in;
      if (r < cells) {
        cell = c0 + r; slot = r;
      } else if (r < cells + H) {
        cell = halo[r - cells]; slot = kStgChunk + (r - cells);
      } else {
        cell = c0 + (r - cells - H); slot = base_row + (r - cells - H); src = psi_base;
      }
      bulk_copy(rowbuf[rb] + (size_t)slot * L.row_bytes, src + (size_t)cell * Mpad + b * W, rbytes, &row_bar[rb]);
    }
    return true;
  };

  if (lane < NQ) {
    wacc[warp][lane] = 0.f;
    wdacc[warp][lane] = 0.0;
  }
  if (threadIdx.x == 0) {
    for (int q = 0; q < 2; ++q) {
      mbar_init(&row_bar[q], kStgWarps);
      s_row_last[q] = -1;
    }
    for (int q = 0; q < kStgMeta; ++q) {
      mbar_init(&meta_bar[q], 1);
      s_meta_last[q] = -1;
    }
    fence_barrier_init();
    for (int i = 0; i < min(n_my, kStgMeta - 1); ++i) issue_meta(i);
  }
  __syncthreads();
  // the first two pairs; afterwards pair j + 2 is issued at the end of pair j
  bool iok = true;
  for (int q = 0; q < min(J, 2); ++q) iok = iok && issue_rows(q);

  bool ok = true;
  float phi_part[kStgCellsPerWarp], bpart[kStgCellsPerWarp];
  int ncell = 0;
  int j = 0;
  for (; j < J; ++j) {
    const int i = j / nb, b = j - i * nb, mb = i % kStgMeta, rb = j & 1;
    const bool rok = mbar_wait_bounded(&row_bar[rb], (uint32_t)((j >> 1) & 1), limit);
    if (__syncthreads_or(!rok || !iok)) {
      ok = false;
      break;
    }
    const int k = it.a + i * G;
    const int c0 = k * kStgChunk;
    const int cells = min(kStgChunk, n_cells - c0);
    if (b == 0) {
      // cell table of the chunk, one thread per cell: the edges' (n.l)/A, sigma_t,
      // the source sigma_s/(2 pi) phi + Q, psi^- per edge, the neighbour slots and
      // whether the cell has a boundary edge
      if (threadIdx.x < cells) {
        const int li = threadIdx.x;
        const int4 nb4 = meta_nbr(mb)[li];
        const float4 g0 = meta_geo(mb)[2 * li], g1 = meta_geo(mb)[2 * li + 1];
        const int m = nb4.w & 255;
        float* t = tab + li * kStgTab;
        t[0] = g0.x; t[1] = g0.z; t[2] = g1.x;   // x components of (n.l)/A for edges 0, 1, 2
        t[3] = g0.y; t[4] = g0.w; t[5] = g1.y;   // y components
        t[6] = d.sig_t[m];
        t[7] = d.sig_s2pi[m] * phi_in[c0 + li] + d.q_src[m];
        const int nbr[3] = {nb4.x, nb4.y, nb4.z};
#pragma unroll
        for (int e = 0; e < 3; ++e) t[8 + e] = (nbr[e] < 0) ? d.ghost[-1 - nbr[e]] : 0.f;
        // neighbour slots (byte e; 255 = boundary edge) and bit 24: a boundary edge exists
        const uint32_t lx = meta_lidx(mb)[li];
        const bool has_bnd = (nbr[0] < 0) | (nbr[1] < 0) | (nbr[2] < 0);
        t[11] = __uint_as_float((lx & 0xffffffu) | (has_bnd ? (1u << 24) : 0u));
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < kStgCellsPerWarp; ++q) {
        phi_part[q] = 0.f;
        bpart[q] = 0.f;
      }
    }
    const T* rows = reinterpret_cast<const T*>(rowbuf[rb]);
    const int kk = b * W + lane * VEC;
    float xi[VEC], eta[VEC], w[VEC];
    ld_row<float, VEC>(d.xi + kk, xi);
    ld_row<float, VEC>(d.eta + kk, eta);
    ld_row<float, VEC>(d.w + kk, w);
#pragma unroll
    for (int q = 0; q < kStgCellsPerWarp; ++q) {
      const int li = warp + q * kStgWarps;
      if (li >= cells) break;
      const int cell = c0 + li;
      const float4 t0 = *reinterpret_cast<const float4*>(tab + li * kStgTab);
      const float4 t1 = *reinterpret_cast<const float4*>(tab + li * kStgTab + 4);
      const float4 t2 = *reinterpret_cast<const float4*>(tab + li * kStgTab + 8);
      const float ax[3] = {t0.x, t0.y, t0.z};
      const float ay[3] = {t0.w, t1.x, t1.y};
      const float sig_t = t1.z, src = t1.w;
      const float gh[3] = {t2.x, t2.y, t2.z};
      const uint32_t lx = __float_as_uint(t2.w);
      const bool has_bnd = (lx >> 24) != 0;
      const int nbr_slot[3] = {(int)(lx & 255u), (int)((lx >> 8) & 255u), (int)((lx >> 16) & 255u)};
      float c[VEC], nbv[3][VEC];
      [[maybe_unused]] float base[VEC];
      ld_row<T, VEC>(rows + (size_t)li * W + lane * VEC, c);
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        if (nbr_slot[e] != 255) {
          ld_row<T, VEC>(rows + (size_t)nbr_slot[e] * W + lane * VEC, nbv[e]);
        } else {
#pragma unroll
          for (int l = 0; l < VEC; ++l) nbv[e][l] = gh[e];
        }
      }
      if constexpr (kBase) ld_row<T, VEC>(rows + (size_t)(base_row + li) * W + lane * VEC, base);
      // BF16 rounding bits of the lane's ordinates kk .. kk+VEC-1 (one group of four)
      [[maybe_unused]] uint2 rb4;
      if constexpr (sizeof(T) == 2) rb4 = sr_bits4((uint32_t)cell, sr_gkey(kk >> 2, salt));
      float out[VEC];
      if constexpr (VEC >= 2) {
        // ordinate pairs: the flux, the update and phi run on FP32 pairs (two values
        // per instruction, each rounded as the scalar operation would be)
        float2 pw = make_float2(0.f, 0.f);
#pragma unroll
        for (int p = 0; p < VEC / 2; ++p) {
          const int l = 2 * p;
          const float2 xi2 = make_float2(xi[l], xi[l + 1]), eta2 = make_float2(eta[l], eta[l + 1]);
          const float2 c2 = make_float2(c[l], c[l + 1]);
          float2 div = make_float2(0.f, 0.f);
#pragma unroll
          for (int e = 0; e < 3; ++e) {
            const float2 on = __ffma2_rn(eta2, make_float2(ay[e], ay[e]), __fmul2_rn(xi2, make_float2(ax[e], ax[e])));
            const float2 up = make_float2(on.x > 0.f ? c2.x : nbv[e][l], on.y > 0.f ? c2.y : nbv[e][l + 1]);
            div = __ffma2_rn(on, up, div);
          }
          const float2 F = __fadd2_rn(__ffma2_rn(make_float2(-sig_t, -sig_t), c2, make_float2(src, src)),
                                      make_float2(-div.x, -div.y));
          float2 o;
          if constexpr (kBase) {
            o = __fmul2_rn(make_float2(0.5f, 0.5f),
                           __ffma2_rn(make_float2(dt, dt), F, __fadd2_rn(make_float2(base[l], base[l + 1]), c2)));
          } else {
            o = __ffma2_rn(make_float2(dt, dt), F, c2);
          }
          if constexpr (sizeof(T) == 2) {
            o.x = Store<T>::round_sr(o.x, sr_elem(rb4, (kk + l) & 3));
            o.y = Store<T>::round_sr(o.y, sr_elem(rb4, (kk + l + 1) & 3));
          }
          out[l] = o.x;
          out[l + 1] = o.y;
          pw = __ffma2_rn(make_float2(w[l], w[l + 1]), o, pw);
        }
        phi_part[q] += pw.x + pw.y;
      } else {
        const float cv = c[0];
        float div = 0.f;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
          const float on = xi[0] * ax[e] + eta[0] * ay[e];
          div += on * ((on > 0.f) ? cv : nbv[e][0]);
        }
        const float F = -div - sig_t * cv + src;
        float o;
        if constexpr (kBase) {
          o = 0.5f * (base[0] + cv + dt * F);
        } else {
          o = cv + dt * F;
        }
        if constexpr (sizeof(T) == 2) o = Store<T>::round_sr(o, sr_elem(rb4, kk & 3));
        out[0] = o;
        phi_part[q] += w[0] * o;
      }
#pragma unroll
      for (int l = 0; l < VEC; ++l) {
        const float o = out[l];
        if (has_bnd) {
#pragma unroll
          for (int e = 0; e < 3; ++e) {
            if (nbr_slot[e] == 255) {
              const float on = xi[l] * ax[e] + eta[l] * ay[e];
              bpart[q] += w[l] * on * ((on > 0.f) ? o : gh[e]);
            }
          }
        }
      }
      st_row<T, VEC>(psi_out + (size_t)cell * Mpad + kk, out);
    }
    if (b == nb - 1) {
      // the chunk is complete: phi and the QoI terms of the warp's cells
#pragma unroll
      for (int q = 0; q < kStgCellsPerWarp; ++q) {
        const int li = warp + q * kStgWarps;
        if (li >= cells) break;
        const int4 nb4 = meta_nbr(mb)[li];
        const bool has_bnd = (nb4.x < 0) | (nb4.y < 0) | (nb4.z < 0);
        const float ph = warp_sum(phi_part[q]);
        float bsum = 0.f;
        if (has_bnd) bsum = warp_sum(bpart[q]);
        if (lane == 0) {
          const int m = nb4.w & 255, reg = (nb4.w >> 8) & 255;
          const float area = meta_geo(mb)[2 * li + 1].z;
          phi_out[c0 + li] = ph;
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
    }
    // every warp is done with row buffer rb (and, at the chunk's end, metadata buffer mb)
    __syncthreads();
    if (b == nb - 1 && threadIdx.x == 0 && i + kStgMeta - 1 < n_my) {
      fence_proxy_async_smem();
      issue_meta(i + kStgMeta - 1);   // into buffer (i - 1) % kStgMeta, free since chunk i - 1 ended
    }
    if (j + 2 < J) {
      fence_proxy_async_smem();
      iok = issue_rows(j + 2) && iok;
    }
  }
  if (!ok) {
    if (threadIdx.x == 0) {
      // drain: the last copies issued into each buffer may still be in flight
      for (int q = 0; q < 2; ++q)
        if (s_row_last[q] >= 0) mbar_wait_bounded(&row_bar[q], (uint32_t)((s_row_last[q] >> 1) & 1), limit);
      for (int q = 0; q < kStgMeta; ++q)
        if (s_meta_last[q] >= 0) mbar_wait_bounded(&meta_bar[q], (uint32_t)((s_meta_last[q] / kStgMeta) & 1), limit);
      atomicCAS(&st->status, DEV_OK, DEV_TIMEOUT);
      st->timeout_where = ((int64_t)blockIdx.x << 32) | (int64_t)j;
    }
  }
  __syncwarp();
  if (lane < nq) wdacc[warp][lane] += (double)wacc[warp][lane];
  __syncthreads();
  if (threadIdx.x < nq) {
    double s = 0.0;
    for (int w2 = 0; w2 < kStgWarps; ++w2) s += wdacc[w2][threadIdx.x];
    red[threadIdx.x] = s;
  }
  __syncthreads();
  finalize_item<kStgThreads>(d, it, red, STAGE, red + NQ);
}

// Ordinates per lane of the staged kernel: those of the instance.
static int stg_vec(int, int vec) { return vec; }

size_t tri_staged_smem_bytes(int vec, int storage, int hmax, int stage) {
  return stg_layout(stg_vec(storage, vec), storage == 1 ? 2 : 4, hmax, stage == STAGE_HEUN2).total;
}

int tri_staged_threads() { return kStgThreads; }

template <int VEC, int STAGE, typename T>
static cudaError_t stg_prepare_one(size_t smem) {
  return cudaFuncSetAttribute(tri_staged_kernel<VEC, STAGE, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <int VEC, int STAGE, typename T>
static cudaError_t stg_launch_one(const InstDesc* d_desc, const WorkItem* d_items, int n_items, size_t smem,
                                  cudaStream_t s) {
  tri_staged_kernel<VEC, STAGE, T><<<n_items, kStgThreads, smem, s>>>(d_desc, d_items);
  return cudaGetLastError();
}

#define RTK_STG_ALL(X, TT)                                                                          \
  X(1, STAGE_EULER, TT) X(1, STAGE_HEUN1, TT) X(1, STAGE_HEUN2, TT) X(2, STAGE_EULER, TT)           \
  X(2, STAGE_HEUN1, TT) X(2, STAGE_HEUN2, TT) X(4, STAGE_EULER, TT) X(4, STAGE_HEUN1, TT)           \
  X(4, STAGE_HEUN2, TT)

// The dynamic shared memory of any instance (the host keeps it below
// kStgSmemCap, else it takes the gathering kernel): every variant's limit is
// raised to that cap once, the same for all instances, so that preparing one
// instance never lowers the limit another one launches with.
constexpr size_t kStgSmemCap = 108 * 1024;   // two CTAs per SM

cudaError_t prepare_tri_staged(int stage, int storage, int vec, int hmax) {
  if (tri_staged_smem_bytes(vec, storage, hmax, stage) > kStgSmemCap) return cudaErrorInvalidValue;
  vec = stg_vec(storage, vec);
  const size_t smem = kStgSmemCap;
#define RTK_P(V, ST, TT) \
  if (vec == V && stage == ST) return stg_prepare_one<V, ST, TT>(smem);
  if (storage == 0) { RTK_STG_ALL(RTK_P, float) } else { RTK_STG_ALL(RTK_P, __nv_bfloat16) }
#undef RTK_P
  return cudaErrorInvalidValue;
}

cudaError_t launch_tri_staged(const InstDesc* d_desc, const WorkItem* d_items, int n_items, int stage, int storage,
                              int vec, int hmax, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  const size_t smem = tri_staged_smem_bytes(vec, storage, hmax, stage);
  vec = stg_vec(storage, vec);
#define RTK_L(V, ST, TT) \
  if (vec == V && stage == ST) return stg_launch_one<V, ST, TT>(d_desc, d_items, n_items, smem, s);
  if (storage == 0) { RTK_STG_ALL(RTK_L, float) } else { RTK_STG_ALL(RTK_L, __nv_bfloat16) }
#undef RTK_L
  return cudaErrorInvalidValue;
}

}  // namespace rtk
