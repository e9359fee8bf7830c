// rt_cart_stage_noalloc: one Cartesian stage on caller-owned device buffers,
// without allocating device memory.
//
// The Cartesian stage kernel needs scratch memory besides its inputs and
// outputs: its descriptor (TMA tensor maps and constants), its work list, a
// small state block (launch ticket, status) and one FP64 row of QoI partial sums
// per work item. rt_create allocates these; this entry point places them in the
// file-scope array below instead, so that callers who cannot allocate device
// memory can still run the kernel. The array has a fixed size (about 1.4 MB,
// for at most RT_NOALLOC_MAX_WORK_ITEMS work items) and stays resident on every
// GPU that loads the library until the process exits. All calls share it: each
// call clears the parts that must start at zero, and calls that overlap on the
// GPU (for example on two streams) race on it.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "host_common.h"

namespace rtk {

namespace {

constexpr size_t round256(size_t n) { return (n + 255) / 256 * 256; }
constexpr int kMaxItems = RT_NOALLOC_MAX_WORK_ITEMS;
constexpr size_t kDescOff = 0;
constexpr size_t kStateOff = kDescOff + round256(sizeof(InstDesc));
constexpr size_t kItemsOff = kStateOff + round256(sizeof(InstState));
constexpr size_t kPartOff = kItemsOff + round256((size_t)kMaxItems * sizeof(WorkItem));
constexpr size_t kScratchBytes = kPartOff + (size_t)kMaxItems * NQ * sizeof(double);

}  // namespace

// Scratch of rt_cart_stage_noalloc: descriptor | state | work items | partial sums.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Write the descriptor and the work list into the scratch array and clear the
// state block (ticket, status, parity and the QoI sums must start at zero),
// then set the step counter to the caller's step index: the stage kernel draws
// the stochastic-rounding bits of BF16 stores from it.
__global__ void noalloc_setup_kernel(const __grid_constant__ InstDesc desc, int n_strips, int n_items,
                                     int64_t step) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const uint32_t* src = reinterpret_cast<const uint32_t*>(&desc);
  uint32_t* dst = reinterpret_cast<uint32_t*>(g_noalloc_scratch + kDescOff);
  for (int i = tid; i < (int)(sizeof(InstDesc) / 4); i += nt) dst[i] = src[i];
  uint32_t* stw = reinterpret_cast<uint32_t*>(g_noalloc_scratch + kStateOff);
  for (int i = tid; i < (int)(sizeof(InstState) / 4); i += nt) stw[i] = 0u;
  __syncthreads();
  if (tid == 0) reinterpret_cast<InstState*>(g_noalloc_scratch + kStateOff)->step = step;
  WorkItem* items = reinterpret_cast<WorkItem*>(g_noalloc_scratch + kItemsOff);
  for (int i = tid; i < n_items; i += nt) {
    WorkItem w;
    w.inst = 0;
    w.a = i % n_strips;
    w.b = i / n_strips;
    w.item = i;
    w.count = n_items;
    w.pad = 0;
    items[i] = w;
  }
  // the tensor maps were written through the generic proxy; the stage kernel
  // reads them through the tensormap proxy
  asm volatile("fence.proxy.tensormap::generic.release.gpu;" ::: "memory");
}

// Copy the output state's QoI integrands and the launch status to the caller.
__global__ void noalloc_copyout_kernel(int stage, int n_regions, double* qoi_out, int32_t* status_out) {
  const InstState* st = reinterpret_cast<const InstState*>(g_noalloc_scratch + kStateOff);
  const double* S = (stage == STAGE_HEUN1) ? st->S_mid : st->S_cur;
  const int t = threadIdx.x;
  if (t < n_regions) qoi_out[t] = S[t];
  if (t == n_regions) qoi_out[t] = S[kQMass];
  if (t == n_regions + 1) qoi_out[t] = S[kQOut];
  if (t == 0 && status_out) *status_out = st->status;
}

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once per device).
rt_status scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_error("cudaGetDevice failed: %s", cudaGetErrorString(e));
    return RT_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device %d is beyond the %d devices this entry point supports", dev, kMaxDevices);
    return RT_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error("cudaGetSymbolAddress of the scratch array failed: %s", cudaGetErrorString(e));
      return RT_ECUDA;
    }
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return RT_OK;
}

rt_status encode_map(CUtensorMap* map, const void* base, int storage, int Mpad, int nx, int ny, int box_k,
                     int box_x) {
  static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  if (!enc) {
    void* fp = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fp, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      set_error("cuTensorMapEncodeTiled is not available from the driver");
      return RT_ECUDA;
    }
    enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fp);
  }
  const size_t es = storage == RT_BF16 ? 2 : 4;
  cuuint64_t dims[3] = {(cuuint64_t)Mpad, (cuuint64_t)nx, (cuuint64_t)ny};
  cuuint64_t strides[2] = {(cuuint64_t)Mpad * es, (cuuint64_t)nx * Mpad * es};
  cuuint32_t box[3] = {(cuuint32_t)box_k, (cuuint32_t)box_x, 1u};
  cuuint32_t estr[3] = {1u, 1u, 1u};
  CUresult r = enc(map, storage == RT_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                   const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return RT_EINVAL;
  }
  return RT_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace
}  // namespace rtk

using namespace rtk;

extern "C" rt_status rt_cart_stage_noalloc(const rt_cart_stage_args* a) {
  clear_error();
  if (!a) { set_error("args is NULL"); return RT_EINVAL; }
  if (a->nx < 1 || a->ny < 1 || !(a->dx > 0.0) || !(a->dy > 0.0) || !std::isfinite(a->dx) || !std::isfinite(a->dy)) {
    set_error("need nx, ny >= 1 and finite dx, dy > 0"); return RT_EINVAL;
  }
  if ((int64_t)a->nx * a->ny > 0x7fffffffLL) { set_error("grid too large"); return RT_EINVAL; }
  const int vec = a->vec == 0 ? 1 : a->vec;
  if (a->M_pad < 32 || a->M_pad % 32 != 0 || a->M_pad > 65536) { set_error("M_pad must be a positive multiple of 32 (at most 65536)"); return RT_EINVAL; }
  if (vec != 1 && vec != 2 && vec != 4) { set_error("vec must be 0, 1, 2 or 4"); return RT_EINVAL; }
  if (a->M_pad % (32 * vec) != 0) { set_error("M_pad must be a multiple of 32*vec"); return RT_EINVAL; }
  if (a->order != 1 && a->order != 2) { set_error("order must be 1 or 2"); return RT_EINVAL; }
  if (a->stage != RT_STAGE_EULER && a->stage != RT_STAGE_HEUN1 && a->stage != RT_STAGE_HEUN2) { set_error("unknown stage %d", a->stage); return RT_EINVAL; }
  if (a->storage != RT_FP32 && a->storage != RT_BF16) { set_error("storage must be RT_FP32 or RT_BF16"); return RT_EINVAL; }
  if (a->n_mat < 1 || a->n_mat > RT_MAX_MATERIALS || a->n_regions < 1 || a->n_regions > RT_MAX_REGIONS) {
    set_error("need 1 <= n_mat <= %d and 1 <= n_regions <= %d", RT_MAX_MATERIALS, RT_MAX_REGIONS); return RT_EINVAL;
  }
  for (int m = 0; m < a->n_mat; ++m)
    if (!(a->sigma_a[m] >= 0.0) || !(a->sigma_s[m] >= 0.0) || !std::isfinite(a->sigma_a[m]) ||
        !std::isfinite(a->sigma_s[m]) || !std::isfinite(a->Q[m])) {
      set_error("material %d: sigma_a, sigma_s must be finite and >= 0, Q finite", m); return RT_EINVAL;
    }
  for (int s = 0; s < 4; ++s)
    if (!std::isfinite(a->inflow[s])) { set_error("inflow[%d] is not finite", s); return RT_EINVAL; }
  if (!(a->dt > 0.0) || !std::isfinite(a->dt)) { set_error("dt must be positive and finite"); return RT_EINVAL; }
  if (!a->psi_in || !a->psi_out || !a->phi_in || !a->phi_out || !a->cell_mat || !a->cell_region || !a->xi ||
      !a->eta || !a->w || !a->qoi_out) {
    set_error("device pointers psi_in, psi_out, phi_in, phi_out, cell_mat, cell_region, xi, eta, w, qoi_out are required");
    return RT_EINVAL;
  }
  if ((a->stage == RT_STAGE_HEUN2) != (a->psi_n != nullptr)) { set_error("psi_n is required for Heun stage 2 and only then"); return RT_EINVAL; }
  if (!aligned16(a->psi_in) || !aligned16(a->psi_out) || (a->psi_n && !aligned16(a->psi_n))) {
    set_error("psi buffers must be 16-byte aligned"); return RT_EINVAL;
  }
  if (a->psi_in == a->psi_out) { set_error("psi_out must not alias psi_in"); return RT_EINVAL; }
  if (a->step < 0 || a->step == INT64_MAX) { set_error("step must be in [0, INT64_MAX)"); return RT_EINVAL; }
  if (a->xi_host) {
    // every group of vec consecutive ordinates must share the sign of xi
    for (int g = 0; g < a->M_pad; g += vec) {
      bool pos = false, neg = false;
      for (int v = 0; v < vec; ++v) {
        const float x = a->xi_host[g + v];
        pos = pos || x > 0.f;
        neg = neg || x < 0.f;
      }
      if (pos && neg) {
        set_error("ordinates %d..%d mix signs of xi; with vec = %d every group of vec consecutive ordinates "
                  "must share one", g, g + vec - 1, vec);
        return RT_EINVAL;
      }
    }
  }

  // work split (strips of 16 cells, rows per segment as rt_create would choose)
  const int run = 2, tx = cart_tile_width(run);
  const int n_strips = (a->nx + tx - 1) / tx;
  int ly = a->tile_y;
  if (ly <= 0) {
    const int target = 2 * device_sm_count();
    const int segs = std::max(1, (target + n_strips - 1) / n_strips);
    ly = std::max(8, std::min((a->ny + segs - 1) / segs, 64));
  }
  ly = std::max(1, std::min(ly, 256));
  const int n_segs = (a->ny + ly - 1) / ly;
  const int64_t n_items = (int64_t)n_strips * n_segs;
  if (n_items > RT_NOALLOC_MAX_WORK_ITEMS) {
    set_error("this grid needs %lld work items but the scratch array of rt_cart_stage_noalloc holds at most %d; "
              "use a larger tile_y or rt_create", (long long)n_items, RT_NOALLOC_MAX_WORK_ITEMS);
    return RT_EINVAL;
  }
  const int kstage = a->stage == RT_STAGE_EULER ? STAGE_EULER : (a->stage == RT_STAGE_HEUN1 ? STAGE_HEUN1 : STAGE_HEUN2);
  if (cart_smem_bytes(a->order, a->storage, run, vec, ly, kstage) > 227 * 1024) {
    set_error("tile_y %d needs more shared memory than a CTA has", ly); return RT_EINVAL;
  }

  unsigned char* base = nullptr;
  rt_status st = scratch_address(&base);
  if (st != RT_OK) return st;

  // descriptor: buffers are arranged as the kernel expects them for this stage
  // (Euler / Heun stage 1 read buffer 0 and write buffer 1; Heun stage 2 reads
  // buffer 1 and psi^n, and writes buffer 0)
  InstDesc D;
  std::memset(&D, 0, sizeof(D));
  const bool s2 = kstage == STAGE_HEUN2;
  const int ib = s2 ? 1 : 0, ob = s2 ? 0 : 1;
  D.psi[ib] = const_cast<void*>(a->psi_in);
  D.psi[ob] = a->psi_out;
  D.phi[ib] = const_cast<float*>(a->phi_in);
  D.phi[ob] = a->phi_out;
  if ((st = encode_map(&D.tm_psi_halo[ib], a->psi_in, a->storage, a->M_pad, a->nx, a->ny, 32 * vec, tx + 2 * a->order)) != RT_OK)
    return st;
  if (s2 && (st = encode_map(&D.tm_psi_center, a->psi_n, a->storage, a->M_pad, a->nx, a->ny, 32 * vec, tx)) != RT_OK)
    return st;
  D.mat = a->cell_mat;
  D.region = a->cell_region;
  D.xi = a->xi;
  D.eta = a->eta;
  D.w = a->w;
  D.st = reinterpret_cast<InstState*>(base + kStateOff);
  D.partials = reinterpret_cast<double*>(base + kPartOff);
  D.kind = KIND_CART;
  D.order = a->order;
  D.integrator = s2 || kstage == STAGE_HEUN1 ? RT_HEUN : RT_EULER;
  D.storage = a->storage;
  D.nx = a->nx;
  D.ny = a->ny;
  D.M = a->M_pad;
  D.Mpad = a->M_pad;
  D.n_chunks = a->M_pad / (32 * vec);
  D.tx = tx;
  D.ly = ly;
  D.n_strips = n_strips;
  D.n_segs = n_segs;
  D.n_items = (int32_t)n_items;
  D.n_regions = a->n_regions;
  D.n_cells = (int64_t)a->nx * a->ny;
  D.n_steps = a->step + 1;   // the kernel skips instances whose step counter reached n_steps
  D.wait_limit = 4000000000LL;
  D.drop_load = -1;
  D.inv_dx = (float)(1.0 / a->dx);
  D.inv_dy = (float)(1.0 / a->dy);
  D.dx_d = a->dx;
  D.dy_d = a->dy;
  D.area_d = a->dx * a->dy;
  D.dt = (float)a->dt;
  D.dt_d = a->dt;
  for (int s = 0; s < 4; ++s) D.ghost[s] = (float)a->inflow[s];
  for (int m = 0; m < kMaxMat; ++m) {
    const bool in = m < a->n_mat;
    const double sa = in ? a->sigma_a[m] : 0.0, ss = in ? a->sigma_s[m] : 0.0, q = in ? a->Q[m] : 0.0;
    D.sig_t[m] = (float)(sa + ss);
    D.sig_s2pi[m] = (float)(ss / (2.0 * M_PI));
    D.q_src[m] = (float)q;
    D.sig_a[m] = sa;
    D.sig_a_f[m] = (float)sa;
  }

  cudaStream_t stream = (cudaStream_t)a->stream;
  cudaError_t e = prepare_cart_stage(kstage, a->order, a->storage, run, vec, ly);
  if (e == cudaSuccess) {
    noalloc_setup_kernel<<<1, 256, 0, stream>>>(D, n_strips, (int)n_items, a->step);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = launch_cart_stage(reinterpret_cast<const InstDesc*>(base + kDescOff),
                          reinterpret_cast<const WorkItem*>(base + kItemsOff), (int)n_items, kstage, a->order,
                          a->storage, run, vec, ly, stream);
  if (e == cudaSuccess) {
    noalloc_copyout_kernel<<<1, 32, 0, stream>>>(kstage, a->n_regions, a->qoi_out, a->status_out);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    set_error("launch failed: %s", cudaGetErrorString(e));
    return RT_ECUDA;
  }
  return RT_OK;
}
