// Host-side building blocks shared by the single-solver and batch entry points:
// error reporting, the caller-provided allocator, and construction of one
// problem instance (validation, mesh metadata, device buffers, tensor maps,
// work items).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "rt.h"
#include "rt_internal.h"

namespace rtk {


void set_error(const char* fmt, ...);
void clear_error();

#define RT_CUDA_TRY(expr)                                                                   \
  do {                                                                                      \
    cudaError_t e_ = (expr);                                                                \
    if (e_ != cudaSuccess) {                                                                \
      ::rtk::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return RT_ECUDA;                                                                      \
    }                                                                                       \
  } while (0)

// Device memory from the caller's allocator (cudaMalloc/cudaFree when none).
struct DeviceArena {
  rt_alloc_fn alloc_fn = nullptr;
  rt_free_fn free_fn = nullptr;
  void* ctx = nullptr;
  std::vector<void*> owned;
  int64_t bytes = 0;

  rt_status get(size_t n, void** out);
  void release(void* p);   // free one block now
  void free_all();
};

struct Instance {
  int32_t kind = 0, order = 1, integrator = RT_EULER, storage = RT_FP32;
  int32_t nx = 0, ny = 0;
  int64_t n_cells = 0;
  int32_t M = 0, Mpad = 0, vec = 1;
  double dt = 0, t_end = 0;
  int64_t n_steps = 0;
  int32_t tx = 16, ly = 32, n_strips = 0, n_segs = 0;
  int32_t run = 2, cvec = 1;        // Cartesian kernel: cells per thread, ordinates per lane
  int32_t uni = 0;                  // Cartesian kernel: chunk-uniform flow directions; triangles (first
                                    // order): 1 = staged kernel (ly then holds the largest chunk halo)
  int32_t staged_ok = 0;            // triangles: the staged kernel's metadata exists (test hook switches)
  // ordinate layout: 0 the caller's order; 1 regrouped by direction quadrant,
  // each quadrant padded to whole chunks (kmap: caller k -> slot; inv: slot ->
  // caller k or -1; device arrays, NULL for the caller's order)
  int32_t regrouped = 0;
  int32_t* kmap = nullptr;
  int32_t* inv = nullptr;
  // triangles: device order of the cells (cell_perm[device index] = caller's
  // index; empty: the caller's order)
  std::vector<int32_t> cell_perm;
  int32_t n_regions = 0;
  double source_rate = 0;   // 2 pi sum_i A_i Q_i
  size_t cart_smem = 0;
  std::vector<WorkItem> stage_items;   // inst field set by the owner
  std::vector<WorkItem> init_items;
  int32_t n_boxes = 0;                 // QoI boxes
  std::vector<WorkItem> box_items;     // box outflow work items (inst field set by the owner)
  // device buffers
  void* psi[2] = {nullptr, nullptr};
  float* phi[2] = {nullptr, nullptr};
  InstState* st = nullptr;
  double* partials = nullptr;
  InstDesc desc;   // host image; pointers are device addresses
  int64_t device_bytes = 0;
};

// Validate the problem and build an instance: derive metadata, allocate and fill
// device buffers (asynchronously on `stream`; the caller synchronises), zero
// psi and phi, encode tensor maps. `d_state_slot` etc. are allocated inside.
rt_status build_instance(const rt_mesh* mesh, const rt_materials* mat, const rt_quadrature* quad,
                         const rt_boundary* bc, int order, int integrator, int storage, double dt, double t_end,
                         int tile_x, int tile_y, DeviceArena& arena, cudaStream_t stream, Instance& inst,
                         std::vector<std::vector<char>>& host_keepalive, int variant = 0, int vec = 0);

int device_sm_count();

// Launch the stage(s) of one time step for the given instances' work items.
// `run`/`cvec` select the Cartesian variant, `vec` the triangle vector width.
// d_box_items/n_box_items: the QoI-box work items of the same instances (one
// launch after the step's last stage).
rt_status launch_step(const InstDesc* d_desc, const WorkItem* d_items, int n_items, int kind, int integrator,
                      int storage, int order, int run, int cvec, int ly_max, int vec, cudaStream_t stream,
                      int uni = 0, const WorkItem* d_box_items = nullptr, int n_box_items = 0);
// Initial-state launches: phi and QoI integrands, then the box outflow.
rt_status launch_init_all(const InstDesc* d_desc, const WorkItem* d_init_items, int n_init_items,
                          const WorkItem* d_box_items, int n_box_items, int vec, int storage, cudaStream_t stream);
rt_status prepare_instance_kernels(const Instance& I, int ly_max);

// Synchronise `stream` and read an instance's device state; maps device status
// codes to RT_ETIMEOUT / RT_ENONFINITE.
rt_status read_inst_state(const Instance& I, cudaStream_t stream, InstState* h);
void fill_qoi(const Instance& I, const InstState& h, rt_qoi_t* out);
// Copy psi of buffer `buf` to host doubles [cell][M] through a bounded device buffer.
rt_status copy_psi_out(const Instance& I, DeviceArena& arena, cudaStream_t stream, int buf, double* host);
rt_status copy_psi_in(const Instance& I, DeviceArena& arena, cudaStream_t stream, int buf, const double* host);
// Copy psi of the given caller's cells of buffer `buf` to host doubles [n][M].
rt_status copy_psi_cells_out(const Instance& I, DeviceArena& arena, cudaStream_t stream, int buf,
                             const int64_t* cells, int64_t n, double* host);

}  // namespace rtk
