// Internal layout shared by the host code and the kernels of the S_N step.
// Device memory of one problem instance (all owned by the solver/batch):
//   psi[2]        psi storage (float or bf16), [n_cells][Mpad], ordinate-innermost
//   phi[2]        scalar flux phi = sum_k w_k psi_k, float [n_cells]
//   mat, region   uint8 per cell (material id, QoI region id)
//   quad          float xi[Mpad], eta[Mpad], w[Mpad] (padding: xi = eta = w = 0)
//   tri_nbr/geo   triangles only: neighbours and (n*l)/A per local edge
//   tri_geo2/lg   triangles, second order: reconstruction vectors, limited gradient
//   desc          InstDesc (tensor maps, pointers, constants)
//   state         InstState (step, buffer parity, status, FP64 QoI sums)
//   partials      FP64 per-work-item QoI partial sums [n_items][NQ]
//   box_tasks     QoI boxes: one record per (face of a box boundary, block of ordinates)
//   box_partials  FP64 per-work-item box outflow partial sums [n_box_items][2 * kMaxBox]
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace rtk {

constexpr int kMaxMat = 64;
constexpr int kMaxReg = 16;
constexpr int kMaxBox = 4;             // QoI boxes (outflow through their boundary)
constexpr int kBoxTasksPerItem = 48;   // box kernel: (face, 128-ordinate block) tasks per work item
constexpr int kQMass = kMaxReg;        // index of the mass in a QoI vector
constexpr int kQOut = kMaxReg + 1;     // index of the boundary outflow
constexpr int NQ = kMaxReg + 2;        // QoI vector: abs[16], mass, outflow
constexpr int kChunk = 32;             // ordinates per chunk (one per lane)
constexpr int kMaxUniChunks = 64;      // chunk-uniform variant: at most this many ordinate chunks
constexpr int kTriStgChunk = 32;       // cells per chunk of the staged first-order triangle kernel

enum Stage : int32_t { STAGE_EULER = 0, STAGE_HEUN1 = 1, STAGE_HEUN2 = 2, STAGE_INIT = 3 };
enum Kind : int32_t { KIND_CART = 0, KIND_TRI = 1 };

// Status codes written by kernels (same values as rt_status).
enum DevStatus : int32_t { DEV_OK = 0, DEV_TIMEOUT = 4, DEV_NONFINITE = 5 };

struct InstState {
  int64_t step;          // completed steps
  int32_t parity;        // Euler: index of the buffer holding psi^n
  int32_t status;        // DevStatus
  uint32_t ticket;       // work items finished in the current launch
  int32_t pad0;
  int64_t timeout_where; // diagnostic: encoded position of a wait that ran out
  double S_cur[NQ];      // integrands at psi^n
  double S_mid[NQ];      // Heun: integrands at psi^(1)
  double I[NQ];          // time integrals (abs, -, outflow)
  // QoI boxes: outflow through each box boundary, updated by the box kernel
  uint32_t box_ticket;   // box work items finished in the current launch
  int32_t pad1;
  int64_t box_step;      // step at the box kernel's last update (tells a masked stage)
  double B_cur[kMaxBox]; // at psi^n
  double B_I[kMaxBox];   // time integrals
};

struct alignas(128) InstDesc {
  // Cartesian tile loads (TMA). 3-D maps over psi: {Mpad, nx, ny}.
  CUtensorMap tm_psi_halo[2];   // box {32, tx + 2h, 1}, per psi buffer
  CUtensorMap tm_psi_center;    // box {32, tx, 1} over psi buffer 0 (Heun stage 2)

  void* psi[2];
  float* phi[2];
  const uint8_t* mat;
  const uint8_t* region;
  const float* xi;
  const float* eta;
  const float* w;
  const int4* tri_nbr;          // {nbr0, nbr1, nbr2, mat | region << 8}; nbr < 0: -1 - side
  const float4* tri_geo;        // 2 per cell: {ax0, ay0, ax1, ay1}, {ax2, ay2, area, eps^2}; a = (n*l)/A,
                                // eps = A^3 (the second-order limiter's, Sec. 4.2)
  InstState* st;
  double* partials;             // [n_items][NQ]

  int32_t kind, order, integrator, storage;
  int32_t nx, ny, M, Mpad;
  int32_t n_chunks, tx, ly, n_strips;
  int32_t n_segs, n_items, n_regions, pad1;
  int64_t n_cells;
  int64_t n_steps;
  int64_t wait_limit;           // device wait bound in clock64 cycles
  int64_t drop_load;            // test hook: skip this load (-1 = none)
  float inv_dx, inv_dy, dt, pad2;
  double dt_d, area_d, dx_d, dy_d;  // Cartesian cell area and sizes (FP64 QoIs)
  float ghost[4];               // inflow value per side (entering ordinates)
  int32_t uni;                  // 1: every ordinate chunk has one sign of xi and one of eta
  int8_t cdir_x[kMaxUniChunks]; // per chunk: sign of xi (+1/-1) when uni
  int8_t cdir_y[kMaxUniChunks]; // per chunk: sign of eta
  float sig_t[kMaxMat];
  float sig_s2pi[kMaxMat];      // sigma_s / (2 pi)
  float q_src[kMaxMat];
  float sig_a_f[kMaxMat];       // sigma_a as float (per-cell QoI terms; no FP64 in hot loops)
  double sig_a[kMaxMat];
  // QoI boxes: task records {inside cell, outside cell, the inside cell's other
  // neighbour along the normal, box | side << 8 | block << 12}, one per face of
  // a box boundary and block of 128 ordinates holding an ordinate that leaves
  // through it (side 0..3: the box's x-, x+, y-, y+ side, named by its outward
  // normal)
  const int4* box_tasks;
  double* box_partials;         // [n_box_items][2 * kMaxBox]
  int32_t n_boxes, n_box_tasks;  // triangles, second order: per cell {r0x, r0y, r1x, r1y}, {r2x, r2y, d0x, d0y},
  // {d1x, d1y, d2x, d2y} (r_e: centroid to edge midpoint; d_e: centroid to the
  // neighbour's centroid, 0 on the boundary), and the limited gradient L g,
  // FP32 [cell][2][Mpad] (x row, then y row)
  const float4* tri_geo2;
  float* tri_lg;
  int32_t periodic_x;           // Cartesian: 1 if the x- and x+ sides are periodic (no boundary faces in x)
  int32_t periodic_y;           // Cartesian: 1 if the y- and y+ sides are periodic
  // triangles, staged first-order kernel: per chunk of kTriStgChunk cells
  // {offset, count} of its halo (the cells outside the chunk that share an edge
  // with it; offsets are multiples of 4), the halo ids, and per cell the slots of
  // its three neighbours among the chunk's staged rows (byte e: 0..31 the chunk's
  // own cells, 32 + h halo cell h, 255 a boundary edge); tri_hmax = the largest
  // halo (multiple of 4)
  const int2* tri_halo_oc;
  const int32_t* tri_halo;
  const uint32_t* tri_lidx;
  int32_t tri_hmax;
  int32_t pad3;
};

struct WorkItem {
  int32_t inst;       // index into the InstDesc array
  int32_t a;          // Cartesian stage: strip; cell-range kernels: first cell
  int32_t b;          // Cartesian stage: segment; cell-range kernels: number of cells
  int32_t item;       // index of this item within its instance (partials row)
  int32_t count;      // items of this instance in this launch (last one finalizes)
  int32_t pad;
};

// Launchers (defined in the .cu files). All enqueue on `stream`.
// Cartesian stage kernel variants: run = cells per thread in x (tile width 8*run),
// vec = ordinates per lane (chunk of 32*vec ordinates).
// uni = 1 selects the chunk-uniform variant (InstDesc::cdir_x/y set per chunk).
cudaError_t launch_cart_stage(const InstDesc* d_desc, const WorkItem* d_items, int n_items, int stage,
                              int order, int storage, int run, int vec, int ly_max, cudaStream_t stream,
                              int uni = 0);
size_t cart_smem_bytes(int order, int storage, int run, int vec, int ly, int stage);
cudaError_t prepare_cart_stage(int stage, int order, int storage, int run, int vec, int ly_max, int uni = 0);
int cart_tile_width(int run);
bool cart_variant_exists(int order, int run, int vec, int uni = 0);
cudaError_t launch_tri_stage(const InstDesc* d_desc, const WorkItem* d_items, int n_items, int stage,
                             int storage, int vec, cudaStream_t stream);
// Staged first-order triangle stage (rows of a chunk's cells and halo in shared
// memory, one 512-thread CTA per SM): hmax = the instances' largest halo.
cudaError_t launch_tri_staged(const InstDesc* d_desc, const WorkItem* d_items, int n_items, int stage, int storage,
                              int vec, int hmax, cudaStream_t stream);
cudaError_t prepare_tri_staged(int stage, int storage, int vec, int hmax);
size_t tri_staged_smem_bytes(int vec, int storage, int hmax, int stage);
cudaError_t launch_init(const InstDesc* d_desc, const WorkItem* d_items, int n_items, int vec,
                        int storage, cudaStream_t stream);
// Second-order triangle stage: the limited-gradient kernel (grad_vec ordinates
// per lane: 1, 2 or 4), then the stage kernel (vec 1 or 2).
cudaError_t launch_tri2_stage(const InstDesc* d_desc, const WorkItem* d_items, int n_items, int stage,
                              int storage, int vec, int grad_vec, cudaStream_t stream);
// Outflow through the QoI boxes after a time step (stage = STAGE_EULER, or
// STAGE_HEUN2 after a whole Heun step) with the step's time-integration
// update, or of the current state (STAGE_INIT). Work items: a = first face,
// b = number of tasks (at most kBoxTasksPerItem).
cudaError_t launch_box_outflow(const InstDesc* d_desc, const WorkItem* d_items, int n_items, int stage,
                               int storage, cudaStream_t stream);
// FP64 [cell][M] (caller's ordinate order) <-> storage [cell][Mpad] (internal
// order); inv: internal slot -> caller ordinate or -1, kmap: caller ordinate ->
// slot (device arrays; NULL when the orders agree).
cudaError_t launch_convert_in(const double* src, void* dst, int64_t n_cells, int M, int Mpad, int storage,
                              const int32_t* inv, cudaStream_t stream);
cudaError_t launch_convert_out(const void* src, double* dst, int64_t n_cells, int M, int Mpad, int storage,
                               const int32_t* kmap, cudaStream_t stream);

}  // namespace rtk
