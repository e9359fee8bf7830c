/*
 * rt.h - C ABI of the GB300 (sm_103a) explicit S_N transport step.
 *
 * One solver advances the 2-D discrete-ordinates system with isotropic
 * scattering (Sec. 4.1, Eq. sn_2d)
 *
 *   d/dt psi_k + xi_k d/dx psi_k + eta_k d/dy psi_k + sigma_t psi_k
 *       = sigma_s/(2 pi) sum_l w_l psi_l + Q,      sum_k w_k = 2 pi,
 *
 * discretised by cell-centred finite volumes with upwind traces (Sec. 4.2,
 * Eq. sn_2d_eqn_fv and Eq. upwind1stOrder; first order, or MUSCL with a
 * minmod limiter on Cartesian grids), ghost cells holding psi^- on boundary
 * faces with first-order boundary fluxes (Sec. 4.2), and forward Euler or
 * Heun's method with uniform dt = T/N_t (Sec. 4.3). Every step runs in CUDA
 * kernels on the caller's stream; the host only validates, derives mesh
 * metadata once and enqueues launches.
 *
 * Conventions
 *   - All array arguments are host pointers unless stated. Inputs are copied
 *     during rt_create; the caller keeps ownership of its arrays.
 *   - Device memory comes only from rt_options.alloc/free (cudaMalloc and
 *     cudaFree when alloc is NULL). Launches and copies go to rt_options.stream
 *     (a cudaStream_t; NULL = legacy default stream) on the device that is
 *     current when rt_create is called.
 *   - psi is stored ordinate-innermost: psi[cell][k], k = 0..M-1, padded on the
 *     device to a multiple of 32 ordinates with zero-weight ordinates.
 *     Cartesian cell id = j*nx + i (x fastest).
 *   - Functions return rt_status; no exception crosses the ABI. The message of
 *     the last failure on the calling thread is rt_last_error().
 *   - After a device error, a wait that ran out (RT_ETIMEOUT) or a non-finite
 *     QoI (RT_ENONFINITE) the solver enters an error state: every later call
 *     but rt_destroy returns RT_ESTATE.
 */
#ifndef RT_GB300_H
#define RT_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RT_OK = 0,
  RT_EINVAL = 1,      /* an argument is invalid; nothing was changed */
  RT_ENOMEM = 2,      /* the allocator returned NULL */
  RT_ECUDA = 3,       /* a CUDA runtime/driver call failed */
  RT_ETIMEOUT = 4,    /* a bounded device-side wait ran out */
  RT_ENONFINITE = 5,  /* the solution became non-finite (NaN/Inf in a QoI) */
  RT_ESTATE = 6       /* the solver is in its error state */
} rt_status;

enum { RT_MESH_CARTESIAN = 0, RT_MESH_TRIANGLES = 1 };
enum { RT_BC_VACUUM = 0, RT_BC_INFLOW = 1, RT_BC_PERIODIC = 2 };
enum { RT_EULER = 0, RT_HEUN = 1 };
enum { RT_FP32 = 0, RT_BF16 = 1 };
enum { RT_SIDE_XMIN = 0, RT_SIDE_XMAX = 1, RT_SIDE_YMIN = 2, RT_SIDE_YMAX = 3 };

#define RT_MAX_MATERIALS 64
#define RT_MAX_REGIONS 16
#define RT_MAX_BOXES 4

/* Spatial mesh (Sec. 4.2).
 *   kind = RT_MESH_CARTESIAN: nx x ny rectangles of size dx x dy with lower-left
 *     corner (x0, y0); cell id j*nx + i.
 *   kind = RT_MESH_TRIANGLES: n_vert vertices vxy[2*v + {0,1}] and n_tri
 *     counter-clockwise triangles tri[3*t + {0,1,2}] (vertex ids). Edges used by
 *     one triangle only are boundary edges; each is assigned to the side
 *     (x-, x+, y-, y+) of the vertices' bounding box nearest to its midpoint.
 *     Local edge e of a triangle runs from its vertex e to vertex (e+1)%3. */
typedef struct {
  int32_t kind;
  int32_t nx, ny;
  double x0, y0, dx, dy;
  int64_t n_vert;
  const double* vxy;
  int64_t n_tri;
  const int32_t* tri;
} rt_mesh;

/* Piecewise-constant materials (Sec. 3.1, 3.2): per material sigma_a, sigma_s
 * (sigma_t = sigma_a + sigma_s) and isotropic source Q; per cell a material id
 * (0..n_mat-1) and a QoI region id (0..n_regions-1). n_mat <= RT_MAX_MATERIALS
 * (64: one material per block of the 7 x 7 lattice, the per-block parameters
 * of Sec. 3.1.3, fits), n_regions <= RT_MAX_REGIONS. */
typedef struct {
  int32_t n_mat;
  const double* sigma_a;
  const double* sigma_s;
  const double* Q;
  const int32_t* cell_mat;
  const int32_t* cell_region;
  int32_t n_regions;
  /* QoI boxes (Sec. 3.1 QoI-1/2: the squares S_l, l in {1.5, 2.5}, of the
   * lattice): n_boxes (0..RT_MAX_BOXES) axis-aligned rectangles
   * boxes[4 b + {0,1,2,3}] = {x_lo, x_hi, y_lo, y_hi}. Cartesian meshes only.
   * Every edge must lie on a grid line (within 1e-9 relative) strictly inside
   * the domain, so that each face of a box has a cell on both sides. For each
   * box the library reports the particle flow leaving it (rt_qoi_t.box_out_*).
   * n_boxes = 0 (boxes may be NULL): none. */
  int32_t n_boxes;
  const double* boxes;
} rt_materials;

/* Ordinates on the upper hemisphere (Sec. 4.1): direction components xi_k,
 * eta_k (|(xi,eta)| <= 1) and weights w_k, k = 0..M-1. The weights should sum
 * to 2 pi (the scattering term uses sigma_s/(2 pi) sum_l w_l psi_l). */
typedef struct {
  int64_t M;
  const double* xi;
  const double* eta;
  const double* w;
} rt_quadrature;

/* Boundary per side (x-, x+, y-, y+): RT_BC_VACUUM (psi^- = 0), RT_BC_INFLOW
 * (isotropic psi^- = inflow[side] for ordinates entering through that side) or
 * RT_BC_PERIODIC. Periodic sides come in pairs (x- with x+, y- with y+) and
 * are supported on Cartesian meshes: the cell across a periodic side is the
 * cell at the other end of the row or column, so the axis has no boundary
 * faces (its fluxes telescope, Sec. 4.2, and nothing leaves through it; MUSCL
 * slopes and faces stay second order there). RT_EINVAL for an unpaired
 * periodic side or a periodic side of a triangle mesh. */
typedef struct {
  int32_t side_kind[4];
  double inflow[4];
} rt_boundary;

typedef void* (*rt_alloc_fn)(size_t bytes, void* ctx);
typedef void (*rt_free_fn)(void* ptr, void* ctx);

/* Solver options.
 *   order: 1 (first-order upwind) or 2: on Cartesian meshes MUSCL with minmod
 *     slopes per dimension; on triangle meshes the paper's reconstruction
 *     (Sec. 4.2): Green-Gauss gradient, Venkatakrishnan limiter with
 *     Delta = g.r/2 and epsilon = A^3, first-order fluxes on boundary edges
 *     (one extra gradient launch per stage and 8 bytes per cell and ordinate
 *     of device memory for the limited gradient).
 *   integrator: RT_EULER or RT_HEUN.  storage: RT_FP32 or RT_BF16 (psi storage;
 *     arithmetic is FP32 either way, QoI accumulation FP64).
 *   dt > 0: target step; N_t = ceil(t_end/dt - 1e-9) and dt = t_end/N_t.
 *   dt <= 0: Cartesian 0.5*min(dx,dy); triangles 0.9*min_i 2 A_i / P_i.
 *   tile_x, tile_y: Cartesian tile: cells per strip in x (16: runs of 2 cells per
 *     warp; 32: runs of 4, which needs chunk-uniform directions with 2 ordinates
 *     per lane) and rows per segment (at most 256); 0 = chosen by the library.
 *   variant: Cartesian kernel variant. 0 = chosen by the library; 1 = per-lane
 *     flow directions (any quadrature); 2 = chunk-uniform directions, usable when
 *     every chunk of ordinates has one sign of xi and one of eta (the product
 *     quadrature's quadrants are contiguous); RT_EINVAL if it is not. The
 *     library takes chunk-uniform directions where the chunks allow them, except
 *     where only 32-cell strips would (2 ordinates per lane) on a grid of at most
 *     1e5 cells: there the per-lane variant measured faster.
 *   vec: Cartesian ordinates per lane (1, 2 or 4; 0 = chosen by the library);
 *     RT_EINVAL if the quadrature does not allow it (see rt_info_t for the choice).
 *   alloc/free/alloc_ctx: device allocator (NULL = cudaMalloc/cudaFree).
 *   stream: cudaStream_t for every launch and copy. */
typedef struct {
  int32_t order;
  int32_t integrator;
  int32_t storage;
  int32_t tile_x;
  int32_t tile_y;
  int32_t variant;
  double dt;
  double t_end;
  rt_alloc_fn alloc;
  rt_free_fn free;
  void* alloc_ctx;
  void* stream;
  int32_t vec;
  int32_t pad;
} rt_options;

/* QoIs (Sec. 3.1 QoI-3..5, Sec. 3.2 QoI-2, QoI-7), FP64:
 *   abs_now[r]  = sum_{i in region r} A_i sigma_a,i phi_i at time t
 *   abs_int[r]  = time integral of abs_now[r] over [0, t]
 *   mass        = sum_i A_i phi_i at time t
 *   outflow_now = sum over boundary faces of l sum_k w_k (omega_k . n) psi_hat_k
 *   outflow_int = its time integral; source_int = t * 2 pi sum_i A_i Q_i.
 * Time integrals use the weights of the scheme (Euler: dt*S(psi^n); Heun:
 * dt/2*(S(psi^n) + S(psi^(1)))), so mass + sum(abs_int) + outflow_int equals
 * mass(0) + source_int up to rounding. */
typedef struct {
  double t;
  int64_t step;
  int64_t n_steps;
  int32_t n_regions;
  int32_t status;
  double abs_now[RT_MAX_REGIONS];
  double abs_int[RT_MAX_REGIONS];
  double mass;
  double outflow_now;
  double outflow_int;
  double source_int;
  /* QoI boxes (rt_materials.boxes), b < n_boxes:
   *   box_out_now[b] = sum over the faces f of the box's boundary of
   *     l_f sum_k w_k max(omega_k . n_f, 0) psi_hat_k,f at time t, n_f the
   *     normal pointing out of the box and psi_hat the scheme's upwind trace
   *     (for a leaving ordinate, the inside cell's value at first order, its
   *     MUSCL-minmod reconstruction at second order): Sec. 3.1 QoI-1;
   *   box_out_int[b] = its time integral with the scheme's weights: QoI-2. */
  int32_t n_boxes;
  int32_t pad;
  double box_out_now[RT_MAX_BOXES];
  double box_out_int[RT_MAX_BOXES];
} rt_qoi_t;

/* Static facts about a solver. */
typedef struct {
  int64_t n_cells;
  int64_t M;
  int64_t M_pad;
  int64_t n_steps;
  double dt;
  double t_end;
  int32_t kind, order, integrator, storage;
  int32_t tile_x, tile_y, n_work_items, stages_per_step;
  int64_t device_bytes;
  int32_t variant;   /* kernel variant in use: Cartesian 1 per-lane, 2 chunk-uniform directions;
                        triangles 3 first order with each chunk's rows staged in shared memory,
                        0 otherwise (rows gathered from global memory) */
  int32_t vec;       /* ordinates per lane */
  int32_t regrouped; /* Cartesian: 1 if the ordinates are stored regrouped by direction quadrant, each
                        quadrant padded with zero-weight ordinates to whole chunks (done when the
                        caller's order does not give sign-uniform chunks and the padding adds at most
                        1/8; M_pad is then the padded count). rt_get_psi / rt_set_psi always use the
                        caller's order; rt_device_state exposes the internal one. */
  int32_t n_box_items; /* QoI boxes: work items of the box-outflow launch that follows each time
                          step's last stage (0: no boxes, no such launch) */
} rt_info_t;

typedef struct rt_solver rt_solver;

/* Product quadrature (Sec. 4.1 with the tensorised Gauss-Legendre rule named in
 * Sec. 5.1.1): n_p Gauss-Legendre points on mu in [0,1] times n_phi azimuths
 * varphi_a = (a + 1/2) 2 pi / n_phi; k = a*n_p + p; xi = sqrt(1-mu^2) cos varphi,
 * eta = sqrt(1-mu^2) sin varphi (Eq. polar_coordinates), w = w_p * 2 pi/n_phi
 * (sum 2 pi). Writes n_p*n_phi values to each host array (mu may be NULL).
 * RT_EINVAL if n_p < 1, n_p > 64, n_phi < 1 or an output pointer is NULL. */
rt_status rt_quad_product(int32_t n_p, int32_t n_phi, double* xi, double* eta, double* mu, double* w);

/* Tessellation quadrature of order N (Sec. 5.1.1, the paper's own choice): each
 * of the four upper faces of the octahedron with vertices (+-1,0,0), (0,+-1,0),
 * (0,0,1) is split into N^2 congruent triangles by dividing its edges into N
 * parts; a triangle's ordinate is its centroid scaled to the unit sphere and
 * its weight the area of the spherical triangle spanned by its corners scaled
 * to the sphere (spherical excess), so the weights sum to 2 pi. M = 4 N^2
 * ordinates in face order (the quadrants xi>0,eta>0; xi<0,eta>0; xi<0,eta<0;
 * xi>0,eta<0, N^2 each); within a face, rows j = 0..N-1 from the equator up and
 * in each row i = 0..N-1-j the upward triangle (i,j), then, if i < N-1-j, the
 * downward one. Writes M values to each host array (mu may be NULL). RT_EINVAL
 * if N < 1, N > 128 or an output pointer is NULL. */
rt_status rt_quad_tessellation(int32_t N, double* xi, double* eta, double* mu, double* w);

/* Create a solver for one problem: validates, derives per-cell metadata
 * (triangles: areas, n*l/A per edge, neighbours, boundary sides), allocates
 * device state, sets psi(0) = 0 and evaluates phi and the QoI integrands of the
 * initial state. RT_EINVAL on invalid input (message in rt_last_error),
 * RT_ENOMEM if the allocator fails, RT_ECUDA on a CUDA failure. On failure
 * *out is NULL and nothing is leaked. */
rt_status rt_create(const rt_mesh* mesh, const rt_materials* mat, const rt_quadrature* quad,
                    const rt_boundary* bc, const rt_options* opts, rt_solver** out);

/* Enqueue n time steps (clamped at N_t) on the solver's stream; returns after
 * enqueueing. Each step is one launch (Euler) or two (Heun stages); second order
 * on triangles adds a gradient launch before each stage, and QoI boxes one
 * launch after the step's last stage. */
rt_status rt_step(rt_solver* s, int64_t n);

/* Synchronise the stream and copy the QoIs to *out (392 bytes). Returns
 * RT_ETIMEOUT / RT_ENONFINITE (and enters the error state) if a kernel
 * reported one. */
rt_status rt_qoi(rt_solver* s, rt_qoi_t* out);

/* Static facts (no synchronisation). */
rt_status rt_info(const rt_solver* s, rt_info_t* out);

/* Copy psi (n = n_cells*M doubles, [cell][k]) or phi (n = n_cells doubles) of the
 * current state to host memory; synchronises. RT_EINVAL if n is wrong. */
rt_status rt_get_psi(rt_solver* s, double* host, int64_t n);

/* Copy psi of n selected cells (caller's cell ids in cells[0..n), any order,
 * repeats allowed) to host[n][M] doubles, ordinates in the caller's order;
 * synchronises. For probing a large state without copying all of it (a
 * 1400^2 x 512 lattice holds 8 GB as doubles). RT_EINVAL if n < 0, a pointer
 * is NULL (with n > 0) or a cell id is out of range (nothing copied then). */
rt_status rt_get_psi_cells(rt_solver* s, const int64_t* cells, int64_t n, double* host);
rt_status rt_get_phi(rt_solver* s, double* host, int64_t n);

/* Replace the current state by psi (n = n_cells*M doubles, [cell][k]); rounds to
 * the storage type, recomputes phi and the QoI integrands. Time, step count and
 * time integrals are kept. Synchronises. */
rt_status rt_set_psi(rt_solver* s, const double* host, int64_t n);

/* Device view of the current state: psi (storage type, [cell][M_pad], ordinates
 * in the internal order: the caller's unless rt_info_t.regrouped) and phi
 * (float, [cell]). Triangle meshes keep their cells in an internal order (the
 * Morton order of the centroids, ties by the caller's index); Cartesian meshes
 * in the caller's. rt_get_psi, rt_set_psi and rt_get_phi always use the
 * caller's orders. Pointers stay owned by the solver and are valid until the
 * next rt_step (Euler alternates two buffers) or rt_destroy. */
rt_status rt_device_state(rt_solver* s, void** psi, void** phi, int32_t* storage);

/* Checkpoint: the full state (psi as stored, phi, step, time integrals, current
 * integrands) as an opaque byte blob of rt_state_size() bytes. rt_set_state
 * restores a blob taken from a solver created with the same arguments; a run
 * resumed from it matches the uninterrupted run bit for bit. Both synchronise. */
rt_status rt_state_size(const rt_solver* s, size_t* bytes);
rt_status rt_get_state(rt_solver* s, void* host, size_t bytes);
rt_status rt_set_state(rt_solver* s, const void* host, size_t bytes);

/* Test hooks, not for production use: key "wait_limit_cycles" bounds every
 * device-side wait (default about two seconds of SM clock); key "drop_load"
 * (value q >= 0) makes the Cartesian kernel skip its q-th tile load, so that the
 * wait for it runs out and the launch reports RT_ETIMEOUT. value < 0 clears.
 * Key "tri_staged" (first-order triangle solvers): 1 runs the stage with the
 * kernel that stages each chunk's rows in shared memory (the default), 0 with
 * the kernel that gathers neighbour rows from global memory; RT_EINVAL for
 * other solvers. */
rt_status rt_debug_set(rt_solver* s, const char* key, int64_t value);

void rt_destroy(rt_solver* s);

/* Message of the last failure on this thread ("" if none). */
const char* rt_last_error(void);

/* ---------------------------------------------------------------------------
 * Autotuner (Cartesian meshes). The paper has no counterpart: it chooses among
 * the library's own kernel configurations. For the problem and options given,
 * each candidate (strip width 16 or 32 cells, segment length in {auto, 16, 24,
 * ..., 64} rows, per-lane or chunk-uniform directions; only those the
 * quadrature and shared memory allow, and opts->variant/vec if set) is built
 * as a full solver with rt_create, advanced one step, then timed with CUDA
 * events over `steps` further steps (at most N_t - 1) on opts->stream, and
 * destroyed. *best receives opts with tile_x, tile_y, variant and vec of the
 * fastest candidate (so rt_create(..., best, ...) builds it), and
 * *best_ms_per_step (may be NULL) its time per step. Device memory: one
 * candidate's state at a time, allocated as rt_create does. When N_t < 2 the
 * library's own choice is returned with time 0. RT_EINVAL for triangle meshes,
 * steps outside 1..1000 or an invalid problem; errors of rt_create, rt_step or
 * a device-side failure of a candidate are returned as they are. Synchronises
 * opts->stream. */
rt_status rt_autotune(const rt_mesh* mesh, const rt_materials* mat, const rt_quadrature* quad, const rt_boundary* bc,
                      const rt_options* opts, int32_t steps, rt_options* best, double* best_ms_per_step);

/* ---------------------------------------------------------------------------
 * Batches: many independent problems advanced together by shared launches.
 * The paper has no batching; the problems are, for example, the lattice
 * design-parameter sweeps of Sec. 3.1.3 (DP-1) or a stream of solve requests.
 * A batch has a fixed number of slots. Each stage of a step is one launch per
 * kernel variant over the work items of every unfinished problem (finished
 * problems are also masked on the device), so many small problems fill the GPU
 * together. Problems may differ in mesh kind, grid, ordinates, order and
 * integrator; they share the storage type, allocator and stream. Problems can
 * be added and removed between steps (continuous batching); each problem's
 * device memory is its own and is freed when it is removed.
 * ------------------------------------------------------------------------- */
typedef struct {
  rt_mesh mesh;
  rt_materials mat;
  rt_quadrature quad;
  rt_boundary bc;
  int32_t order;
  int32_t integrator;
  double dt;       /* as rt_options.dt */
  double t_end;
  int32_t tile_y;  /* as rt_options; 0 = the batch options' value */
  int32_t variant;
  int32_t vec;
  int32_t pad;
} rt_problem;

typedef struct rt_batch rt_batch;

/* Create a batch with `capacity` slots (0 = k) holding the k problems given
 * (slots 0..k-1, k may be 0). Storage, allocator, stream and default kernel
 * options come from opts (its order/integrator/dt/t_end are not used).
 * Errors as rt_create; on failure *out is NULL and nothing is leaked. */
rt_status rt_batch_create(int32_t k, const rt_problem* problems, int32_t capacity, const rt_options* opts,
                          rt_batch** out);

/* Add a problem in a free slot; *slot receives its index. Creates and
 * initialises its device state (synchronises the stream). RT_EINVAL if the
 * problem is invalid or no slot is free, RT_ENOMEM if the allocator fails;
 * the batch is unchanged then. */
rt_status rt_batch_add(rt_batch* b, const rt_problem* problem, int32_t* slot);

/* Remove the problem in `slot` and free its device memory (synchronises). */
rt_status rt_batch_remove(rt_batch* b, int32_t slot);

/* Enqueue up to n steps of every unfinished problem (each stops at its own
 * N_t) and return. While the set of unfinished problems and n stay the same,
 * calls replay one captured CUDA graph. */
rt_status rt_batch_step(rt_batch* b, int64_t n);

/* Advance every problem to its own N_t (at most max_steps steps per problem
 * when max_steps > 0); enqueues and returns. */
rt_status rt_batch_run(rt_batch* b, int64_t max_steps);

/* Hold (hold != 0) or release (hold = 0) the problem in `slot`: a held problem
 * keeps its state on the device but is left out of rt_batch_step and
 * rt_batch_run until released, so a scheduler can choose which problems the
 * shared launches advance (the serving loop gives the GPU to the oldest
 * requests first). The paper has no counterpart. Takes effect at the next
 * step (the work list is rebuilt then); no synchronisation. RT_EINVAL for an
 * empty slot. */
rt_status rt_batch_hold(rt_batch* b, int32_t slot, int32_t hold);

/* Steps enqueued so far for the problem in `slot` and its N_t (no
 * synchronisation). RT_EINVAL for an empty slot. */
rt_status rt_batch_progress(const rt_batch* b, int32_t slot, int64_t* steps_done, int64_t* n_steps);

/* Kernel launches this batch has issued so far, counted as they are enqueued:
 * one initial-state launch per added problem (plus one QoI-box launch if it
 * has boxes), then per step the stage launches of every kernel-variant group
 * (two with Heun, one with Euler) and one QoI-box launch per run of groups
 * ending on the same stage; a graph replay counts every launch it holds. For
 * reports of the work done on the device; no synchronisation. RT_EINVAL for
 * NULL arguments. The paper has no counterpart. */
rt_status rt_batch_launches(const rt_batch* b, int64_t* n);

/* Synchronise and copy the QoIs of the problem in `slot`. */
rt_status rt_batch_qoi(rt_batch* b, int32_t slot, rt_qoi_t* out);

/* Copy psi of the problem in `slot` ([cell][k] doubles, n = n_cells*M). */
rt_status rt_batch_get_psi(rt_batch* b, int32_t slot, double* host, int64_t n);

void rt_batch_destroy(rt_batch* b);

/* ---------------------------------------------------------------------------
 * One Cartesian stage without device allocation.
 *
 * The paper has no counterpart of this call. Some callers cannot let a library
 * allocate GPU memory: applications whose device memory is fully reserved by
 * their own allocator or memory pool (a library cudaMalloc would fail there, or
 * bypass their accounting), and loops that must not take the implicit device
 * synchronisation of cudaMalloc/cudaFree. rt_cart_stage_noalloc runs the same
 * Cartesian stage kernel as rt_step on buffers the caller owns, and allocates
 * nothing: the kernel's scratch memory (descriptor with TMA tensor maps, work
 * list, launch state and FP64 partial sums) lives in a fixed file-scope device
 * array of about 1.4 MB, which every GPU that loads the library keeps until the
 * process exits. Consequences:
 *   - grids needing more than RT_NOALLOC_MAX_WORK_ITEMS work items (strips of
 *     16 cells x tile_y rows) are rejected with RT_EINVAL;
 *   - every call shares the array; each call clears the parts that must start
 *     at zero, but calls that overlap on the GPU (e.g. on two streams) race;
 *   - the first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 * Arguments (all device pointers unless stated; layout as rt_device_state):
 *   nx, ny, dx, dy: Cartesian grid; M_pad: ordinates per cell in the psi layout
 *   [cell][M_pad] (a multiple of 32; padding ordinates must have xi = eta = w = 0);
 *   vec: ordinates per lane (1, 2 or 4; 0 means 1) - every group of vec
 *   consecutive ordinates must share the sign of xi (the kernel takes each
 *   lane's upwind direction in x from the group's summed xi, so a group that
 *   mixes signs gives wrong results, not an error, unless xi_host is given);
 *   order 1 or 2; stage
 *   RT_STAGE_EULER / RT_STAGE_HEUN1 (psi_out = psi_in + dt F(psi_in)) or
 *   RT_STAGE_HEUN2 (psi_out = (psi_n + psi_in + dt F(psi_in))/2; psi_out may be
 *   psi_n); storage RT_FP32 or RT_BF16; tile_y rows per work item (0 = default);
 *   material table on the host (n_mat <= 64, n_regions <= 16); inflow psi^- per
 *   side (x-, x+, y-, y+; 0 = vacuum); dt; psi_in, psi_n, psi_out (16-byte
 *   aligned, psi_out distinct from psi_in); phi_in = sum_k w_k psi_in,k and
 *   phi_out (float [cell]); cell_mat, cell_region (uint8 [cell]); xi, eta, w
 *   (float [M_pad]); qoi_out (double [n_regions + 2]: absorption per region,
 *   mass, boundary outflow of the output state); status_out (int32, optional:
 *   0, RT_ETIMEOUT or RT_ENONFINITE once the stream reaches it; every call
 *   starts from status 0, so a failed call does not carry over); stream;
 *   step: index of the time step this stage belongs to (n for the stages that
 *   advance psi^n; Heun's two stages share it). BF16 storage rounds
 *   stochastically with random bits drawn from (element, step, stage), so
 *   successive steps must pass successive indices: the same index on every
 *   step would reuse the same bits and bias the rounding. With the indices of
 *   rt_step (0, 1, 2, ...) the stored results match rt_step's. FP32 ignores it.
 *   xi_host (host pointer, optional): a host copy of xi[0..M_pad); when given,
 *   the call first checks that every group of vec consecutive ordinates
 *   shares the sign of xi and returns RT_EINVAL if one does not.
 * Enqueues on `stream` and returns; RT_EINVAL on invalid arguments (nothing is
 * launched), RT_ECUDA if a launch fails. */
#define RT_NOALLOC_MAX_WORK_ITEMS 8192
enum { RT_STAGE_EULER = 0, RT_STAGE_HEUN1 = 1, RT_STAGE_HEUN2 = 2 };
typedef struct {
  int32_t nx, ny;
  double dx, dy;
  int32_t M_pad, vec;
  int32_t order, stage, storage, tile_y;
  int32_t n_mat, n_regions;
  double sigma_a[RT_MAX_MATERIALS], sigma_s[RT_MAX_MATERIALS], Q[RT_MAX_MATERIALS];
  double inflow[4];
  double dt;
  const void* psi_in;
  const void* psi_n;
  void* psi_out;
  const float* phi_in;
  float* phi_out;
  const uint8_t* cell_mat;
  const uint8_t* cell_region;
  const float* xi;
  const float* eta;
  const float* w;
  double* qoi_out;
  int32_t* status_out;
  void* stream;
  int64_t step;
  const float* xi_host;
} rt_cart_stage_args;

rt_status rt_cart_stage_noalloc(const rt_cart_stage_args* args);

#ifdef __cplusplus
}
#endif
#endif /* RT_GB300_H */
