// Autotuner of the Cartesian stage kernel: times candidate configurations
// (strip width, segment length, direction family) of one problem on the
// current device and returns the fastest. Each candidate is a complete solver
// built through the public entry points, so what is timed is what rt_step runs.
#include <cmath>
#include <cstring>
#include <tuple>
#include <vector>

#include "host_common.h"

using namespace rtk;

extern "C" rt_status rt_autotune(const rt_mesh* mesh, const rt_materials* mat, const rt_quadrature* quad,
                                 const rt_boundary* bc, const rt_options* opts, int32_t steps, rt_options* best,
                                 double* best_ms_per_step) {
  clear_error();
  if (!mesh || !opts || !best) { set_error("mesh, opts and best are required"); return RT_EINVAL; }
  if (mesh->kind != RT_MESH_CARTESIAN) {
    set_error("the autotuner covers Cartesian meshes (triangle meshes have one configuration)");
    return RT_EINVAL;
  }
  if (steps < 1 || steps > 1000) { set_error("steps must be in 1..1000"); return RT_EINVAL; }
  const cudaStream_t stream = (cudaStream_t)opts->stream;

  struct Cand { int tile_x, tile_y, variant; };
  std::vector<Cand> cands;
  const int lys[] = {0, 16, 24, 32, 40, 48, 56, 64};
  for (int tx : {16, 32})
    for (int var : {0, 1}) {
      if (tx == 32 && var == 1) continue;   // 32-cell strips exist for chunk-uniform directions only
      if (opts->variant != 0 && var != 0 && var != opts->variant) continue;
      for (int ly : lys) cands.push_back({tx, ly, var != 0 ? var : opts->variant});
    }

  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    (void)cudaGetLastError();
    set_error("event creation failed");
    return RT_ECUDA;
  }
  std::vector<std::tuple<int, int, int, int>> seen;
  double best_ms = INFINITY;
  rt_options best_opts = *opts;
  rt_status result = RT_OK;
  for (const Cand& c : cands) {
    rt_options o = *opts;
    o.tile_x = c.tile_x;
    o.tile_y = c.tile_y;
    o.variant = c.variant;
    rt_solver* s = nullptr;
    rt_status st = rt_create(mesh, mat, quad, bc, &o, &s);
    if (st == RT_EINVAL) continue;   // not available for this problem (quadrature, shared memory)
    if (st != RT_OK) { result = st; break; }
    rt_info_t info;
    rt_info(s, &info);
    const auto key = std::make_tuple(info.tile_x, info.tile_y, info.variant, info.vec);
    bool dup = false;
    for (const auto& k : seen) dup = dup || (k == key);
    const int64_t n = std::min<int64_t>(steps, info.n_steps - 1);
    if (dup || n < 1) {
      rt_destroy(s);
      if (n < 1 && !dup && std::isinf(best_ms)) {   // too few steps to time: keep the library's choice
        best_opts = o;
        best_opts.tile_x = info.tile_x;
        best_opts.tile_y = info.tile_y;
        best_opts.variant = info.variant;
        best_opts.vec = info.vec;
        best_ms = 0.0;
        break;
      }
      continue;
    }
    seen.push_back(key);
    float ms = 0.f;
    if ((st = rt_step(s, 1)) == RT_OK) {
      cudaEventRecord(e0, stream);
      st = rt_step(s, n);
      cudaEventRecord(e1, stream);
      if (st == RT_OK && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) {
        rt_qoi_t q;
        st = rt_qoi(s, &q);   // reports a device-side timeout or a non-finite state
      } else if (st == RT_OK) {
        set_error("timing a candidate failed: %s", cudaGetErrorString(cudaGetLastError()));
        st = RT_ECUDA;
      }
    }
    rt_destroy(s);
    if (st != RT_OK) { result = st; break; }
    const double per = (double)ms / (double)n;
    if (per < best_ms) {
      best_ms = per;
      best_opts = o;
      best_opts.tile_x = info.tile_x;
      best_opts.tile_y = info.tile_y;
      best_opts.variant = info.variant;
      best_opts.vec = info.vec;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (result != RT_OK) return result;
  if (std::isinf(best_ms)) { set_error("no candidate configuration could be built for this problem"); return RT_EINVAL; }
  *best = best_opts;
  if (best_ms_per_step) *best_ms_per_step = best_ms;
  return RT_OK;
}
