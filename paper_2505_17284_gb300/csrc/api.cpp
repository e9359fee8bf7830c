// C ABI of the single-problem solver: create, step (direct launches or CUDA
// graph replays on the caller's stream), QoIs, state access and checkpoints.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "host_common.h"

namespace rtk {
const char* last_error_cstr();
}

using namespace rtk;

struct rt_solver {
  DeviceArena arena;
  Instance I;
  cudaStream_t stream = nullptr;       // caller's stream
  cudaStream_t cap_stream = nullptr;   // private stream used only to capture graphs
  InstDesc* d_desc = nullptr;
  WorkItem* d_stage_items = nullptr;
  WorkItem* d_init_items = nullptr;
  WorkItem* d_box_items = nullptr;     // QoI boxes (none: nullptr)
  int64_t host_step = 0;               // steps enqueued
  bool failed = false;
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
};

namespace {

constexpr int kGraphSteps = 16;

rt_status fail(rt_solver* s, rt_status st) {
  if (s && st != RT_OK && st != RT_EINVAL) s->failed = true;
  return st;
}

rt_status launch_steps_direct(rt_solver* s, int64_t n, cudaStream_t stream) {
  const Instance& I = s->I;
  for (int64_t i = 0; i < n; ++i) {
    rt_status st = launch_step(s->d_desc, s->d_stage_items, (int)I.stage_items.size(), I.kind, I.integrator,
                               I.storage, I.order, I.run, I.cvec, I.ly, I.vec, stream, I.uni, s->d_box_items,
                               (int)I.box_items.size());
    if (st != RT_OK) return st;
  }
  return RT_OK;
}

rt_status ensure_graph(rt_solver* s) {
  if (s->graph) return RT_OK;
  if (!s->cap_stream) RT_CUDA_TRY(cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  RT_CUDA_TRY(cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
  rt_status st = launch_steps_direct(s, kGraphSteps, s->cap_stream);
  cudaError_t e = cudaStreamEndCapture(s->cap_stream, &g);
  if (st != RT_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) {
    set_error("graph capture failed: %s", cudaGetErrorString(e));
    return RT_ECUDA;
  }
  e = cudaGraphInstantiate(&s->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    s->graph = nullptr;
    set_error("graph instantiation failed: %s", cudaGetErrorString(e));
    return RT_ECUDA;
  }
  s->graph_steps = kGraphSteps;
  return RT_OK;
}

rt_status read_state(rt_solver* s, InstState* h) { return read_inst_state(s->I, s->stream, h); }

rt_status run_init(rt_solver* s) {
  const Instance& I = s->I;
  return launch_init_all(s->d_desc, s->d_init_items, (int)I.init_items.size(), s->d_box_items,
                         (int)I.box_items.size(), I.vec, I.storage, s->stream);
}

size_t elem_size(const Instance& I) { return I.storage == RT_BF16 ? 2 : 4; }

}  // namespace

extern "C" {

const char* rt_last_error(void) { return last_error_cstr(); }

rt_status rt_create(const rt_mesh* mesh, const rt_materials* mat, const rt_quadrature* quad, const rt_boundary* bc,
                    const rt_options* opts, rt_solver** out) {
  clear_error();
  if (!out) { set_error("out is NULL"); return RT_EINVAL; }
  *out = nullptr;
  if (!opts) { set_error("options are NULL"); return RT_EINVAL; }
  if ((opts->alloc == nullptr) != (opts->free == nullptr)) { set_error("alloc and free must both be set or both NULL"); return RT_EINVAL; }
  rt_solver* s = new rt_solver();
  s->arena.alloc_fn = opts->alloc;
  s->arena.free_fn = opts->free;
  s->arena.ctx = opts->alloc_ctx;
  s->stream = (cudaStream_t)opts->stream;
  std::vector<std::vector<char>> keep;
  rt_status st = build_instance(mesh, mat, quad, bc, opts->order, opts->integrator, opts->storage, opts->dt,
                                opts->t_end, opts->tile_x, opts->tile_y, s->arena, s->stream, s->I, keep,
                                opts->variant, opts->vec);
  auto bail = [&](rt_status code) {
    cudaStreamSynchronize(s->stream);
    (void)cudaGetLastError();
    s->arena.free_all();
    delete s;
    return code;
  };
  if (st != RT_OK) return bail(st);
  Instance& I = s->I;
  void* p = nullptr;
  if ((st = s->arena.get(sizeof(InstDesc), &p)) != RT_OK) return bail(st);
  s->d_desc = (InstDesc*)p;
  if ((st = s->arena.get(I.stage_items.size() * sizeof(WorkItem), &p)) != RT_OK) return bail(st);
  s->d_stage_items = (WorkItem*)p;
  if ((st = s->arena.get(I.init_items.size() * sizeof(WorkItem), &p)) != RT_OK) return bail(st);
  s->d_init_items = (WorkItem*)p;
  if (!I.box_items.empty()) {
    if ((st = s->arena.get(I.box_items.size() * sizeof(WorkItem), &p)) != RT_OK) return bail(st);
    s->d_box_items = (WorkItem*)p;
  }
  I.device_bytes = s->arena.bytes;
  if (cudaMemcpyAsync(s->d_desc, &I.desc, sizeof(InstDesc), cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
      cudaMemcpyAsync(s->d_stage_items, I.stage_items.data(), I.stage_items.size() * sizeof(WorkItem),
                      cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
      cudaMemcpyAsync(s->d_init_items, I.init_items.data(), I.init_items.size() * sizeof(WorkItem),
                      cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
      (s->d_box_items && cudaMemcpyAsync(s->d_box_items, I.box_items.data(), I.box_items.size() * sizeof(WorkItem),
                                         cudaMemcpyHostToDevice, s->stream) != cudaSuccess)) {
    set_error("copying the solver descriptor failed: %s", cudaGetErrorString(cudaGetLastError()));
    return bail(RT_ECUDA);
  }
  if ((st = prepare_instance_kernels(I, I.ly)) != RT_OK) return bail(st);
  if ((st = run_init(s)) != RT_OK) return bail(st);
  InstState h;
  if ((st = read_state(s, &h)) != RT_OK) return bail(st);
  *out = s;
  return RT_OK;
}

rt_status rt_step(rt_solver* s, int64_t n) {
  clear_error();
  if (!s) { set_error("solver is NULL"); return RT_EINVAL; }
  if (s->failed) { set_error("solver is in its error state"); return RT_ESTATE; }
  if (n < 0) { set_error("n must be >= 0"); return RT_EINVAL; }
  n = std::min(n, s->I.n_steps - s->host_step);
  if (n <= 0) return RT_OK;
  int64_t done = 0;
  if (n >= 2 * kGraphSteps) {
    rt_status st = ensure_graph(s);
    if (st != RT_OK) return fail(s, st);
    while (n - done >= s->graph_steps) {
      cudaError_t e = cudaGraphLaunch(s->graph, s->stream);
      if (e != cudaSuccess) {
        set_error("graph launch failed: %s", cudaGetErrorString(e));
        return fail(s, RT_ECUDA);
      }
      done += s->graph_steps;
    }
  }
  rt_status st = launch_steps_direct(s, n - done, s->stream);
  if (st != RT_OK) return fail(s, st);
  s->host_step += n;
  return RT_OK;
}

rt_status rt_qoi(rt_solver* s, rt_qoi_t* out) {
  clear_error();
  if (!s || !out) { set_error("solver and out are required"); return RT_EINVAL; }
  if (s->failed) { set_error("solver is in its error state"); return RT_ESTATE; }
  InstState h;
  rt_status st = read_state(s, &h);
  if (st != RT_OK) return fail(s, st);
  fill_qoi(s->I, h, out);
  return RT_OK;
}

rt_status rt_info(const rt_solver* s, rt_info_t* out) {
  clear_error();
  if (!s || !out) { set_error("solver and out are required"); return RT_EINVAL; }
  const Instance& I = s->I;
  std::memset(out, 0, sizeof(*out));
  out->n_cells = I.n_cells;
  out->M = I.M;
  out->M_pad = I.Mpad;
  out->n_steps = I.n_steps;
  out->dt = I.dt;
  out->t_end = I.t_end;
  out->kind = I.kind;
  out->order = I.order;
  out->integrator = I.integrator;
  out->storage = I.storage;
  out->tile_x = I.kind == RT_MESH_CARTESIAN ? I.tx : 0;
  out->tile_y = I.kind == RT_MESH_CARTESIAN ? I.ly : 0;
  out->n_work_items = (int32_t)I.stage_items.size();
  out->stages_per_step = I.integrator == RT_HEUN ? 2 : 1;
  out->device_bytes = s->arena.bytes;
  out->variant = I.kind == RT_MESH_CARTESIAN ? (I.uni ? 2 : 1) : (I.uni ? 3 : 0);
  out->vec = I.kind == RT_MESH_CARTESIAN ? I.cvec : I.vec;
  out->regrouped = I.regrouped;
  out->n_box_items = (int32_t)I.box_items.size();
  return RT_OK;
}

static rt_status current_buffers(rt_solver* s, int* buf) {
  InstState h;
  rt_status st = read_state(s, &h);
  if (st != RT_OK) return fail(s, st);
  *buf = h.parity;
  return RT_OK;
}

rt_status rt_get_psi(rt_solver* s, double* host, int64_t n) {
  clear_error();
  if (!s || !host) { set_error("solver and host are required"); return RT_EINVAL; }
  if (s->failed) { set_error("solver is in its error state"); return RT_ESTATE; }
  const Instance& I = s->I;
  if (n != I.n_cells * I.M) { set_error("n must be n_cells*M = %lld", (long long)(I.n_cells * I.M)); return RT_EINVAL; }
  int buf = 0;
  rt_status st = current_buffers(s, &buf);
  if (st != RT_OK) return st;
  st = copy_psi_out(I, s->arena, s->stream, buf, host);
  return st == RT_OK ? RT_OK : fail(s, st);
}

rt_status rt_get_psi_cells(rt_solver* s, const int64_t* cells, int64_t n, double* host) {
  clear_error();
  if (!s || n < 0 || (n > 0 && (!cells || !host))) { set_error("solver, cells and host are required (n >= 0)"); return RT_EINVAL; }
  if (s->failed) { set_error("solver is in its error state"); return RT_ESTATE; }
  int buf = 0;
  rt_status st = current_buffers(s, &buf);
  if (st != RT_OK) return st;
  st = copy_psi_cells_out(s->I, s->arena, s->stream, buf, cells, n, host);
  return (st == RT_OK || st == RT_EINVAL) ? st : fail(s, st);
}

rt_status rt_get_phi(rt_solver* s, double* host, int64_t n) {
  clear_error();
  if (!s || !host) { set_error("solver and host are required"); return RT_EINVAL; }
  if (s->failed) { set_error("solver is in its error state"); return RT_ESTATE; }
  const Instance& I = s->I;
  if (n != I.n_cells) { set_error("n must be n_cells = %lld", (long long)I.n_cells); return RT_EINVAL; }
  int buf = 0;
  rt_status st = current_buffers(s, &buf);
  if (st != RT_OK) return st;
  std::vector<float> tmp((size_t)I.n_cells);
  cudaError_t e = cudaMemcpyAsync(tmp.data(), I.phi[buf], (size_t)I.n_cells * 4, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) {
    set_error("reading phi failed: %s", cudaGetErrorString(e));
    return fail(s, RT_ECUDA);
  }
  if (I.cell_perm.empty()) {
    for (int64_t i = 0; i < I.n_cells; ++i) host[i] = tmp[i];
  } else {
    for (int64_t i = 0; i < I.n_cells; ++i) host[I.cell_perm[i]] = tmp[i];
  }
  return RT_OK;
}

rt_status rt_set_psi(rt_solver* s, const double* host, int64_t n) {
  clear_error();
  if (!s || !host) { set_error("solver and host are required"); return RT_EINVAL; }
  if (s->failed) { set_error("solver is in its error state"); return RT_ESTATE; }
  const Instance& I = s->I;
  if (n != I.n_cells * I.M) { set_error("n must be n_cells*M = %lld", (long long)(I.n_cells * I.M)); return RT_EINVAL; }
  for (int64_t i = 0; i < n; ++i)
    if (!std::isfinite(host[i])) { set_error("psi[%lld] is not finite", (long long)i); return RT_EINVAL; }
  int buf = 0;
  rt_status st = current_buffers(s, &buf);
  if (st != RT_OK) return st;
  if ((st = copy_psi_in(I, s->arena, s->stream, buf, host)) != RT_OK) return fail(s, st);
  if ((st = run_init(s)) != RT_OK) return fail(s, st);
  InstState h;
  if ((st = read_state(s, &h)) != RT_OK) return fail(s, st);
  return RT_OK;
}

rt_status rt_device_state(rt_solver* s, void** psi, void** phi, int32_t* storage) {
  clear_error();
  if (!s) { set_error("solver is NULL"); return RT_EINVAL; }
  if (s->failed) { set_error("solver is in its error state"); return RT_ESTATE; }
  int buf = 0;
  rt_status st = current_buffers(s, &buf);
  if (st != RT_OK) return st;
  if (psi) *psi = s->I.psi[buf];
  if (phi) *phi = s->I.phi[buf];
  if (storage) *storage = s->I.storage;
  return RT_OK;
}

// ---- checkpoints: header | InstState | psi (storage bytes, [cell][Mpad]) | phi (float)
struct StateHeader {
  char magic[8];
  int64_t n_cells, M, Mpad;
  int32_t storage, kind, integrator, order;
};

rt_status rt_state_size(const rt_solver* s, size_t* bytes) {
  clear_error();
  if (!s || !bytes) { set_error("solver and bytes are required"); return RT_EINVAL; }
  const Instance& I = s->I;
  *bytes = sizeof(StateHeader) + sizeof(InstState) + (size_t)I.n_cells * I.Mpad * elem_size(I) + (size_t)I.n_cells * 4;
  return RT_OK;
}

rt_status rt_get_state(rt_solver* s, void* host, size_t bytes) {
  clear_error();
  size_t need = 0;
  if (!s || !host) { set_error("solver and host are required"); return RT_EINVAL; }
  if (s->failed) { set_error("solver is in its error state"); return RT_ESTATE; }
  rt_state_size(s, &need);
  if (bytes != need) { set_error("state blob must be %zu bytes", need); return RT_EINVAL; }
  const Instance& I = s->I;
  InstState h;
  rt_status st = read_state(s, &h);
  if (st != RT_OK) return fail(s, st);
  char* p = (char*)host;
  StateHeader hd{};
  std::memcpy(hd.magic, "RTSTATE1", 8);
  hd.n_cells = I.n_cells; hd.M = I.M; hd.Mpad = I.Mpad;
  hd.storage = I.storage; hd.kind = I.kind; hd.integrator = I.integrator; hd.order = I.order;
  std::memcpy(p, &hd, sizeof(hd));
  p += sizeof(hd);
  std::memcpy(p, &h, sizeof(h));
  p += sizeof(h);
  const size_t pb = (size_t)I.n_cells * I.Mpad * elem_size(I);
  cudaError_t e = cudaMemcpyAsync(p, I.psi[h.parity], pb, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(p + pb, I.phi[h.parity], (size_t)I.n_cells * 4, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) {
    set_error("reading the state failed: %s", cudaGetErrorString(e));
    return fail(s, RT_ECUDA);
  }
  return RT_OK;
}

rt_status rt_set_state(rt_solver* s, const void* host, size_t bytes) {
  clear_error();
  size_t need = 0;
  if (!s || !host) { set_error("solver and host are required"); return RT_EINVAL; }
  if (s->failed) { set_error("solver is in its error state"); return RT_ESTATE; }
  rt_state_size(s, &need);
  if (bytes != need) { set_error("state blob must be %zu bytes", need); return RT_EINVAL; }
  const Instance& I = s->I;
  const char* p = (const char*)host;
  StateHeader hd;
  std::memcpy(&hd, p, sizeof(hd));
  if (std::memcmp(hd.magic, "RTSTATE1", 8) != 0 || hd.n_cells != I.n_cells || hd.M != I.M || hd.Mpad != I.Mpad ||
      hd.storage != I.storage || hd.kind != I.kind || hd.integrator != I.integrator || hd.order != I.order) {
    set_error("state blob does not match this solver");
    return RT_EINVAL;
  }
  p += sizeof(hd);
  InstState h;
  std::memcpy(&h, p, sizeof(h));
  p += sizeof(h);
  if (h.status != DEV_OK || h.step < 0 || h.step > I.n_steps || (h.parity != 0 && h.parity != 1)) {
    set_error("state blob holds an invalid state");
    return RT_EINVAL;
  }
  h.ticket = 0;
  const size_t pb = (size_t)I.n_cells * I.Mpad * elem_size(I);
  cudaError_t e = cudaMemcpyAsync(I.psi[h.parity], p, pb, cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(I.phi[h.parity], p + pb, (size_t)I.n_cells * 4, cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(I.st, &h, sizeof(h), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) {
    set_error("writing the state failed: %s", cudaGetErrorString(e));
    return fail(s, RT_ECUDA);
  }
  s->host_step = h.step;
  return RT_OK;
}

rt_status rt_debug_set(rt_solver* s, const char* key, int64_t value) {
  clear_error();
  if (!s || !key) { set_error("solver and key are required"); return RT_EINVAL; }
  InstDesc& D = s->I.desc;
  size_t off = 0;
  int64_t v = value;
  if (std::strcmp(key, "wait_limit_cycles") == 0) {
    if (v <= 0) v = 4000000000LL;
    D.wait_limit = v;
    off = offsetof(InstDesc, wait_limit);
  } else if (std::strcmp(key, "drop_load") == 0) {
    if (v < 0) v = -1;
    D.drop_load = v;
    off = offsetof(InstDesc, drop_load);
  } else if (std::strcmp(key, "tri_staged") == 0) {
    // first-order triangles: 1 = the staged kernel, 0 = the gathering kernel (host-side choice)
    if (s->I.kind != RT_MESH_TRIANGLES || s->I.order != 1 || !s->I.staged_ok) {
      set_error("tri_staged applies to first-order triangle solvers with chunk halos");
      return RT_EINVAL;
    }
    cudaStreamSynchronize(s->stream);
    if (s->graph) {
      cudaGraphExecDestroy(s->graph);
      s->graph = nullptr;
    }
    s->I.uni = value != 0 ? 1 : 0;
    return RT_OK;
  } else {
    set_error("unknown debug key '%s'", key);
    return RT_EINVAL;
  }
  cudaError_t e = cudaMemcpyAsync((char*)s->d_desc + off, &v, sizeof(int64_t), cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) {
    set_error("debug update failed: %s", cudaGetErrorString(e));
    return fail(s, RT_ECUDA);
  }
  return RT_OK;
}

void rt_destroy(rt_solver* s) {
  if (!s) return;
  cudaStreamSynchronize(s->stream);
  (void)cudaGetLastError();
  if (s->graph) cudaGraphExecDestroy(s->graph);
  if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
  s->arena.free_all();
  delete s;
}

}  // extern "C"
