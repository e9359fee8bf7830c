// Batches of independent S_N problems advanced by shared launches.
//
// All problems' descriptors sit in one device array; a stage launch covers the
// work items of every unfinished problem of one kernel variant (mesh kind,
// order, tile width, vector width), so many small problems fill the GPU
// together instead of one launch each. rt_batch_run proceeds in phases: a phase
// lasts until the next problem reaches its own N_t, its work list holds only
// unfinished problems, and its steps replay a captured CUDA graph of
// kBatchGraphSteps steps (plus direct launches for the remainder). The kernels
// also mask finished problems on the device.
#include <algorithm>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "host_common.h"

using namespace rtk;

namespace {
constexpr int kBatchGraphSteps = 8;

struct Group {
  int kind, order, run, cvec, vec, uni, ly_max;
  int offset, count;
};
}  // namespace

struct rt_batch {
  DeviceArena arena;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  std::vector<Instance> inst;
  InstDesc* d_desc = nullptr;
  WorkItem* d_items = nullptr;        // capacity: all stage items of all problems
  WorkItem* d_init_items = nullptr;
  std::vector<int> init_offset;
  std::vector<int64_t> done;          // steps enqueued per problem
  int integrator = RT_EULER, storage = RT_FP32;
  bool failed = false;
};

static rt_status batch_fail(rt_batch* b, rt_status st) {
  if (b && st != RT_OK && st != RT_EINVAL) b->failed = true;
  return st;
}

static rt_status enqueue_phase_steps(rt_batch* b, const std::vector<Group>& groups, int64_t n, cudaStream_t stream) {
  for (int64_t i = 0; i < n; ++i) {
    for (const Group& g : groups) {
      rt_status st = launch_step(b->d_desc, b->d_items + g.offset, g.count, g.kind, b->integrator, b->storage,
                                 g.order, g.run, g.cvec, g.ly_max, g.vec, stream, g.uni);
      if (st != RT_OK) return st;
    }
  }
  return RT_OK;
}

extern "C" {

rt_status rt_batch_create(int32_t k, const rt_problem* problems, const rt_options* opts, rt_batch** out) {
  clear_error();
  if (!out) { set_error("out is NULL"); return RT_EINVAL; }
  *out = nullptr;
  if (k < 1 || !problems || !opts) { set_error("need k >= 1, problems and options"); return RT_EINVAL; }
  if ((opts->alloc == nullptr) != (opts->free == nullptr)) { set_error("alloc and free must both be set or both NULL"); return RT_EINVAL; }
  for (int i = 1; i < k; ++i)
    if (problems[i].integrator != problems[0].integrator) { set_error("all problems of a batch must use the same integrator"); return RT_EINVAL; }
  rt_batch* b = new rt_batch();
  b->arena.alloc_fn = opts->alloc;
  b->arena.free_fn = opts->free;
  b->arena.ctx = opts->alloc_ctx;
  b->stream = (cudaStream_t)opts->stream;
  b->integrator = problems[0].integrator;
  b->storage = opts->storage;
  b->inst.resize(k);
  b->done.assign(k, 0);
  auto bail = [&](rt_status code) {
    cudaStreamSynchronize(b->stream);
    (void)cudaGetLastError();
    b->arena.free_all();
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    delete b;
    return code;
  };
  std::vector<std::vector<char>> keep;
  size_t n_stage = 0, n_init = 0;
  for (int i = 0; i < k; ++i) {
    const rt_problem& P = problems[i];
    rt_status st = build_instance(&P.mesh, &P.mat, &P.quad, &P.bc, P.order, P.integrator, opts->storage, P.dt,
                                  P.t_end, opts->tile_x, opts->tile_y, b->arena, b->stream, b->inst[i], keep,
                                  opts->variant);
    if (st != RT_OK) {
      char msg[1200];
      snprintf(msg, sizeof(msg), "problem %d: %s", i, rt_last_error());
      set_error("%s", msg);
      return bail(st);
    }
    n_stage += b->inst[i].stage_items.size();
    b->init_offset.push_back((int)n_init);
    n_init += b->inst[i].init_items.size();
    // host copies of per-problem arrays are already on the stream; sync to bound host memory
    if (keep.size() > 64) {
      if (cudaStreamSynchronize(b->stream) != cudaSuccess) { set_error("stream failed during create"); return bail(RT_ECUDA); }
      keep.clear();
    }
  }
  void* p = nullptr;
  rt_status st;
  if ((st = b->arena.get((size_t)k * sizeof(InstDesc), &p)) != RT_OK) return bail(st);
  b->d_desc = (InstDesc*)p;
  if ((st = b->arena.get(n_stage * sizeof(WorkItem), &p)) != RT_OK) return bail(st);
  b->d_items = (WorkItem*)p;
  if ((st = b->arena.get(n_init * sizeof(WorkItem), &p)) != RT_OK) return bail(st);
  b->d_init_items = (WorkItem*)p;
  std::vector<InstDesc> hd(k);
  std::vector<WorkItem> hi;
  hi.reserve(n_init);
  for (int i = 0; i < k; ++i) {
    hd[i] = b->inst[i].desc;
    for (WorkItem w : b->inst[i].init_items) {
      w.inst = 0;   // init launches are per problem (descriptor pointer offset by i)
      hi.push_back(w);
    }
  }
  if (cudaMemcpyAsync(b->d_desc, hd.data(), (size_t)k * sizeof(InstDesc), cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
      cudaMemcpyAsync(b->d_init_items, hi.data(), hi.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, b->stream) != cudaSuccess) {
    set_error("copying batch descriptors failed");
    return bail(RT_ECUDA);
  }
  for (int i = 0; i < k; ++i) {
    const Instance& I = b->inst[i];
    if ((st = prepare_instance_kernels(I, I.ly)) != RT_OK) return bail(st);
    cudaError_t e = launch_init(b->d_desc + i, b->d_init_items + b->init_offset[i], (int)I.init_items.size(), I.vec,
                                I.storage, b->stream);
    if (e != cudaSuccess) {
      set_error("init launch failed: %s", cudaGetErrorString(e));
      return bail(RT_ECUDA);
    }
  }
  for (int i = 0; i < k; ++i) {
    InstState h;
    if ((st = read_inst_state(b->inst[i], b->stream, &h)) != RT_OK) return bail(st);
  }
  if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    set_error("stream creation failed");
    return bail(RT_ECUDA);
  }
  *out = b;
  return RT_OK;
}

rt_status rt_batch_run(rt_batch* b, int64_t max_steps) {
  clear_error();
  if (!b) { set_error("batch is NULL"); return RT_EINVAL; }
  if (b->failed) { set_error("batch is in its error state"); return RT_ESTATE; }
  const int k = (int)b->inst.size();
  std::vector<int64_t> target(k);
  for (int i = 0; i < k; ++i) {
    target[i] = b->inst[i].n_steps;
    if (max_steps > 0) target[i] = std::min(target[i], b->done[i] + max_steps);
  }
  while (true) {
    int64_t phase = INT64_MAX;
    for (int i = 0; i < k; ++i)
      if (b->done[i] < target[i]) phase = std::min(phase, target[i] - b->done[i]);
    if (phase == INT64_MAX) break;
    // work list of the unfinished problems, grouped by kernel variant
    std::map<std::tuple<int, int, int, int, int, int>, std::vector<int>> by_variant;
    for (int i = 0; i < k; ++i) {
      if (b->done[i] >= target[i]) continue;
      const Instance& I = b->inst[i];
      by_variant[std::make_tuple(I.kind, I.order, I.run, I.cvec, I.vec, I.uni)].push_back(i);
    }
    std::vector<WorkItem> items;
    std::vector<Group> groups;
    for (auto& kv : by_variant) {
      Group g{};
      std::tie(g.kind, g.order, g.run, g.cvec, g.vec, g.uni) = kv.first;
      g.offset = (int)items.size();
      g.ly_max = 1;
      for (int i : kv.second) {
        const Instance& I = b->inst[i];
        g.ly_max = std::max(g.ly_max, I.ly);
        for (WorkItem w : I.stage_items) {
          w.inst = i;
          items.push_back(w);
        }
      }
      g.count = (int)items.size() - g.offset;
      groups.push_back(g);
      rt_status pst = prepare_instance_kernels(b->inst[kv.second[0]], g.ly_max);
      if (pst != RT_OK) return batch_fail(b, pst);
    }
    cudaError_t e = cudaMemcpyAsync(b->d_items, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice,
                                    b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);   // the host list is freed at the end of the phase
    if (e != cudaSuccess) {
      set_error("copying the work list failed: %s", cudaGetErrorString(e));
      return batch_fail(b, RT_ECUDA);
    }
    int64_t left = phase;
    if (phase >= 2 * kBatchGraphSteps) {
      cudaGraph_t g = nullptr;
      cudaGraphExec_t ge = nullptr;
      if (cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        set_error("graph capture could not start");
        return batch_fail(b, RT_ECUDA);
      }
      rt_status st = enqueue_phase_steps(b, groups, kBatchGraphSteps, b->cap_stream);
      e = cudaStreamEndCapture(b->cap_stream, &g);
      if (st != RT_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        if (st == RT_OK) set_error("graph capture failed: %s", cudaGetErrorString(e));
        return batch_fail(b, st != RT_OK ? st : RT_ECUDA);
      }
      e = cudaGraphInstantiate(&ge, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        set_error("graph instantiation failed: %s", cudaGetErrorString(e));
        return batch_fail(b, RT_ECUDA);
      }
      while (left >= kBatchGraphSteps) {
        e = cudaGraphLaunch(ge, b->stream);
        if (e != cudaSuccess) break;
        left -= kBatchGraphSteps;
      }
      // keep the executable graph alive until its replays have been consumed
      cudaError_t e2 = cudaStreamSynchronize(b->stream);
      cudaGraphExecDestroy(ge);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        set_error("graph replay failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
        return batch_fail(b, RT_ECUDA);
      }
    }
    rt_status st = enqueue_phase_steps(b, groups, left, b->stream);
    if (st != RT_OK) return batch_fail(b, st);
    for (int i = 0; i < k; ++i)
      if (b->done[i] < target[i]) b->done[i] += phase;
  }
  return RT_OK;
}

rt_status rt_batch_qoi(rt_batch* b, int32_t i, rt_qoi_t* out) {
  clear_error();
  if (!b || !out) { set_error("batch and out are required"); return RT_EINVAL; }
  if (i < 0 || i >= (int)b->inst.size()) { set_error("problem index %d out of range", i); return RT_EINVAL; }
  if (b->failed) { set_error("batch is in its error state"); return RT_ESTATE; }
  InstState h;
  rt_status st = read_inst_state(b->inst[i], b->stream, &h);
  if (st != RT_OK) return batch_fail(b, st);
  fill_qoi(b->inst[i], h, out);
  return RT_OK;
}

rt_status rt_batch_get_psi(rt_batch* b, int32_t i, double* host, int64_t n) {
  clear_error();
  if (!b || !host) { set_error("batch and host are required"); return RT_EINVAL; }
  if (i < 0 || i >= (int)b->inst.size()) { set_error("problem index %d out of range", i); return RT_EINVAL; }
  if (b->failed) { set_error("batch is in its error state"); return RT_ESTATE; }
  const Instance& I = b->inst[i];
  if (n != I.n_cells * I.M) { set_error("n must be n_cells*M = %lld", (long long)(I.n_cells * I.M)); return RT_EINVAL; }
  InstState h;
  rt_status st = read_inst_state(I, b->stream, &h);
  if (st != RT_OK) return batch_fail(b, st);
  st = copy_psi_out(I, b->arena, b->stream, h.parity, host);
  return st == RT_OK ? RT_OK : batch_fail(b, st);
}

void rt_batch_destroy(rt_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  (void)cudaGetLastError();
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  b->arena.free_all();
  delete b;
}

}  // extern "C"
