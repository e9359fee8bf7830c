// Batches of independent S_N problems advanced by shared launches.
//
// A batch has `capacity` slots. The descriptors of all slots sit in one device
// array; a stage launch covers the work items of every unfinished problem of
// one kernel variant (mesh kind, order, integrator and the Cartesian or
// triangle variant knobs), so many small problems fill the GPU together
// instead of one launch each. Problems can be added and removed between steps;
// each slot owns its device memory (its own allocation list), freed on removal.
// rt_batch_step enqueues up to n steps for the unfinished problems; while the
// membership and n stay the same it replays one captured CUDA graph (captured
// at the second call with the same membership: a call right after a change
// launches directly, since a serving loop may change the membership at every
// call). Membership changes do not drain the stream: the new work list is
// copied from pinned staging buffers behind the launches already queued, and a
// replaced graph is destroyed at the next point where the stream is
// synchronised anyway. Problems
// past their own N_t are dropped from the work list at the next step and are
// also masked on the device.
#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <tuple>
#include <vector>

#include "host_common.h"

using namespace rtk;

namespace {

struct Group {
  int kind, order, integrator, run, cvec, vec, uni, ly_max;
  int offset, count;
  int box_offset, box_count;   // QoI-box work items of the group's problems
};

struct Slot {
  bool used = false;
  bool held = false;   // left out of the work list until released (rt_batch_hold)
  std::unique_ptr<DeviceArena> arena;
  Instance inst;
  WorkItem* d_init_items = nullptr;
  WorkItem* d_box_items = nullptr;   // for the initial state (descriptor pointer offset by slot)
  int64_t done = 0;   // steps enqueued
};

}  // namespace

struct rt_batch {
  rt_alloc_fn alloc_fn = nullptr;
  rt_free_fn free_fn = nullptr;
  void* alloc_ctx = nullptr;
  DeviceArena shared;                 // descriptor array and work list
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  int storage = RT_FP32;
  int tile_x = 0, tile_y = 0, variant = 0, vec = 0;
  std::vector<Slot> slots;
  InstDesc* d_desc = nullptr;         // [capacity]
  WorkItem* d_items = nullptr;
  size_t items_cap = 0;
  WorkItem* d_box_list = nullptr;     // QoI-box work items of the current membership
  size_t box_cap = 0;
  // work list and graph of the current membership
  bool dirty = true;
  std::vector<Group> groups;
  std::vector<int> members;           // slots in the current work list
  cudaGraphExec_t graph = nullptr;
  int64_t graph_n = 0;
  int64_t graph_launches = 0;          // kernel launches in one replay of the graph
  int64_t launches = 0;                // kernel launches issued or replayed so far (rt_batch_launches)
  bool fresh = false;                  // the work list was rebuilt at the last step call
  std::vector<cudaGraphExec_t> old_graphs;   // replaced, destroyed once the stream is synchronised
  // pinned staging of the work lists (a ring, so a copy still queued is not overwritten)
  static constexpr int kStage = 4;
  char* h_stage[kStage] = {};
  size_t h_stage_cap[kStage] = {};
  cudaEvent_t h_stage_ev[kStage] = {};
  int h_next = 0;
  bool failed = false;
};

namespace {

rt_status batch_fail(rt_batch* b, rt_status st) {
  if (b && st != RT_OK && st != RT_EINVAL) b->failed = true;
  return st;
}

// Retire the current graph; launches of it may still be queued, so it is
// destroyed by release_graphs once the stream has been synchronised.
void release_graphs(rt_batch* b);

void drop_graph(rt_batch* b) {
  if (b->graph) {
    b->old_graphs.push_back(b->graph);
    b->graph = nullptr;
  }
  b->graph_n = 0;
  if (b->old_graphs.size() > 64) {   // bound the retired list
    cudaStreamSynchronize(b->stream);
    release_graphs(b);
  }
}

// Destroy retired graphs. Call only after the stream has been synchronised.
void release_graphs(rt_batch* b) {
  for (cudaGraphExec_t g : b->old_graphs) cudaGraphExecDestroy(g);
  b->old_graphs.clear();
}

// Copy `bytes` from host memory to `dst` on the batch's stream through the next
// pinned staging buffer, without synchronising with the work already queued.
rt_status stage_copy(rt_batch* b, void* dst, const void* src, size_t bytes) {
  if (bytes == 0) return RT_OK;
  const int k = b->h_next;
  b->h_next = (k + 1) % rt_batch::kStage;
  if (!b->h_stage_ev[k] && cudaEventCreateWithFlags(&b->h_stage_ev[k], cudaEventDisableTiming) != cudaSuccess) {
    set_error("event creation failed");
    return RT_ECUDA;
  }
  // the last copy out of this buffer must have been done (rarely still queued)
  if (b->h_stage[k] && cudaEventSynchronize(b->h_stage_ev[k]) != cudaSuccess) {
    set_error("waiting for a staging copy failed");
    return RT_ECUDA;
  }
  if (b->h_stage_cap[k] < bytes) {
    if (b->h_stage[k]) cudaFreeHost(b->h_stage[k]);
    b->h_stage[k] = nullptr;
    b->h_stage_cap[k] = 0;
    const size_t cap = std::max<size_t>(bytes * 2, 64 << 10);
    if (cudaHostAlloc((void**)&b->h_stage[k], cap, cudaHostAllocDefault) != cudaSuccess) {
      b->h_stage[k] = nullptr;
      set_error("pinned staging allocation of %zu bytes failed", cap);
      return RT_ECUDA;
    }
    b->h_stage_cap[k] = cap;
  }
  std::memcpy(b->h_stage[k], src, bytes);
  if (cudaMemcpyAsync(dst, b->h_stage[k], bytes, cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
      cudaEventRecord(b->h_stage_ev[k], b->stream) != cudaSuccess) {
    set_error("copying a work list failed");
    return RT_ECUDA;
  }
  return RT_OK;
}

void free_staging(rt_batch* b) {
  for (int k = 0; k < rt_batch::kStage; ++k) {
    if (b->h_stage[k]) cudaFreeHost(b->h_stage[k]);
    if (b->h_stage_ev[k]) cudaEventDestroy(b->h_stage_ev[k]);
    b->h_stage[k] = nullptr;
    b->h_stage_ev[k] = nullptr;
  }
}

// Build, validate and initialise a problem in slot `i`.
rt_status add_in_slot(rt_batch* b, const rt_problem& P, int i) {
  Slot& S = b->slots[i];
  S.arena.reset(new DeviceArena());
  S.arena->alloc_fn = b->alloc_fn;
  S.arena->free_fn = b->free_fn;
  S.arena->ctx = b->alloc_ctx;
  S.inst = Instance();
  std::vector<std::vector<char>> keep;
  const int ty = P.tile_y ? P.tile_y : b->tile_y;
  const int var = P.variant ? P.variant : b->variant;
  const int vec = P.vec ? P.vec : b->vec;
  rt_status st = build_instance(&P.mesh, &P.mat, &P.quad, &P.bc, P.order, P.integrator, b->storage, P.dt, P.t_end,
                                b->tile_x, ty, *S.arena, b->stream, S.inst, keep, var, vec);
  auto undo = [&](rt_status code) {
    cudaStreamSynchronize(b->stream);
    (void)cudaGetLastError();
    S.arena->free_all();
    S.arena.reset();
    S.used = false;
    return code;
  };
  if (st != RT_OK) return undo(st);
  Instance& I = S.inst;
  void* p = nullptr;
  if ((st = S.arena->get(I.init_items.size() * sizeof(WorkItem), &p)) != RT_OK) return undo(st);
  S.d_init_items = (WorkItem*)p;
  std::vector<WorkItem> hi = I.init_items;
  for (WorkItem& w : hi) w.inst = 0;   // init launches are per problem (descriptor pointer offset by slot)
  std::vector<WorkItem> hb = I.box_items;
  for (WorkItem& w : hb) w.inst = 0;
  if (!hb.empty()) {
    if ((st = S.arena->get(hb.size() * sizeof(WorkItem), &p)) != RT_OK) return undo(st);
    S.d_box_items = (WorkItem*)p;
    if (cudaMemcpyAsync(S.d_box_items, hb.data(), hb.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, b->stream) !=
        cudaSuccess) {
      set_error("copying a problem's box work items failed");
      return undo(RT_ECUDA);
    }
  } else {
    S.d_box_items = nullptr;
  }
  if (cudaMemcpyAsync(S.d_init_items, hi.data(), hi.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, b->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(b->d_desc + i, &I.desc, sizeof(InstDesc), cudaMemcpyHostToDevice, b->stream) != cudaSuccess) {
    set_error("copying a problem's descriptor failed");
    return undo(RT_ECUDA);
  }
  if ((st = prepare_instance_kernels(I, I.ly)) != RT_OK) return undo(st);
  if ((st = launch_init_all(b->d_desc + i, S.d_init_items, (int)I.init_items.size(), S.d_box_items, (int)hb.size(),
                            I.vec, I.storage, b->stream)) != RT_OK)
    return undo(st);
  b->launches += hb.empty() ? 1 : 2;
  InstState h;
  if ((st = read_inst_state(I, b->stream, &h)) != RT_OK) return undo(st);
  S.used = true;
  S.done = 0;
  b->dirty = true;
  return RT_OK;
}

// Rebuild the work list of the unfinished problems, grouped by kernel variant.
rt_status rebuild(rt_batch* b) {
  drop_graph(b);
  std::map<std::tuple<int, int, int, int, int, int, int>, std::vector<int>> by_variant;
  b->members.clear();
  for (int i = 0; i < (int)b->slots.size(); ++i) {
    const Slot& S = b->slots[i];
    if (!S.used || S.held || S.done >= S.inst.n_steps) continue;
    const Instance& I = S.inst;
    by_variant[std::make_tuple(I.kind, I.order, I.integrator, I.run, I.cvec, I.vec, I.uni)].push_back(i);
    b->members.push_back(i);
  }
  std::vector<WorkItem> items, box_items;
  b->groups.clear();
  for (auto& kv : by_variant) {
    Group g{};
    std::tie(g.kind, g.order, g.integrator, g.run, g.cvec, g.vec, g.uni) = kv.first;
    g.offset = (int)items.size();
    g.box_offset = (int)box_items.size();
    g.ly_max = 1;
    for (int i : kv.second) {
      const Instance& I = b->slots[i].inst;
      g.ly_max = std::max(g.ly_max, I.ly);
      for (WorkItem w : I.stage_items) {
        w.inst = i;
        items.push_back(w);
      }
      for (WorkItem w : I.box_items) {
        w.inst = i;
        box_items.push_back(w);
      }
    }
    g.count = (int)items.size() - g.offset;
    g.box_count = (int)box_items.size() - g.box_offset;
    rt_status pst = prepare_instance_kernels(b->slots[kv.second[0]].inst, g.ly_max);
    if (pst != RT_OK) return pst;
    b->groups.push_back(g);
  }
  if (items.size() > b->items_cap) {
    cudaStreamSynchronize(b->stream);
    release_graphs(b);
    if (b->d_items) b->shared.release(b->d_items);
    b->d_items = nullptr;
    b->items_cap = 0;
    void* p = nullptr;
    const size_t cap = std::max<size_t>(items.size() * 2, 1024);
    rt_status st = b->shared.get(cap * sizeof(WorkItem), &p);
    if (st != RT_OK) return st;
    b->d_items = (WorkItem*)p;
    b->items_cap = cap;
  }
  if (box_items.size() > b->box_cap) {
    cudaStreamSynchronize(b->stream);
    release_graphs(b);
    if (b->d_box_list) b->shared.release(b->d_box_list);
    b->d_box_list = nullptr;
    b->box_cap = 0;
    void* p = nullptr;
    const size_t cap = std::max<size_t>(box_items.size() * 2, 256);
    rt_status st = b->shared.get(cap * sizeof(WorkItem), &p);
    if (st != RT_OK) return st;
    b->d_box_list = (WorkItem*)p;
    b->box_cap = cap;
  }
  // the launches already queued read the old lists before these copies (stream order)
  rt_status cst = stage_copy(b, b->d_box_list, box_items.data(), box_items.size() * sizeof(WorkItem));
  if (cst == RT_OK) cst = stage_copy(b, b->d_items, items.data(), items.size() * sizeof(WorkItem));
  if (cst != RT_OK) return cst;
  b->dirty = false;
  b->fresh = true;
  return RT_OK;
}

// Enqueue n steps of the current work list on `stream`; *launched counts the
// kernel launches enqueued (also when a launch fails part way).
rt_status enqueue_steps(rt_batch* b, int64_t n, cudaStream_t stream, int64_t* launched) {
  const size_t ng = b->groups.size();
  *launched = 0;
  auto last_stage = [&](size_t j) { return b->groups[j].integrator == RT_HEUN ? STAGE_HEUN2 : STAGE_EULER; };
  for (int64_t i = 0; i < n; ++i) {
    for (const Group& g : b->groups) {
      rt_status st = launch_step(b->d_desc, b->d_items + g.offset, g.count, g.kind, g.integrator, b->storage, g.order,
                                 g.run, g.cvec, g.ly_max, g.vec, stream, g.uni, nullptr, 0);
      if (st != RT_OK) return st;
      *launched += g.integrator == RT_HEUN ? 2 : 1;
    }
    // QoI boxes once every group has stepped: one launch per run of consecutive
    // groups that end the step with the same stage (their box items are
    // contiguous in the list); each box reads only its own problem's state
    for (size_t j = 0; j < ng;) {
      const int stage = last_stage(j);
      const int first = b->groups[j].box_offset;
      int n_box = 0;
      size_t k = j;
      for (; k < ng && last_stage(k) == stage; ++k) n_box += b->groups[k].box_count;
      if (n_box > 0) {
        const cudaError_t e = launch_box_outflow(b->d_desc, b->d_box_list + first, n_box, stage, b->storage, stream);
        if (e != cudaSuccess) {
          set_error("box outflow launch failed: %s", cudaGetErrorString(e));
          return RT_ECUDA;
        }
        ++*launched;
      }
      j = k;
    }
  }
  return RT_OK;
}

constexpr int64_t kGraphMinSteps = 4;

rt_status step_members(rt_batch* b, int64_t n) {
  if (b->dirty) {
    rt_status st = rebuild(b);
    if (st != RT_OK) return st;
  }
  if (b->members.empty() || n <= 0) return RT_OK;
  const bool fresh = b->fresh;
  b->fresh = false;
  if (n >= kGraphMinSteps && !fresh) {
    if (!b->graph || b->graph_n != n) {
      drop_graph(b);
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        set_error("graph capture could not start");
        return RT_ECUDA;
      }
      int64_t cnt = 0;
      rt_status st = enqueue_steps(b, n, b->cap_stream, &cnt);
      cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
      if (st != RT_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        if (st == RT_OK) set_error("graph capture failed: %s", cudaGetErrorString(e));
        return st != RT_OK ? st : RT_ECUDA;
      }
      e = cudaGraphInstantiate(&b->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        b->graph = nullptr;
        set_error("graph instantiation failed: %s", cudaGetErrorString(e));
        return RT_ECUDA;
      }
      b->graph_n = n;
      b->graph_launches = cnt;
    }
    cudaError_t e = cudaGraphLaunch(b->graph, b->stream);
    if (e != cudaSuccess) {
      set_error("graph launch failed: %s", cudaGetErrorString(e));
      return RT_ECUDA;
    }
    b->launches += b->graph_launches;
  } else {
    int64_t cnt = 0;
    rt_status st = enqueue_steps(b, n, b->stream, &cnt);
    b->launches += cnt;
    if (st != RT_OK) return st;
  }
  for (int i : b->members) {
    Slot& S = b->slots[i];
    S.done = std::min(S.inst.n_steps, S.done + n);
    if (S.done >= S.inst.n_steps) b->dirty = true;   // drop it from the work list next time
  }
  return RT_OK;
}

bool slot_ok(const rt_batch* b, int32_t i) { return i >= 0 && i < (int)b->slots.size() && b->slots[i].used; }

}  // namespace

extern "C" {

rt_status rt_batch_create(int32_t k, const rt_problem* problems, int32_t capacity, const rt_options* opts,
                          rt_batch** out) {
  clear_error();
  if (!out) { set_error("out is NULL"); return RT_EINVAL; }
  *out = nullptr;
  if (k < 0 || (k > 0 && !problems) || !opts) { set_error("need k >= 0, problems (when k > 0) and options"); return RT_EINVAL; }
  if (capacity == 0) capacity = k;
  if (capacity < k || capacity < 1 || capacity > (1 << 20)) { set_error("capacity must be in max(k,1)..2^20"); return RT_EINVAL; }
  if ((opts->alloc == nullptr) != (opts->free == nullptr)) { set_error("alloc and free must both be set or both NULL"); return RT_EINVAL; }
  if (opts->storage != RT_FP32 && opts->storage != RT_BF16) { set_error("storage must be RT_FP32 or RT_BF16"); return RT_EINVAL; }
  rt_batch* b = new rt_batch();
  b->alloc_fn = opts->alloc;
  b->free_fn = opts->free;
  b->alloc_ctx = opts->alloc_ctx;
  b->shared.alloc_fn = opts->alloc;
  b->shared.free_fn = opts->free;
  b->shared.ctx = opts->alloc_ctx;
  b->stream = (cudaStream_t)opts->stream;
  b->storage = opts->storage;
  b->tile_x = opts->tile_x;
  b->tile_y = opts->tile_y;
  b->variant = opts->variant;
  b->vec = opts->vec;
  b->slots.resize(capacity);
  auto bail = [&](rt_status code) {
    cudaStreamSynchronize(b->stream);
    (void)cudaGetLastError();
    for (Slot& S : b->slots)
      if (S.arena) S.arena->free_all();
    b->shared.free_all();
    release_graphs(b);
    free_staging(b);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    delete b;
    return code;
  };
  void* p = nullptr;
  rt_status st = b->shared.get((size_t)capacity * sizeof(InstDesc), &p);
  if (st != RT_OK) return bail(st);
  b->d_desc = (InstDesc*)p;
  if (cudaMemsetAsync(b->d_desc, 0, (size_t)capacity * sizeof(InstDesc), b->stream) != cudaSuccess) {
    set_error("clearing the descriptor array failed");
    return bail(RT_ECUDA);
  }
  if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    set_error("stream creation failed");
    return bail(RT_ECUDA);
  }
  for (int i = 0; i < k; ++i) {
    if ((st = add_in_slot(b, problems[i], i)) != RT_OK) {
      char msg[1200];
      snprintf(msg, sizeof(msg), "problem %d: %s", i, rt_last_error());
      set_error("%s", msg);
      return bail(st);
    }
  }
  *out = b;
  return RT_OK;
}

rt_status rt_batch_add(rt_batch* b, const rt_problem* problem, int32_t* slot) {
  clear_error();
  if (!b || !problem || !slot) { set_error("batch, problem and slot are required"); return RT_EINVAL; }
  if (b->failed) { set_error("batch is in its error state"); return RT_ESTATE; }
  int i = 0;
  while (i < (int)b->slots.size() && b->slots[i].used) ++i;
  if (i == (int)b->slots.size()) { set_error("no free slot (capacity %d)", (int)b->slots.size()); return RT_EINVAL; }
  rt_status st = add_in_slot(b, *problem, i);
  if (st != RT_OK) return st == RT_ECUDA ? batch_fail(b, st) : st;
  *slot = i;
  return RT_OK;
}

rt_status rt_batch_remove(rt_batch* b, int32_t i) {
  clear_error();
  if (!b) { set_error("batch is NULL"); return RT_EINVAL; }
  if (!slot_ok(b, i)) { set_error("slot %d is empty or out of range", i); return RT_EINVAL; }
  drop_graph(b);
  cudaStreamSynchronize(b->stream);
  release_graphs(b);
  Slot& S = b->slots[i];
  S.arena->free_all();
  S.arena.reset();
  S.used = false;
  S.held = false;
  S.done = 0;
  b->dirty = true;
  return RT_OK;
}

rt_status rt_batch_hold(rt_batch* b, int32_t i, int32_t hold) {
  clear_error();
  if (!b) { set_error("batch is NULL"); return RT_EINVAL; }
  if (!slot_ok(b, i)) { set_error("slot %d is empty or out of range", i); return RT_EINVAL; }
  const bool h = hold != 0;
  if (b->slots[i].held != h) {
    b->slots[i].held = h;
    b->dirty = true;   // the work list (and its graph) changes at the next step
  }
  return RT_OK;
}

rt_status rt_batch_step(rt_batch* b, int64_t n) {
  clear_error();
  if (!b) { set_error("batch is NULL"); return RT_EINVAL; }
  if (b->failed) { set_error("batch is in its error state"); return RT_ESTATE; }
  if (n < 0) { set_error("n must be >= 0"); return RT_EINVAL; }
  rt_status st = step_members(b, n);
  return st == RT_OK ? RT_OK : batch_fail(b, st);
}

rt_status rt_batch_run(rt_batch* b, int64_t max_steps) {
  clear_error();
  if (!b) { set_error("batch is NULL"); return RT_EINVAL; }
  if (b->failed) { set_error("batch is in its error state"); return RT_ESTATE; }
  constexpr int64_t kChunkSteps = 8;
  int64_t budget = max_steps > 0 ? max_steps : INT64_MAX;
  while (budget > 0) {
    // steps until the next problem finishes
    int64_t phase = INT64_MAX;
    for (const Slot& S : b->slots)
      if (S.used && !S.held && S.done < S.inst.n_steps) phase = std::min(phase, S.inst.n_steps - S.done);
    if (phase == INT64_MAX) break;
    phase = std::min(phase, budget);
    int64_t left = phase;
    while (left > 0) {
      const int64_t n = left >= kChunkSteps ? kChunkSteps : left;
      rt_status st = step_members(b, n);
      if (st != RT_OK) return batch_fail(b, st);
      left -= n;
    }
    budget -= phase;
  }
  return RT_OK;
}

rt_status rt_batch_launches(const rt_batch* b, int64_t* n) {
  clear_error();
  if (!b || !n) { set_error("batch or output is NULL"); return RT_EINVAL; }
  *n = b->launches;
  return RT_OK;
}

rt_status rt_batch_progress(const rt_batch* b, int32_t i, int64_t* steps_done, int64_t* n_steps) {
  clear_error();
  if (!b) { set_error("batch is NULL"); return RT_EINVAL; }
  if (!slot_ok(b, i)) { set_error("slot %d is empty or out of range", i); return RT_EINVAL; }
  if (steps_done) *steps_done = b->slots[i].done;
  if (n_steps) *n_steps = b->slots[i].inst.n_steps;
  return RT_OK;
}

rt_status rt_batch_qoi(rt_batch* b, int32_t i, rt_qoi_t* out) {
  clear_error();
  if (!b || !out) { set_error("batch and out are required"); return RT_EINVAL; }
  if (!slot_ok(b, i)) { set_error("slot %d is empty or out of range", i); return RT_EINVAL; }
  if (b->failed) { set_error("batch is in its error state"); return RT_ESTATE; }
  InstState h;
  rt_status st = read_inst_state(b->slots[i].inst, b->stream, &h);   // synchronises the stream
  if (st != RT_OK) return batch_fail(b, st);
  release_graphs(b);
  fill_qoi(b->slots[i].inst, h, out);
  return RT_OK;
}

rt_status rt_batch_get_psi(rt_batch* b, int32_t i, double* host, int64_t n) {
  clear_error();
  if (!b || !host) { set_error("batch and host are required"); return RT_EINVAL; }
  if (!slot_ok(b, i)) { set_error("slot %d is empty or out of range", i); return RT_EINVAL; }
  if (b->failed) { set_error("batch is in its error state"); return RT_ESTATE; }
  Slot& S = b->slots[i];
  const Instance& I = S.inst;
  if (n != I.n_cells * I.M) { set_error("n must be n_cells*M = %lld", (long long)(I.n_cells * I.M)); return RT_EINVAL; }
  InstState h;
  rt_status st = read_inst_state(I, b->stream, &h);
  if (st != RT_OK) return batch_fail(b, st);
  st = copy_psi_out(I, *S.arena, b->stream, h.parity, host);
  return st == RT_OK ? RT_OK : batch_fail(b, st);
}

void rt_batch_destroy(rt_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  (void)cudaGetLastError();
  if (b->graph) cudaGraphExecDestroy(b->graph);
  release_graphs(b);
  free_staging(b);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  for (Slot& S : b->slots)
    if (S.arena) S.arena->free_all();
  b->shared.free_all();
  delete b;
}

}  // extern "C"
