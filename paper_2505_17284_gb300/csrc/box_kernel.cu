// Read-back evaluation of the QoI-box outflow (Sec. 3.1 QoI-1) of the current
// state. The time integral (QoI-2) is accumulated by the stage launches
// themselves (box work items of the Cartesian stage kernel, on each stage's
// input state); this kernel only fills the box columns of InstState::S_cur
// when the QoIs are read. Partial sums are FP64 per work item, reduced by the
// last item in item order (deterministic); it borrows the instance's ticket
// and partial rows, which are idle between launches.
#include "box_device.cuh"

namespace rtk {

namespace {

constexpr int kBoxThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kBoxThreads, 4)
    box_eval_kernel(const InstDesc* __restrict__ descs, const WorkItem* __restrict__ items) {
  __shared__ double red[(kBoxThreads / 32) * kMaxBox];
  __shared__ uint32_t s_last;
  const WorkItem it = items[blockIdx.x];
  const InstDesc& d = descs[it.inst];
  InstState* st = d.st;
  // current state: Euler keeps it in the buffer named by the parity, Heun in 0
  const T* psi = reinterpret_cast<const T*>(d.psi[st->parity]);
  double part[kMaxBox];
  box_face_sums<kBoxThreads, T>(d, it, psi, red, part);
  if (threadIdx.x < kMaxBox) d.partials[(size_t)it.item * NQ + threadIdx.x] = part[threadIdx.x];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t t = atomicAdd(&st->ticket, 1u);
    s_last = (t == static_cast<uint32_t>(it.count - 1)) ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x < kMaxBox) {
    double v = 0.0;
    for (int i = 0; i < it.count; ++i) v += __ldcg(d.partials + (size_t)i * NQ + threadIdx.x);
    st->S_cur[kQBox + threadIdx.x] = (threadIdx.x < d.n_boxes) ? v : 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    st->ticket = 0u;
    __threadfence();
  }
}

}  // namespace

cudaError_t launch_box_eval(const InstDesc* d_desc, const WorkItem* d_items, int n_items, int storage,
                            cudaStream_t stream) {
  if (n_items <= 0) return cudaSuccess;
  if (storage == 1)
    box_eval_kernel<__nv_bfloat16><<<n_items, kBoxThreads, 0, stream>>>(d_desc, d_items);
  else
    box_eval_kernel<float><<<n_items, kBoxThreads, 0, stream>>>(d_desc, d_items);
  return cudaGetLastError();
}

}  // namespace rtk
