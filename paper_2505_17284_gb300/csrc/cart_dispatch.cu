// Dispatch over the Cartesian kernel's instantiation units and the static facts
// the host needs about the variants (tile width, shared memory per CTA).
#include "cart_kernel.cuh"

namespace rtk {

cudaError_t cart_prepare_f32_lane(int, int, int, int);
cudaError_t cart_prepare_f32_uni(int, int, int, int);
cudaError_t cart_prepare_bf16_lane(int, int, int, int);
cudaError_t cart_prepare_bf16_uni(int, int, int, int);
cudaError_t cart_launch_f32_lane(const InstDesc*, const WorkItem*, int, int, int, int, int, cudaStream_t);
cudaError_t cart_launch_f32_uni(const InstDesc*, const WorkItem*, int, int, int, int, int, cudaStream_t);
cudaError_t cart_launch_bf16_lane(const InstDesc*, const WorkItem*, int, int, int, int, int, cudaStream_t);
cudaError_t cart_launch_bf16_uni(const InstDesc*, const WorkItem*, int, int, int, int, int, cudaStream_t);

int cart_tile_width(int run) { return kCartWarps * run; }

bool cart_variant_exists(int order, int run, int vec, int uni) {
  if (order != 1 && order != 2) return false;
  if (run != 2) return false;
  if (uni) return vec == 2 || vec == 4;
  return vec == 1 || vec == 2 || vec == 4;
}

cudaError_t prepare_cart_stage(int stage, int order, int storage, int run, int vec, int ly_max, int uni) {
  if (!cart_variant_exists(order, run, vec, uni)) return cudaErrorInvalidValue;
  if (storage == 0) return uni ? cart_prepare_f32_uni(stage, order, vec, ly_max) : cart_prepare_f32_lane(stage, order, vec, ly_max);
  return uni ? cart_prepare_bf16_uni(stage, order, vec, ly_max) : cart_prepare_bf16_lane(stage, order, vec, ly_max);
}

cudaError_t launch_cart_stage(const InstDesc* d_desc, const WorkItem* d_items, int n_items, int stage, int order,
                              int storage, int run, int vec, int ly_max, cudaStream_t stream, int uni) {
  if (n_items <= 0) return cudaSuccess;
  if (!cart_variant_exists(order, run, vec, uni)) return cudaErrorInvalidValue;
  if (storage == 0)
    return uni ? cart_launch_f32_uni(d_desc, d_items, n_items, stage, order, vec, ly_max, stream)
               : cart_launch_f32_lane(d_desc, d_items, n_items, stage, order, vec, ly_max, stream);
  return uni ? cart_launch_bf16_uni(d_desc, d_items, n_items, stage, order, vec, ly_max, stream)
             : cart_launch_bf16_lane(d_desc, d_items, n_items, stage, order, vec, ly_max, stream);
}

template <typename T>
static size_t smem_of(int order, int vec, int ly, int stage) {
#define RTK_SMC(O, VV, ST) \
  if (order == O && vec == VV && stage == ST) return cart_smem_for<O, 2, VV, ST, T>(ly);
#define RTK_SMO(O) RTK_SMC(O, 1, STAGE_EULER) RTK_SMC(O, 1, STAGE_HEUN1) RTK_SMC(O, 1, STAGE_HEUN2) \
  RTK_SMC(O, 2, STAGE_EULER) RTK_SMC(O, 2, STAGE_HEUN1) RTK_SMC(O, 2, STAGE_HEUN2)                 \
  RTK_SMC(O, 4, STAGE_EULER) RTK_SMC(O, 4, STAGE_HEUN1) RTK_SMC(O, 4, STAGE_HEUN2)
  RTK_SMO(1) RTK_SMO(2)
#undef RTK_SMO
#undef RTK_SMC
  return 0;
}

size_t cart_smem_bytes(int order, int storage, int run, int vec, int ly, int stage) {
  if (run != 2) return 0;
  return storage == 0 ? smem_of<float>(order, vec, ly, stage) : smem_of<__nv_bfloat16>(order, vec, ly, stage);
}

}  // namespace rtk
