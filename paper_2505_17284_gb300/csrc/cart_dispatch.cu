// Dispatch over the Cartesian kernel's instantiation units and the static facts
// the host needs about the variants (tile width, shared memory per CTA).
#include "cart_kernel.cuh"

namespace rtk {

#define RTK_UNIT_DECL(NAME)                                                                     \
  cudaError_t cart_prepare_##NAME(int, int, int, int, int);                                     \
  cudaError_t cart_launch_##NAME(const InstDesc*, const WorkItem*, int, int, int, int, int, int, \
                                 cudaStream_t);
RTK_UNIT_DECL(f32_lane)
RTK_UNIT_DECL(f32_uni2v2)
RTK_UNIT_DECL(f32_uni2v4)
RTK_UNIT_DECL(f32_uni4)
RTK_UNIT_DECL(bf16_lane)
RTK_UNIT_DECL(bf16_uni2v2)
RTK_UNIT_DECL(bf16_uni2v4)
RTK_UNIT_DECL(bf16_uni4)
#undef RTK_UNIT_DECL

int cart_tile_width(int run) { return kCartWarps * run; }

// (run, vec) pairs built: per-lane directions (2, 1), (2, 2), (2, 4); chunk-uniform
// directions (2, 2), (2, 4), (4, 2).
bool cart_variant_exists(int order, int run, int vec, int uni) {
  if (order != 1 && order != 2) return false;
  if (run == 4) return uni && vec == 2;
  if (run != 2) return false;
  if (uni) return vec == 2 || vec == 4;
  return vec == 1 || vec == 2 || vec == 4;
}

cudaError_t prepare_cart_stage(int stage, int order, int storage, int run, int vec, int ly_max, int uni) {
  if (!cart_variant_exists(order, run, vec, uni)) return cudaErrorInvalidValue;
  if (storage == 0) {
    if (!uni) return cart_prepare_f32_lane(stage, order, run, vec, ly_max);
    return run == 4 ? cart_prepare_f32_uni4(stage, order, run, vec, ly_max)
                    : (vec == 4 ? cart_prepare_f32_uni2v4 : cart_prepare_f32_uni2v2)(stage, order, run, vec, ly_max);
  }
  if (!uni) return cart_prepare_bf16_lane(stage, order, run, vec, ly_max);
  return run == 4 ? cart_prepare_bf16_uni4(stage, order, run, vec, ly_max)
                  : (vec == 4 ? cart_prepare_bf16_uni2v4 : cart_prepare_bf16_uni2v2)(stage, order, run, vec, ly_max);
}

cudaError_t launch_cart_stage(const InstDesc* d_desc, const WorkItem* d_items, int n_items, int stage, int order,
                              int storage, int run, int vec, int ly_max, cudaStream_t stream, int uni) {
  if (n_items <= 0) return cudaSuccess;
  if (!cart_variant_exists(order, run, vec, uni)) return cudaErrorInvalidValue;
  if (storage == 0) {
    if (!uni) return cart_launch_f32_lane(d_desc, d_items, n_items, stage, order, run, vec, ly_max, stream);
    return run == 4 ? cart_launch_f32_uni4(d_desc, d_items, n_items, stage, order, run, vec, ly_max, stream)
                    : (vec == 4 ? cart_launch_f32_uni2v4 : cart_launch_f32_uni2v2)(d_desc, d_items, n_items, stage, order, run, vec, ly_max, stream);
  }
  if (!uni) return cart_launch_bf16_lane(d_desc, d_items, n_items, stage, order, run, vec, ly_max, stream);
  return run == 4 ? cart_launch_bf16_uni4(d_desc, d_items, n_items, stage, order, run, vec, ly_max, stream)
                  : (vec == 4 ? cart_launch_bf16_uni2v4 : cart_launch_bf16_uni2v2)(d_desc, d_items, n_items, stage, order, run, vec, ly_max, stream);
}

template <typename T>
static size_t smem_of(int order, int run, int vec, int ly, int stage) {
#define RTK_SMC(O, RR, VV, ST) \
  if (order == O && run == RR && vec == VV && stage == ST) return cart_smem_for<O, RR, VV, ST, T>(ly);
#define RTK_SMV(O, RR, VV) RTK_SMC(O, RR, VV, STAGE_EULER) RTK_SMC(O, RR, VV, STAGE_HEUN1) RTK_SMC(O, RR, VV, STAGE_HEUN2)
#define RTK_SMO(O) RTK_SMV(O, 2, 1) RTK_SMV(O, 2, 2) RTK_SMV(O, 2, 4) RTK_SMV(O, 4, 2)
  RTK_SMO(1) RTK_SMO(2)
#undef RTK_SMO
#undef RTK_SMV
#undef RTK_SMC
  return 0;
}

size_t cart_smem_bytes(int order, int storage, int run, int vec, int ly, int stage) {
  if (run != 2 && run != 4) return 0;
  return storage == 0 ? smem_of<float>(order, run, vec, ly, stage) : smem_of<__nv_bfloat16>(order, run, vec, ly, stage);
}

}  // namespace rtk
