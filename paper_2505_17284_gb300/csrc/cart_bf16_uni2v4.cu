// Instantiation unit of the Cartesian stage kernel: storage __nv_bfloat16, chunk-uniform flow
// directions, runs of 2 cells per warp, 4 ordinates per lane. Units are compiled in parallel; the dispatcher is cart_dispatch.cu.
#include "cart_kernel.cuh"

namespace rtk {
#define RTK_CART_UNIT_LIST(X, TT, U) RTK_CART_STAGES(X, 1, 2, 4, U, TT) RTK_CART_STAGES(X, 2, 2, 4, U, TT)
RTK_CART_DEFINE_UNIT(bf16_uni2v4, __nv_bfloat16, true)
#undef RTK_CART_UNIT_LIST
}  // namespace rtk
