// Instantiation unit of the Cartesian stage kernel: storage float, per-lane flow
// directions. Units are compiled in parallel; the dispatcher is cart_dispatch.cu.
#include "cart_kernel.cuh"

namespace rtk {
#define RTK_CART_UNIT_LIST(X, TT, U) RTK_CART_STAGES(X, 1, 2, 1, U, TT) RTK_CART_STAGES(X, 1, 2, 2, U, TT) RTK_CART_STAGES(X, 1, 2, 4, U, TT) \
  RTK_CART_STAGES(X, 2, 2, 1, U, TT) RTK_CART_STAGES(X, 2, 2, 2, U, TT) RTK_CART_STAGES(X, 2, 2, 4, U, TT)
RTK_CART_DEFINE_UNIT(f32_lane, float, false)
#undef RTK_CART_UNIT_LIST
}  // namespace rtk
