// Instantiation of the one-CTA-per-system variant of the one-warp tridiagonal
// propagator (tri_warp.cuh): one system per CTA of C warps, FP32 and FP64.
#define LRP_TRI_WARP_KERNEL
#include "tri_warp.cuh"

namespace lrp {
template lrp_status tri_launch_warp_block<float>(Ctx* c, ClPlan* pl, ClKArgs& a);
template lrp_status tri_launch_warp_block<double>(Ctx* c, ClPlan* pl, ClKArgs& a);
}  // namespace lrp
