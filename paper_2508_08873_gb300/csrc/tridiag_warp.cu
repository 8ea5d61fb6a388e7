// Instantiation of the one-warp cluster tridiagonal propagator (tri_warp.cuh)
// with the last third of the backward rows after the barrier's wait (the default).
#define LRP_TRI_WARP_KERNEL
#include "tri_warp.cuh"

namespace lrp {
template lrp_status tri_launch_warp<1>(Ctx* c, ClPlan* pl, ClKArgs& a);
}  // namespace lrp
