// Instantiation of the one-warp cluster tridiagonal propagator (tri_warp.cuh)
// with all of the chunk-interior solve between the barrier's arrive and wait.
#define LRP_TRI_WARP_KERNEL
#include "tri_warp.cuh"

namespace lrp {
template lrp_status tri_launch_warp<0>(Ctx* c, ClPlan* pl, ClKArgs& a);
}  // namespace lrp
