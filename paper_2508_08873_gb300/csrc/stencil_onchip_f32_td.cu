// FP32 instantiations of the on-chip CG kernel (stencil_onchip.cuh) for
// time-dependent operators (every fine step its own couplings and scales):
// grid pitch 64..512 columns, 16 or 32 rows per CTA.
#include "stencil_onchip.cuh"

namespace lrp {
namespace oc {
Variant variant_f32_td(int pitch, int rpt) {
  switch (pitch * 100 + rpt) {
    case 6416: return make_variant<float, 64, 16, false, 12, true>();
    case 6432: return make_variant<float, 64, 32, true, 16, true>();
    case 12816: return make_variant<float, 128, 16, false, 12, true>();
    case 12832: return make_variant<float, 128, 32, true, 16, true>();
    case 25616: return make_variant<float, 256, 16, false, 12, true>();
    case 25632: return make_variant<float, 256, 32, true, 16, true>();
    case 51216: return make_variant<float, 512, 16, false, 12, true>();
    case 51232: return make_variant<float, 512, 32, true, 16, true>();
    default: return Variant{nullptr, 0};
  }
}
}  // namespace oc
}  // namespace lrp
