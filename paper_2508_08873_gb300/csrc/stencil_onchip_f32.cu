// FP32 instantiations of the on-chip CG kernel (stencil_onchip.cuh): grid
// pitch 64..512 columns, 16 or 32 rows per CTA.
#include "stencil_onchip.cuh"

namespace lrp {
namespace oc {
Variant variant_f32(int pitch, int rpt) {
  switch (pitch * 100 + rpt) {
    case 6416: return make_variant<float, 64, 16, false, 12>();
    case 6432: return make_variant<float, 64, 32, true, 16>();
    case 12816: return make_variant<float, 128, 16, false, 12>();
    case 12832: return make_variant<float, 128, 32, true, 16>();
    case 25616: return make_variant<float, 256, 16, false, 12>();
    case 25632: return make_variant<float, 256, 32, true, 16>();
    case 51216: return make_variant<float, 512, 16, false, 12>();
    case 51232: return make_variant<float, 512, 32, true, 16>();
    default: return Variant{nullptr, 0};
  }
}
}  // namespace oc
}  // namespace lrp
