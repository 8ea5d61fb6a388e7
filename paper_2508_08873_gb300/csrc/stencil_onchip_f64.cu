// FP64 instantiations of the on-chip CG kernel (stencil_onchip.cuh): grid
// pitch 64..512 columns, 8 or 16 rows per CTA.
#include "stencil_onchip.cuh"

namespace lrp {
namespace oc {
Variant variant_f64(int pitch, int rpt) {
  switch (pitch * 100 + rpt) {
    case 6408: return make_variant<double, 64, 8, false, 8>();
    case 6416: return make_variant<double, 64, 16, true, 8>();
    case 12808: return make_variant<double, 128, 8, false, 8>();
    case 12816: return make_variant<double, 128, 16, true, 8>();
    case 25608: return make_variant<double, 256, 8, false, 8>();
    case 25616: return make_variant<double, 256, 16, true, 8>();
    case 51208: return make_variant<double, 512, 8, false, 8>();
    case 51216: return make_variant<double, 512, 16, true, 8>();
    default: return Variant{nullptr, 0};
  }
}
}  // namespace oc
}  // namespace lrp
