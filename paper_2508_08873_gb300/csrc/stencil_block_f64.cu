// FP64 instantiations of the block CG kernel (stencil_block.cuh): grids of
// up to 256 columns, four systems per block, 32 rows per CTA.
#include "stencil_block.cuh"

namespace lrp {
namespace bk {

Variant variant_f64(int pitch) {
  switch (pitch) {
    case 64: return make_variant<double, 4, 64, 32>();
    case 128: return make_variant<double, 4, 128, 32>();
    case 256: return make_variant<double, 4, 256, 32>();
    default: return Variant{nullptr, 0, 0, 0, 0, 0};
  }
}

}  // namespace bk
}  // namespace lrp
