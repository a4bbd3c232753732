// Batched-apply kernels of degrees 5..8 (N = 6..9, all launch variants).
#include "dg_batch_kernels.cuh"

namespace dgbt {
VariantInfo variant_info_hi(int N, int v) {
  switch (N) {
    case 6: return variant_info_n<6>(v);
    case 7: return variant_info_n<7>(v);
    case 8: return variant_info_n<8>(v);
    default: return variant_info_n<9>(v);
  }
}
}  // namespace dgbt
