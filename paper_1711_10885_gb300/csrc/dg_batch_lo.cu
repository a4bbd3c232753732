// Batched-apply kernels of degrees 1..4 (N = 2..5, all launch variants).
#include "dg_batch_kernels.cuh"

namespace dgbt {
VariantInfo variant_info_lo(int N, int v) {
  switch (N) {
    case 2: return variant_info_n<2>(v);
    case 3: return variant_info_n<3>(v);
    case 4: return variant_info_n<4>(v);
    default: return variant_info_n<5>(v);
  }
}
}  // namespace dgbt
