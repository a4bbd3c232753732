// Double-float instantiations of the point-wise coefficient kernels (FP64 vectors, every operation on pairs
// of FP32 numbers; degrees 1..8, q = 2p or 2p+4).
#include "dg_launch.cuh"

namespace dgi {
int launch_apply_pwx(const dg_handle* h, const double* z, double* y, int mode, int stages, const StageArgs* st,
                     cudaStream_t s) {
  return pw_dispatch<dgk::dfl>(h, z, y, mode, stages, st, nullptr, s, false);
}
}  // namespace dgi
