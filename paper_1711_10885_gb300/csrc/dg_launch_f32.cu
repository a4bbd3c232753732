// FP32 instantiations of the operator kernels (degrees 1..10).
#include "dg_launch.cuh"

namespace dgi {
int launch_apply_f32(const dg_handle* h, const float* z, float* y, int mode, int stages, cudaStream_t s) {
  return apply_dispatch<float>(h, z, y, mode, stages, s);
}
}  // namespace dgi
