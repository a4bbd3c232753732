// FP64 instantiations of the point-wise coefficient kernels (Problem B of Sec. 5.1: coefficients at the
// quadrature points, affine cells, q = 2p or 2p+4; degrees 1..8).
#include "dg_launch.cuh"

namespace dgi {
int launch_apply_pw(const dg_handle* h, const double* z, double* y, int mode, int stages, const StageArgs* st,
                    cudaStream_t s) {
  return pw_dispatch<double>(h, z, y, mode, stages, st, nullptr, s, false);
}
int launch_rhs_pw(const dg_handle* h, const double* f, const double* const g[6], double* F, cudaStream_t s,
                  bool project) {
  return pw_dispatch<double>(h, f, F, 2, 2, nullptr, g, s, project);
}
}  // namespace dgi
