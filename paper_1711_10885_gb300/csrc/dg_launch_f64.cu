// FP64 instantiations of the operator kernels (degrees 1..10).
#include "dg_launch.cuh"

namespace dgi {
int launch_apply_f64(const dg_handle* h, const double* z, double* y, int mode, int stages, cudaStream_t s) {
  return apply_dispatch<double>(h, z, y, mode, stages, s);
}
int launch_rhs_f64(const dg_handle* h, const double* f, const double* const g[6], double* F, cudaStream_t s) {
  return rhs_dispatch<double>(h, f, g, F, s);
}
int launch_diag_blocks_f64(const dg_handle* h, double* out, int cell_base, int ncells, double* V, double* tr,
                           cudaStream_t s) {
  return diag_blocks_dispatch(h, out, cell_base, ncells, V, tr, s);
}
}  // namespace dgi
