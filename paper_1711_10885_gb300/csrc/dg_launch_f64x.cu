// Double-float instantiations of the operator kernels (degrees 1..10): FP64 vectors in and out, every
// operation on pairs of FP32 numbers (about 48 significand bits) so that the work runs on the FP32 pipes.
#include "dg_launch.cuh"

namespace dgi {
int launch_apply_f64x(const dg_handle* h, const double* z, double* y, int mode, int stages, cudaStream_t s) {
  if (h->pw) return launch_apply_pwx(h, z, y, mode, stages, nullptr, s);
  if (h->td) return launch_apply_td(h, z, y, mode, stages, nullptr, true, s);
  if (h->vb) return launch_apply_f64x_vb(h, z, y, mode, stages, nullptr, s);
  return apply_dispatch<dgk::dfl, double>(h, z, y, mode, stages, s);
}
int launch_stage_f64x(const dg_handle* h, const double* u, double* y, const StageArgs& st, cudaStream_t s) {
  if (h->pw) return launch_apply_pwx(h, u, y, 3, 3, &st, s);
  if (h->td) return launch_apply_td(h, u, y, 3, 3, &st, true, s);
  if (h->vb) return launch_apply_f64x_vb(h, u, y, 3, 3, &st, s);
  return apply_dispatch<dgk::dfl, double>(h, u, y, 3, 3, s, &st);
}
}  // namespace dgi
