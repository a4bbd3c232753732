// Double-float instantiations of the velocity field kernels (M = k+1 or k+3 points, degrees 1..8): the
// transport example of Sec. 5.3 with FP64 vectors and the operator on the FP32 pipes.
#include "dg_launch.cuh"

namespace dgi {
int launch_apply_f64x_vb(const dg_handle* h, const double* z, double* y, int mode, int stages, const StageArgs* st,
                         cudaStream_t s) {
  switch (h->N) {
    case 2: return apply_vb_n<2, dgk::dfl>(h, z, y, mode, stages, st, s);
    case 3: return apply_vb_n<3, dgk::dfl>(h, z, y, mode, stages, st, s);
    case 4: return apply_vb_n<4, dgk::dfl>(h, z, y, mode, stages, st, s);
    case 5: return apply_vb_n<5, dgk::dfl>(h, z, y, mode, stages, st, s);
    case 6: return apply_vb_n<6, dgk::dfl>(h, z, y, mode, stages, st, s);
    case 7: return apply_vb_n<7, dgk::dfl>(h, z, y, mode, stages, st, s);
    case 8: return apply_vb_n<8, dgk::dfl>(h, z, y, mode, stages, st, s);
    case 9: return apply_vb_n<9, dgk::dfl>(h, z, y, mode, stages, st, s);
    default: set_error("velocity field kernels support degrees 1..8"); return DG_ERR_INVALID_ARG;
  }
}
}  // namespace dgi
