// FP64 instantiations of the velocity field kernels (a flow field b(x) at the quadrature points,
// M = k+1 or k+3 Gauss points per direction; degrees 1..8), used by the transport example of Sec. 5.3.
#include "dg_launch.cuh"

namespace dgi {
int launch_apply_f64_vb(const dg_handle* h, const double* z, double* y, int mode, int stages, const StageArgs* st,
                        cudaStream_t s) {
  switch (h->N) {
    case 2: return apply_vb_n<2>(h, z, y, mode, stages, st, s);
    case 3: return apply_vb_n<3>(h, z, y, mode, stages, st, s);
    case 4: return apply_vb_n<4>(h, z, y, mode, stages, st, s);
    case 5: return apply_vb_n<5>(h, z, y, mode, stages, st, s);
    case 6: return apply_vb_n<6>(h, z, y, mode, stages, st, s);
    case 7: return apply_vb_n<7>(h, z, y, mode, stages, st, s);
    case 8: return apply_vb_n<8>(h, z, y, mode, stages, st, s);
    case 9: return apply_vb_n<9>(h, z, y, mode, stages, st, s);
    default: set_error("velocity field kernels support degrees 1..8"); return DG_ERR_INVALID_ARG;
  }
}
int launch_rhs_f64_vb(const dg_handle* h, const double* f, const double* const g[6], double* F, cudaStream_t s,
                      bool project) {
  switch (h->N) {
    case 2: return rhs_vb_n<2>(h, f, g, F, s, project);
    case 3: return rhs_vb_n<3>(h, f, g, F, s, project);
    case 4: return rhs_vb_n<4>(h, f, g, F, s, project);
    case 5: return rhs_vb_n<5>(h, f, g, F, s, project);
    case 6: return rhs_vb_n<6>(h, f, g, F, s, project);
    case 7: return rhs_vb_n<7>(h, f, g, F, s, project);
    case 8: return rhs_vb_n<8>(h, f, g, F, s, project);
    case 9: return rhs_vb_n<9>(h, f, g, F, s, project);
    default: set_error("velocity field kernels support degrees 1..8"); return DG_ERR_INVALID_ARG;
  }
}
}  // namespace dgi
