// Instantiations of the tensor-diffusion / affine-geometry kernels (the paper's tensor-valued D of
// Problem A and the affine cells of Problem B, Sec. 5.1): degrees 1..8, M = N, FP64 and double-float.
#include "dg_launch.cuh"

namespace dgi {

template <typename T>
static int td_dispatch(const dg_handle* h, const double* z, double* y, int mode, int stages, const StageArgs* st,
                       const double* const g6[6], cudaStream_t s, bool project) {
  switch (h->N) {
    case 2: return apply_td_n<2, T>(h, z, y, mode, stages, st, g6, s, project);
    case 3: return apply_td_n<3, T>(h, z, y, mode, stages, st, g6, s, project);
    case 4: return apply_td_n<4, T>(h, z, y, mode, stages, st, g6, s, project);
    case 5: return apply_td_n<5, T>(h, z, y, mode, stages, st, g6, s, project);
    case 6: return apply_td_n<6, T>(h, z, y, mode, stages, st, g6, s, project);
    case 7: return apply_td_n<7, T>(h, z, y, mode, stages, st, g6, s, project);
    case 8: return apply_td_n<8, T>(h, z, y, mode, stages, st, g6, s, project);
    case 9: return apply_td_n<9, T>(h, z, y, mode, stages, st, g6, s, project);
    default: set_error("tensor-diffusion kernels support degrees 1..8"); return DG_ERR_INVALID_ARG;
  }
}

int launch_apply_td(const dg_handle* h, const double* z, double* y, int mode, int stages, const StageArgs* st,
                    bool pairs, cudaStream_t s) {
  if (pairs) return td_dispatch<dgk::dfl>(h, z, y, mode, stages, st, nullptr, s, false);
  return td_dispatch<double>(h, z, y, mode, stages, st, nullptr, s, false);
}

int launch_rhs_td(const dg_handle* h, const double* f, const double* const g[6], double* F, cudaStream_t s,
                  bool project) {
  return td_dispatch<double>(h, f, F, 2, 2, nullptr, g, s, project);
}

}  // namespace dgi
