// FP64 instantiations of the operator kernels (degrees 1..10).
#include "dg_launch.cuh"

namespace dgi {
static int diag_blocks_dispatch(const dg_handle* h, double* out, int cell_base, int ncells, double* V, double* tr,
                                cudaStream_t s) {
  switch (h->N) {
    case 2: return diag_blocks_n<2>(h, out, cell_base, ncells, V, tr, s);
    case 3: return diag_blocks_n<3>(h, out, cell_base, ncells, V, tr, s);
    case 4: return diag_blocks_n<4>(h, out, cell_base, ncells, V, tr, s);
    case 5: return diag_blocks_n<5>(h, out, cell_base, ncells, V, tr, s);
    case 6: return diag_blocks_n<6>(h, out, cell_base, ncells, V, tr, s);
    case 7: return diag_blocks_n<7>(h, out, cell_base, ncells, V, tr, s);
    case 8: return diag_blocks_n<8>(h, out, cell_base, ncells, V, tr, s);
    case 9: return diag_blocks_n<9>(h, out, cell_base, ncells, V, tr, s);
    case 10: return diag_blocks_n<10>(h, out, cell_base, ncells, V, tr, s);
    case 11: return diag_blocks_n<11>(h, out, cell_base, ncells, V, tr, s);
    default: set_error("unsupported degree"); return DG_ERR_INVALID_ARG;
  }
}

int launch_apply_f64(const dg_handle* h, const double* z, double* y, int mode, int stages, cudaStream_t s) {
  if (h->pw) return launch_apply_pw(h, z, y, mode, stages, nullptr, s);
  if (h->td) return launch_apply_td(h, z, y, mode, stages, nullptr, false, s);
  if (h->vb) return launch_apply_f64_vb(h, z, y, mode, stages, nullptr, s);
  return apply_dispatch<double>(h, z, y, mode, stages, s);
}
int launch_stage_f64(const dg_handle* h, const double* u, double* y, const StageArgs& st, cudaStream_t s) {
  if (h->pw) return launch_apply_pw(h, u, y, 3, 3, &st, s);
  if (h->td) return launch_apply_td(h, u, y, 3, 3, &st, false, s);
  if (h->vb) return launch_apply_f64_vb(h, u, y, 3, 3, &st, s);
  return apply_dispatch<double>(h, u, y, 3, 3, s, &st);
}
int launch_rhs_f64(const dg_handle* h, const double* f, const double* const g[6], double* F, cudaStream_t s,
                   bool project) {
  if (h->pw) return launch_rhs_pw(h, f, g, F, s, project);
  if (h->td) return launch_rhs_td(h, f, g, F, s, project);
  if (h->vb) return launch_rhs_f64_vb(h, f, g, F, s, project);
  return rhs_dispatch<double>(h, f, g, F, s, project);
}
int launch_diag_blocks_f64(const dg_handle* h, double* out, int cell_base, int ncells, double* V, double* tr,
                           cudaStream_t s) {
  return diag_blocks_dispatch(h, out, cell_base, ncells, V, tr, s);
}
}  // namespace dgi
