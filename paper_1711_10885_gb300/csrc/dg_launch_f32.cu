// FP32 instantiations of the operator kernels (degrees 1..10).
#include "dg_launch.cuh"

namespace dgi {
int launch_apply_f32(const dg_handle* h, const float* z, float* y, int mode, int stages, cudaStream_t s) {
  return apply_dispatch<float>(h, z, y, mode, stages, s);
}
bool has_offdiag_f32(const dg_handle* h) { return (h->N == 5 || h->N == 6) && !h->vb && !h->td && !h->pw; }
int launch_offdiag_f32(const dg_handle* h, const float* z, float* t, const int* from, int64_t nfrom, const int* to,
                       int64_t nto, cudaStream_t s) {
  if (!has_offdiag_f32(h)) {
    set_error("off-diagonal FP32 apply: degrees 4 and 5, axis-parallel handles only");
    return DG_ERR_INVALID_ARG;
  }
  if (h->N == 5) return apply_plane_offdiag<5>(h, z, t, from, (int)nfrom, to, (int)nto, s);
  return apply_plane_offdiag<6>(h, z, t, from, (int)nfrom, to, (int)nto, s);
}
}  // namespace dgi
