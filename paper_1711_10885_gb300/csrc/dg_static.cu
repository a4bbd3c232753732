// dg_static.cu -- Jacobian application that allocates nothing: its work buffers (point-space
// residual, face traces, face coefficients) live in one file-scope device array instead of in
// memory obtained from cudaMalloc by dg_setup.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include "dg_internal.h"

namespace {

// Shared by every call on a device and kept until the process exits.
static __device__ __align__(256) unsigned char g_static_scratch[DG_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
void* g_static_ptr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device, looked up once per device; *dev_out receives
// the current device's index.
int static_scratch(void** out, int* dev_out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return dgi::cuda_fail(e, "dg_apply_jacobian_static: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) {
    dgi::set_error("dg_apply_jacobian_static: device index out of range");
    return DG_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_static_mutex);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return dgi::cuda_fail(e, "dg_apply_jacobian_static: cudaGetSymbolAddress");
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  *dev_out = dev;
  return DG_OK;
}

// Face coefficients of every cell, the same quantities dg_setup computes on the host:
// interior (w_own D_own / h, w_nbr D_nbr / h, gamma_F), Dirichlet boundary (D_own / h, 1, gamma_F).
__global__ void static_face_coeffs(const double* __restrict__ D, int nx, int ny, int nz, double hx, double hy,
                                   double hz, double sigma, double* __restrict__ fc) {
  const int64_t ncell = (int64_t)nx * ny * nz;
  for (int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < ncell;
       cell += (int64_t)gridDim.x * blockDim.x) {
    const int ic[3] = {(int)(cell % nx), (int)((cell / nx) % ny), (int)(cell / ((int64_t)nx * ny))};
    const int n[3] = {nx, ny, nz};
    const double hh[3] = {hx, hy, hz};
    const int64_t strides[3] = {1, nx, (int64_t)nx * ny};
    const double Do = D[cell];
    for (int dir = 0; dir < 3; ++dir)
      for (int side = 0; side < 2; ++side) {
        double* c3 = fc + (cell * 6 + 2 * dir + side) * 3;
        const double hq = hh[dir];
        const bool boundary = side ? ic[dir] == n[dir] - 1 : ic[dir] == 0;
        if (boundary) {
          c3[0] = Do / hq;
          c3[1] = 1.0;  // the upwind flux of a Dirichlet face
          c3[2] = Do * sigma / hq;
        } else {
          const double Dn = D[side ? cell + strides[dir] : cell - strides[dir]];
          const double sum = Do + Dn;
          c3[0] = (Dn / sum) * Do / hq;
          c3[1] = (Do / sum) * Dn / hq;
          c3[2] = (2.0 * Do * Dn / sum) * sigma / hq;
        }
      }
  }
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" {

int dg_apply_jacobian_static(const dg_mesh* mesh, int32_t k, const double* D_dev, const double b[3], double c,
                             double sigma, const double* z_dev, double* y_dev, void* stream) {
  using namespace dgi;
  if (!mesh || !D_dev || !b || !z_dev || !y_dev || z_dev == y_dev) {
    set_error("dg_apply_jacobian_static: null pointer, or z and y alias");
    return DG_ERR_INVALID_ARG;
  }
  if (k < 1 || k > DG_MAX_DEGREE) {
    set_error("dg_apply_jacobian_static: degree k must be in [1, 10]");
    return DG_ERR_INVALID_ARG;
  }
  int64_t ncell = 1;
  for (int r = 0; r < 3; ++r) {
    if (mesh->n[r] < 1 || !std::isfinite(mesh->lo[r]) || !std::isfinite(mesh->hi[r]) ||
        !(mesh->hi[r] > mesh->lo[r]) || !std::isfinite(b[r])) {
      set_error("dg_apply_jacobian_static: each axis needs n >= 1, finite lo < hi and a finite velocity");
      return DG_ERR_INVALID_ARG;
    }
    if (ncell > ((int64_t)1 << 30) / mesh->n[r]) {
      set_error("dg_apply_jacobian_static: more than 2^30 cells");
      return DG_ERR_INVALID_ARG;
    }
    ncell *= mesh->n[r];
  }
  if (!std::isfinite(c) || !std::isfinite(sigma) || sigma < 0) {
    set_error("dg_apply_jacobian_static: c must be finite and sigma finite and >= 0");
    return DG_ERR_INVALID_ARG;
  }
  const int N = k + 1;
  const size_t bytes_V = align256((size_t)ncell * N * N * N * sizeof(double));
  const size_t bytes_tr = align256((size_t)ncell * 12 * N * N * sizeof(double));
  const size_t bytes_fc = align256((size_t)ncell * 18 * sizeof(double));
  if (ncell > ((int64_t)1 << 30) || bytes_V + bytes_tr + bytes_fc > (size_t)DG_STATIC_SCRATCH_BYTES) {
    set_error("dg_apply_jacobian_static: problem needs " + std::to_string(bytes_V + bytes_tr + bytes_fc) +
              " bytes of work space, more than the fixed " + std::to_string((size_t)DG_STATIC_SCRATCH_BYTES) +
              " bytes; use dg_setup / dg_apply_jacobian");
    return DG_ERR_INVALID_ARG;
  }
  void* base = nullptr;
  int dev = 0;
  if (int rc = static_scratch(&base, &dev)) return rc;
  unsigned char* p = static_cast<unsigned char*>(base);

  // A handle on the stack that points into the fixed array; nothing in it is owned or freed.
  dg_handle h;
  h.k = k;
  h.N = N;
  h.M = N;
  h.ncell = ncell;
  for (int r = 0; r < 3; ++r) {
    h.n[r] = mesh->n[r];
    h.lo[r] = mesh->lo[r];
    h.hi[r] = mesh->hi[r];
    h.h[r] = (mesh->hi[r] - mesh->lo[r]) / mesh->n[r];
    h.b[r] = b[r];
  }
  h.c = c;
  h.sigma = sigma;
  build_tables(N, N, &h.tab);
  h.work_V = p;
  h.work_tr = p + bytes_V;
  h.p64.fc = p + bytes_V + bytes_tr;
  h.p64.D = const_cast<double*>(D_dev);
  h.device = dev;

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const unsigned fgrid = (unsigned)std::min<int64_t>((ncell + 127) / 128, (int64_t)sm_count() * 4);
  static_face_coeffs<<<fgrid, 128, 0, s>>>(D_dev, h.n[0], h.n[1], h.n[2], h.h[0], h.h[1], h.h[2], sigma,
                                            static_cast<double*>(h.p64.fc));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "dg_apply_jacobian_static: face coefficient kernel");
  return launch_apply_f64(&h, z_dev, y_dev, 0, 3, s);
}

}  // extern "C"
