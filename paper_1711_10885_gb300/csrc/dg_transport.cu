// dg_transport.cu -- the transport example of Sec. 5.3: velocity field tables at the quadrature points,
// L2 projection of the initial value, and explicit strong-stability-preserving Runge-Kutta stages.
#include <cmath>
#include <string>

#include "dg_dfloat.cuh"
#include "dg_internal.h"

namespace {

using dgi::MAXM;

struct PointGeo {
  double lo[3], h[3];
  int n[3];
  int M;
  double xi[MAXM];  // Gauss points on [0,1]
  double w[MAXM];   // Gauss weights
};

// the fixed flow field of Sec. 5.3
__device__ __forceinline__ void taylor_green(const double x[3], double b[3]) {
  double s1, c1, s2, c2, s3, c3;
  sincos(x[0], &s1, &c1);
  sincos(-x[1], &s2, &c2);
  sincos(-x[2], &s3, &c3);
  b[0] = c1 * s2 * s3;
  b[1] = 0.5 * s1 * c2 * s3;
  b[2] = 0.5 * s1 * s2 * c3;
}

// b at every volume point, raw[(cell*M^3 + q)*3 + r], q = i1 + M (i2 + M i3) (TAYLOR_GREEN or CONSTANT)
__global__ void velocity_points(PointGeo pg, int kind, double b0, double b1, double b2, double* __restrict__ raw,
                                int64_t npts) {
  const int M = pg.M, M3 = M * M * M;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < npts; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = e / M3;
    const int q = (int)(e - cell * M3);
    const int ic[3] = {(int)(cell % pg.n[0]), (int)((cell / pg.n[0]) % pg.n[1]),
                       (int)(cell / ((int64_t)pg.n[0] * pg.n[1]))};
    const int iq[3] = {q % M, (q / M) % M, q / (M * M)};
    double b[3] = {b0, b1, b2};
    if (kind == DG_VELOCITY_TAYLOR_GREEN) {
      double x[3];
      for (int r = 0; r < 3; ++r) x[r] = pg.lo[r] + pg.h[r] * (ic[r] + pg.xi[iq[r]]);
      taylor_green(x, b);
    }
    for (int r = 0; r < 3; ++r) raw[e * 3 + r] = b[r];
  }
}

// b . e_dir at the face points of every face of every cell, bface[(cell*6 + face)*M^2 + pa + M pb]
__global__ void velocity_faces(PointGeo pg, int kind, double b0, double b1, double b2, double* __restrict__ bface,
                               int64_t nvals) {
  const int M = pg.M, MM = M * M;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nvals; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cf = e / MM;
    const int p = (int)(e - cf * MM);
    const int64_t cell = cf / 6;
    const int face = (int)(cf - cell * 6), dir = face / 2, side = face % 2;
    const int ta = dir == 0 ? 1 : 0, tb = dir == 2 ? 1 : 2;
    const int ic[3] = {(int)(cell % pg.n[0]), (int)((cell / pg.n[0]) % pg.n[1]),
                       (int)(cell / ((int64_t)pg.n[0] * pg.n[1]))};
    double b[3] = {b0, b1, b2};
    if (kind == DG_VELOCITY_TAYLOR_GREEN) {
      double x[3];
      x[dir] = pg.lo[dir] + pg.h[dir] * (ic[dir] + side);
      x[ta] = pg.lo[ta] + pg.h[ta] * (ic[ta] + pg.xi[p % M]);
      x[tb] = pg.lo[tb] + pg.h[tb] * (ic[tb] + pg.xi[p / M]);
      taylor_green(x, b);
    }
    bface[e] = b[dir];
  }
}

// pre-scaled volume velocity of the kernels: bsc[((cell*3 + r)*M + l)*M^2 + a + M b] = -b_r |T| / h_r w_a w_b
// at the point with index l along axis r and (a, b) along the other two axes in increasing order
__global__ void scale_velocity(PointGeo pg, const double* __restrict__ raw, double* __restrict__ bsc,
                               int64_t nvals) {
  const int M = pg.M, MM = M * M, M3 = MM * M;
  const double vol = pg.h[0] * pg.h[1] * pg.h[2];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nvals; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cr = e / M3;
    const int rem = (int)(e - cr * M3);
    const int64_t cell = cr / 3;
    const int r = (int)(cr - cell * 3);
    const int l = rem / MM, t = rem - l * MM, a = t % M, b = t / M;
    int i[3];
    i[r] = l;
    i[r == 0 ? 1 : 0] = a;
    i[r == 2 ? 1 : 2] = b;
    const int q = i[0] + M * (i[1] + M * i[2]);
    bsc[e] = -raw[(cell * M3 + q) * 3 + r] * (vol / pg.h[r]) * (pg.w[a] * pg.w[b]);
  }
}

// double-float copy of a table (DG_F64X applies of the velocity field kernels)
__global__ void to_pairs(const double* __restrict__ a, dgk::dfl* __restrict__ x, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = dgk::dfl_from_double(a[i]);
}

unsigned grid_for(int64_t n) {
  const int64_t blocks = (n + 255) / 256, cap = (int64_t)dgi::sm_count() * 16;
  return (unsigned)(blocks > cap ? cap : (blocks > 0 ? blocks : 1));
}

}  // namespace

namespace dgi {

int copy_to_pairs(const double* a, void* x_pairs, int64_t n, cudaStream_t s) {
  to_pairs<<<grid_for(n), 256, 0, s>>>(a, static_cast<dgk::dfl*>(x_pairs), n);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : cuda_fail(e, "to_pairs launch");
}

int setup_velocity(dg_handle* h, int kind, const double b[3], const double* b_qp, const double* b_face,
                   cudaStream_t s) {
  const int M = h->M;
  const int64_t npts = h->ncell * M * M * M, nface = h->ncell * 6 * M * M;
  PointGeo pg;
  for (int r = 0; r < 3; ++r) {
    pg.lo[r] = h->lo[r];
    pg.h[r] = h->h[r];
    pg.n[r] = h->n[r];
  }
  pg.M = M;
  for (int i = 0; i < M; ++i) {
    pg.xi[i] = h->tab.xi[i];
    pg.w[i] = h->tab.w[i];
  }
  double* raw = nullptr;
  cudaError_t e = cudaMalloc(&h->bsc, npts * 3 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&h->bface, nface * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&h->bscX, npts * 3 * sizeof(dgk::dfl));
  if (e == cudaSuccess) e = cudaMalloc(&h->bfaceX, nface * sizeof(dgk::dfl));
  if (e == cudaSuccess) e = cudaMalloc(&raw, npts * 3 * sizeof(double));
  if (e != cudaSuccess) {
    cudaFree(raw);
    return cuda_fail(e, "dg_setup: velocity tables");
  }
  if (kind == DG_VELOCITY_POINTS) {
    e = cudaMemcpyAsync(raw, b_qp, npts * 3 * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h->bface, b_face, nface * sizeof(double), cudaMemcpyHostToDevice, s);
  } else {
    velocity_points<<<grid_for(npts), 256, 0, s>>>(pg, kind, b[0], b[1], b[2], raw, npts);
    velocity_faces<<<grid_for(nface), 256, 0, s>>>(pg, kind, b[0], b[1], b[2], static_cast<double*>(h->bface),
                                                   nface);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    scale_velocity<<<grid_for(npts * 3), 256, 0, s>>>(pg, raw, static_cast<double*>(h->bsc), npts * 3);
    to_pairs<<<grid_for(npts * 3), 256, 0, s>>>(static_cast<const double*>(h->bsc), static_cast<dgk::dfl*>(h->bscX),
                                                npts * 3);
    to_pairs<<<grid_for(nface), 256, 0, s>>>(static_cast<const double*>(h->bface),
                                             static_cast<dgk::dfl*>(h->bfaceX), nface);
    e = cudaGetLastError();
  }
  // the temporary field is released once the kernels that read it are done
  cudaError_t es = cudaStreamSynchronize(s);
  cudaFree(raw);
  if (e != cudaSuccess) return cuda_fail(e, "dg_setup: velocity kernels");
  if (es != cudaSuccess) return cuda_fail(es, "dg_setup: velocity synchronize");
  return DG_OK;
}

}  // namespace dgi

using namespace dgi;

extern "C" {

int dg_project(dg_handle* h, const double* u_qp, double* z, void* stream) {
  if (!h || !u_qp || !z) {
    set_error("dg_project: null argument");
    return DG_ERR_INVALID_ARG;
  }
  if (h->ml) {
    set_error("dg_project: the mass matrix of multilinear cells is not |T| I");
    return DG_ERR_INVALID_ARG;
  }
  const double* none[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  return launch_rhs_f64(h, u_qp, none, z, static_cast<cudaStream_t>(stream), true);
}

static int stage(const dg_handle* h, const double* u, double* y, const StageArgs& st, int32_t precision,
                 cudaStream_t s) {
  if (h->ml) {
    set_error("Runge-Kutta stages: the mass matrix of multilinear cells is not |T| I");
    return DG_ERR_INVALID_ARG;
  }
  return precision == DG_F64X ? launch_stage_f64x(h, u, y, st, s) : launch_stage_f64(h, u, y, st, s);
}

int dg_rk_stage(dg_handle* h, const double* u, const double* z0, double* y, double cz, double cu, double cdt,
                int32_t precision, void* stream) {
  if (!h || !u || !z0 || !y) {
    set_error("dg_rk_stage: null argument");
    return DG_ERR_INVALID_ARG;
  }
  if (precision != DG_F64 && precision != DG_F64X) {
    set_error("dg_rk_stage: precision must be DG_F64 or DG_F64X");
    return DG_ERR_INVALID_ARG;
  }
  if (!std::isfinite(cz) || !std::isfinite(cu) || !std::isfinite(cdt)) {
    set_error("dg_rk_stage: coefficients must be finite");
    return DG_ERR_INVALID_ARG;
  }
  const double vol = h->detJ;  // |T|: the mass matrix is |T| I
  const StageArgs st{z0, cz, cu, cdt / vol};  // M^{-1} = I / |T|
  return stage(h, u, y, st, precision, static_cast<cudaStream_t>(stream));
}

int dg_ssprk2(dg_handle* h, double* z, double dt, int32_t nsteps, int32_t precision, void* stream) {
  if (!h || !z || nsteps < 0 || !std::isfinite(dt) || (precision != DG_F64 && precision != DG_F64X)) {
    set_error("dg_ssprk2: bad arguments (precision DG_F64 or DG_F64X, nsteps >= 0, finite dt)");
    return DG_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!h->rk_tmp) {
    const int64_t ndof = h->ncell * h->N * h->N * h->N;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMalloc(&h->rk_tmp, ndof * sizeof(double));
    if (e != cudaSuccess) return cuda_fail(e, "dg_ssprk2: stage vector");
  }
  double* z1 = static_cast<double*>(h->rk_tmp);
  const double vol = h->detJ;  // |T|: the mass matrix is |T| I
  const StageArgs st1{z, 0.0, 1.0, dt / vol};
  const StageArgs st2{z, 0.5, 0.5, 0.5 * dt / vol};
  for (int32_t i = 0; i < nsteps; ++i) {
    if (int rc = stage(h, z, z1, st1, precision, s)) return rc;   // z1 = z - dt M^{-1}(A z - F)
    if (int rc = stage(h, z1, z, st2, precision, s)) return rc;   // z = (z + z1 - dt M^{-1}(A z1 - F)) / 2
  }
  return DG_OK;
}

}  // extern "C"
