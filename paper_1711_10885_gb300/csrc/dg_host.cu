// dg_host.cu -- C ABI entry points: setup (1D tables, coefficients, right hand side), apply, teardown.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <new>
#include <string>
#include <vector>

#include "dg_dfloat.cuh"
#include "dg_internal.h"

namespace dgi {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

int cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA;
}

int sm_count() {
  static std::atomic<int> cache[64];  // 0 = not queried yet
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  const bool cached = dev >= 0 && dev < 64;
  if (cached) {
    const int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
  if (cached) cache[dev].store(sms, std::memory_order_relaxed);
  return sms;
}

// P_j(2x-1) and its x-derivative for j = 0..jmax (three-term recurrence, differentiated term by term)
static void shifted_legendre(int jmax, double x, double* p, double* dp) {
  const double t = 2.0 * x - 1.0;
  p[0] = 1.0;
  dp[0] = 0.0;
  if (jmax >= 1) {
    p[1] = t;
    dp[1] = 2.0;
  }
  for (int j = 1; j < jmax; ++j) {
    p[j + 1] = ((2 * j + 1) * t * p[j] - j * p[j - 1]) / (j + 1);
    dp[j + 1] = ((2 * j + 1) * (2.0 * p[j] + t * dp[j]) - j * dp[j - 1]) / (j + 1);
  }
}

// Gauss-Legendre nodes/weights on [0,1] with M points (Sec. 3.1) and the 1D matrices of the kernels for
// N = k+1 modes.
void build_tables(int N, int M, Tables1D* tb) {
  tb->N = N;
  tb->M = M;
  double p[MAXM + 2], dp[MAXM + 2];
  // Newton on P_M(2x-1) for the lower half of the nodes; the rule is symmetric about 1/2, and the
  // kernels rely on that symmetry exactly (even-odd form), so the upper half is mirrored
  for (int i = 0; i < (M + 1) / 2; ++i) {
    double x = 0.5 * (1.0 - std::cos(M_PI * (i + 0.75) / (M + 0.5)));
    if (2 * i + 1 == M) {
      x = 0.5;
    } else {
      for (int it = 0; it < 60; ++it) {
        shifted_legendre(M, x, p, dp);
        const double dx = p[M] / dp[M];
        x -= dx;
        if (std::fabs(dx) < 1e-16) break;
      }
    }
    shifted_legendre(M, x, p, dp);
    tb->xi[i] = x;
    tb->w[i] = 1.0 / (x * (1.0 - x) * dp[M] * dp[M]);
    tb->xi[M - 1 - i] = 1.0 - x;
    tb->w[M - 1 - i] = tb->w[i];
  }
  // theta_j(x) = sqrt(2j+1) P_j(2x-1), j < M: values / derivatives at the nodes and at the end points
  double th[MAXM][MAXM], dth[MAXM][MAXM], te[2][MAXM], dte[2][MAXM];
  for (int i = 0; i < M; ++i) {
    shifted_legendre(M - 1, tb->xi[i], p, dp);
    for (int j = 0; j < M; ++j) {
      th[i][j] = std::sqrt(2.0 * j + 1.0) * p[j];
      dth[i][j] = std::sqrt(2.0 * j + 1.0) * dp[j];
    }
  }
  for (int s = 0; s < 2; ++s) {
    shifted_legendre(M - 1, (double)s, p, dp);
    for (int j = 0; j < M; ++j) {
      te[s][j] = std::sqrt(2.0 * j + 1.0) * p[j];
      dte[s][j] = std::sqrt(2.0 * j + 1.0) * dp[j];
    }
  }
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < N; ++j) tb->A[i][j] = th[i][j];
  // Lagrange basis on the M Gauss points through the orthonormal expansion
  //   l_l(x) = sum_{j<M} theta_j(x) theta_j(xi_l) w_l   (exact: the M-point rule integrates degree 2M-1)
  for (int l = 0; l < M; ++l) {
    for (int i = 0; i < M; ++i) {
      double acc = 0.0;
      for (int j = 0; j < M; ++j) acc += dth[i][j] * th[l][j];
      tb->Dt[i][l] = acc * tb->w[l];
    }
    for (int s = 0; s < 2; ++s) {
      double av = 0.0, ad = 0.0;
      for (int j = 0; j < M; ++j) {
        av += te[s][j] * th[l][j];
        ad += dte[s][j] * th[l][j];
      }
      tb->L[s][l] = av * tb->w[l];
      tb->P[s][l] = ad * tb->w[l];
    }
  }
}

__global__ void cast_f64_to_f32(const double* __restrict__ a, float* __restrict__ b, dgk::dfl* __restrict__ x,
                                int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    b[i] = (float)a[i];
    x[i] = dgk::dfl_from_double(a[i]);
  }
}

static int cast_launch(const double* a, float* b, dgk::dfl* x, int64_t n, cudaStream_t s) {
  const int64_t blocks64 = (n + 255) / 256;
  const int64_t cap = (int64_t)sm_count() * 32;
  const unsigned blocks = (unsigned)(blocks64 > cap ? cap : (blocks64 > 0 ? blocks64 : 1));
  cast_f64_to_f32<<<blocks, 256, 0, s>>>(a, b, x, n);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : cuda_fail(e, "cast kernel");
}

static bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

static void free_buffers(Buffers& b) {
  cudaFree(b.D);
  cudaFree(b.fc);
  cudaFree(b.F);
  b = Buffers();
}

}  // namespace dgi

using namespace dgi;

extern "C" {

const char* dg_last_error(void) { return g_err.c_str(); }

double dg_penalty_sigma(int32_t k, int32_t mode) {
  if (mode == 1) return 2.0 * k * (k + 2);  // alpha p (p + d - 1), alpha = 2, d = 3
  return 2.0 * k * (k + 1);
}

int dg_destroy(dg_handle* h) {
  if (!h) return DG_OK;
  free_buffers(h->p64);
  free_buffers(h->p32);
  free_buffers(h->pX);
  cudaFree(h->work_V);
  cudaFree(h->work_tr);
  cudaFree(h->bj64);
  cudaFree(h->bj32);
  cudaFree(h->bj16);
  cudaFree(h->bj16s);
  for (void* q : {h->fdm.re32, h->fdm.re64, h->fdm.cx32, h->fdm.cx64, (void*)h->fdm.re_cells, (void*)h->fdm.cx_cells,
                  (void*)h->fdm.red32, (void*)h->fdm.black32})
    cudaFree(q);
  cudaFree(h->bsc);
  cudaFree(h->bface);
  cudaFree(h->bscX);
  cudaFree(h->bfaceX);
  cudaFree(h->kq64);
  cudaFree(h->kqX);
  cudaFree(h->kf64);
  cudaFree(h->kfX);
  delete[] h->verts;
  cudaFree(h->rk_tmp);
  cudaFree(h->ws);
  if (h->ws_host) cudaFreeHost(h->ws_host);
  delete h;
  return DG_OK;
}

int dg_sizes(const dg_handle* h, int64_t* ncells, int32_t* dofs_per_cell, int64_t* ndofs) {
  if (!h) {
    set_error("dg_sizes: null handle");
    return DG_ERR_INVALID_ARG;
  }
  if (ncells) *ncells = h->ncell;
  if (dofs_per_cell) *dofs_per_cell = h->N * h->N * h->N;
  if (ndofs) *ndofs = h->ncell * h->N * h->N * h->N;
  return DG_OK;
}

int dg_setup(const dg_mesh* mesh, int32_t k, const dg_coeffs* co, const dg_bc* bc, const double* f_qp,
             void* stream, dg_handle** out) {
  return dg_setup_ex(mesh, k, co, bc, f_qp, nullptr, stream, out);
}

int dg_setup_ex(const dg_mesh* mesh, int32_t k, const dg_coeffs* co, const dg_bc* bc, const double* f_qp,
                const dg_setup_ext* ext, void* stream, dg_handle** out) {
  if (!out) {
    set_error("dg_setup: out is null");
    return DG_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (!mesh || !co) {
    set_error("dg_setup: mesh and coefficients are required");
    return DG_ERR_INVALID_ARG;
  }
  if (k < 1 || k > DG_MAX_DEGREE) {
    set_error("dg_setup: degree k must be in [1, " + std::to_string(DG_MAX_DEGREE) + "]");
    return DG_ERR_INVALID_ARG;
  }
  int64_t ncell = 1;
  for (int r = 0; r < 3; ++r) {
    if (mesh->n[r] < 1 || !std::isfinite(mesh->lo[r]) || !std::isfinite(mesh->hi[r]) ||
        !(mesh->hi[r] > mesh->lo[r])) {
      set_error("dg_setup: each axis needs n >= 1 and finite lo < hi");
      return DG_ERR_INVALID_ARG;
    }
    if (ncell > ((int64_t)1 << 30) / mesh->n[r]) {
      set_error("dg_setup: too many cells");
      return DG_ERR_INVALID_ARG;
    }
    ncell *= mesh->n[r];
  }
  if (ncell > (int64_t)1 << 30) {
    set_error("dg_setup: too many cells");
    return DG_ERR_INVALID_ARG;
  }
  for (int r = 0; r < 3; ++r)
    if (!std::isfinite(co->b[r])) {
      set_error("dg_setup: velocity must be finite");
      return DG_ERR_INVALID_ARG;
    }
  if (!std::isfinite(co->c) || !std::isfinite(co->sigma) || co->sigma < 0) {
    set_error("dg_setup: c must be finite and sigma finite and >= 0");
    return DG_ERR_INVALID_ARG;
  }
  const int M = (ext && ext->m) ? ext->m : k + 1;
  const int velocity = ext ? ext->velocity : DG_VELOCITY_CONSTANT;
  if (M != k + 1 && M != k + 3) {
    set_error("dg_setup: m must be k+1 or k+3 Gauss points per direction");
    return DG_ERR_INVALID_ARG;
  }
  if (velocity != DG_VELOCITY_CONSTANT && velocity != DG_VELOCITY_POINTS && velocity != DG_VELOCITY_TAYLOR_GREEN) {
    set_error("dg_setup: unknown velocity kind");
    return DG_ERR_INVALID_ARG;
  }
  if (velocity == DG_VELOCITY_POINTS && (!ext->b_qp || !ext->b_face)) {
    set_error("dg_setup: DG_VELOCITY_POINTS needs b_qp and b_face");
    return DG_ERR_INVALID_ARG;
  }
  const bool vb = velocity != DG_VELOCITY_CONSTANT || M != k + 1;
  if (vb && k > 8) {
    set_error("dg_setup: a velocity field or m = k+3 needs degree k <= 8");
    return DG_ERR_INVALID_ARG;
  }
  const bool ml = ext && ext->vertices;
  const bool pw_given = ext && (ext->D_qp || ext->D_face);
  if (pw_given && (!ext->D_qp || !ext->D_face)) {
    set_error("dg_setup: point-wise coefficients need both D_qp and D_face");
    return DG_ERR_INVALID_ARG;
  }
  const bool pw = pw_given || ml;
  if (pw && (k > 8 || velocity == DG_VELOCITY_TAYLOR_GREEN)) {
    set_error("dg_setup: point-wise coefficients and multilinear cells need degree k <= 8 and a constant or "
              "point-wise velocity");
    return DG_ERR_INVALID_ARG;
  }
  if (ml && (ext->jacobian || ext->periodic[0] || ext->periodic[1] || ext->periodic[2])) {
    set_error("dg_setup: multilinear cells (vertices) exclude an affine jacobian and periodic axes");
    return DG_ERR_INVALID_ARG;
  }
  if (ml) {
    const int64_t nv = (int64_t)(mesh->n[0] + 1) * (mesh->n[1] + 1) * (mesh->n[2] + 1);
    for (int64_t i = 0; i < 3 * nv; ++i)
      if (!std::isfinite(ext->vertices[i])) {
        set_error("dg_setup: vertices must be finite");
        return DG_ERR_INVALID_ARG;
      }
  }
  if (!pw && ext && ext->c_qp) {
    set_error("dg_setup: c_qp needs the point-wise coefficients D_qp and D_face");
    return DG_ERR_INVALID_ARG;
  }
  const bool td = ext && (ext->D_tensor || ext->jacobian || pw);
  if (td && !pw && (vb || k > 8)) {
    set_error("dg_setup: a diffusion tensor or an affine geometry needs a constant velocity, m = k+1 and k <= 8");
    return DG_ERR_INVALID_ARG;
  }
  double Jm[3][3];
  if (td && ext->jacobian) {
    for (int a = 0; a < 3; ++a)
      for (int r = 0; r < 3; ++r) {
        Jm[a][r] = ext->jacobian[3 * a + r];
        if (!std::isfinite(Jm[a][r])) {
          set_error("dg_setup: the Jacobian must be finite");
          return DG_ERR_INVALID_ARG;
        }
      }
  }
  int bc_type[6] = {0, 0, 0, 0, 0, 0};
  for (int f = 0; f < 6; ++f) {
    bc_type[f] = ext ? ext->bc_type[f] : DG_BC_DIRICHLET;
    if (bc_type[f] != DG_BC_DIRICHLET && bc_type[f] != DG_BC_NEUMANN && bc_type[f] != DG_BC_OUTFLOW) {
      set_error("dg_setup: bc_type must be DG_BC_DIRICHLET, DG_BC_NEUMANN or DG_BC_OUTFLOW");
      return DG_ERR_INVALID_ARG;
    }
  }
  int periodic[3] = {0, 0, 0};
  for (int r = 0; r < 3; ++r) {
    if (ext && ext->periodic[r] != 0 && ext->periodic[r] != 1) {
      set_error("dg_setup: periodic flags must be 0 or 1");
      return DG_ERR_INVALID_ARG;
    }
    periodic[r] = ext ? ext->periodic[r] : 0;
  }
  std::vector<double> D(ncell);
  const bool tensor_given = td && ext->D_tensor && !pw_given;
  for (int64_t i = 0; i < ncell; ++i) {
    if (pw_given) {
      D[i] = 1.0;  // unused: the point tables carry the coefficients
      continue;
    }
    if (tensor_given) {
      // symmetric positive definite: positive leading principal minors (Sylvester's criterion)
      const double* t = ext->D_tensor + 6 * i;
      bool ok = true;
      for (int q = 0; q < 6; ++q) ok = ok && std::isfinite(t[q]);
      const double m2 = t[0] * t[1] - t[3] * t[3];
      const double m3 = t[0] * (t[1] * t[2] - t[5] * t[5]) - t[3] * (t[3] * t[2] - t[5] * t[4]) +
                        t[4] * (t[3] * t[5] - t[1] * t[4]);
      if (!ok || !(t[0] > 0) || !(m2 > 0) || !(m3 > 0)) {
        set_error("dg_setup: every D_T must be symmetric positive definite (cell " + std::to_string(i) + ")");
        return DG_ERR_INVALID_ARG;
      }
      D[i] = t[0];
      continue;
    }
    D[i] = co->D_cell ? co->D_cell[i] : co->D_const;
    if (!finite_pos(D[i])) {
      set_error("dg_setup: every D_T must be finite and > 0 (cell " + std::to_string(i) + ")");
      return DG_ERR_INVALID_ARG;
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  dg_handle* h = new (std::nothrow) dg_handle();
  if (!h) {
    set_error("dg_setup: host allocation failed");
    return DG_ERR_OOM;
  }
  cudaGetDevice(&h->device);
  h->k = k;
  h->N = k + 1;
  h->ncell = ncell;
  for (int r = 0; r < 3; ++r) {
    h->n[r] = mesh->n[r];
    h->lo[r] = mesh->lo[r];
    h->hi[r] = mesh->hi[r];
    h->h[r] = (mesh->hi[r] - mesh->lo[r]) / mesh->n[r];
    h->b[r] = co->b[r];
  }
  h->c = co->c;
  h->sigma = co->sigma;
  h->M = M;
  h->vb = vb;
  h->td = td;
  h->pw = pw;
  h->ml = ml;
  h->affine = td && ext->jacobian;
  if (ml) {
    const size_t nv = (size_t)(h->n[0] + 1) * (h->n[1] + 1) * (h->n[2] + 1) * 3;
    h->verts = new (std::nothrow) double[nv];
    if (!h->verts) {
      delete h;
      set_error("dg_setup: host allocation failed");
      return DG_ERR_OOM;
    }
    std::memcpy(h->verts, ext->vertices, nv * sizeof(double));
  }
  for (int r = 0; r < 3; ++r) h->periodic[r] = periodic[r];
  for (int f = 0; f < 6; ++f) h->bc_type[f] = periodic[f / 2] ? DG_BC_DIRICHLET : bc_type[f];
  // cell Jacobian: the affine map, or diag(h) for the axis-parallel grid
  for (int a = 0; a < 3; ++a)
    for (int r = 0; r < 3; ++r) h->J[a][r] = h->affine ? Jm[a][r] : (a == r ? h->h[r] : 0.0);
  {
    const double(*J)[3] = h->J;
    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    if (!(std::fabs(det) > 0) || !std::isfinite(det)) {
      delete h;
      set_error("dg_setup: the Jacobian must be invertible");
      return DG_ERR_INVALID_ARG;
    }
    h->Jinv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
    h->Jinv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    h->Jinv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    h->Jinv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
    h->Jinv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    h->Jinv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    h->Jinv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
    h->Jinv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    h->Jinv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    h->detJ = std::fabs(det);
    for (int r = 0; r < 3; ++r)
      h->fscale[r] = std::sqrt(h->Jinv[r][0] * h->Jinv[r][0] + h->Jinv[r][1] * h->Jinv[r][1] +
                               h->Jinv[r][2] * h->Jinv[r][2]);
  }
  build_tables(h->N, M, &h->tab);

  const int N = h->N;
  const int64_t nb = (int64_t)N * N * N;
  const int64_t ndof = ncell * nb;
  const int64_t npts = ncell * M * M * M;  // volume quadrature points
  // face coefficients per cell and face (Sec. 2: weights w+- = delta-+/(delta- + delta+), gamma_F)
  std::vector<double> fc(ncell * 18);
  for (int64_t cell = 0; cell < ncell; ++cell) {
    int ic[3] = {(int)(cell % h->n[0]), (int)((cell / h->n[0]) % h->n[1]), (int)(cell / ((int64_t)h->n[0] * h->n[1]))};
    const int64_t strides[3] = {1, h->n[0], (int64_t)h->n[0] * h->n[1]};
    for (int dir = 0; dir < 3; ++dir)
      for (int side = 0; side < 2; ++side) {
        double* c3 = &fc[(cell * 6 + 2 * dir + side) * 3];
        const double hq = h->h[dir];
        const double Do = D[cell];
        const bool at_end = side ? ic[dir] == h->n[dir] - 1 : ic[dir] == 0;
        const bool boundary = at_end && !h->periodic[dir];
        if (boundary) {
          // Dirichlet: (D_own / h, upwind factor 1, delta- sigma |F| / |T-|); outflow: upwind flux only;
          // Neumann: no term in a_h
          const int bt = h->bc_type[2 * dir + side];
          c3[0] = bt == DG_BC_DIRICHLET ? Do / hq : 0.0;
          c3[1] = bt == DG_BC_NEUMANN ? 0.0 : 1.0;
          c3[2] = bt == DG_BC_DIRICHLET ? Do * h->sigma / hq : 0.0;
        } else {
          // the neighbour; across the end faces of a periodic axis it is the cell at the other end
          const int64_t wrap = (int64_t)(h->n[dir] - 1) * strides[dir];
          const int64_t nbr = side ? (at_end ? cell - wrap : cell + strides[dir])
                                   : (at_end ? cell + wrap : cell - strides[dir]);
          const double Dn = D[nbr];
          const double sum = Do + Dn;
          c3[0] = (Dn / sum) * Do / hq;  // w_own D_own / h
          c3[1] = (Do / sum) * Dn / hq;  // w_nbr D_nbr / h
          c3[2] = (2.0 * Do * Dn / sum) * h->sigma / hq;
        }
      }
  }
  if (td) {
    // K = |det J| J^{-1} D_T J^{-T} per cell (D_T the tensor, or D_T I), and per face (w_own, w_nbr, gamma,
    // kn, kt1, kt2): delta = nu^T D nu is proportional to K_rr on every cell (one Jacobian), so the weights
    // are w_own = K_nbr,rr / (K_own,rr + K_nbr,rr); gamma = <delta-, delta+> sigma |F| / |T| with
    // delta = K_rr / (|det J| |J^{-T} e_r|^2) and |F| / |T| = |J^{-T} e_r|; kn, kt = w_own K_r. / |F_r|
    std::vector<double> K(ncell * 6);
    for (int64_t cell = 0; cell < ncell; ++cell) {
      double Dt[3][3];
      if (tensor_given) {
        const double* t = ext->D_tensor + 6 * cell;
        Dt[0][0] = t[0], Dt[1][1] = t[1], Dt[2][2] = t[2];
        Dt[0][1] = Dt[1][0] = t[3];
        Dt[0][2] = Dt[2][0] = t[4];
        Dt[1][2] = Dt[2][1] = t[5];
      } else {
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) Dt[a][b] = a == b ? D[cell] : 0.0;
      }
      double Km[3][3];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          double acc = 0.0;
          for (int p = 0; p < 3; ++p)
            for (int q = 0; q < 3; ++q) acc += h->Jinv[a][p] * Dt[p][q] * h->Jinv[b][q];
          Km[a][b] = h->detJ * acc;
        }
      double* k6 = &K[cell * 6];
      k6[0] = Km[0][0], k6[1] = Km[1][1], k6[2] = Km[2][2], k6[3] = Km[0][1], k6[4] = Km[0][2], k6[5] = Km[1][2];
    }
    auto Kat = [&](int64_t cell, int a, int b) {
      const double* k6 = &K[cell * 6];
      if (a == b) return k6[a];
      const int lo_ = a < b ? a : b, hi_ = a < b ? b : a;
      return lo_ == 0 ? (hi_ == 1 ? k6[3] : k6[4]) : k6[5];
    };
    fc.assign(ncell * 36, 0.0);
    for (int64_t cell = 0; cell < ncell; ++cell) {
      int ic[3] = {(int)(cell % h->n[0]), (int)((cell / h->n[0]) % h->n[1]),
                   (int)(cell / ((int64_t)h->n[0] * h->n[1]))};
      const int64_t strides[3] = {1, h->n[0], (int64_t)h->n[0] * h->n[1]};
      for (int dir = 0; dir < 3; ++dir)
        for (int side = 0; side < 2; ++side) {
          double* c6 = &fc[(cell * 6 + 2 * dir + side) * 6];
          const int ta = dir == 0 ? 1 : 0, tb = dir == 2 ? 1 : 2;
          const double area = h->detJ * h->fscale[dir];
          const double dscale = 1.0 / (h->detJ * h->fscale[dir] * h->fscale[dir]);  // delta = K_rr * dscale
          const double ko = Kat(cell, dir, dir);
          const bool at_end = side ? ic[dir] == h->n[dir] - 1 : ic[dir] == 0;
          const bool boundary = at_end && !h->periodic[dir];
          double wo = 1.0, wn = 0.0, gam;
          if (boundary) {
            gam = ko * dscale * h->sigma * h->fscale[dir];
          } else {
            const int64_t wrap = (int64_t)(h->n[dir] - 1) * strides[dir];
            const int64_t nbr = side ? (at_end ? cell - wrap : cell + strides[dir])
                                     : (at_end ? cell + wrap : cell - strides[dir]);
            const double kn_ = Kat(nbr, dir, dir);
            wo = kn_ / (ko + kn_);
            wn = ko / (ko + kn_);
            gam = (2.0 * ko * kn_ / (ko + kn_)) * dscale * h->sigma * h->fscale[dir];
          }
          c6[0] = wo;
          c6[1] = wn;
          c6[2] = gam;
          c6[3] = wo * ko / area;
          c6[4] = wo * Kat(cell, dir, ta) / area;
          c6[5] = wo * Kat(cell, dir, tb) / area;
          if (boundary) {
            // the second coefficient multiplies the upwind flux on a boundary face; outflow and Neumann faces
            // have no diffusion or penalty term
            const int bt = h->bc_type[2 * dir + side];
            c6[1] = bt == DG_BC_NEUMANN ? 0.0 : 1.0;
            if (bt != DG_BC_DIRICHLET) c6[0] = c6[2] = c6[3] = c6[4] = c6[5] = 0.0;
          }
        }
    }
    D.swap(K);
  }
  std::vector<double> kq, kf, bface_pw;
  if (pw) {
    // multilinear cells with per-cell coefficients: repeat each cell's tensor at its points
    std::vector<double> Dq, Df;
    const double* Dqp = pw_given ? ext->D_qp : nullptr;
    const double* Dfp = pw_given ? ext->D_face : nullptr;
    if (!pw_given) {
      const int64_t M3 = (int64_t)M * M * M, MM = (int64_t)M * M;
      Dq.resize((size_t)ncell * M3 * 6);
      Df.resize((size_t)ncell * 6 * MM * 6);
      for (int64_t cell = 0; cell < ncell; ++cell) {
        double t6[6];
        if (tensor_given) {
          for (int q = 0; q < 6; ++q) t6[q] = ext->D_tensor[6 * cell + q];
        } else {
          // (D itself holds the per-cell metric by now)
          t6[0] = t6[1] = t6[2] = co->D_cell ? co->D_cell[cell] : co->D_const;
          t6[3] = t6[4] = t6[5] = 0.0;
        }
        for (int64_t q = 0; q < M3; ++q) std::memcpy(&Dq[(cell * M3 + q) * 6], t6, sizeof(t6));
        for (int64_t q = 0; q < 6 * MM; ++q) std::memcpy(&Df[(cell * 6 * MM + q) * 6], t6, sizeof(t6));
      }
      Dqp = Dq.data();
      Dfp = Df.data();
    }
    const int prc = build_pointwise_tables(h, Dqp, Dfp, ext->c_qp, co->c, co->b,
                                           velocity == DG_VELOCITY_POINTS ? ext->b_qp : nullptr,
                                           velocity == DG_VELOCITY_POINTS ? ext->b_face : nullptr, kq, kf, fc,
                                           bface_pw);
    if (prc != DG_OK) {
      dg_destroy(h);
      return prc;
    }
  }
  std::vector<float> D32(D.begin(), D.end()), fc32(fc.begin(), fc.end());
  std::vector<dgk::dfl> DX(D.size()), fcX(fc.size());
  for (size_t i = 0; i < D.size(); ++i) DX[i] = dgk::dfl(D[i]);
  for (size_t i = 0; i < fc.size(); ++i) fcX[i] = dgk::dfl(fc[i]);

  int rc = DG_OK;
  cudaError_t e = cudaSuccess;
  double* gdev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
#define DG_TRY(call, what)            \
  do {                                \
    e = (call);                       \
    if (e != cudaSuccess) {           \
      rc = cuda_fail(e, what);        \
      goto fail;                      \
    }                                 \
  } while (0)
  {
    const size_t nD = D.size(), nfc = fc.size();  // per cell 1 and 18 values, or 6 and 36 (td)
    DG_TRY(cudaMalloc(&h->p64.D, nD * sizeof(double)), "cudaMalloc(D)");
    DG_TRY(cudaMalloc(&h->p32.D, nD * sizeof(float)), "cudaMalloc(D32)");
    DG_TRY(cudaMalloc(&h->p64.fc, nfc * sizeof(double)), "cudaMalloc(fc)");
    DG_TRY(cudaMalloc(&h->p32.fc, nfc * sizeof(float)), "cudaMalloc(fc32)");
    DG_TRY(cudaMalloc(&h->pX.D, nD * sizeof(dgk::dfl)), "cudaMalloc(D pairs)");
    DG_TRY(cudaMalloc(&h->pX.fc, nfc * sizeof(dgk::dfl)), "cudaMalloc(fc pairs)");
    DG_TRY(cudaMalloc(&h->p64.F, ndof * sizeof(double)), "cudaMalloc(F)");
    DG_TRY(cudaMalloc(&h->p32.F, ndof * sizeof(float)), "cudaMalloc(F32)");
    DG_TRY(cudaMalloc(&h->pX.F, ndof * sizeof(dgk::dfl)), "cudaMalloc(F pairs)");
    DG_TRY(cudaMalloc(&h->work_V, npts * sizeof(double)), "cudaMalloc(work V)");
    DG_TRY(cudaMalloc(&h->work_tr, ncell * 12 * M * M * sizeof(double)), "cudaMalloc(work traces)");
    DG_TRY(cudaMemcpyAsync(h->p64.D, D.data(), nD * sizeof(double), cudaMemcpyHostToDevice, s), "copy D");
    DG_TRY(cudaMemcpyAsync(h->p32.D, D32.data(), nD * sizeof(float), cudaMemcpyHostToDevice, s), "copy D32");
    DG_TRY(cudaMemcpyAsync(h->p64.fc, fc.data(), nfc * sizeof(double), cudaMemcpyHostToDevice, s), "copy fc");
    DG_TRY(cudaMemcpyAsync(h->p32.fc, fc32.data(), nfc * sizeof(float), cudaMemcpyHostToDevice, s), "copy fc32");
    DG_TRY(cudaMemcpyAsync(h->pX.D, DX.data(), nD * sizeof(dgk::dfl), cudaMemcpyHostToDevice, s), "copy D pairs");
    DG_TRY(cudaMemcpyAsync(h->pX.fc, fcX.data(), nfc * sizeof(dgk::dfl), cudaMemcpyHostToDevice, s),
           "copy fc pairs");
    if (pw) {
      // point tables, FP64 and double-float (the face coefficients went with fc above)
      const int64_t nkq = (int64_t)kq.size(), nkf = (int64_t)kf.size(), nbf = (int64_t)bface_pw.size();
      DG_TRY(cudaMalloc(&h->kq64, nkq * sizeof(double)), "cudaMalloc(point table)");
      DG_TRY(cudaMalloc(&h->kqX, nkq * sizeof(dgk::dfl)), "cudaMalloc(point table pairs)");
      DG_TRY(cudaMalloc(&h->kf64, nkf * sizeof(double)), "cudaMalloc(face metric)");
      DG_TRY(cudaMalloc(&h->kfX, nkf * sizeof(dgk::dfl)), "cudaMalloc(face metric pairs)");
      DG_TRY(cudaMalloc(&h->bface, nbf * sizeof(double)), "cudaMalloc(normal velocity)");
      DG_TRY(cudaMalloc(&h->bfaceX, nbf * sizeof(dgk::dfl)), "cudaMalloc(normal velocity pairs)");
      DG_TRY(cudaMemcpyAsync(h->kq64, kq.data(), nkq * sizeof(double), cudaMemcpyHostToDevice, s), "copy kq");
      DG_TRY(cudaMemcpyAsync(h->kf64, kf.data(), nkf * sizeof(double), cudaMemcpyHostToDevice, s), "copy kf");
      DG_TRY(cudaMemcpyAsync(h->bface, bface_pw.data(), nbf * sizeof(double), cudaMemcpyHostToDevice, s),
             "copy bface");
      if ((rc = copy_to_pairs(static_cast<const double*>(h->kq64), h->kqX, nkq, s)) != DG_OK) goto fail;
      if ((rc = copy_to_pairs(static_cast<const double*>(h->kf64), h->kfX, nkf, s)) != DG_OK) goto fail;
      if ((rc = copy_to_pairs(static_cast<const double*>(h->bface), h->bfaceX, nbf, s)) != DG_OK) goto fail;
      // the host tables must outlive the asynchronous copies
      DG_TRY(cudaStreamSynchronize(s), "dg_setup synchronize");
    }
    // velocity field tables (before the right hand side, whose inflow terms read b . nu)
    if (vb && !pw) {
      rc = setup_velocity(h, velocity, co->b, ext ? ext->b_qp : nullptr, ext ? ext->b_face : nullptr, s);
      if (rc != DG_OK) goto fail;
    }
    // right hand side: f at the volume points goes through the work buffer (on multilinear cells times the
    // volume element |det J| of each point: the kernels then see |T| = 1)
    if (f_qp && ml) {
      std::vector<double> fs(f_qp, f_qp + npts);
      const int64_t M3 = (int64_t)M * M * M;
      for (int64_t e = 0; e < npts; ++e) {
        const int q = (int)(e % M3);
        const double xi[3] = {h->tab.xi[q % M], h->tab.xi[(q / M) % M], h->tab.xi[q / (M * M)]};
        MapGeo g;
        if ((rc = point_geometry(h, e / M3, xi, &g)) != DG_OK) goto fail;
        fs[e] *= g.det;
      }
      DG_TRY(cudaMemcpyAsync(h->work_V, fs.data(), npts * sizeof(double), cudaMemcpyHostToDevice, s), "copy f");
      DG_TRY(cudaStreamSynchronize(s), "dg_setup synchronize");
    } else if (f_qp) {
      DG_TRY(cudaMemcpyAsync(h->work_V, f_qp, npts * sizeof(double), cudaMemcpyHostToDevice, s), "copy f");
    } else {
      DG_TRY(cudaMemsetAsync(h->work_V, 0, npts * sizeof(double), s), "memset f");
    }
    int64_t gsize[6];
    for (int sd = 0; sd < 6; ++sd) {
      const int dir = sd / 2, ta = dir == 0 ? 1 : 0, tb = dir == 2 ? 1 : 2;
      gsize[sd] = (int64_t)h->n[ta] * h->n[tb] * M * M;
      if (bc && bc->g_qp[sd] && !h->periodic[dir]) {
        DG_TRY(cudaMalloc(&gdev[sd], gsize[sd] * sizeof(double)), "cudaMalloc(g)");
        if (ml && h->bc_type[sd] == DG_BC_NEUMANN) {
          // Neumann flux times the face's area element (the kernels see a unit face measure)
          std::vector<double> js(bc->g_qp[sd], bc->g_qp[sd] + gsize[sd]);
          const int MM = M * M;
          for (int64_t e = 0; e < gsize[sd]; ++e) {
            const int64_t fidx = e / MM;
            const int p = (int)(e % MM);
            int ic3[3];
            ic3[dir] = (sd % 2) ? h->n[dir] - 1 : 0;
            ic3[ta] = (int)(fidx % h->n[ta]);
            ic3[tb] = (int)(fidx / h->n[ta]);
            const int64_t cell = ic3[0] + (int64_t)h->n[0] * (ic3[1] + (int64_t)h->n[1] * ic3[2]);
            double xi[3], nu[3];
            face_xi(h, sd, p, xi);
            MapGeo g;
            if ((rc = point_geometry(h, cell, xi, &g)) != DG_OK) goto fail;
            js[e] *= face_frame(g, dir, nu);
          }
          DG_TRY(cudaMemcpyAsync(gdev[sd], js.data(), gsize[sd] * sizeof(double), cudaMemcpyHostToDevice, s),
                 "copy j");
          DG_TRY(cudaStreamSynchronize(s), "dg_setup synchronize");
        } else {
          DG_TRY(cudaMemcpyAsync(gdev[sd], bc->g_qp[sd], gsize[sd] * sizeof(double), cudaMemcpyHostToDevice, s),
                 "copy g");
        }
      }
    }
    rc = launch_rhs_f64(h, static_cast<const double*>(h->work_V), gdev, static_cast<double*>(h->p64.F), s);
    if (rc == DG_OK)
      rc = cast_launch(static_cast<const double*>(h->p64.F), static_cast<float*>(h->p32.F),
                       static_cast<dgk::dfl*>(h->pX.F), ndof, s);
    e = cudaStreamSynchronize(s);
    for (int sd = 0; sd < 6; ++sd) {
      cudaFree(gdev[sd]);
      gdev[sd] = nullptr;
    }
    if (rc != DG_OK) goto fail;
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "dg_setup synchronize");
      goto fail;
    }
  }
#undef DG_TRY
  *out = h;
  return DG_OK;
fail:
  cudaStreamSynchronize(s);
  for (int sd = 0; sd < 6; ++sd) cudaFree(gdev[sd]);
  dg_destroy(h);
  return rc;
}

int dg_quadrature_points(const dg_handle* h, int32_t which, double* xyz) {
  if (!h || !xyz || which < 0 || which > 7) {
    set_error("dg_quadrature_points: bad arguments");
    return DG_ERR_INVALID_ARG;
  }
  const int N = h->M;  // points per direction
  const double* x = h->tab.xi;
  // x = lo + J xi for a point xi of the structured reference grid (J = diag(h) without an affine map); on
  // multilinear cells the trilinear map of the cell that holds xi (a point on a face between two cells is
  // mapped by the upper one; both maps give the same point)
  auto map = [&](const double xi[3], double* out) {
    if (h->ml) {
      int ic[3];
      double t[3];
      for (int r = 0; r < 3; ++r) {
        ic[r] = (int)std::floor(xi[r]);
        if (ic[r] > h->n[r] - 1) ic[r] = h->n[r] - 1;
        if (ic[r] < 0) ic[r] = 0;
        t[r] = xi[r] - ic[r];
      }
      for (int a = 0; a < 3; ++a) out[a] = 0.0;
      for (int c = 0; c < 2; ++c)
        for (int b = 0; b < 2; ++b)
          for (int a = 0; a < 2; ++a) {
            const double Nw = (a ? t[0] : 1.0 - t[0]) * (b ? t[1] : 1.0 - t[1]) * (c ? t[2] : 1.0 - t[2]);
            const int64_t v =
                (ic[0] + a) + (int64_t)(h->n[0] + 1) * ((ic[1] + b) + (int64_t)(h->n[1] + 1) * (ic[2] + c));
            for (int r = 0; r < 3; ++r) out[r] += Nw * h->verts[3 * v + r];
          }
      return;
    }
    for (int a = 0; a < 3; ++a)
      out[a] = h->affine ? h->lo[a] + h->J[a][0] * xi[0] + h->J[a][1] * xi[1] + h->J[a][2] * xi[2]
                         : h->lo[a] + h->h[a] * xi[a];
  };
  size_t o = 0;
  if (which == 0) {
    for (int iz = 0; iz < h->n[2]; ++iz)
      for (int iy = 0; iy < h->n[1]; ++iy)
        for (int ix = 0; ix < h->n[0]; ++ix)
          for (int i3 = 0; i3 < N; ++i3)
            for (int i2 = 0; i2 < N; ++i2)
              for (int i1 = 0; i1 < N; ++i1) {
                const double xi[3] = {ix + x[i1], iy + x[i2], iz + x[i3]};
                map(xi, xyz + o);
                o += 3;
              }
    return DG_OK;
  }
  if (which == 7) {
    // every face of every cell: face 2*dir+side at xi_dir = ic_dir + side, points (pa, pb) tangential
    for (int64_t cell = 0; cell < h->ncell; ++cell) {
      const int ic[3] = {(int)(cell % h->n[0]), (int)((cell / h->n[0]) % h->n[1]),
                         (int)(cell / ((int64_t)h->n[0] * h->n[1]))};
      for (int face = 0; face < 6; ++face) {
        const int dir = face / 2, side = face % 2, ta = dir == 0 ? 1 : 0, tb = dir == 2 ? 1 : 2;
        for (int pb = 0; pb < N; ++pb)
          for (int pa = 0; pa < N; ++pa) {
            double xi[3];
            xi[dir] = ic[dir] + side;
            xi[ta] = ic[ta] + x[pa];
            xi[tb] = ic[tb] + x[pb];
            map(xi, xyz + o);
            o += 3;
          }
      }
    }
    return DG_OK;
  }
  const int sd = which - 1, dir = sd / 2, side = sd % 2;
  const int ta = dir == 0 ? 1 : 0, tb = dir == 2 ? 1 : 2;
  for (int cb = 0; cb < h->n[tb]; ++cb)
    for (int ca = 0; ca < h->n[ta]; ++ca)
      for (int pb = 0; pb < N; ++pb)
        for (int pa = 0; pa < N; ++pa) {
          double xi[3];
          xi[dir] = side ? h->n[dir] : 0;
          xi[ta] = ca + x[pa];
          xi[tb] = cb + x[pb];
          if (!h->affine && !h->ml && side) {
            // the upper boundary exactly at hi
            double pt[3];
            map(xi, pt);
            pt[dir] = h->hi[dir];
            xyz[o++] = pt[0];
            xyz[o++] = pt[1];
            xyz[o++] = pt[2];
            continue;
          }
          map(xi, xyz + o);
          o += 3;
        }
  return DG_OK;
}

static int check_apply(dg_handle* h, const void* in, void* out, int32_t precision, const char* name) {
  if (!h || !in || !out) {
    set_error(std::string(name) + ": null handle or vector");
    return DG_ERR_INVALID_ARG;
  }
  if (in == out) {
    set_error(std::string(name) + ": input and output must not alias");
    return DG_ERR_INVALID_ARG;
  }
  if (precision != DG_F64 && precision != DG_F32 && precision != DG_F64X) {
    set_error(std::string(name) + ": precision must be DG_F64, DG_F32 or DG_F64X");
    return DG_ERR_INVALID_ARG;
  }
  if ((h->vb || h->td) && precision == DG_F32) {
    set_error(std::string(name) + ": a handle with a velocity field, m = k+3, a diffusion tensor or an affine "
                                  "geometry applies in DG_F64 or DG_F64X only");
    return DG_ERR_INVALID_ARG;
  }
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != h->device) {
    set_error(std::string(name) + ": current device differs from the handle's device");
    return DG_ERR_INVALID_ARG;
  }
  return DG_OK;
}

int dg_apply_jacobian(dg_handle* h, const void* z, void* y, int32_t precision, void* stream) {
  if (int rc = check_apply(h, z, y, precision, "dg_apply_jacobian")) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision == DG_F64)
    return launch_apply_f64(h, static_cast<const double*>(z), static_cast<double*>(y), 0, 3, s);
  if (precision == DG_F64X)
    return launch_apply_f64x(h, static_cast<const double*>(z), static_cast<double*>(y), 0, 3, s);
  return launch_apply_f32(h, static_cast<const float*>(z), static_cast<float*>(y), 0, 3, s);
}

int dg_apply_residual(dg_handle* h, const void* u, void* r, int32_t precision, void* stream) {
  if (int rc = check_apply(h, u, r, precision, "dg_apply_residual")) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision == DG_F64)
    return launch_apply_f64(h, static_cast<const double*>(u), static_cast<double*>(r), 1, 3, s);
  if (precision == DG_F64X)
    return launch_apply_f64x(h, static_cast<const double*>(u), static_cast<double*>(r), 1, 3, s);
  return launch_apply_f32(h, static_cast<const float*>(u), static_cast<float*>(r), 1, 3, s);
}

int dg_apply_stage(dg_handle* h, int32_t stage, const void* in, void* out, int32_t precision, int32_t residual,
                   void* stream) {
  if (stage != 0 && stage != 1) {
    set_error("dg_apply_stage: stage must be 0 (cell kernel) or 1 (face kernel)");
    return DG_ERR_INVALID_ARG;
  }
  // stage 0 reads `in` only, stage 1 writes `out` only; the unused pointer may be anything non-null
  if (int rc = check_apply(h, stage == 0 ? in : (const void*)h, stage == 1 ? out : (void*)h, precision,
                           "dg_apply_stage"))
    return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int mode = residual ? 1 : 0, stages = stage == 0 ? 1 : 2;
  if (precision == DG_F64)
    return launch_apply_f64(h, static_cast<const double*>(in), static_cast<double*>(out), mode, stages, s);
  if (precision == DG_F64X)
    return launch_apply_f64x(h, static_cast<const double*>(in), static_cast<double*>(out), mode, stages, s);
  return launch_apply_f32(h, static_cast<const float*>(in), static_cast<float*>(out), mode, stages, s);
}

int dg_rhs(dg_handle* h, void* F, int32_t precision, void* stream) {
  if (!h || !F || (precision != DG_F64 && precision != DG_F32) || ((h->vb || h->td) && precision != DG_F64)) {
    set_error("dg_rhs: bad arguments");
    return DG_ERR_INVALID_ARG;
  }
  const int64_t ndof = h->ncell * h->N * h->N * h->N;
  const void* src = precision == DG_F64 ? h->p64.F : h->p32.F;
  const size_t bytes = ndof * (precision == DG_F64 ? sizeof(double) : sizeof(float));
  cudaError_t e = cudaMemcpyAsync(F, src, bytes, cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? DG_OK : cuda_fail(e, "dg_rhs copy");
}

}  // extern "C"
