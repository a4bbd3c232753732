// dg_internal.h -- host-side state of a dg_handle and the per-precision launchers.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/dg.h"

namespace dgi {

constexpr int MAXN = DG_MAX_DEGREE + 1;
constexpr int MAXM = MAXN + 2;  // Gauss points per direction: k+1 (q = 2p) or k+3 (q = 2p+4)

// 1D tables in FP64 for N modes and M Gauss points (Sec. 3.1), computed once per handle
struct Tables1D {
  int N, M;
  double xi[MAXM], w[MAXM];      // Gauss-Legendre nodes / weights on [0,1]
  double A[MAXM][MAXN];          // A[i][j] = theta_j(xi_i)
  double Dt[MAXM][MAXM];         // Dt[i][l] = l_l'(xi_i), Lagrange basis on the M points
  double L[2][MAXM], P[2][MAXM]; // l_l(s), l_l'(s) for s = 0, 1
};

struct Buffers {
  void* D = nullptr;       // per-cell diffusion            [ncell]
  void* fc = nullptr;      // per-cell face coefficients    [ncell][6][3]
  void* F = nullptr;       // right hand side               [ncell][N^3]
};

}  // namespace dgi

// Tables of the fast-diagonalisation block inverse.  A cell whose three 1D operators have real eigenvalues and
// eigenvectors gets real tables, the others complex ones (3 (2 n^2 + n) + 1 entries per cell either way, in the
// order of their group); each group lists its cells, red before black, each colour in ascending order.
struct FdmTables {
  bool built = false;
  int64_t nre = 0, ncx = 0;
  // each group lists its red cells (ix + iy + iz even) first, then its black ones: nre_red / ncx_red red cells
  int64_t nre_red = 0, ncx_red = 0;
  void* re32 = nullptr;  // [nre][TS] float
  void* re64 = nullptr;  // [nre][TS] double
  void* cx32 = nullptr;  // [ncx][TS] float2
  void* cx64 = nullptr;  // [ncx][TS] double2
  int64_t* re_cells = nullptr;
  int64_t* cx_cells = nullptr;
  // every red and every black cell (int32, ascending), for the operator restricted to one colour
  int* red32 = nullptr;
  int* black32 = nullptr;
  int64_t nred = 0, nblack = 0;
  bool two_cyclic = false;  // no face joins two cells of one colour (no periodic axis of odd length)
};

struct dg_handle {
  int k = 0, N = 0;
  int M = 0;                 // Gauss points per direction (N or N + 2)
  int n[3] = {0, 0, 0};
  int periodic[3] = {0, 0, 0};
  int bc_type[6] = {0, 0, 0, 0, 0, 0};  // DG_BC_* per boundary side (0 = Dirichlet)
  // velocity field kernels (a field b(x) or M != N; FP64 only): pre-scaled volume velocity
  // [ncell][3][M][M^2] and normal velocity at the face points [ncell][6][M^2] (layouts of dgk::Geo)
  bool vb = false;
  void* bsc = nullptr;
  void* bface = nullptr;
  void* bscX = nullptr;      // double-float copies of the two tables (DG_F64X applies)
  void* bfaceX = nullptr;
  void* rk_tmp = nullptr;    // Runge-Kutta stage vector (FP64, allocated by the first dg_ssprk2 call)
  // tensor diffusion / affine geometry kernels (td): Buffers::D then holds K = |det J| J^{-1} D_T J^{-T}
  // ([ncell][6]) and Buffers::fc six coefficients per face; J is the cell Jacobian (diag(h) unless affine)
  bool td = false;
  bool affine = false;
  // point-wise coefficients (pw, a td handle with Problem B's coefficients at the quadrature points):
  // kq [ncell][10][M^3] = (K00, K11, K22, K01, K02, K12, beta_0..2, c |det J| w) at every volume point,
  // kf [ncell][6][3][M^2] = row dir of K / |F_dir| at every face point, Buffers::fc [ncell][6][6][M^2] the
  // face coefficients of every face point, bface the normal velocity; FP64 and double-float copies
  bool pw = false;
  // multilinear cells (ml, a pw handle, Problem C): host copy of the vertex coordinates
  // [(n0+1)(n1+1)(n2+1)][3]; the kernels then see a unit face measure and |T| = 1 (both folded into the tables)
  bool ml = false;
  double* verts = nullptr;
  void* kq64 = nullptr;
  void* kqX = nullptr;
  void* kf64 = nullptr;
  void* kfX = nullptr;
  double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  double Jinv[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  double detJ = 0;           // |det J| = |T|
  double fscale[3] = {0, 0, 0};  // |J^{-T} e_r| = |F_r| / |T|
  int64_t ncell = 0;
  double lo[3], hi[3], h[3];
  double b[3] = {0, 0, 0};
  double c = 0, sigma = 0;
  dgi::Tables1D tab;
  dgi::Buffers p64, p32;   // FP64 and FP32 copies of the coefficient data
  dgi::Buffers pX;         // double-float copies (D and face coefficients; F is read from p64)
  void* work_V = nullptr;  // point-space residual scratch [ncell][M^3] (sized for FP64)
  void* work_tr = nullptr; // face trace scratch [ncell][6][2][M^2] (sized for FP64)
  int device = 0;
  // block-Jacobi preconditioner: per cell (A_TT^{-1})^T, row-major [ncell][N^3][N^3], FP64 and FP32
  void* bj64 = nullptr;
  void* bj32 = nullptr;
  // FP16 copy divided by each block's largest |entry| (bj16s: the FP32 factors), rows padded to a multiple of 8;
  // used by the FP32 inner solves of DG_SOLVE_MIXED
  void* bj16 = nullptr;
  void* bj16s = nullptr;
  // exact block inverse by fast diagonalisation (tables built on the host, see dg_precond.cu)
  FdmTables fdm;
  // Krylov workspace (grown on demand, freed by dg_destroy)
  void* ws = nullptr;
  size_t ws_bytes = 0;
  double* ws_host = nullptr;  // pinned host staging for reduction results
};

namespace dgi {

void set_error(const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

// Streaming multiprocessors of the current device (queried once per device); grids of the memory-bound and
// persistent kernels are sized from it.
int sm_count();

// A one-time setting per device and function (cudaFuncSetAttribute acts on the current device only): run(f)
// calls f on the first use on each device and records success there.  Two threads that first meet a device at
// once may both call f, which is harmless for the idempotent attribute settings it guards.
class DeviceOnce {
 public:
  template <class F>
  int run(F&& f) {
    int dev = 0;
    const cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return f();
    const uint64_t bit = 1ull << dev;
    if (done_.load(std::memory_order_acquire) & bit) return 0;
    const int rc = f();
    if (rc == 0) done_.fetch_or(bit, std::memory_order_acq_rel);
    return rc;
  }

 private:
  std::atomic<uint64_t> done_{0};
};
// Gauss-Legendre nodes/weights (M points) and the 1D matrices for N = k+1 modes (host, FP64)
void build_tables(int N, int M, Tables1D* tb);

// mode 0: y = A z, mode 1: y = A z - F; stages: bit 0 cell kernel, bit 1 face kernel (3 = full apply)
int launch_apply_f64(const dg_handle* h, const double* z, double* y, int mode, int stages, cudaStream_t s);
int launch_apply_f32(const dg_handle* h, const float* z, float* y, int mode, int stages, cudaStream_t s);
// t = (A z)_to for z vanishing outside the cells `from` (two colours of the red-black colouring); t written on
// `to` only.  Available where has_offdiag_f32 (degree 5, axis-parallel scalar coefficients)
bool has_offdiag_f32(const dg_handle* h);
int launch_offdiag_f32(const dg_handle* h, const float* z, float* t, const int* from, int64_t nfrom, const int* to,
                       int64_t nto, cudaStream_t s);
// FP64 vectors, operator evaluated in double-float arithmetic (pairs of FP32)
int launch_apply_f64x(const dg_handle* h, const double* z, double* y, int mode, int stages, cudaStream_t s);
int launch_diag_blocks_f64(const dg_handle* h, double* out, int cell_base, int ncells, double* V, double* tr,
                           cudaStream_t s);
// block-Jacobi application z = M r (precision by type), M from dg_precond_setup
int precond_bj_f64(const dg_handle* h, const double* r, double* z, cudaStream_t s);
int precond_bj_f32(const dg_handle* h, const float* r, float* z, cudaStream_t s);
int precond_bj_f16(const dg_handle* h, const float* r, float* z, cudaStream_t s);
int precond_fdm_f32(const dg_handle* h, const float* r, float* z, cudaStream_t s);
// z = block inverse of (scale * r) for a scaled FP16 r; tmp: n FP32 values of scratch, 16-byte aligned
int precond_fdm_f32_half(const dg_handle* h, const __half* r, float scale, float* z, float* tmp, cudaStream_t s,
                         int color = -1);
// red-black block Gauss-Seidel (t: n values of scratch; tmp as for precond_fdm_f32_half)
int precond_rbgs_f32(const dg_handle* h, const float* r, float* z, float* t, cudaStream_t s);
int precond_rbgs_f64(const dg_handle* h, const double* r, double* z, double* t, cudaStream_t s);
int precond_rbgs_f32_half(const dg_handle* h, const __half* r, float scale, float* z, float* t, float* tmp,
                          cudaStream_t s);
// z = M^{-1} u with red-black Gauss-Seidel and w = A z = u + U z together (FP32, two-cyclic colouring, a
// one-colour operator available): u FP32 or a scaled FP16 row
bool has_rbgs_eisenstat(const dg_handle* h);
int precond_rbgs_eisenstat_f32(const dg_handle* h, const float* u, float* z, float* w, float* t, cudaStream_t s);
int precond_rbgs_eisenstat_f32_half(const dg_handle* h, const __half* u, float scale, float* z, float* w, float* t,
                                    float* tmp, cudaStream_t s);
// F = l_h(phi_i) from f at the volume points (device, may not be null) and g per side (device or null);
// with vol = 1 instead of |T| and no g this is the L2 projection z_i = (f, phi_i)_T / |T|
int launch_rhs_f64(const dg_handle* h, const double* f, const double* const g[6], double* F, cudaStream_t s,
                   bool project = false);
// explicit Runge-Kutta stage y = cz z0 + cu u - cr (A u - F) (mode 3 of the face kernel)
struct StageArgs {
  const double* z0;
  double cz, cu, cr;
};
int launch_stage_f64(const dg_handle* h, const double* u, double* y, const StageArgs& st, cudaStream_t s);
int launch_stage_f64x(const dg_handle* h, const double* u, double* y, const StageArgs& st, cudaStream_t s);
// velocity field tables of a vb handle (allocates h->bsc and h->bface): kind DG_VELOCITY_*, the constant b,
// or host arrays b_qp [ncell][M^3][3] and b_face [ncell][6][M^2]
int setup_velocity(dg_handle* h, int kind, const double b[3], const double* b_qp, const double* b_face,
                   cudaStream_t s);
// the velocity field kernels (h->vb): same launches for the FP64 operator
int launch_apply_f64_vb(const dg_handle* h, const double* z, double* y, int mode, int stages, const StageArgs* st,
                        cudaStream_t s);
int launch_rhs_f64_vb(const dg_handle* h, const double* f, const double* const g[6], double* F, cudaStream_t s,
                      bool project);
int launch_apply_f64x_vb(const dg_handle* h, const double* z, double* y, int mode, int stages, const StageArgs* st,
                         cudaStream_t s);
// tensor diffusion / affine kernels (h->td): FP64 and double-float operators, FP64 vectors
int launch_apply_td(const dg_handle* h, const double* z, double* y, int mode, int stages, const StageArgs* st,
                    bool pairs, cudaStream_t s);
int launch_rhs_td(const dg_handle* h, const double* f, const double* const g[6], double* F, cudaStream_t s,
                  bool project);
// point-wise coefficient kernels (h->pw): FP64 (dg_launch_pw.cu) and double-float (dg_launch_pwx.cu) operators
int launch_apply_pw(const dg_handle* h, const double* z, double* y, int mode, int stages, const StageArgs* st,
                    cudaStream_t s);
int launch_apply_pwx(const dg_handle* h, const double* z, double* y, int mode, int stages, const StageArgs* st,
                     cudaStream_t s);
int launch_rhs_pw(const dg_handle* h, const double* f, const double* const g[6], double* F, cudaStream_t s,
                  bool project);
// host tables of a pw handle (h->J, h->M, mesh, sigma set): kq, kf, fc and bface in the layouts above; the
// velocity is b (constant) or b_qp [ncell][M^3][3] and b_face [ncell][6][M^2] (normal velocity) when given
int build_pointwise_tables(const dg_handle* h, const double* D_qp, const double* D_face, const double* c_qp,
                           double c_const, const double b[3], const double* b_qp, const double* b_face,
                           std::vector<double>& kq, std::vector<double>& kf, std::vector<double>& fc,
                           std::vector<double>& bface);
// geometry of a cell's map at a local reference point xi in [0,1]^3: J^{-1} and |det J| (constant unless the
// cells are multilinear); face_frame: unit normal along +reference axis r and the area element
// |det J| |J^{-T} e_r|; face_xi: the local coordinates of point p of face 2*dir+side
struct MapGeo {
  double Jinv[3][3];
  double det;   // |det J|
  double sdet;  // det J (its sign is the cell map's orientation)
};
int point_geometry(const dg_handle* h, int64_t cell, const double xi[3], MapGeo* g);
double face_frame(const MapGeo& g, int r, double nu[3]);
void face_xi(const dg_handle* h, int face, int p, double xi[3]);
// x[i] = pair of FP32 numbers closest to a[i] (double-float copies of the coefficient tables)
int copy_to_pairs(const double* a, void* x_pairs, int64_t n, cudaStream_t s);

}  // namespace dgi
