// dg_solve.cu -- flexible GMRES on the matrix-free operator: plain FP64, or an FP64 outer FGMRES whose
// preconditioner is an FP32 inner FGMRES on the FP32 operator (mixed precision).  The residual, the
// defect updates and the outer orthogonalisation stay in FP64.
#include <chrono>
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <initializer_list>
#include <string>
#include <type_traits>
#include <vector>

#include "dg_blas.cuh"
#include "dg_internal.h"

namespace dgi {

bool mlp_matches(const dg_mlp* m, const dg_handle* h);
int mlp_apply_impl(dg_mlp* m, const dg_handle* h, const void* r, void* z, int32_t precision, int accumulate,
                   cudaStream_t s);

namespace {

// Arnoldi steps of the inner FP32 solve between two reads of its device-side state (a step costs about a
// millisecond at the benchmark sizes, a read a few microseconds; steps past a convergence are wasted)
constexpr int kInnerCheckEvery = 5;

struct Ctx {
  dg_handle* h;
  cudaStream_t s;
  size_t n;
  double* part;   // PART_ROWS rows of block sums (up to max(dots2_blocks, red_blocks) per row)
  double* hdev;   // 128 results of a dot pass
  double* ydev;   // 64 coefficients of the solution update
  double* cdev;   // 2 MAX_ROWS + 3 coefficients of the second basis pass
  double* hhost;  // pinned, 512: reduction results at 0, the Arnoldi state's head at 448
  dgb::ArnState* arn[2] = {nullptr, nullptr};  // device Arnoldi state of the outer (0) and inner (1) FGMRES
  int depth = 0;                               // nesting level of the running fgmres call
  int applies64 = 0, applies32 = 0;
  bool f64x = false;  // FP64 vectors with the double-float operator
  // grids, sized from the device's SM count: the element-wise kernels, the basis passes (one wave at their
  // resident-CTA bound) and the two-row dot pass
  int red_blocks = 0, pass_blocks = 0, dots2_blocks = 0;
  void set_grids(int sms) {
    red_blocks = sms * 4;
    pass_blocks = sms * dgb::PASS_MINB;
    dots2_blocks = sms * dgb::DOTS2_MINB;
  }
};

int cuda_check(cudaError_t e, const char* what) { return e == cudaSuccess ? 0 : cuda_fail(e, what); }

// 16-byte packs when the length and every row start allow them, else one element per load
template <typename T>
bool packable(size_t n, std::initializer_list<const void*> ptrs) {
  constexpr size_t W = 16 / sizeof(T);
  if (n % W) return false;
  for (const void* q : ptrs)
    if (reinterpret_cast<uintptr_t>(q) % 16) return false;
  return true;
}

// the per-thread partial sums of a dot pass take up to MAX_ROWS columns of shared memory (128 KB in FP64), beyond
// the 48 KB a launch gets without opting in: opt in once per kernel
template <typename T, int W>
int basis_smem_attr() {
  static DeviceOnce once;
  return once.run([] {
    return cuda_check(cudaFuncSetAttribute(dgb::basis_dots<T, W, dgb::PASS_MINB, dgb::PASS_LOADS>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           dgb::MAX_ROWS * dgb::RED_THREADS * (int)sizeof(T)),
                      "basis pass shared memory");
  });
}

// dst[q] = V_q . w (q < nv) on the device
template <typename T>
int basis_dots(Ctx& c, const T* V, int nv, const T* w, double* dst) {
  const size_t smem = (size_t)nv * dgb::RED_THREADS * sizeof(T);
  if (packable<T>(c.n, {V, w})) {
    constexpr int W = 16 / sizeof(T);
    if (int rc = basis_smem_attr<T, W>()) return rc;
    dgb::basis_dots<T, W, dgb::PASS_MINB, dgb::PASS_LOADS>
        <<<c.pass_blocks, dgb::RED_THREADS, smem, c.s>>>(V, c.n, nv, w, c.n / W, c.part);
  } else {
    if (int rc = basis_smem_attr<T, 1>()) return rc;
    dgb::basis_dots<T, 1, dgb::PASS_MINB, dgb::PASS_LOADS>
        <<<c.pass_blocks, dgb::RED_THREADS, smem, c.s>>>(V, c.n, nv, w, c.n, c.part);
  }
  dgb::mdot_final<<<nv, dgb::RED_THREADS, 0, c.s>>>(c.part, c.pass_blocks, dst);
  return cuda_check(cudaGetLastError(), "basis dot kernels");
}

// x <- x + sum_q y[q] Z_q, y on the device
template <typename T>
int lincomb_add(Ctx& c, const T* Z, int nv, const double* y, T* x) {
  if (packable<T>(c.n, {Z, x})) {
    constexpr int W = 16 / sizeof(T);
    dgb::lincomb_add<T, W, dgb::PASS_MINB, dgb::PASS_LOADS><<<c.pass_blocks, dgb::RED_THREADS, 0, c.s>>>(Z, c.n, nv, y, x, c.n / W);
  } else {
    dgb::lincomb_add<T, 1, dgb::PASS_MINB, dgb::PASS_LOADS><<<c.pass_blocks, dgb::RED_THREADS, 0, c.s>>>(Z, c.n, nv, y, x, c.n);
  }
  return cuda_check(cudaGetLastError(), "solution update");
}

// out_host[q] = V_q . w for q < nv (synchronises)
template <typename T>
int dots(Ctx& c, const T* V, int nv, const T* w, double* out_host) {
  if (int rc = basis_dots<T>(c, V, nv, w, c.hdev)) return rc;
  if (int rc = cuda_check(cudaMemcpyAsync(c.hhost, c.hdev, nv * sizeof(double), cudaMemcpyDeviceToHost, c.s),
                          "dot copy"))
    return rc;
  if (int rc = cuda_check(cudaStreamSynchronize(c.s), "dot sync")) return rc;
  std::memcpy(out_host, c.hhost, nv * sizeof(double));
  return 0;
}

template <typename T>
int scale(Ctx& c, T* v, double a) {
  dgb::scale_copy<T, T><<<c.red_blocks, dgb::RED_THREADS, 0, c.s>>>(v, v, a, c.n);
  return cuda_check(cudaGetLastError(), "scale");
}

// y = A x in precision T
template <typename T>
int apply_A(Ctx& c, const T* x, T* y);
template <>
int apply_A<double>(Ctx& c, const double* x, double* y) {
  ++c.applies64;
  return c.f64x ? launch_apply_f64x(c.h, x, y, 0, 3, c.s) : launch_apply_f64(c.h, x, y, 0, 3, c.s);
}
template <>
int apply_A<float>(Ctx& c, const float* x, float* y) {
  ++c.applies32;
  return launch_apply_f32(c.h, x, y, 0, 3, c.s);
}

struct Result {
  int iterations = 0;
  double res = 0;     // last (estimated or true) residual norm
  double beta0 = 0;   // initial residual norm
  bool converged = false;
};

// Pass 1 of the lagged Arnoldi step: dst[0 .. 2 nr] = (V_q . u, q < nr; V_q . w, q < nr; w . w), u = V_{nr-1}
template <typename T>
int basis_dots2(Ctx& c, const T* V, int nr, const T* w, double* dst) {
  const int rows = 2 * nr + 1;
  const size_t smem = (size_t)rows * dgb::DOTS2_THREADS * sizeof(T);
  static DeviceOnce attr_packed, attr_scalar;
  const bool pk = packable<T>(c.n, {V, w});
  constexpr int W = 16 / sizeof(T);
  const int most = dgb::PART_ROWS * dgb::DOTS2_THREADS * (int)sizeof(T);
  if (int rc = (pk ? attr_packed : attr_scalar).run([&] {
        return cuda_check(pk ? cudaFuncSetAttribute(dgb::basis_dots2<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    most)
                             : cudaFuncSetAttribute(dgb::basis_dots2<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    most),
                          "basis pass shared memory");
      }))
    return rc;
  if (pk)
    dgb::basis_dots2<T, W><<<c.dots2_blocks, dgb::DOTS2_THREADS, smem, c.s>>>(V, c.n, nr, w, c.n / W, c.part);
  else
    dgb::basis_dots2<T, 1><<<c.dots2_blocks, dgb::DOTS2_THREADS, smem, c.s>>>(V, c.n, nr, w, c.n, c.part);
  dgb::mdot_final<<<rows, dgb::RED_THREADS, 0, c.s>>>(c.part, c.dots2_blocks, dst);
  return cuda_check(cudaGetLastError(), "basis dot kernels");
}

// Pass 2 with the coefficients the device-side Arnoldi step wrote to c.cdev (skipped once the cycle stopped)
template <typename T>
int basis_update2(Ctx& c, T* V, int nr, bool write_u, T* w, const int* stop) {
  if (packable<T>(c.n, {V, w})) {
    constexpr int W = 16 / sizeof(T);
    dgb::basis_update2<T, W><<<c.pass_blocks, dgb::RED_THREADS, 0, c.s>>>(V, c.n, nr, c.cdev, write_u, w,
                                                                           c.n / W, stop);
  } else {
    dgb::basis_update2<T, 1><<<c.pass_blocks, dgb::RED_THREADS, 0, c.s>>>(V, c.n, nr, c.cdev, write_u, w, c.n,
                                                                           stop);
  }
  return cuda_check(cudaGetLastError(), "basis update");
}

// The same three passes over an FP16 basis (rows scaled by dgb::HB_SCALE) of the FP32 inner solve; w is an FP32
// vector of its own.  The caller guarantees n % 8 == 0 and 16-byte aligned rows.
int basis_dots2(Ctx& c, const __half* V, int nr, const float* w, double* dst) {
  const int rows = 2 * nr + 1;
  static DeviceOnce attr;
  if (int rc = attr.run([] {
        return cuda_check(cudaFuncSetAttribute(dgb::basis_dots2_h, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               dgb::PART_ROWS * dgb::DOTS2_THREADS * (int)sizeof(float)),
                          "basis pass shared memory");
      }))
    return rc;
  dgb::basis_dots2_h<<<c.dots2_blocks, dgb::DOTS2_THREADS, (size_t)rows * dgb::DOTS2_THREADS * sizeof(float), c.s>>>(
      V, c.n, nr, w, c.n / 8, c.part);
  dgb::mdot_final<<<rows, dgb::RED_THREADS, 0, c.s>>>(c.part, c.dots2_blocks, dst);
  return cuda_check(cudaGetLastError(), "basis dot kernels");
}

int basis_update2(Ctx& c, __half* V, int nr, bool write_u, const float* w, const int* stop) {
  dgb::basis_update2_h<<<c.pass_blocks, dgb::RED_THREADS, 0, c.s>>>(V, c.n, nr, c.cdev, write_u, w, c.n / 8, stop);
  return cuda_check(cudaGetLastError(), "basis update");
}

int basis_dots(Ctx& c, const __half* V, int nv, const __half* x, double* dst) {
  static DeviceOnce attr;
  if (int rc = attr.run([] {
        return cuda_check(cudaFuncSetAttribute(dgb::basis_dots_h, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               dgb::MAX_ROWS * dgb::RED_THREADS * (int)sizeof(float)),
                          "basis pass shared memory");
      }))
    return rc;
  dgb::basis_dots_h<<<c.pass_blocks, dgb::RED_THREADS, (size_t)nv * dgb::RED_THREADS * sizeof(float), c.s>>>(
      V, c.n, nv, x, c.n / 8, c.part);
  dgb::mdot_final<<<nv, dgb::RED_THREADS, 0, c.s>>>(c.part, c.pass_blocks, dst);
  return cuda_check(cudaGetLastError(), "basis dot kernels");
}

// Flexible GMRES(m) on A x = b in precision T with right preconditioner M (nullptr: none, z_j = v_j).
// V: (m+1) n, Z: m n.  x holds the initial guess unless x0_zero.
//
// Arnoldi by classical Gram-Schmidt with the reorthogonalisation delayed by one step (two passes over the basis
// per step instead of three).  At step j the rows V_0 .. V_{j-1} are final and V_j holds a provisional u_j (u_0 =
// r0 / ||r0|| is final).  The step preconditions the provisional vector, z_j = M(u_j), forms w = A z_j and in
// pass 1 takes a = V_{<j}^T u_j, ||u_j||^2, V_{<=j}^T w and ||w||^2.  The final v_j = (u_j - V_{<j} a) / alpha,
// alpha^2 = ||u_j||^2 - ||a||^2, so the coefficients of w on the final basis are c_i = V_i . w (i < j) and
// c_j = (u_j . w - a . c_{<j}) / alpha, and the projection of w leaves beta^2 = ||w||^2 - ||c||^2.  Pass 2
// writes v_j and the next provisional row u_{j+1} = (w - V_{<=j} c) / beta (with v_j expressed through u_j).
// Column j of H follows one step later, from w = V_{<=j} c + beta u_{j+1} and u_{j+1}'s own reorthogonalisation
// (a', alpha'): H[0..j][j] = c + beta a', H[j+1][j] = beta alpha'.  FGMRES needs only A Z = V H with V
// orthonormal, and z_j = M(u_j) is such a direction whatever the later correction of u_j.
//
// The scalar work of a step (finalising column j - 1, the Givens rotations, the residual estimate, the stop test,
// the provisional estimate after column j and the coefficients of pass 2) runs on the device (dgb::arn_step),
// so the host launches the steps of a cycle without waiting; it reads the state back every check_every steps
// and at the end of the cycle (one synchronisation each).  When the provisional estimate has met the
// tolerance, one more dot pass (the reorthogonalisation of u_{j+1}) finalises column j and decides; a cycle
// that stops between two reads is confirmed by the next step's pass 1, whose operator application is then
// unused.  The outer solve reads every step (its steps are whole inner solves); the inner one less often.
//
// B = __half (T = float only): the basis V is stored in scaled FP16 and `tmp` holds two FP32 vectors, the new
// operator product w and the FP32 copy of u_j that the preconditioner reads; a preconditioner MB that reads
// the FP16 row itself takes the place of that copy and of M.
template <typename T, typename B = T>
int fgmres(Ctx& c, const std::function<int(const T*, T*)>& M, const T* b, T* x, bool x0_zero, B* V, T* Z, int m,
           double tol_abs, int maxit, int max_cycles, bool true_residual_check, Result* out,
           const std::function<void(double, double)>& cycle_hook = {},
           const std::function<int(const T*, T*)>& M0 = {}, int check_every = 1, T* tmp = nullptr,
           const std::function<int(const B*, T*)>& MB = {}, const std::function<int(const B*, T*, T*)>& MA = {}) {
  constexpr bool half_basis = !std::is_same<T, B>::value;
  static_assert(!half_basis || (std::is_same<T, float>::value && std::is_same<B, __half>::value),
                "FP16 basis storage is for the FP32 solve");
  const size_t n = c.n;
  if (c.depth > 1) {
    set_error("FGMRES: nested deeper than outer and inner solve");
    return DG_ERR_INVALID_ARG;
  }
  dgb::ArnState* st = c.arn[c.depth];
  ++c.depth;
  struct DepthGuard {
    Ctx& c;
    ~DepthGuard() { --c.depth; }
  } guard{c};
  const int* stop = &st->stop;
  double* head = c.hhost + 448;  // pinned copy of the state's head (ARN_HEAD_BYTES)
  dgb::ArnState hd;
  auto read_head = [&]() -> int {
    if (int rc = cuda_check(cudaMemcpyAsync(head, st, dgb::ARN_HEAD_BYTES, cudaMemcpyDeviceToHost, c.s),
                            "Arnoldi state copy"))
      return rc;
    if (int rc = cuda_check(cudaStreamSynchronize(c.s), "Arnoldi sync")) return rc;
    std::memcpy(&hd, head, dgb::ARN_HEAD_BYTES);
    if (hd.err) {
      set_error("FGMRES: non-finite Arnoldi vector");
      return DG_ERR_NAN;
    }
    return 0;
  };
  Result r;
  for (int cycle = 0; cycle < max_cycles; ++cycle) {
    T* v0;  // the residual, normalised in place (or, with an FP16 basis, stored scaled into row 0)
    if constexpr (half_basis) v0 = tmp;
    else v0 = V;
    if (x0_zero && cycle == 0) {
      if (int rc = cuda_check(cudaMemcpyAsync(v0, b, n * sizeof(T), cudaMemcpyDeviceToDevice, c.s), "copy b"))
        return rc;
    } else {
      if (int rc = apply_A<T>(c, x, v0)) return rc;
      dgb::sub<T><<<c.red_blocks, dgb::RED_THREADS, 0, c.s>>>(b, v0, v0, n);
    }
    double nrm2;
    if (int rc = dots<T>(c, v0, 1, v0, &nrm2)) return rc;
    const double beta = std::sqrt(nrm2);
    if (!std::isfinite(beta)) {
      set_error("FGMRES: non-finite residual");
      return DG_ERR_NAN;
    }
    if (cycle == 0) r.beta0 = beta;
    r.res = beta;
    if (beta <= tol_abs) {
      r.converged = true;
      break;
    }
    if (r.iterations >= maxit) break;
    if (cycle > 0 && !true_residual_check) break;
    if constexpr (half_basis) {
      dgb::h_store_scaled<<<c.red_blocks, dgb::RED_THREADS, 0, c.s>>>(v0, (float)(1.0 / beta), V, n / 8);
      if (int rc = cuda_check(cudaGetLastError(), "basis row store")) return rc;
    } else if (int rc = scale<T>(c, v0, 1.0 / beta)) {
      return rc;
    }
    dgb::arn_init<<<1, 1, 0, c.s>>>(st, m, tol_abs, beta);
    const int steps = std::min(m, maxit - r.iterations);
    int last = steps - 1;  // the step after which the cycle's last column is finalised
    bool finalised = false;
    for (int j = 0; j < steps; ++j) {
      const T* uj = nullptr;
      T* w;
      T* zj = Z + (size_t)j * n;
      bool applied = false;  // z_j formed straight from the FP16 row
      bool have_w = false;   // z_j and w = A z_j formed together (MA)
      if (MA && !(j == 0 && M0)) {
        if constexpr (half_basis) w = tmp;
        else w = V + (size_t)(j + 1) * n;
        if (int rc = MA(V + (size_t)j * n, zj, w)) return rc;
        applied = have_w = true;
      } else if constexpr (half_basis) {
        w = tmp;
        if (MB && !(j == 0 && M0)) {
          if (int rc = MB(V + (size_t)j * n, zj)) return rc;
          applied = true;
        } else {
          dgb::h_load<<<c.red_blocks, dgb::RED_THREADS, 0, c.s>>>(V + (size_t)j * n, tmp + n, n / 8);
          if (int rc = cuda_check(cudaGetLastError(), "basis row load")) return rc;
          uj = tmp + n;
        }
      } else {
        uj = V + (size_t)j * n;
        w = V + (size_t)(j + 1) * n;
      }
      if (applied) {
      } else if (j == 0 && M0) {
        if (int rc = M0(uj, zj)) return rc;
      } else if (M) {
        if (int rc = M(uj, zj)) return rc;
      } else {
        if (int rc = cuda_check(cudaMemcpyAsync(zj, uj, n * sizeof(T), cudaMemcpyDeviceToDevice, c.s), "copy v"))
          return rc;
      }
      if (!have_w)
        if (int rc = apply_A<T>(c, zj, w)) return rc;
      if (int rc = basis_dots2(c, V, j + 1, w, c.hdev)) return rc;  // pass 1
      dgb::arn_step<<<1, 32, 0, c.s>>>(st, c.hdev, j, c.cdev);
      if (int rc = basis_update2(c, V, j + 1, j > 0, w, stop)) return rc;  // pass 2
      if (j == steps - 1 || (j + 1) % check_every != 0) continue;
      if (int rc = read_head()) return rc;
      if (hd.stop) {  // converged or broke down at an earlier column: nothing left to finalise
        last = j;
        finalised = true;
        break;
      }
      if (hd.prov <= tol_abs) {
        // finalise column j now: the reorthogonalisation of u_{j+1} against rows 0 .. j
        if (int rc = basis_dots(c, V, j + 2, V + (size_t)(j + 1) * n, c.hdev)) return rc;
        dgb::arn_final<<<1, 32, 0, c.s>>>(st, c.hdev, j);
        if (int rc = read_head()) return rc;
        if (hd.res <= tol_abs) {
          last = j;
          finalised = true;
          break;
        }
      }
    }
    // finalise the last column: the reorthogonalisation of u_steps against rows 0 .. steps - 1
    if (!finalised) {
      if (int rc = basis_dots(c, V, last + 2, V + (size_t)(last + 1) * n, c.hdev)) return rc;
      dgb::arn_final<<<1, 32, 0, c.s>>>(st, c.hdev, last);
    }
    dgb::arn_solve<<<1, 1, 0, c.s>>>(st, c.ydev);
    if (int rc = read_head()) return rc;
    if (hd.fin != hd.jend) {
      set_error("FGMRES: internal error (Hessenberg column not finalised)");
      return DG_ERR_INVALID_ARG;
    }
    const int jend = hd.jend;
    r.iterations += jend;
    r.res = hd.res;
    const bool est_conv = hd.stop || hd.res <= tol_abs;
    // x += Z y
    if (jend > 0)
      if (int rc = lincomb_add<T>(c, Z, jend, c.ydev, x)) return rc;
    if (cycle_hook) cycle_hook(beta, r.res);
    if (est_conv && !true_residual_check) {
      r.converged = true;
      break;
    }
  }
  *out = r;
  return 0;
}

int ensure_ws(dg_handle* h, size_t bytes) {
  if (h->ws_bytes >= bytes) return 0;
  cudaFree(h->ws);
  h->ws = nullptr;
  h->ws_bytes = 0;
  cudaError_t e = cudaMalloc(&h->ws, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(solver workspace)");
  h->ws_bytes = bytes;
  if (!h->ws_host) {
    e = cudaMallocHost(&h->ws_host, 512 * sizeof(double));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocHost(solver staging)");
  }
  return 0;
}

}  // namespace

}  // namespace dgi

using namespace dgi;

extern "C" {

int dg_solve(dg_handle* h, const double* b_dev, double* x_dev, const dg_solve_opts* o, dg_solve_stats* st,
             void* stream) {
  if (!h || !x_dev || !o) {
    set_error("dg_solve: null handle, x or options");
    return DG_ERR_INVALID_ARG;
  }
  const int m = o->restart > 0 ? o->restart : 30;
  const int mo = o->outer_restart > 0 ? o->outer_restart : 20;
  if (m > 60 || mo > 60 || (o->mode != DG_SOLVE_FP64 && o->mode != DG_SOLVE_MIXED) ||
      (o->inner_block_precision < 0 || o->inner_block_precision > 2) ||
      (o->outer_precision < 0 || o->outer_precision > 1) ||
      (o->inner_basis_precision < 0 || o->inner_basis_precision > 1) ||
      (o->preconditioner != DG_PRECOND_NONE && o->preconditioner != DG_PRECOND_BLOCK_JACOBI &&
       o->preconditioner != DG_PRECOND_MLP && o->preconditioner != DG_PRECOND_BJ_MLP &&
       o->preconditioner != DG_PRECOND_RB_GS) ||
      !(o->rtol > 0) || (o->mode == DG_SOLVE_MIXED && !(o->inner_rtol > 0 && o->inner_rtol < 1))) {
    set_error("dg_solve: bad options (restart <= 60, mode, preconditioner, rtol > 0, 0 < inner_rtol < 1)");
    return DG_ERR_INVALID_ARG;
  }
  if ((h->vb || h->td) && o->mode != DG_SOLVE_FP64) {
    set_error("dg_solve: a handle with a velocity field, m = k+3, a diffusion tensor or an affine geometry solves "
              "in DG_SOLVE_FP64 only");
    return DG_ERR_INVALID_ARG;
  }
  if ((o->preconditioner == DG_PRECOND_BLOCK_JACOBI || o->preconditioner == DG_PRECOND_BJ_MLP) && !h->bj64 &&
      !h->fdm.built) {
    set_error("dg_solve: block-Jacobi requested but dg_precond_setup was not called");
    return DG_ERR_INVALID_ARG;
  }
  if (o->preconditioner == DG_PRECOND_RB_GS && !h->fdm.built) {
    set_error("dg_solve: red-black Gauss-Seidel requested but dg_precond_setup was not called");
    return DG_ERR_INVALID_ARG;
  }
  if ((o->preconditioner == DG_PRECOND_MLP || o->preconditioner == DG_PRECOND_BJ_MLP) && !mlp_matches(o->mlp, h)) {
    set_error("dg_solve: DG_PRECOND_MLP / DG_PRECOND_BJ_MLP need opts->mlp for the handle's degree");
    return DG_ERR_INVALID_ARG;
  }
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t n = (size_t)h->ncell * h->N * h->N * h->N;
  const bool pc = o->preconditioner != DG_PRECOND_NONE;
  const bool rbgs = o->preconditioner == DG_PRECOND_RB_GS;  // one more vector: the sweep's A z_red
  // MLP preconditioner, with a switch to block-Jacobi when a cycle stagnates (if blocks exist)
  bool use_mlp = o->preconditioner == DG_PRECOND_MLP || o->preconditioner == DG_PRECOND_BJ_MLP;
  const bool with_bj = o->preconditioner == DG_PRECOND_BJ_MLP;
  // placement 1: the network only acts on the first direction of each (outer) FGMRES cycle, where the
  // direction is the true residual r / ||r|| -- the kind of input it was trained on
  const bool first_only = use_mlp && o->mlp_placement == 1;
  int fallback = 0;
  dg_mlp* mlp = const_cast<dg_mlp*>(o->mlp);
  auto maybe_fallback = [&](double start, double end) {
    if (use_mlp && o->fallback_ratio > 0 && (h->bj64 || h->fdm.built) && start > 0 && end > o->fallback_ratio * start) {
      use_mlp = false;
      fallback = 1;
    }
  };
  // workspace: reductions, r/b copy, FP64 basis (V, Z), FP32 basis for the inner solve
  // partial sums (rows x blocks of the widest pass), then the dot results (128), y (128) and the pass
  // coefficients (2 MAX_ROWS + 3 = 131); 400 keeps what follows 16-byte aligned
  Ctx c;
  c.set_grids(sm_count());
  const size_t part_size = (size_t)dgb::PART_ROWS * std::max(c.dots2_blocks, c.red_blocks);
  const size_t arn_words = (sizeof(dgb::ArnState) + 255) / 256 * 32;  // one state, rounded to 256 bytes
  const size_t small = part_size + 400 + 2 * arn_words;
  // FP16 storage of the inner basis: FP32 Z, rhs, e, w and u (m + 4 vectors), then the m + 1 FP16 rows
  const bool half_basis = o->mode == DG_SOLVE_MIXED && o->inner_basis_precision == 1 && n % 8 == 0;
  size_t v64 = 0, v32 = 0;
  if (o->mode == DG_SOLVE_FP64) {
    v64 = (size_t)(2 * m + 1 + (rbgs ? 1 : 0)) * n;  // V and Z (Z = V's provisional rows without a preconditioner)
  } else {
    v64 = (size_t)(2 * mo + 1) * n;
    v32 = half_basis ? (size_t)(m + 4) * n + (size_t)(m + 1) * n / 2 : (size_t)(2 * m + 1 + 2) * n;
    if (rbgs) v32 += n;
  }
  const size_t bytes = (small + n + v64) * sizeof(double) + v32 * sizeof(float) + 256;
  if (int rc = ensure_ws(h, bytes)) return rc;
  c.h = h;
  c.s = s;
  c.n = n;
  double* base = static_cast<double*>(h->ws);
  c.part = base;
  c.hdev = base + part_size;  // up to 2 * 61 + 1 results of a pass
  c.ydev = c.hdev + 128;
  c.cdev = c.ydev + 128;
  c.arn[0] = reinterpret_cast<dgb::ArnState*>(base + part_size + 400);
  c.arn[1] = reinterpret_cast<dgb::ArnState*>(base + part_size + 400 + arn_words);
  double* bcopy = base + small;
  double* V64 = bcopy + n;
  // the FP32 / FP16 vectors start on a 256-byte boundary (the 256 spare bytes of the workspace)
  float* f32 = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(V64 + v64) + 255) / 256 * 256);
  c.hhost = h->ws_host;

  int rc = 0;
  if (b_dev)
    rc = cuda_check(cudaMemcpyAsync(bcopy, b_dev, n * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy b");
  else
    rc = cuda_check(cudaMemcpyAsync(bcopy, h->p64.F, n * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy F");
  if (rc) return rc;
  double bn2;
  if ((rc = dots<double>(c, bcopy, 1, bcopy, &bn2))) return rc;
  const double bnorm = std::sqrt(bn2);
  const double tol = o->rtol * (bnorm > 0 ? bnorm : 1.0);
  const int maxit = o->max_iterations > 0 ? o->max_iterations : 10000;
  Result res;
  int inner_total = 0;
  if (o->mode == DG_SOLVE_FP64) {
    std::function<int(const double*, double*)> M, M0;
    double* gs64 = V64 + (size_t)(2 * m + 1) * n;  // scratch of the Gauss-Seidel sweep
    if (rbgs)
      M = [&](const double* r, double* z) {
        ++c.applies64;
        return precond_rbgs_f64(h, r, z, gs64, s);
      };
    else if (pc && !first_only)
      M = [&](const double* r, double* z) {
        if (!use_mlp) return precond_bj_f64(h, r, z, s);
        if (!with_bj) return mlp_apply_impl(mlp, h, r, z, DG_F64, 0, s);
        int e2 = precond_bj_f64(h, r, z, s);
        return e2 ? e2 : mlp_apply_impl(mlp, h, r, z, DG_F64, 1, s);
      };
    if (first_only) {
      if (with_bj) M = [&](const double* r, double* z) { return precond_bj_f64(h, r, z, s); };
      M0 = [&](const double* r, double* z) {
        if (!use_mlp) return M ? M(r, z) : cuda_check(cudaMemcpyAsync(z, r, n * sizeof(double),
                                                                      cudaMemcpyDeviceToDevice, s), "copy");
        if (!with_bj) return mlp_apply_impl(mlp, h, r, z, DG_F64, 0, s);
        int e2 = precond_bj_f64(h, r, z, s);
        return e2 ? e2 : mlp_apply_impl(mlp, h, r, z, DG_F64, 1, s);
      };
    }
    rc = fgmres<double>(c, M, bcopy, x_dev, false, V64, V64 + (size_t)(m + 1) * n, m, tol, maxit, 1 << 20, true,
                        &res, maybe_fallback, M0);
    inner_total = res.iterations;
  } else {
    // inner FP32 FGMRES(m) on the FP32 operator, x0 = 0, one cycle or until inner_rtol: z = P(v)
    float *V32, *Z32, *rhs32, *e32, *tmp32 = nullptr;
    __half* V16 = nullptr;
    if (half_basis) {
      Z32 = f32;
      rhs32 = Z32 + (size_t)m * n;
      e32 = rhs32 + n;
      tmp32 = e32 + n;
      V16 = reinterpret_cast<__half*>(tmp32 + 2 * n);
      V32 = nullptr;
    } else {
      V32 = f32;
      Z32 = V32 + (size_t)(m + 1) * n;
      rhs32 = Z32 + (size_t)m * n;
      e32 = rhs32 + n;
    }
    float* gs32 = f32 + v32 - n;  // scratch of the Gauss-Seidel sweep (the last FP32 vector)
    std::function<int(const float*, float*)> M32;
    // block-Jacobi inside the FP32 inner solve: the FP16 blocks (half the bytes of this HBM-bound product) unless
    // the caller asked for the FP32 ones
    auto bj_inner = [&](const float* r, float* z) {
      if (o->inner_block_precision == 1) return precond_bj_f32(h, r, z, s);
      if (o->inner_block_precision == 0 && h->fdm.built) return precond_fdm_f32(h, r, z, s);
      return precond_bj_f16(h, r, z, s);
    };
    if (rbgs)
      M32 = [&](const float* r, float* z) {
        ++c.applies32;
        return precond_rbgs_f32(h, r, z, gs32, s);
      };
    else if (pc)
      M32 = [&](const float* r, float* z) {
        if (!use_mlp || first_only) return with_bj || !use_mlp ? bj_inner(r, z)
                                                             : cuda_check(cudaMemcpyAsync(z, r, n * sizeof(float),
                                                                                          cudaMemcpyDeviceToDevice, s),
                                                                          "copy");
        if (!with_bj) return mlp_apply_impl(mlp, h, r, z, DG_F32, 0, s);
        int e2 = bj_inner(r, z);
        return e2 ? e2 : mlp_apply_impl(mlp, h, r, z, DG_F32, 1, s);
      };
    // with the FP16 basis and the fast-diagonalisation block inverse alone (no network), the block inverse reads
    // the basis rows itself (the FP32 copy of u_j goes away)
    std::function<int(const __half*, float*)> M16;
    if (half_basis && rbgs)
      M16 = [&](const __half* r, float* z) {
        ++c.applies32;
        return precond_rbgs_f32_half(h, r, dgb::HB_INV, z, gs32, tmp32 + n, s);
      };
    else if (half_basis && pc && !use_mlp && o->inner_block_precision == 0 && h->fdm.built)
      M16 = [&](const __half* r, float* z) {
        return precond_fdm_f32_half(h, r, dgb::HB_INV, z, tmp32 + n, s);
      };
    // red-black Gauss-Seidel with a two-cyclic colouring: the sweep and the Krylov step's operator together,
    // A z = u + U z (half an operator instead of a whole one)
    std::function<int(const float*, float*, float*)> MA32;
    std::function<int(const __half*, float*, float*)> MA16;
    if (rbgs && has_rbgs_eisenstat(h)) {
      MA32 = [&](const float* u, float* z, float* w) {
        c.applies32 += 2;
        return precond_rbgs_eisenstat_f32(h, u, z, w, gs32, s);
      };
      MA16 = [&](const __half* u, float* z, float* w) {
        c.applies32 += 2;
        return precond_rbgs_eisenstat_f32_half(h, u, dgb::HB_INV, z, w, gs32, tmp32 + n, s);
      };
    }
    std::function<int(const double*, double*)> P = [&](const double* v, double* z) -> int {
      dgb::scale_copy<double, float><<<c.red_blocks, dgb::RED_THREADS, 0, s>>>(v, rhs32, 1.0, n);
      cudaMemsetAsync(e32, 0, n * sizeof(float), s);
      Result ri;
      double vn2;
      int rc2 = dots<float>(c, rhs32, 1, rhs32, &vn2);
      if (rc2) return rc2;
      const double itol = o->inner_rtol * std::sqrt(vn2);
      rc2 = half_basis ? fgmres<float, __half>(c, M32, rhs32, e32, true, V16, Z32, m, itol, m, 1, false, &ri, {}, {},
                                               kInnerCheckEvery, tmp32, M16, MA16)
                       : fgmres<float>(c, M32, rhs32, e32, true, V32, Z32, m, itol, m, 1, false, &ri, {}, {},
                                       kInnerCheckEvery, nullptr, {}, MA32);
      if (rc2) return rc2;
      maybe_fallback(ri.beta0, ri.res);
      inner_total += ri.iterations;
      dgb::scale_copy<float, double><<<c.red_blocks, dgb::RED_THREADS, 0, s>>>(e32, z, 1.0, n);
      return cuda_check(cudaGetLastError(), "inner solve casts");
    };
    std::function<int(const double*, double*)> P0;
    if (first_only)
      P0 = [&](const double* v, double* z) -> int {
        // the inner solve, plus the network's correction of the true residual direction
        if (int rc2 = P(v, z)) return rc2;
        return use_mlp ? mlp_apply_impl(mlp, h, v, z, DG_F64, 1, s) : 0;
      };
    // the outer operator in double-float; once its FGMRES stops, the true residual with the FP64 operator
    // decides, and the solve continues in FP64 from the current x if that residual is still above tol
    c.f64x = o->outer_precision == 0;
    for (bool first = true;; first = false) {
      Result part;
      rc = fgmres<double>(c, P, bcopy, x_dev, false, V64, V64 + (size_t)(mo + 1) * n, mo, tol,
                          maxit - res.iterations, 1 << 20, true, &part, {}, P0);
      res.iterations += part.iterations;
      res.res = part.res;
      res.converged = part.converged;
      if (first) res.beta0 = part.beta0;
      if (rc || !part.converged || !c.f64x) break;
      c.f64x = false;
      double* r64 = V64;  // the basis is free between calls
      if ((rc = apply_A<double>(c, x_dev, r64))) break;
      dgb::sub<double><<<c.red_blocks, dgb::RED_THREADS, 0, s>>>(bcopy, r64, r64, n);
      double rn2;
      if ((rc = dots<double>(c, r64, 1, r64, &rn2))) break;
      res.res = std::sqrt(rn2);
      res.converged = res.res <= tol;
      if (res.converged || res.iterations >= maxit) break;
    }
  }
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (st) {
    st->status = rc ? rc : (res.converged ? DG_OK : DG_ERR_NOT_CONVERGED);
    st->iterations = res.iterations;
    st->inner_iterations = inner_total;
    st->applies_f64 = c.applies64;
    st->applies_f32 = c.applies32;
    st->rel_residual = res.res / (bnorm > 0 ? bnorm : 1.0);
    st->seconds = secs;
    st->fallback = fallback;
  }
  if (rc) return rc;
  if (!res.converged) {
    set_error("dg_solve: not converged (relative residual " + std::to_string(res.res / (bnorm > 0 ? bnorm : 1.0)) +
              ")");
    return DG_ERR_NOT_CONVERGED;
  }
  return DG_OK;
}

}  // extern "C"
