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
#include <vector>

#include "dg_blas.cuh"
#include "dg_internal.h"

namespace dgi {

bool mlp_matches(const dg_mlp* m, const dg_handle* h);
int mlp_apply_impl(dg_mlp* m, const dg_handle* h, const void* r, void* z, int32_t precision, int accumulate,
                   cudaStream_t s);

namespace {

struct Ctx {
  dg_handle* h;
  cudaStream_t s;
  size_t n;
  double* part;   // MAX_ROWS rows of RED_BLOCKS block sums
  double* hdev;   // 64 results of the first projection (and of plain dot products)
  double* ydev;   // 64 coefficients of the solution update
  double* h2dev;  // 64 results of the second projection, then w . w
  double* hhost;  // pinned, 256
  int applies64 = 0, applies32 = 0;
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

// the per-thread partial sums of a basis pass take up to MAX_ROWS columns of shared memory (128 KB in FP64),
// beyond the 48 KB (static plus dynamic) a launch gets without opting in: opt in once per kernel
template <typename T, bool UPDATE>
constexpr int dots_loads() { return UPDATE ? dgb::FUSED_LOADS : dgb::PASS_LOADS; }

template <typename T, int W, bool UPDATE>
int basis_smem_attr() {
  static bool done = false;
  if (done) return 0;
  if (int rc = cuda_check(cudaFuncSetAttribute(dgb::basis_dots<T, W, UPDATE, dgb::PASS_MINB, dots_loads<T, UPDATE>()>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               dgb::MAX_ROWS * dgb::RED_THREADS * (int)sizeof(T)),
                          "basis pass shared memory"))
    return rc;
  done = true;
  return 0;
}

// dst[q] = V_q . w (q < nv) on the device; with UPDATE, w <- w - sum_q h[q] V_q first and dst[nv] = w . w
template <typename T, bool UPDATE>
int basis_dots(Ctx& c, const T* V, int nv, const double* h, T* w, double* dst) {
  const int rows = nv + (UPDATE ? 1 : 0);
  const size_t smem = (size_t)rows * dgb::RED_THREADS * sizeof(T);
  if (packable<T>(c.n, {V, w})) {
    constexpr int W = 16 / sizeof(T);
    if (int rc = basis_smem_attr<T, W, UPDATE>()) return rc;
    dgb::basis_dots<T, W, UPDATE, dgb::PASS_MINB, dots_loads<T, UPDATE>()>
        <<<dgb::PASS_BLOCKS, dgb::RED_THREADS, smem, c.s>>>(V, c.n, nv, h, w, c.n / W, c.part);
  } else {
    if (int rc = basis_smem_attr<T, 1, UPDATE>()) return rc;
    dgb::basis_dots<T, 1, UPDATE, dgb::PASS_MINB, dots_loads<T, UPDATE>()>
        <<<dgb::PASS_BLOCKS, dgb::RED_THREADS, smem, c.s>>>(V, c.n, nv, h, w, c.n, c.part);
  }
  dgb::mdot_final<<<rows, dgb::RED_THREADS, 0, c.s>>>(c.part, dgb::PASS_BLOCKS, dst);
  return cuda_check(cudaGetLastError(), "basis dot kernels");
}

// w <- alpha (w - sum_q h[q] V_q), alpha the inverse norm of the result from h when normalise
template <typename T>
int basis_update(Ctx& c, const T* V, int nv, const double* h, bool normalise, T* w) {
  if (packable<T>(c.n, {V, w})) {
    constexpr int W = 16 / sizeof(T);
    dgb::basis_update<T, W, dgb::PASS_MINB, dgb::PASS_LOADS><<<dgb::PASS_BLOCKS, dgb::RED_THREADS, 0, c.s>>>(V, c.n, nv, h, normalise, w, c.n / W);
  } else {
    dgb::basis_update<T, 1, dgb::PASS_MINB, dgb::PASS_LOADS><<<dgb::PASS_BLOCKS, dgb::RED_THREADS, 0, c.s>>>(V, c.n, nv, h, normalise, w, c.n);
  }
  return cuda_check(cudaGetLastError(), "basis update");
}

// x <- x + sum_q y[q] Z_q, y on the device
template <typename T>
int lincomb_add(Ctx& c, const T* Z, int nv, const double* y, T* x) {
  if (packable<T>(c.n, {Z, x})) {
    constexpr int W = 16 / sizeof(T);
    dgb::lincomb_add<T, W, dgb::PASS_MINB, dgb::PASS_LOADS><<<dgb::PASS_BLOCKS, dgb::RED_THREADS, 0, c.s>>>(Z, c.n, nv, y, x, c.n / W);
  } else {
    dgb::lincomb_add<T, 1, dgb::PASS_MINB, dgb::PASS_LOADS><<<dgb::PASS_BLOCKS, dgb::RED_THREADS, 0, c.s>>>(Z, c.n, nv, y, x, c.n);
  }
  return cuda_check(cudaGetLastError(), "solution update");
}

// out_host[q] = V_q . w for q < nv (synchronises)
template <typename T>
int dots(Ctx& c, const T* V, int nv, const T* w, double* out_host) {
  if (int rc = basis_dots<T, false>(c, V, nv, nullptr, const_cast<T*>(w), c.hdev)) return rc;
  if (int rc = cuda_check(cudaMemcpyAsync(c.hhost, c.hdev, nv * sizeof(double), cudaMemcpyDeviceToHost, c.s),
                          "dot copy"))
    return rc;
  if (int rc = cuda_check(cudaStreamSynchronize(c.s), "dot sync")) return rc;
  std::memcpy(out_host, c.hhost, nv * sizeof(double));
  return 0;
}

template <typename T>
int scale(Ctx& c, T* v, double a) {
  dgb::scale_copy<T, T><<<dgb::RED_BLOCKS, dgb::RED_THREADS, 0, c.s>>>(v, v, a, c.n);
  return cuda_check(cudaGetLastError(), "scale");
}

// y = A x in precision T
template <typename T>
int apply_A(Ctx& c, const T* x, T* y);
template <>
int apply_A<double>(Ctx& c, const double* x, double* y) {
  ++c.applies64;
  return launch_apply_f64(c.h, x, y, 0, 3, c.s);
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

// Flexible GMRES(m) on A x = b in precision T with right preconditioner M (nullptr: none).
// V: (m+1) n, Z: m n (ignored without M).  x holds the initial guess unless x0_zero.
template <typename T>
int fgmres(Ctx& c, const std::function<int(const T*, T*)>& M, const T* b, T* x, bool x0_zero, T* V, T* Z, int m,
           double tol_abs, int maxit, int max_cycles, bool true_residual_check, Result* out,
           const std::function<void(double, double)>& cycle_hook = {},
           const std::function<int(const T*, T*)>& M0 = {}) {
  const size_t n = c.n;
  std::vector<double> H((m + 1) * m), cs(m), sn(m), g(m + 1), hv(m + 2), h2(m + 2), y(m);
  Result r;
  for (int cycle = 0; cycle < max_cycles; ++cycle) {
    T* v0 = V;
    if (x0_zero && cycle == 0) {
      if (int rc = cuda_check(cudaMemcpyAsync(v0, b, n * sizeof(T), cudaMemcpyDeviceToDevice, c.s), "copy b"))
        return rc;
    } else {
      if (int rc = apply_A<T>(c, x, v0)) return rc;
      dgb::sub<T><<<dgb::RED_BLOCKS, dgb::RED_THREADS, 0, c.s>>>(b, v0, v0, n);
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
    if (int rc = scale<T>(c, v0, 1.0 / beta)) return rc;
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int jend = 0;
    bool est_conv = false;
    for (int j = 0; j < m; ++j) {
      T* vj = V + (size_t)j * n;
      T* zj = (M || M0) ? Z + (size_t)j * n : vj;
      T* w = V + (size_t)(j + 1) * n;
      if (j == 0 && M0) {
        if (int rc = M0(vj, zj)) return rc;
      } else if (M) {
        if (int rc = M(vj, zj)) return rc;
      } else if (M0) {
        if (int rc = cuda_check(cudaMemcpyAsync(zj, vj, n * sizeof(T), cudaMemcpyDeviceToDevice, c.s), "copy v"))
          return rc;
      }
      if (int rc = apply_A<T>(c, zj, w)) return rc;
      // classical Gram-Schmidt, twice, in three passes over the basis with the coefficients kept on the device:
      // h = V^T w; then w -= V h together with h2 = V^T w and ||w||^2; then w = (w - V h2) / ||w - V h2||, the
      // norm by Pythagoras.  One synchronisation fetches h and h2 for the Hessenberg column.
      if (int rc = basis_dots<T, false>(c, V, j + 1, nullptr, w, c.hdev)) return rc;
      if (int rc = basis_dots<T, true>(c, V, j + 1, c.hdev, w, c.h2dev)) return rc;
      if (int rc = basis_update<T>(c, V, j + 1, c.h2dev, true, w)) return rc;
      if (int rc = cuda_check(cudaMemcpyAsync(c.hhost, c.hdev, (j + 1) * sizeof(double), cudaMemcpyDeviceToHost,
                                              c.s), "h copy"))
        return rc;
      if (int rc = cuda_check(cudaMemcpyAsync(c.hhost + 128, c.h2dev, (j + 2) * sizeof(double),
                                              cudaMemcpyDeviceToHost, c.s), "h2 copy"))
        return rc;
      if (int rc = cuda_check(cudaStreamSynchronize(c.s), "Arnoldi sync")) return rc;
      std::memcpy(hv.data(), c.hhost, (j + 1) * sizeof(double));
      std::memcpy(h2.data(), c.hhost + 128, (j + 2) * sizeof(double));
      double s2 = h2[j + 1];  // ||w||^2 after the first projection
      for (int i = 0; i <= j; ++i) {
        H[i * m + j] = hv[i] + h2[i];
        s2 -= h2[i] * h2[i];
      }
      const double hn = std::sqrt(std::max(s2, 0.0));
      if (!std::isfinite(hn)) {
        set_error("FGMRES: non-finite Arnoldi vector");
        return DG_ERR_NAN;
      }
      H[(j + 1) * m + j] = hn;  // (w was scaled by 1 / hn on the device when hn > 0)
      // Givens rotations
      for (int i = 0; i < j; ++i) {
        const double a = H[i * m + j], bb = H[(i + 1) * m + j];
        H[i * m + j] = cs[i] * a + sn[i] * bb;
        H[(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
      }
      const double a = H[j * m + j], bb = H[(j + 1) * m + j];
      const double rr = std::hypot(a, bb);
      cs[j] = rr > 0 ? a / rr : 1.0;
      sn[j] = rr > 0 ? bb / rr : 0.0;
      H[j * m + j] = rr;
      H[(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++r.iterations;
      jend = j + 1;
      r.res = std::fabs(g[j + 1]);
      if (r.res <= tol_abs) {
        est_conv = true;
        break;
      }
      if (r.iterations >= maxit || hn == 0.0) break;
    }
    // y = H^{-1} g (upper triangular), x += Z y
    for (int i = jend - 1; i >= 0; --i) {
      double acc = g[i];
      for (int k = i + 1; k < jend; ++k) acc -= H[i * m + k] * y[k];
      y[i] = H[i * m + i] != 0 ? acc / H[i * m + i] : 0.0;
    }
    std::memcpy(c.hhost, y.data(), jend * sizeof(double));
    if (int rc = cuda_check(cudaMemcpyAsync(c.ydev, c.hhost, jend * sizeof(double), cudaMemcpyHostToDevice, c.s),
                            "y copy"))
      return rc;
    const T* basis = (M || M0) ? Z : V;
    if (int rc = lincomb_add<T>(c, basis, jend, c.ydev, x)) return rc;
    if (int rc = cuda_check(cudaStreamSynchronize(c.s), "solution update")) return rc;
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
    e = cudaMallocHost(&h->ws_host, 256 * sizeof(double));
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
  const int mo = o->outer_restart > 0 ? o->outer_restart : 10;
  if (m > 60 || mo > 60 || (o->mode != DG_SOLVE_FP64 && o->mode != DG_SOLVE_MIXED) ||
      (o->inner_block_precision < 0 || o->inner_block_precision > 2) ||
      (o->preconditioner != DG_PRECOND_NONE && o->preconditioner != DG_PRECOND_BLOCK_JACOBI &&
       o->preconditioner != DG_PRECOND_MLP && o->preconditioner != DG_PRECOND_BJ_MLP) ||
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
      !h->fdm64) {
    set_error("dg_solve: block-Jacobi requested but dg_precond_setup was not called");
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
  // MLP preconditioner, with a switch to block-Jacobi when a cycle stagnates (if blocks exist)
  bool use_mlp = o->preconditioner == DG_PRECOND_MLP || o->preconditioner == DG_PRECOND_BJ_MLP;
  const bool with_bj = o->preconditioner == DG_PRECOND_BJ_MLP;
  // placement 1: the network only acts on the first direction of each (outer) FGMRES cycle, where the
  // direction is the true residual r / ||r|| -- the kind of input it was trained on
  const bool first_only = use_mlp && o->mlp_placement == 1;
  int fallback = 0;
  dg_mlp* mlp = const_cast<dg_mlp*>(o->mlp);
  auto maybe_fallback = [&](double start, double end) {
    if (use_mlp && o->fallback_ratio > 0 && (h->bj64 || h->fdm64) && start > 0 && end > o->fallback_ratio * start) {
      use_mlp = false;
      fallback = 1;
    }
  };
  // workspace: reductions, r/b copy, FP64 basis (V, Z), FP32 basis for the inner solve
  const size_t small = (size_t)dgb::RED_BLOCKS * dgb::MAX_ROWS + 192;
  size_t v64 = 0, v32 = 0;
  if (o->mode == DG_SOLVE_FP64) {
    v64 = (size_t)(m + 1 + (pc ? m : 0)) * n;
  } else {
    v64 = (size_t)(2 * mo + 1) * n;
    v32 = (size_t)(m + 1 + (pc ? m : 0) + 2) * n;
  }
  const size_t bytes = (small + n + v64) * sizeof(double) + v32 * sizeof(float) + 256;
  if (int rc = ensure_ws(h, bytes)) return rc;
  Ctx c;
  c.h = h;
  c.s = s;
  c.n = n;
  double* base = static_cast<double*>(h->ws);
  c.part = base;
  c.hdev = base + (size_t)dgb::RED_BLOCKS * 64;
  c.ydev = c.hdev + 64;
  c.h2dev = c.ydev + 64;
  double* bcopy = base + small;
  double* V64 = bcopy + n;
  float* f32 = reinterpret_cast<float*>(V64 + v64);
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
    if (pc && !first_only)
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
    float* V32 = f32;
    float* Z32 = V32 + (size_t)(m + 1) * n;
    float* rhs32 = Z32 + (pc ? (size_t)m * n : 0);
    float* e32 = rhs32 + n;
    std::function<int(const float*, float*)> M32;
    // block-Jacobi inside the FP32 inner solve: the FP16 blocks (half the bytes of this HBM-bound product) unless
    // the caller asked for the FP32 ones
    auto bj_inner = [&](const float* r, float* z) {
      if (o->inner_block_precision == 1) return precond_bj_f32(h, r, z, s);
      if (o->inner_block_precision == 0 && h->fdm) return precond_fdm_f32(h, r, z, s);
      return precond_bj_f16(h, r, z, s);
    };
    if (pc)
      M32 = [&](const float* r, float* z) {
        if (!use_mlp || first_only) return with_bj || !use_mlp ? bj_inner(r, z)
                                                             : cuda_check(cudaMemcpyAsync(z, r, n * sizeof(float),
                                                                                          cudaMemcpyDeviceToDevice, s),
                                                                          "copy");
        if (!with_bj) return mlp_apply_impl(mlp, h, r, z, DG_F32, 0, s);
        int e2 = bj_inner(r, z);
        return e2 ? e2 : mlp_apply_impl(mlp, h, r, z, DG_F32, 1, s);
      };
    std::function<int(const double*, double*)> P = [&](const double* v, double* z) -> int {
      dgb::scale_copy<double, float><<<dgb::RED_BLOCKS, dgb::RED_THREADS, 0, s>>>(v, rhs32, 1.0, n);
      cudaMemsetAsync(e32, 0, n * sizeof(float), s);
      Result ri;
      double vn2;
      int rc2 = dots<float>(c, rhs32, 1, rhs32, &vn2);
      if (rc2) return rc2;
      rc2 = fgmres<float>(c, M32, rhs32, e32, true, V32, Z32, m, o->inner_rtol * std::sqrt(vn2), m, 1, false, &ri);
      if (rc2) return rc2;
      maybe_fallback(ri.beta0, ri.res);
      inner_total += ri.iterations;
      dgb::scale_copy<float, double><<<dgb::RED_BLOCKS, dgb::RED_THREADS, 0, s>>>(e32, z, 1.0, n);
      return cuda_check(cudaGetLastError(), "inner solve casts");
    };
    std::function<int(const double*, double*)> P0;
    if (first_only)
      P0 = [&](const double* v, double* z) -> int {
        // the inner solve, plus the network's correction of the true residual direction
        if (int rc2 = P(v, z)) return rc2;
        return use_mlp ? mlp_apply_impl(mlp, h, v, z, DG_F64, 1, s) : 0;
      };
    rc = fgmres<double>(c, P, bcopy, x_dev, false, V64, V64 + (size_t)(mo + 1) * n, mo, tol, maxit, 1 << 20, true,
                        &res, {}, P0);
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
