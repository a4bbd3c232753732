// dg_eig.h -- eigen-decomposition of small real non-symmetric matrices (host code, n <= 16).
//
// Used by the fast-diagonalisation block-Jacobi preconditioner: on an axis-parallel cell with per-cell
// coefficients, the diagonal block of the operator is a Kronecker sum of three 1D operators (one per axis), so
// its inverse follows from their eigen-decompositions A_r = V_r diag(lambda_r) V_r^{-1}.
//
// Method: Householder reduction to upper Hessenberg form, then complex single-shift QR iterations with
// Wilkinson shifts (Givens rotations on the active block, deflation on negligible subdiagonal entries) to the
// Schur form A = Q T Q^H; the eigenvectors of the triangular T by back substitution, mapped back with Q; and
// V^{-1} by Gauss-Jordan elimination with partial pivoting; when every eigenvalue is real, the same
// decomposition in real arithmetic (real_decomposition).  Plain C++ (no CUDA), so that a host test can check it
// against a library eigen-solver.
#pragma once

#include <cmath>
#include <complex>
#include <utility>

namespace dge {

using cd = std::complex<double>;

// A: row-major n x n real.  Outputs (row-major n x n): V (columns are eigenvectors, unit 2-norm), Vinv, and lam.
// Returns false when the QR iteration does not converge or V is numerically singular (cond > 1e12).
inline bool eig_general(int n, const double* A, cd* V, cd* Vinv, cd* lam) {
  constexpr int NMAX = 16;
  if (n < 1 || n > NMAX) return false;
  cd H[NMAX][NMAX], Q[NMAX][NMAX];
  double anorm = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      H[i][j] = A[i * n + j];
      Q[i][j] = i == j ? 1.0 : 0.0;
      anorm = std::fmax(anorm, std::fabs(A[i * n + j]));
    }
  if (!(anorm > 0.0) || !std::isfinite(anorm)) return false;
  // Householder reduction to Hessenberg form: H = P H P, Q = Q P with P = I - 2 v v^H
  for (int k = 0; k + 2 < n; ++k) {
    double xn = 0.0;
    for (int i = k + 1; i < n; ++i) xn += std::norm(H[i][k]);
    xn = std::sqrt(xn);
    if (xn == 0.0) continue;
    cd v[NMAX];
    const cd x0 = H[k + 1][k];
    const cd phase = std::abs(x0) > 0.0 ? x0 / std::abs(x0) : cd(1.0);
    for (int i = 0; i < n; ++i) v[i] = 0.0;
    for (int i = k + 1; i < n; ++i) v[i] = H[i][k];
    v[k + 1] += phase * xn;
    double vn = 0.0;
    for (int i = k + 1; i < n; ++i) vn += std::norm(v[i]);
    vn = std::sqrt(vn);
    if (vn == 0.0) continue;
    for (int i = k + 1; i < n; ++i) v[i] /= vn;
    for (int j = 0; j < n; ++j) {  // H = (I - 2 v v^H) H
      cd s = 0.0;
      for (int i = k + 1; i < n; ++i) s += std::conj(v[i]) * H[i][j];
      for (int i = k + 1; i < n; ++i) H[i][j] -= 2.0 * v[i] * s;
    }
    for (int i = 0; i < n; ++i) {  // H = H (I - 2 v v^H), Q = Q (I - 2 v v^H)
      cd s = 0.0, t = 0.0;
      for (int j = k + 1; j < n; ++j) {
        s += H[i][j] * v[j];
        t += Q[i][j] * v[j];
      }
      for (int j = k + 1; j < n; ++j) {
        H[i][j] -= 2.0 * s * std::conj(v[j]);
        Q[i][j] -= 2.0 * t * std::conj(v[j]);
      }
    }
    for (int i = k + 2; i < n; ++i) H[i][k] = 0.0;
  }
  // shifted QR iterations on the active block [lo, hi]
  const double eps = 1e-15;
  int hi = n - 1, iter = 0, total = 0;
  while (hi > 0) {
    int lo = hi;
    while (lo > 0) {
      const double sub = std::abs(H[lo][lo - 1]);
      if (sub <= eps * (std::abs(H[lo][lo]) + std::abs(H[lo - 1][lo - 1])) || sub <= 1e-300 * anorm) {
        H[lo][lo - 1] = 0.0;
        break;
      }
      --lo;
    }
    if (lo == hi) {  // H[hi][hi] has converged
      --hi;
      iter = 0;
      continue;
    }
    if (++total > 100 * n) return false;
    ++iter;
    // Wilkinson shift: the eigenvalue of the trailing 2 x 2 block nearer to H[hi][hi] (an exceptional shift
    // every 10 iterations without deflation)
    cd mu;
    if (iter % 10 == 0) {
      mu = H[hi][hi] + 0.75 * std::abs(H[hi][hi - 1]);
    } else {
      const cd a = H[hi - 1][hi - 1], b = H[hi - 1][hi], c = H[hi][hi - 1], d = H[hi][hi];
      const cd tr = a + d, det = a * d - b * c;
      const cd disc = std::sqrt(tr * tr - 4.0 * det);
      const cd l1 = 0.5 * (tr + disc), l2 = 0.5 * (tr - disc);
      mu = std::abs(l1 - d) < std::abs(l2 - d) ? l1 : l2;
    }
    // one QR step on H[lo..hi][lo..hi] - mu I with Givens rotations, applied to the whole matrix (rows lo..hi of
    // columns lo..n-1, columns lo..hi of rows 0..hi) and accumulated in Q
    for (int i = lo; i <= hi; ++i) H[i][i] -= mu;
    double gc[NMAX];
    cd gs[NMAX];
    for (int k = lo; k < hi; ++k) {
      const cd a = H[k][k], b = H[k + 1][k];
      const double r = std::sqrt(std::norm(a) + std::norm(b));
      double c;
      cd s;
      if (r == 0.0) {
        c = 1.0;
        s = 0.0;
      } else if (std::abs(a) == 0.0) {
        c = 0.0;
        s = std::conj(b) / std::abs(b);
      } else {
        c = std::abs(a) / r;
        s = (a / std::abs(a)) * std::conj(b) / r;
      }
      gc[k] = c;
      gs[k] = s;
      for (int j = k; j < n; ++j) {  // rows k, k+1: [c s; -conj(s) c]
        const cd x = H[k][j], y = H[k + 1][j];
        H[k][j] = c * x + s * y;
        H[k + 1][j] = -std::conj(s) * x + c * y;
      }
    }
    for (int k = lo; k < hi; ++k) {  // columns k, k+1 with the conjugate transposed rotation
      const double c = gc[k];
      const cd s = gs[k];
      for (int i = 0; i <= std::min(hi, k + 2); ++i) {
        const cd x = H[i][k], y = H[i][k + 1];
        H[i][k] = c * x + std::conj(s) * y;
        H[i][k + 1] = -s * x + c * y;
      }
      for (int i = 0; i < n; ++i) {
        const cd x = Q[i][k], y = Q[i][k + 1];
        Q[i][k] = c * x + std::conj(s) * y;
        Q[i][k + 1] = -s * x + c * y;
      }
    }
    for (int i = lo; i <= hi; ++i) H[i][i] += mu;
  }
  for (int k = 0; k < n; ++k) lam[k] = H[k][k];
  // eigenvectors of the triangular T = H: (T - lam_k I) y = 0 with y_k = 1, y_j = 0 for j > k
  double tnorm = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = i; j < n; ++j) tnorm = std::fmax(tnorm, std::abs(H[i][j]));
  for (int k = 0; k < n; ++k) {
    cd y[NMAX];
    for (int j = 0; j < n; ++j) y[j] = 0.0;
    y[k] = 1.0;
    for (int j = k - 1; j >= 0; --j) {
      cd s = 0.0;
      for (int l = j + 1; l <= k; ++l) s += H[j][l] * y[l];
      cd den = H[j][j] - lam[k];
      if (std::abs(den) < 1e-14 * tnorm) den = 1e-14 * tnorm;
      y[j] = -s / den;
    }
    double nv = 0.0;
    for (int i = 0; i < n; ++i) {
      cd s = 0.0;
      for (int j = 0; j <= k; ++j) s += Q[i][j] * y[j];
      V[i * n + k] = s;
      nv += std::norm(s);
    }
    nv = std::sqrt(nv);
    for (int i = 0; i < n; ++i) V[i * n + k] /= nv;
  }
  // V^{-1} by Gauss-Jordan with partial pivoting
  cd M[NMAX][2 * NMAX];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j) M[i][j] = j < n ? V[i * n + j] : (j - n == i ? cd(1.0) : cd(0.0));
  for (int p = 0; p < n; ++p) {
    int piv = p;
    for (int i = p + 1; i < n; ++i)
      if (std::abs(M[i][p]) > std::abs(M[piv][p])) piv = i;
    if (!(std::abs(M[piv][p]) > 1e-13)) return false;
    if (piv != p)
      for (int j = 0; j < 2 * n; ++j) std::swap(M[p][j], M[piv][j]);
    const cd d = M[p][p];
    for (int j = 0; j < 2 * n; ++j) M[p][j] /= d;
    for (int i = 0; i < n; ++i) {
      if (i == p) continue;
      const cd f = M[i][p];
      if (f == cd(0.0)) continue;
      for (int j = 0; j < 2 * n; ++j) M[i][j] -= f * M[p][j];
    }
  }
  double vinv_max = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      Vinv[i * n + j] = M[i][j + n];
      vinv_max = std::fmax(vinv_max, std::abs(M[i][j + n]));
    }
  return vinv_max < 1e12;
}

// Real form of a decomposition from eig_general when every eigenvalue is real (|Im lambda| <= 1e-13 max |lambda|):
// each eigenvector column is rotated by the conjugate phase of its largest entry (a real simple eigenvalue has a
// real eigenvector up to a complex factor), which must leave imaginary parts below 1e-9 of the column's norm; the
// real parts, renormalised to unit 2-norm, give Vr, and Wr = Vr^{-1} by Gauss-Jordan with partial pivoting.
// Returns false (outputs unspecified) when an eigenvalue is complex, a column does not become real (a defective
// or repeated eigenvalue with a complex basis of its eigenspace), or Vr is numerically singular.
inline bool real_decomposition(int n, const cd* V, const cd* lam, double* Vr, double* Wr, double* lr) {
  constexpr int NMAX = 16;
  if (n < 1 || n > NMAX) return false;
  double lmax = 0.0;
  for (int k = 0; k < n; ++k) lmax = std::fmax(lmax, std::abs(lam[k]));
  for (int k = 0; k < n; ++k) {
    if (std::fabs(lam[k].imag()) > 1e-13 * lmax) return false;
    lr[k] = lam[k].real();
  }
  for (int k = 0; k < n; ++k) {
    int big = 0;
    for (int i = 1; i < n; ++i)
      if (std::abs(V[i * n + k]) > std::abs(V[big * n + k])) big = i;
    const double vb = std::abs(V[big * n + k]);
    if (!(vb > 0.0)) return false;
    const cd rot = std::conj(V[big * n + k]) / vb;
    double nrm = 0.0, imax = 0.0;
    for (int i = 0; i < n; ++i) {
      const cd v = V[i * n + k] * rot;
      Vr[i * n + k] = v.real();
      nrm += v.real() * v.real();
      imax = std::fmax(imax, std::fabs(v.imag()));
    }
    nrm = std::sqrt(nrm);
    if (imax > 1e-9 * nrm) return false;
    for (int i = 0; i < n; ++i) Vr[i * n + k] /= nrm;
  }
  double M[NMAX][2 * NMAX];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j) M[i][j] = j < n ? Vr[i * n + j] : (j - n == i ? 1.0 : 0.0);
  for (int p = 0; p < n; ++p) {
    int piv = p;
    for (int i = p + 1; i < n; ++i)
      if (std::fabs(M[i][p]) > std::fabs(M[piv][p])) piv = i;
    if (!(std::fabs(M[piv][p]) > 1e-13)) return false;
    if (piv != p)
      for (int j = 0; j < 2 * n; ++j) std::swap(M[p][j], M[piv][j]);
    const double d = M[p][p];
    for (int j = 0; j < 2 * n; ++j) M[p][j] /= d;
    for (int i = 0; i < n; ++i) {
      if (i == p) continue;
      const double f = M[i][p];
      if (f == 0.0) continue;
      for (int j = 0; j < 2 * n; ++j) M[i][j] -= f * M[p][j];
    }
  }
  double wmax = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      Wr[i * n + j] = M[i][j + n];
      wmax = std::fmax(wmax, std::fabs(M[i][j + n]));
    }
  return wmax < 1e12;
}

}  // namespace dge
