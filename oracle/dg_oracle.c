/*
 * dg_oracle.c -- plain, slow, FP64 CPU oracle for the weighted symmetric interior
 * penalty (WSIPG) DG operator of Muething, Piatkowski & Bastian (arXiv 1711.10885).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is used by the test suite, by the
 * smoke check and by the CPU-baseline leg of the benchmark.  The product path
 * (the CUDA library) never links, loads or calls it, and it shares no code,
 * headers or tables with the library.
 *
 * What it computes (Sec. 2, eq. blf and the right hand side functional l_h):
 *   (A u)_i = a_h(u, phi_i),   F_i = l_h(phi_i)
 * for every basis function phi_i of the DG space Q_k on an axis-parallel
 * uniform cuboid mesh, by DIRECT quadrature: at every quadrature point the
 * finite element function and its gradient are summed over all (k+1)^3 basis
 * functions, and every integral is accumulated point by point for every test
 * function.  No sum factorisation, no 1D factorisation reuse (Sec. 3 is the
 * method being checked; this is the definition it must reproduce).
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *  - weighted average {v}_w = w- v- + w+ v+ (the printed minus sign
 *    contradicts w- + w+ = 1 and the convex-average definition it cites);
 *  - orthonormal shifted Legendre basis on the reference interval [0,1]:
 *    theta_j(x) = sqrt(2j+1) P_j(2x-1)  ("L2-orthogonal Legendre", Sec. 2);
 *  - tensor Gauss-Legendre rule with m points per direction (Sec. 3.1);
 *  - diffusion constant per cell, either scalar D_T * I or a full symmetric
 *    tensor D_T (the "tensor-valued diffusion coefficients" of Sec. 5.1), with
 *    delta = nu^T D nu in the face weights and the penalty; constant c; and
 *    either a constant b (Problem A) or b given at the quadrature points (the
 *    Taylor-Green transport problem of Sec. 5.3, evaluated by the caller);
 *  - coefficients given at the quadrature points instead (Problem B of Sec. 5.1:
 *    "coefficients that are polynomials in the coordinates", evaluated by the
 *    caller): D at the volume points and at each cell's face points, c at the
 *    volume points; on a face, delta, the weights and the penalty are then
 *    taken point by point from the two cells' tensors at that point;
 *  - geometry: axis-parallel cells, an affine image of the structured grid
 *    (every cell T = lo + J (ic + [0,1]^3) with one constant Jacobian J, as in
 *    Problem B of Sec. 5.1), or multilinear cells (Problem C): each cell the
 *    trilinear image of [0,1]^3 through its 8 corner vertices, J = J(x) taken
 *    at every quadrature point; gradients map as J^{-T}, the volume element is
 *    |det J|, a face across reference axis r has the unit normal
 *    nu = J^{-T} e_r / |J^{-T} e_r| and the area element |det J| |J^{-T} e_r|;
 *    the penalty's |F| and |T| are the face area and cell volume (integrals of
 *    those elements by the same rule);
 *  - a periodic axis makes its two end faces interior faces between the last
 *    and the first cell (Sec. 5.1, 5.3);
 *  - penalty gamma_F = <delta-,delta+> * sigma * |F| / min(|T-|,|T+|) where the
 *    caller passes sigma (the paper's alpha*p*(p+d-1), or 2k(k+1));
 *    on boundary faces <delta-,delta+> -> delta- and min|T| -> |T-|;
 *  - boundary faces are Dirichlet unless a side is declared Neumann (no term
 *    in a_h, -(j, v) in l_h with the total flux j = (b u - D grad u) . nu) or
 *    outflow (only the upwind flux Phi(u, 0, b_nu) in a_h, nothing in l_h), as
 *    the face sets F^D, F^N, F^O of eq. blf and l_h split them; interior faces
 *    are oriented from the cell with the lower index along the face normal (T-)
 *    to the upper (T+);
 *  - upwind tie b_nu = 0 takes the u- branch (value 0 either way).
 *
 * Layouts (shared with the library only as a documented interface):
 *   cells lexicographic, x fastest: cell = ix + nx*(iy + ny*iz);
 *   DOF within a cell: J = j1 + n*(j2 + n*j3), n = k+1 (x-degree fastest);
 *   volume quadrature points within a cell: q = i1 + m*(i2 + m*i3);
 *   boundary side s = 2*dir + (0 lower | 1 upper); its faces enumerate the
 *   cells of that boundary layer lexicographically in the two tangential
 *   cell indices (lower axis fastest), and the m*m face points of each face
 *   with the lower tangential axis fastest.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* 1D ingredients                                                      */
/* ------------------------------------------------------------------ */

/* Legendre polynomial P_j(t) and derivative on [-1,1] by the three-term
 * (Bonnet) recurrence; returns values for j = 0..jmax. */
static void legendre_all(int jmax, double t, double* P, double* dP) {
  P[0] = 1.0;
  dP[0] = 0.0;
  if (jmax >= 1) {
    P[1] = t;
    dP[1] = 1.0;
  }
  for (int j = 1; j < jmax; ++j) {
    P[j + 1] = ((2.0 * j + 1.0) * t * P[j] - j * P[j - 1]) / (j + 1.0);
    /* P'_{j+1} = P'_{j-1} + (2j+1) P_j */
    dP[j + 1] = dP[j - 1] + (2.0 * j + 1.0) * P[j];
  }
}

/* Gauss-Legendre rule with m points on [0,1] (ascending), Sec. 3.1.  Newton
 * iteration on P_m from the Chebyshev-like initial guesses. */
int oracle_gauss_legendre(int m, double* x, double* w) {
  if (m < 1 || m > 64) return -1;
  double P[66], dP[66];
  for (int i = 0; i < m; ++i) {
    double t = -cos(M_PI * (i + 0.75) / (m + 0.5));
    for (int it = 0; it < 100; ++it) {
      legendre_all(m, t, P, dP);
      double dt = P[m] / dP[m];
      t -= dt;
      if (fabs(dt) < 1e-17) break;
    }
    legendre_all(m, t, P, dP);
    x[i] = 0.5 * (1.0 + t);
    w[i] = 1.0 / ((1.0 - t * t) * dP[m] * dP[m]); /* = (2/((1-t^2)P'^2)) / 2 */
  }
  return 0;
}

/* Orthonormal shifted Legendre basis on [0,1] and its derivative, j = 0..k. */
void oracle_basis_1d(int k, double x, double* val, double* der) {
  double P[66], dP[66];
  legendre_all(k, 2.0 * x - 1.0, P, dP);
  for (int j = 0; j <= k; ++j) {
    double s = sqrt(2.0 * j + 1.0);
    val[j] = s * P[j];
    der[j] = 2.0 * s * dP[j];
  }
}

/* ------------------------------------------------------------------ */
/* Problem description                                                 */
/* ------------------------------------------------------------------ */

typedef struct {
  int n[3];            /* cells per direction                               */
  double lo[3], hi[3]; /* domain [lo, hi]                                    */
  int k;               /* polynomial degree; n = k+1 shape functions / dir   */
  int m;               /* Gauss points per direction                         */
  const double* D;     /* [ncells] scalar diffusion per cell                 */
  double b[3];         /* constant velocity                                  */
  double c;            /* reaction                                           */
  double sigma;        /* penalty factor, gamma = <d-,d+> sigma |F|/min|T|   */
  int periodic[3];     /* 1: the axis wraps around (its end faces are interior faces) */
  const double* b_vol;  /* NULL, or b at the volume points [ncells][m^3][3]          */
  const double* b_face; /* NULL, or b . nu_dir at each cell's face points [ncells][6][m^2] */
  const double* Dten;   /* NULL, or [ncells][6] diffusion tensor (xx, yy, zz, xy, xz, yz); replaces D */
  int affine;           /* 1: cells are lo + J (ic + [0,1]^3) with the Jacobian J below; 0: J = diag(h) */
  double J[3][3];
  const double* D_vol;  /* NULL, or the tensor at the volume points [ncells][m^3][6]            */
  const double* D_face; /* NULL, or the tensor at each cell's face points [ncells][6][m^2][6]   */
  const double* c_vol;  /* NULL, or c at the volume points [ncells][m^3]                      */
  int bc[6];            /* boundary type of side 2*dir + (0 lower | 1 upper): BC_DIRICHLET, BC_NEUMANN or
                           BC_OUTFLOW (eq. modelproblem: Gamma_D, Gamma_N, Gamma_O)                     */
  const double* vertices; /* NULL, or multilinear cells (Problem C of Sec. 5.1): the grid's vertex coordinates
                             [(n0+1)(n1+1)(n2+1)][3], vertex (i, j, l) at i + (n0+1)(j + (n1+1) l); cell (ix, iy,
                             iz) is the trilinear image of [0,1]^3 through its 8 corner vertices            */
} oracle_problem;

enum { BC_DIRICHLET = 0, BC_NEUMANN = 1, BC_OUTFLOW = 2 };

/* Full 3D tables at one set of points: phi[p*nb + J], grad[(p*nb + J)*3 + r]
 * are the reference-cube basis values and reference gradients. */
typedef struct {
  int np, nb;
  double* phi;
  double* grad;
  double* wgt; /* quadrature weight per point (reference measure) */
  double* xi;  /* local reference coordinates of each point in [0,1]^3, xi[p*3 + r] */
} table3d;

static void table_free(table3d* t) {
  free(t->phi);
  free(t->grad);
  free(t->wgt);
  free(t->xi);
}

/* Points given by three per-axis coordinate lists; point p = a + na*(b + nb_*c)
 * enumerates axis0 fastest.  A face is an axis list with one fixed entry. */
static int table_build(int k, const double* ax[3], const double* aw[3], const int na[3], table3d* t) {
  int n = k + 1;
  t->nb = n * n * n;
  t->np = na[0] * na[1] * na[2];
  t->phi = (double*)malloc(sizeof(double) * t->np * t->nb);
  t->grad = (double*)malloc(sizeof(double) * t->np * t->nb * 3);
  t->wgt = (double*)malloc(sizeof(double) * t->np);
  t->xi = (double*)malloc(sizeof(double) * t->np * 3);
  if (!t->phi || !t->grad || !t->wgt || !t->xi) return -1;
  double v[3][66], d[3][66];
  for (int p2 = 0; p2 < na[2]; ++p2)
    for (int p1 = 0; p1 < na[1]; ++p1)
      for (int p0 = 0; p0 < na[0]; ++p0) {
        int p = p0 + na[0] * (p1 + na[1] * p2);
        oracle_basis_1d(k, ax[0][p0], v[0], d[0]);
        oracle_basis_1d(k, ax[1][p1], v[1], d[1]);
        oracle_basis_1d(k, ax[2][p2], v[2], d[2]);
        t->wgt[p] = aw[0][p0] * aw[1][p1] * aw[2][p2];
        t->xi[3 * p + 0] = ax[0][p0];
        t->xi[3 * p + 1] = ax[1][p1];
        t->xi[3 * p + 2] = ax[2][p2];
        for (int j3 = 0; j3 < n; ++j3)
          for (int j2 = 0; j2 < n; ++j2)
            for (int j1 = 0; j1 < n; ++j1) {
              int J = j1 + n * (j2 + n * j3);
              size_t o = (size_t)p * t->nb + J;
              t->phi[o] = v[0][j1] * v[1][j2] * v[2][j3];
              t->grad[o * 3 + 0] = d[0][j1] * v[1][j2] * v[2][j3];
              t->grad[o * 3 + 1] = v[0][j1] * d[1][j2] * v[2][j3];
              t->grad[o * 3 + 2] = v[0][j1] * v[1][j2] * d[2][j3];
            }
      }
  return 0;
}

typedef struct {
  table3d vol;
  table3d face[6]; /* face s = 2*dir + side, side 0 at xi_dir = 0, side 1 at 1 */
  double J[3][3], Jinv[3][3];
  double vol_T;    /* |T| = |det J| */
  double nrm[3][3]; /* nrm[r]: unit normal of the faces across reference axis r, J^{-T} e_r / |J^{-T} e_r| */
  double area[3];  /* |F| of a face across reference axis r: |det J| |J^{-T} e_r| */
  int ncell;
} oracle_ctx;

static int ctx_build(const oracle_problem* pr, oracle_ctx* cx) {
  memset(cx, 0, sizeof(*cx));
  int m = pr->m;
  double* x = (double*)malloc(sizeof(double) * m);
  double* w = (double*)malloc(sizeof(double) * m);
  if (!x || !w || oracle_gauss_legendre(m, x, w)) return -1;
  static const double zero = 0.0, one = 1.0, unitw = 1.0;
  const double* ax[3] = {x, x, x};
  const double* aw[3] = {w, w, w};
  int na[3] = {m, m, m};
  if (table_build(pr->k, ax, aw, na, &cx->vol)) return -1;
  for (int dir = 0; dir < 3; ++dir)
    for (int side = 0; side < 2; ++side) {
      const double* fx[3] = {x, x, x};
      const double* fw[3] = {w, w, w};
      int fn[3] = {m, m, m};
      fx[dir] = side ? &one : &zero;
      fw[dir] = &unitw;
      fn[dir] = 1;
      if (table_build(pr->k, fx, fw, fn, &cx->face[2 * dir + side])) return -1;
    }
  free(x);
  free(w);
  /* the cell Jacobian: diag(h) for the axis-parallel mesh, else the given affine map */
  for (int a = 0; a < 3; ++a)
    for (int r = 0; r < 3; ++r)
      cx->J[a][r] = pr->affine ? pr->J[a][r] : (a == r ? (pr->hi[r] - pr->lo[r]) / pr->n[r] : 0.0);
  const double (*J)[3] = cx->J;
  double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
               J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  if (det == 0.0) return -1;
  /* inverse by cofactors */
  cx->Jinv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
  cx->Jinv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  cx->Jinv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  cx->Jinv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
  cx->Jinv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  cx->Jinv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  cx->Jinv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
  cx->Jinv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  cx->Jinv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  cx->vol_T = fabs(det);
  for (int r = 0; r < 3; ++r) {
    /* J^{-T} e_r is row r of J^{-1} */
    double len = sqrt(cx->Jinv[r][0] * cx->Jinv[r][0] + cx->Jinv[r][1] * cx->Jinv[r][1] + cx->Jinv[r][2] * cx->Jinv[r][2]);
    for (int a = 0; a < 3; ++a) cx->nrm[r][a] = cx->Jinv[r][a] / len;
    cx->area[r] = cx->vol_T * len;
  }
  cx->ncell = pr->n[0] * pr->n[1] * pr->n[2];
  return 0;
}

static void ctx_free(oracle_ctx* cx) {
  table_free(&cx->vol);
  for (int s = 0; s < 6; ++s) table_free(&cx->face[s]);
}

/* Geometry of the cell map at one point (Sec. 3.2: gradients map with S = J^{-T}, volumes with Delta = |det J|) */
typedef struct {
  double Jinv[3][3];
  double det; /* |det J| */
} pgeo;

/* physical gradient from a reference gradient: g = J^{-T} gref */
static void phys_grad(const double Jinv[3][3], const double gref[3], double g[3]) {
  for (int a = 0; a < 3; ++a) {
    g[a] = 0.0;
    for (int r = 0; r < 3; ++r) g[a] += Jinv[r][a] * gref[r];
  }
}

/* u and physical gradient of the FE function with coefficients zc at point p of table t (J^{-1} at the point) */
static void eval_fe(const table3d* t, int p, const double* zc, const double Jinv[3][3], double* u, double g[3]) {
  double uu = 0, gr3[3] = {0, 0, 0};
  const double* ph = t->phi + (size_t)p * t->nb;
  const double* gr = t->grad + (size_t)p * t->nb * 3;
  for (int J = 0; J < t->nb; ++J) {
    uu += zc[J] * ph[J];
    gr3[0] += zc[J] * gr[3 * J + 0];
    gr3[1] += zc[J] * gr[3 * J + 1];
    gr3[2] += zc[J] * gr[3 * J + 2];
  }
  *u = uu;
  phys_grad(Jinv, gr3, g);
}

/* a packed symmetric tensor (xx, yy, zz, xy, xz, yz) as a 3x3 matrix */
static void unpack6(const double* t, double Dm[3][3]) {
  Dm[0][0] = t[0];
  Dm[1][1] = t[1];
  Dm[2][2] = t[2];
  Dm[0][1] = Dm[1][0] = t[3];
  Dm[0][2] = Dm[2][0] = t[4];
  Dm[1][2] = Dm[2][1] = t[5];
}

/* diffusion tensor of a cell: the given symmetric tensor, or D_T * I */
static void diff_tensor(const oracle_problem* pr, int cell, double Dm[3][3]) {
  if (pr->Dten) {
    unpack6(pr->Dten + (size_t)cell * 6, Dm);
  } else {
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < 3; ++c) Dm[a][c] = a == c ? pr->D[cell] : 0.0;
  }
}

/* nu . (D w) */
static double flux_along(const double nu[3], const double Dm[3][3], const double w[3]) {
  double s = 0.0;
  for (int a = 0; a < 3; ++a) s += nu[a] * (Dm[a][0] * w[0] + Dm[a][1] * w[1] + Dm[a][2] * w[2]);
  return s;
}

/* physical gradient of test function i at point p of table t */
static void test_grad(const table3d* t, int p, int i, const double Jinv[3][3], double g[3]) {
  const double* gr = t->grad + ((size_t)p * t->nb + i) * 3;
  phys_grad(Jinv, gr, g);
}

static double upwind(double um, double up, double bnu) { return bnu >= 0.0 ? um * bnu : up * bnu; }

static double harmonic(double a, double b) { return 2.0 * a * b / (a + b); }

static void cell_coords(const oracle_problem* pr, int cell, int ic[3]) {
  ic[0] = cell % pr->n[0];
  ic[1] = (cell / pr->n[0]) % pr->n[1];
  ic[2] = cell / (pr->n[0] * pr->n[1]);
}

static int cell_index(const oracle_problem* pr, const int ic[3]) {
  return ic[0] + pr->n[0] * (ic[1] + pr->n[1] * ic[2]);
}

/* inverse and |determinant| of a 3x3 matrix, by cofactors */
static void invert3(const double J[3][3], double Jinv[3][3], double* absdet) {
  double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
               J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  Jinv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
  Jinv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  Jinv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  Jinv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
  Jinv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  Jinv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  Jinv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
  Jinv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  Jinv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  *absdet = fabs(det);
}

/* The cell map's geometry at the local reference point xi of a cell: the constant J of the axis-parallel or
 * affine grid, or, for multilinear cells, the derivative of the trilinear map
 *   x(xi) = sum over the corners (a, b, c) in {0,1}^3 of N_a(xi_0) N_b(xi_1) N_c(xi_2) X_abc,
 *   N_0(t) = 1 - t, N_1(t) = t,  J[row][r] = d x_row / d xi_r. */
static void point_geo(const oracle_problem* pr, const oracle_ctx* cx, int cell, const double xi[3], pgeo* g) {
  if (!pr->vertices) {
    memcpy(g->Jinv, cx->Jinv, sizeof(g->Jinv));
    g->det = cx->vol_T;
    return;
  }
  int ic[3];
  cell_coords(pr, cell, ic);
  double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int c = 0; c < 2; ++c)
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) {
        const int corner[3] = {a, b, c};
        double N[3], dN[3];
        for (int r = 0; r < 3; ++r) {
          N[r] = corner[r] ? xi[r] : 1.0 - xi[r];
          dN[r] = corner[r] ? 1.0 : -1.0;
        }
        const double d[3] = {dN[0] * N[1] * N[2], N[0] * dN[1] * N[2], N[0] * N[1] * dN[2]};
        const size_t v = (size_t)(ic[0] + a) + (size_t)(pr->n[0] + 1) * ((ic[1] + b) + (size_t)(pr->n[1] + 1) * (ic[2] + c));
        const double* X = pr->vertices + 3 * v;
        for (int row = 0; row < 3; ++row)
          for (int r = 0; r < 3; ++r) J[row][r] += X[row] * d[r];
      }
  invert3(J, g->Jinv, &g->det);
}

/* unit normal nu along +reference axis r at a point of a face across r, and the face's area element
 * |det J| |J^{-T} e_r| there (J^{-T} e_r is row r of J^{-1}) */
static double face_normal(const pgeo* g, int r, double nu[3]) {
  const double len = sqrt(g->Jinv[r][0] * g->Jinv[r][0] + g->Jinv[r][1] * g->Jinv[r][1] + g->Jinv[r][2] * g->Jinv[r][2]);
  for (int a = 0; a < 3; ++a) nu[a] = g->Jinv[r][a] / len;
  return g->det * len;
}

/* |T|: the cell's volume by the volume rule (exact for multilinear cells: |det J| has degree 2 per direction) */
static double cell_volume(const oracle_problem* pr, const oracle_ctx* cx, int cell) {
  if (!pr->vertices) return cx->vol_T;
  double v = 0.0;
  for (int p = 0; p < cx->vol.np; ++p) {
    pgeo g;
    point_geo(pr, cx, cell, cx->vol.xi + 3 * p, &g);
    v += cx->vol.wgt[p] * g.det;
  }
  return v;
}

/* |F|: the area of face s = 2*dir + side of a cell, by the face rule */
static double face_area(const oracle_problem* pr, const oracle_ctx* cx, int cell, int s) {
  if (!pr->vertices) return cx->area[s / 2];
  const table3d* ft = &cx->face[s];
  double a = 0.0;
  for (int p = 0; p < ft->np; ++p) {
    pgeo g;
    double nu[3];
    point_geo(pr, cx, cell, ft->xi + 3 * p, &g);
    a += ft->wgt[p] * face_normal(&g, s / 2, nu);
  }
  return a;
}

/* a_h(u, phi_i) for all test functions phi_i supported on one cell: the
 * cell's volume term plus every face of the cell (eq. blf).  Gradients, normals,
 * area and volume elements are taken at each quadrature point from the cell
 * map (constant for the axis-parallel and affine grids). */
static void apply_cell(const oracle_problem* pr, const oracle_ctx* cx, const double* u, int cell, double* y) {
  const int nb = cx->vol.nb;
  const double* zc = u + (size_t)cell * nb;
  double DT[3][3];
  diff_tensor(pr, cell, DT);
  for (int i = 0; i < nb; ++i) y[i] = 0.0;

  /* volume: (D grad u - b u, grad v)_T + (c u, v)_T */
  for (int p = 0; p < cx->vol.np; ++p) {
    pgeo G;
    point_geo(pr, cx, cell, cx->vol.xi + 3 * p, &G);
    double uq, g[3];
    eval_fe(&cx->vol, p, zc, G.Jinv, &uq, g);
    double dx = cx->vol.wgt[p] * G.det; /* Delta_T * w_i */
    double Dp_[3][3];
    if (pr->D_vol) unpack6(pr->D_vol + ((size_t)cell * cx->vol.np + p) * 6, Dp_);
    const double(*Dq)[3] = pr->D_vol ? Dp_ : DT;   /* D at this point */
    const double cq = pr->c_vol ? pr->c_vol[(size_t)cell * cx->vol.np + p] : pr->c;
    double Dg[3], fl[3];
    for (int a = 0; a < 3; ++a) Dg[a] = Dq[a][0] * g[0] + Dq[a][1] * g[1] + Dq[a][2] * g[2];
    for (int r = 0; r < 3; ++r) {
      const double br = pr->b_vol ? pr->b_vol[((size_t)cell * cx->vol.np + p) * 3 + r] : pr->b[r];
      fl[r] = Dg[r] - br * uq;
    }
    const double* ph = cx->vol.phi + (size_t)p * nb;
    for (int i = 0; i < nb; ++i) {
      double gv[3];
      test_grad(&cx->vol, p, i, G.Jinv, gv);
      y[i] += dx * (fl[0] * gv[0] + fl[1] * gv[1] + fl[2] * gv[2] + cq * uq * ph[i]);
    }
  }

  int ic[3];
  cell_coords(pr, cell, ic);
  const double volT = cell_volume(pr, cx, cell);
  for (int dir = 0; dir < 3; ++dir)
    for (int side = 0; side < 2; ++side) {
      const table3d* ft = &cx->face[2 * dir + side]; /* this cell's trace at the face */
      int nic[3] = {ic[0], ic[1], ic[2]};
      nic[dir] += side ? 1 : -1;
      if (pr->periodic[dir]) nic[dir] = (nic[dir] + pr->n[dir]) % pr->n[dir];
      int interior = nic[dir] >= 0 && nic[dir] < pr->n[dir];
      const double areaF = face_area(pr, cx, cell, 2 * dir + side); /* |F| of the penalty */
      /* normal velocity b . nu at face point p of this face */
      const double* bfp = pr->b_face ? pr->b_face + ((size_t)cell * 6 + 2 * dir + side) * ft->np : 0;
      if (interior) {
        /* T- is the lower cell along dir, nu from T- to T+ */
        int nbr = cell_index(pr, nic);
        const double* zn = u + (size_t)nbr * nb;
        const table3d* nt = &cx->face[2 * dir + (1 - side)]; /* neighbour's trace */
        int this_is_minus = side == 1;
        double DN[3][3];
        diff_tensor(pr, nbr, DN);
        const double volN = cell_volume(pr, cx, nbr);
        const double vmin = volT < volN ? volT : volN; /* min(|T-|, |T+|) */
        const int oface = 2 * dir + (1 - side); /* the same face seen from the neighbour */
        for (int p = 0; p < ft->np; ++p) {
          pgeo Go, Gn;
          point_geo(pr, cx, cell, ft->xi + 3 * p, &Go);
          point_geo(pr, cx, nbr, nt->xi + 3 * p, &Gn);
          double nu[3]; /* unit normal pointing along +reference axis dir */
          const double dA = face_normal(&Go, dir, nu);
          const double bdotn = pr->b[0] * nu[0] + pr->b[1] * nu[1] + pr->b[2] * nu[2];
          /* the two cells' tensors at this face point (constant per cell unless given point-wise) */
          double Do_[3][3], Dn_[3][3];
          if (pr->D_face) {
            unpack6(pr->D_face + (((size_t)cell * 6 + 2 * dir + side) * ft->np + p) * 6, Do_);
            unpack6(pr->D_face + (((size_t)nbr * 6 + oface) * ft->np + p) * 6, Dn_);
          }
          const double(*Dow)[3] = pr->D_face ? Do_ : DT;
          const double(*Dnb)[3] = pr->D_face ? Dn_ : DN;
          const double(*Dm)[3] = this_is_minus ? Dow : Dnb;
          const double(*Dp)[3] = this_is_minus ? Dnb : Dow;
          double dm = flux_along(nu, Dm, nu), dp = flux_along(nu, Dp, nu); /* delta = nu^T D nu */
          double wm = dp / (dm + dp), wp = dm / (dm + dp);
          double gam = harmonic(dm, dp) * pr->sigma * areaF / vmin;
          double bnu = bfp ? bfp[p] : bdotn;
          double us, gs[3], un, gn[3];
          eval_fe(ft, p, zc, Go.Jinv, &us, gs);
          eval_fe(nt, p, zn, Gn.Jinv, &un, gn);
          double um = this_is_minus ? us : un, up = this_is_minus ? un : us;
          double dnum = flux_along(nu, Dm, this_is_minus ? gs : gn); /* nu . D- grad u- */
          double dnup = flux_along(nu, Dp, this_is_minus ? gn : gs);
          double jump_u = um - up;
          double avg_flux = wm * dnum + wp * dnup; /* nu . {D grad u}_w */
          double phi_flux = upwind(um, up, bnu);
          double dx = ft->wgt[p] * dA;
          const double* ph = ft->phi + (size_t)p * nb;
          for (int i = 0; i < nb; ++i) {
            double gv[3];
            test_grad(ft, p, i, Go.Jinv, gv);
            double v = ph[i], dv = flux_along(nu, Dow, gv); /* nu . D grad v on this cell */
            /* jump and weighted average of the test function supported on this cell */
            double jump_v = this_is_minus ? v : -v;
            double avg_dv = this_is_minus ? wm * dv : wp * dv;
            y[i] += dx * (phi_flux * jump_v - avg_flux * jump_v - avg_dv * jump_u + gam * jump_u * jump_v);
          }
        }
      } else if (pr->bc[2 * dir + side] == BC_NEUMANN) {
        /* Neumann face: eq. blf has no term on F^N; the prescribed total flux j enters l_h */
      } else if (pr->bc[2 * dir + side] == BC_OUTFLOW) {
        /* outflow face (F^O, (D grad u) . nu = 0): only the upwind convective flux Phi(u, 0, b_nu) */
        double sgn = side ? 1.0 : -1.0;
        for (int p = 0; p < ft->np; ++p) {
          pgeo Go;
          point_geo(pr, cx, cell, ft->xi + 3 * p, &Go);
          double nu[3];
          const double dA = face_normal(&Go, dir, nu);
          const double bdotn = pr->b[0] * nu[0] + pr->b[1] * nu[1] + pr->b[2] * nu[2];
          double bnu = sgn * (bfp ? bfp[p] : bdotn);
          double us, gs[3];
          eval_fe(ft, p, zc, Go.Jinv, &us, gs);
          double dx = ft->wgt[p] * dA;
          const double* ph = ft->phi + (size_t)p * nb;
          for (int i = 0; i < nb; ++i) y[i] += dx * upwind(us, 0.0, bnu) * ph[i];
        }
      } else {
        /* Dirichlet boundary face, outward normal sgn * nu */
        double sgn = side ? 1.0 : -1.0;
        for (int p = 0; p < ft->np; ++p) {
          pgeo Go;
          point_geo(pr, cx, cell, ft->xi + 3 * p, &Go);
          double nu[3];
          const double dA = face_normal(&Go, dir, nu);
          const double bdotn = pr->b[0] * nu[0] + pr->b[1] * nu[1] + pr->b[2] * nu[2];
          double nout[3] = {sgn * nu[0], sgn * nu[1], sgn * nu[2]};
          double Db_[3][3];
          if (pr->D_face) unpack6(pr->D_face + (((size_t)cell * 6 + 2 * dir + side) * ft->np + p) * 6, Db_);
          const double(*DB)[3] = pr->D_face ? Db_ : DT;
          double gam = flux_along(nout, DB, nout) * pr->sigma * areaF / volT;
          double bnu = sgn * (bfp ? bfp[p] : bdotn);
          double us, gs[3];
          eval_fe(ft, p, zc, Go.Jinv, &us, gs);
          double dnu = flux_along(nout, DB, gs);
          double dx = ft->wgt[p] * dA;
          const double* ph = ft->phi + (size_t)p * nb;
          for (int i = 0; i < nb; ++i) {
            double gv[3];
            test_grad(ft, p, i, Go.Jinv, gv);
            double v = ph[i], dnv = flux_along(nout, DB, gv);
            y[i] += dx * (upwind(us, 0.0, bnu) * v - dnu * v - dnv * us + gam * us * v);
          }
        }
      }
    }
}

static int fill_problem(oracle_problem* pr, const int* n, const double* lo, const double* hi, int k, int m,
                        const double* D, const double* b, double c, double sigma) {
  for (int r = 0; r < 3; ++r) {
    pr->n[r] = n[r];
    pr->lo[r] = lo[r];
    pr->hi[r] = hi[r];
    pr->b[r] = b[r];
    if (n[r] < 1 || !(hi[r] > lo[r])) return -1;
  }
  if (k < 0 || k > 20 || m < 1 || m > 40) return -1;
  pr->k = k;
  pr->m = m;
  pr->D = D;
  pr->c = c;
  pr->sigma = sigma;
  pr->periodic[0] = pr->periodic[1] = pr->periodic[2] = 0;
  pr->b_vol = 0;
  pr->b_face = 0;
  pr->Dten = 0;
  pr->D_vol = 0;
  pr->D_face = 0;
  pr->c_vol = 0;
  for (int s = 0; s < 6; ++s) pr->bc[s] = BC_DIRICHLET;
  pr->vertices = 0;
  pr->affine = 0;
  memset(pr->J, 0, sizeof(pr->J));
  return 0;
}

/* boundary types per side (bc == NULL: all Dirichlet); a periodic axis has no boundary sides */
static int set_bc(oracle_problem* pr, const int* bc) {
  for (int s = 0; s < 6; ++s) {
    pr->bc[s] = bc ? bc[s] : BC_DIRICHLET;
    if (pr->bc[s] < BC_DIRICHLET || pr->bc[s] > BC_OUTFLOW) return -1;
  }
  return 0;
}

/* tensor diffusion and affine geometry options shared by the _ex entry points */
static void set_general(oracle_problem* pr, const double* Dten, const double* Jmap, const double* D_vol,
                        const double* D_face, const double* c_vol) {
  pr->Dten = Dten;
  pr->D_vol = D_vol;
  pr->D_face = D_face;
  pr->c_vol = c_vol;
  if (Jmap) {
    pr->affine = 1;
    for (int a = 0; a < 3; ++a)
      for (int r = 0; r < 3; ++r) pr->J[a][r] = Jmap[3 * a + r];
  }
}

/* y = A u restricted to the listed cells (cells == NULL: all cells, in order).
 * y holds ncell_out blocks of (k+1)^3 values, one per listed cell. */
static int apply_impl(oracle_problem* pr_in, const double* u, double* y, const int* cells, int ncells_out);

int oracle_apply(const int* n, const double* lo, const double* hi, int k, int m, const double* D, const double* b,
                 double c, double sigma, const double* u, double* y, const int* cells, int ncells_out) {
  oracle_problem pr;
  if (fill_problem(&pr, n, lo, hi, k, m, D, b, c, sigma)) return -1;
  return apply_impl(&pr, u, y, cells, ncells_out);
}

/* oracle_apply with periodic axes, a velocity field given at the quadrature points, a tensor diffusion
 * coefficient and an affine geometry:
 *   b_vol [ncells][m^3][3] (NULL: constant b), b_face [ncells][6][m^2] = b . nu at each face point of each
 *   cell, nu the unit normal along +reference axis (NULL: constant b);
 *   Dten [ncells][6] = (xx, yy, zz, xy, xz, yz) (NULL: D_T * I from D);
 *   Jmap [9] row-major cell Jacobian, cells lo + J (ic + [0,1]^3) (NULL: the axis-parallel [lo, hi] grid);
 *   D_vol [ncells][m^3][6], D_face [ncells][6][m^2][6], c_vol [ncells][m^3]: coefficients at the quadrature
 *   points (NULL: per cell / constant).
 * On a periodic axis the end faces couple the first and last cells. */
int oracle_apply_ex(const int* n, const double* lo, const double* hi, int k, int m, const double* D, const double* b,
                    double c, double sigma, const int* periodic, const int* bc, const double* b_vol,
                    const double* b_face, const double* Dten, const double* Jmap, const double* verts,
                    const double* D_vol, const double* D_face, const double* c_vol, const double* u, double* y,
                    const int* cells, int ncells_out) {
  oracle_problem pr;
  if (fill_problem(&pr, n, lo, hi, k, m, D, b, c, sigma)) return -1;
  for (int r = 0; r < 3; ++r) pr.periodic[r] = periodic ? periodic[r] != 0 : 0;
  if (set_bc(&pr, bc)) return -1;
  pr.b_vol = b_vol;
  pr.b_face = b_face;
  set_general(&pr, Dten, Jmap, D_vol, D_face, c_vol);
  pr.vertices = verts;
  return apply_impl(&pr, u, y, cells, ncells_out);
}

static int apply_impl(oracle_problem* pr_in, const double* u, double* y, const int* cells, int ncells_out) {
  oracle_problem pr = *pr_in;
  oracle_ctx cx;
  if (ctx_build(&pr, &cx)) return -2;
  int nb = cx.vol.nb;
  int count = cells ? ncells_out : cx.ncell;
  for (int t = 0; t < count; ++t) {
    int cell = cells ? cells[t] : t;
    if (cell < 0 || cell >= cx.ncell) {
      ctx_free(&cx);
      return -3;
    }
    apply_cell(&pr, &cx, u, cell, y + (size_t)t * nb);
  }
  ctx_free(&cx);
  return 0;
}

/* F_i = l_h(phi_i): (f, v)_T from f given at the volume quadrature points
 * (f_qp: [ncells][m^3], NULL means f = 0) plus, on Dirichlet sides, the terms
 * -(Phi(0,g,b_nu), v)_F - (nu . D grad v, g)_F + gamma_F (g, v)_F from g given
 * at the boundary face points (g_qp[s]: side s array, NULL means g = 0), and on
 * Neumann sides -(j, v)_F with j given in the same per-side array. */
static int rhs_impl(oracle_problem* pr_in, const double* f_qp, const double* const* g_qp, double* F);

int oracle_rhs(const int* n, const double* lo, const double* hi, int k, int m, const double* D, const double* b,
               double c, double sigma, const double* f_qp, const double* const* g_qp, double* F) {
  oracle_problem pr;
  if (fill_problem(&pr, n, lo, hi, k, m, D, b, c, sigma)) return -1;
  return rhs_impl(&pr, f_qp, g_qp, F);
}

/* oracle_rhs with periodic axes (no Dirichlet faces there), b . nu at the face points, a tensor diffusion
 * coefficient and an affine geometry (arguments as in oracle_apply_ex). */
int oracle_rhs_ex(const int* n, const double* lo, const double* hi, int k, int m, const double* D, const double* b,
                  double c, double sigma, const int* periodic, const int* bc, const double* b_face,
                  const double* Dten, const double* Jmap, const double* verts, const double* D_face,
                  const double* f_qp, const double* const* g_qp, double* F) {
  oracle_problem pr;
  if (fill_problem(&pr, n, lo, hi, k, m, D, b, c, sigma)) return -1;
  for (int r = 0; r < 3; ++r) pr.periodic[r] = periodic ? periodic[r] != 0 : 0;
  if (set_bc(&pr, bc)) return -1;
  pr.b_face = b_face;
  set_general(&pr, Dten, Jmap, 0, D_face, 0);
  pr.vertices = verts;
  return rhs_impl(&pr, f_qp, g_qp, F);
}

static int rhs_impl(oracle_problem* pr_in, const double* f_qp, const double* const* g_qp, double* F) {
  oracle_problem pr = *pr_in;
  oracle_ctx cx;
  if (ctx_build(&pr, &cx)) return -2;
  int nb = cx.vol.nb, npv = cx.vol.np;
  for (int cell = 0; cell < cx.ncell; ++cell) {
    double* y = F + (size_t)cell * nb;
    for (int i = 0; i < nb; ++i) y[i] = 0.0;
    if (f_qp) {
      for (int p = 0; p < npv; ++p) {
        pgeo G;
        point_geo(&pr, &cx, cell, cx.vol.xi + 3 * p, &G);
        double fx = f_qp[(size_t)cell * npv + p] * cx.vol.wgt[p] * G.det;
        const double* ph = cx.vol.phi + (size_t)p * nb;
        for (int i = 0; i < nb; ++i) y[i] += fx * ph[i];
      }
    }
    int ic[3];
    cell_coords(&pr, cell, ic);
    for (int dir = 0; dir < 3; ++dir)
      for (int side = 0; side < 2; ++side) {
        int s = 2 * dir + side;
        int on_boundary = side ? ic[dir] == pr.n[dir] - 1 : ic[dir] == 0;
        if (pr.periodic[dir] || !on_boundary || !g_qp || !g_qp[s]) continue;
        if (pr.bc[s] == BC_OUTFLOW) continue; /* no outflow term in l_h */
        /* face index within the boundary layer: tangential cell indices, lower axis fastest */
        int ta = dir == 0 ? 1 : 0, tb = dir == 2 ? 1 : 2;
        int fidx = ic[ta] + pr.n[ta] * ic[tb];
        const table3d* ft = &cx.face[s];
        double sgn = side ? 1.0 : -1.0;
        const double* bfp = pr.b_face ? pr.b_face + ((size_t)cell * 6 + s) * ft->np : 0;
        double DT[3][3];
        diff_tensor(&pr, cell, DT);
        const double areaF = face_area(&pr, &cx, cell, s), volT = cell_volume(&pr, &cx, cell);
        for (int p = 0; p < ft->np; ++p) {
          pgeo Go;
          point_geo(&pr, &cx, cell, ft->xi + 3 * p, &Go);
          double nu[3];
          const double dA = face_normal(&Go, dir, nu);
          double dx = ft->wgt[p] * dA;
          const double* ph = ft->phi + (size_t)p * nb;
          if (pr.bc[s] == BC_NEUMANN) {
            /* -(j, v)_F with the prescribed total flux j = (b u - D grad u) . nu_out at the face points */
            double jf = g_qp[s][(size_t)fidx * ft->np + p];
            for (int i = 0; i < nb; ++i) y[i] -= dx * jf * ph[i];
            continue;
          }
          double nout[3] = {sgn * nu[0], sgn * nu[1], sgn * nu[2]};
          const double bdotn = pr.b[0] * nu[0] + pr.b[1] * nu[1] + pr.b[2] * nu[2];
          double Db_[3][3];
          if (pr.D_face) unpack6(pr.D_face + (((size_t)cell * 6 + s) * ft->np + p) * 6, Db_);
          const double(*DB)[3] = pr.D_face ? Db_ : DT;
          double gam = flux_along(nout, DB, nout) * pr.sigma * areaF / volT;
          double g = g_qp[s][(size_t)fidx * ft->np + p];
          double bnu = sgn * (bfp ? bfp[p] : bdotn);
          for (int i = 0; i < nb; ++i) {
            double gv[3];
            test_grad(ft, p, i, Go.Jinv, gv);
            double v = ph[i], dnv = flux_along(nout, DB, gv);
            y[i] += dx * (-upwind(0.0, g, bnu) * v - dnv * g + gam * g * v);
          }
        }
      }
  }
  ctx_free(&cx);
  return 0;
}

/* x = lo + J xi for a point xi of the structured reference grid (xi_r = cell index + local coordinate);
 * J = diag((hi - lo) / n) without an affine map; with vertices, the trilinear map of the cell that holds xi
 * (a point on a face between two cells is mapped by the lower one; both give the same point) */
static void map_point_v(const int* n, const double* lo, const double* hi, const double* Jmap, const double* verts,
                        const double xi[3], double* out) {
  if (verts) {
    int ic[3];
    double t[3];
    for (int r = 0; r < 3; ++r) {
      ic[r] = (int)floor(xi[r]);
      if (ic[r] > n[r] - 1) ic[r] = n[r] - 1;
      if (ic[r] < 0) ic[r] = 0;
      t[r] = xi[r] - ic[r];
    }
    for (int a = 0; a < 3; ++a) out[a] = 0.0;
    for (int c = 0; c < 2; ++c)
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) {
          const double N = (a ? t[0] : 1.0 - t[0]) * (b ? t[1] : 1.0 - t[1]) * (c ? t[2] : 1.0 - t[2]);
          const size_t v = (size_t)(ic[0] + a) + (size_t)(n[0] + 1) * ((ic[1] + b) + (size_t)(n[1] + 1) * (ic[2] + c));
          for (int r = 0; r < 3; ++r) out[r] += N * verts[3 * v + r];
        }
    return;
  }
  for (int a = 0; a < 3; ++a) {
    if (Jmap) {
      out[a] = lo[a] + Jmap[3 * a] * xi[0] + Jmap[3 * a + 1] * xi[1] + Jmap[3 * a + 2] * xi[2];
    } else {
      out[a] = lo[a] + (hi[a] - lo[a]) / n[a] * xi[a];
    }
  }
}

/* Physical coordinates of the volume quadrature points: xyz[(cell*m^3 + q)*3 + r]. */
int oracle_volume_points_ex(const int* n, const double* lo, const double* hi, const double* Jmap,
                            const double* verts, int m, double* xyz) {
  double* x = (double*)malloc(sizeof(double) * m);
  double* w = (double*)malloc(sizeof(double) * m);
  if (!x || !w || oracle_gauss_legendre(m, x, w)) return -1;
  size_t o = 0;
  for (int iz = 0; iz < n[2]; ++iz)
    for (int iy = 0; iy < n[1]; ++iy)
      for (int ix = 0; ix < n[0]; ++ix)
        for (int i3 = 0; i3 < m; ++i3)
          for (int i2 = 0; i2 < m; ++i2)
            for (int i1 = 0; i1 < m; ++i1) {
              const double xi[3] = {ix + x[i1], iy + x[i2], iz + x[i3]};
              map_point_v(n, lo, hi, Jmap, verts, xi, xyz + o);
              o += 3;
            }
  free(x);
  free(w);
  return 0;
}

int oracle_volume_points(const int* n, const double* lo, const double* hi, int m, double* xyz) {
  return oracle_volume_points_ex(n, lo, hi, 0, 0, m, xyz);
}

/* Physical coordinates of the boundary face points of side s = 2*dir + side:
 * xyz[(face*m^2 + p)*3 + r], faces and points ordered as documented above. */
int oracle_face_points_ex(const int* n, const double* lo, const double* hi, const double* Jmap,
                          const double* verts, int m, int s, double* xyz) {
  if (s < 0 || s > 5) return -1;
  double* x = (double*)malloc(sizeof(double) * m);
  double* w = (double*)malloc(sizeof(double) * m);
  if (!x || !w || oracle_gauss_legendre(m, x, w)) return -1;
  int dir = s / 2, side = s % 2;
  int ta = dir == 0 ? 1 : 0, tb = dir == 2 ? 1 : 2;
  size_t o = 0;
  for (int cb = 0; cb < n[tb]; ++cb)
    for (int ca = 0; ca < n[ta]; ++ca)
      for (int pb = 0; pb < m; ++pb)
        for (int pa = 0; pa < m; ++pa) {
          double xi[3];
          xi[dir] = side ? n[dir] : 0;
          xi[ta] = ca + x[pa];
          xi[tb] = cb + x[pb];
          map_point_v(n, lo, hi, Jmap, verts, xi, xyz + o);
          o += 3;
        }
  free(x);
  free(w);
  return 0;
}

int oracle_face_points(const int* n, const double* lo, const double* hi, int m, int s, double* xyz) {
  return oracle_face_points_ex(n, lo, hi, 0, 0, m, s, xyz);
}

/* Physical coordinates of the face points of every face of every cell:
 * xyz[((cell*6 + s)*m^2 + p)*3 + r], s = 2*dir + side, points ordered as in the face tables
 * (lower tangential axis fastest). */
int oracle_cell_face_points_ex(const int* n, const double* lo, const double* hi, const double* Jmap,
                               const double* verts, int m, double* xyz) {
  double* x = (double*)malloc(sizeof(double) * m);
  double* w = (double*)malloc(sizeof(double) * m);
  if (!x || !w || oracle_gauss_legendre(m, x, w)) return -1;
  size_t o = 0;
  for (int iz = 0; iz < n[2]; ++iz)
    for (int iy = 0; iy < n[1]; ++iy)
      for (int ix = 0; ix < n[0]; ++ix) {
        const int ic[3] = {ix, iy, iz};
        for (int dir = 0; dir < 3; ++dir)
          for (int side = 0; side < 2; ++side) {
            int ta = dir == 0 ? 1 : 0, tb = dir == 2 ? 1 : 2;
            for (int pb = 0; pb < m; ++pb)
              for (int pa = 0; pa < m; ++pa) {
                double xi[3];
                xi[dir] = ic[dir] + side;
                xi[ta] = ic[ta] + x[pa];
                xi[tb] = ic[tb] + x[pb];
                map_point_v(n, lo, hi, Jmap, verts, xi, xyz + o);
                o += 3;
              }
          }
      }
  free(x);
  free(w);
  return 0;
}

int oracle_cell_face_points(const int* n, const double* lo, const double* hi, int m, double* xyz) {
  return oracle_cell_face_points_ex(n, lo, hi, 0, 0, m, xyz);
}
