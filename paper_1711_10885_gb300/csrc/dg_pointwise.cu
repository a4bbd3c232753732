// dg_pointwise.cu -- coefficient and geometry tables of the point-wise kernels: Problem B of Sec. 5.1 (affine
// cells with a diffusion tensor, velocity and reaction given at the quadrature points, the paper's
// "coefficients that are polynomials in the coordinates", integrated with q = 2p+4) and Problem C
// (multilinear cells: each cell the trilinear image of the reference cube through its 8 corner vertices).
//
// Everything is moved to reference coordinates once, at set-up (Sec. 3.2: S_T = J^{-T}, Delta_T = |det J|),
// with the cell Jacobian J taken at each point (constant on the axis-parallel and affine grids):
//   volume point:  K = |det J| J^{-1} D(x) J^{-T},  beta = -|det J| J^{-1} b(x),  c |det J| w
//   face point of a face across reference axis r, with the area element |F_r| = |det J| |J^{-T} e_r| and the
//   unit normal nu = J^{-T} e_r / |J^{-T} e_r|:  nu . D grad u = (K grad u)_r / |F_r|,  delta = nu^T D nu.
// On an interior face the weights w+- = delta-+/(delta- + delta+) and the penalty
// gamma = <delta-, delta+> sigma |F| / min(|T-|, |T+|) come from the two cells' tensors at the same face point
// (Sec. 2); |F| and |T| are the face area and the cell volumes.  On multilinear cells the area element varies
// over a face; it is folded into the face coefficients and the normal velocity (the kernels then use a unit
// face measure).
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "dg_internal.h"

namespace {

// symmetric 3x3 from (xx, yy, zz, xy, xz, yz)
void unpack6(const double* t, double D[3][3]) {
  D[0][0] = t[0], D[1][1] = t[1], D[2][2] = t[2];
  D[0][1] = D[1][0] = t[3];
  D[0][2] = D[2][0] = t[4];
  D[1][2] = D[2][1] = t[5];
}

// Sylvester's criterion, and every entry finite
bool spd(const double* t) {
  for (int q = 0; q < 6; ++q)
    if (!std::isfinite(t[q])) return false;
  const double m2 = t[0] * t[1] - t[3] * t[3];
  const double m3 = t[0] * (t[1] * t[2] - t[5] * t[5]) - t[3] * (t[3] * t[2] - t[5] * t[4]) +
                    t[4] * (t[3] * t[5] - t[1] * t[4]);
  return t[0] > 0 && m2 > 0 && m3 > 0;
}

// K = |det J| J^{-1} D J^{-T} at a point
void metric(const dgi::MapGeo& g, const double* t, double K[3][3]) {
  double D[3][3];
  unpack6(t, D);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double acc = 0.0;
      for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) acc += g.Jinv[a][p] * D[p][q] * g.Jinv[b][q];
      K[a][b] = g.det * acc;
    }
}

// nu^T D nu
double along(const double nu[3], const double* t) {
  double D[3][3];
  unpack6(t, D);
  double s = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) s += nu[a] * D[a][b] * nu[b];
  return s;
}

}  // namespace

namespace dgi {

int point_geometry(const dg_handle* h, int64_t cell, const double xi[3], MapGeo* g) {
  if (!h->ml) {
    for (int a = 0; a < 3; ++a)
      for (int r = 0; r < 3; ++r) g->Jinv[a][r] = h->Jinv[a][r];
    g->det = h->detJ;
    g->sdet = h->detJ;
    return DG_OK;
  }
  const int ic[3] = {(int)(cell % h->n[0]), (int)((cell / h->n[0]) % h->n[1]),
                     (int)(cell / ((int64_t)h->n[0] * h->n[1]))};
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
        const int64_t v = (ic[0] + a) + (int64_t)(h->n[0] + 1) * ((ic[1] + b) + (int64_t)(h->n[1] + 1) * (ic[2] + c));
        const double* X = h->verts + 3 * v;
        for (int row = 0; row < 3; ++row)
          for (int r = 0; r < 3; ++r) J[row][r] += X[row] * d[r];
      }
  const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                     J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                     J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  if (!(std::fabs(det) > 0) || !std::isfinite(det)) {
    set_error("dg_setup: a multilinear cell's map is singular or not finite (cell " + std::to_string(cell) + ")");
    return DG_ERR_INVALID_ARG;
  }
  g->Jinv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
  g->Jinv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  g->Jinv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  g->Jinv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
  g->Jinv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  g->Jinv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  g->Jinv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
  g->Jinv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  g->Jinv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  g->det = std::fabs(det);
  g->sdet = det;
  return DG_OK;
}

double face_frame(const MapGeo& g, int r, double nu[3]) {
  const double len = std::sqrt(g.Jinv[r][0] * g.Jinv[r][0] + g.Jinv[r][1] * g.Jinv[r][1] + g.Jinv[r][2] * g.Jinv[r][2]);
  for (int a = 0; a < 3; ++a) nu[a] = g.Jinv[r][a] / len;
  return g.det * len;
}

void face_xi(const dg_handle* h, int face, int p, double xi[3]) {
  const int dir = face / 2, side = face % 2, ta = dir == 0 ? 1 : 0, tb = dir == 2 ? 1 : 2;
  xi[dir] = side;
  xi[ta] = h->tab.xi[p % h->M];
  xi[tb] = h->tab.xi[p / h->M];
}

int build_pointwise_tables(const dg_handle* h, const double* D_qp, const double* D_face, const double* c_qp,
                           double c_const, const double b[3], const double* b_qp, const double* b_face,
                           std::vector<double>& kq, std::vector<double>& kf, std::vector<double>& fc,
                           std::vector<double>& bface) {
  const int M = h->M, MM = M * M, M3 = MM * M;
  const int64_t ncell = h->ncell;
  const double* w = h->tab.w;
  const double* x = h->tab.xi;
  kq.assign((size_t)ncell * 10 * M3, 0.0);
  kf.assign((size_t)ncell * 18 * MM, 0.0);
  fc.assign((size_t)ncell * 36 * MM, 0.0);
  bface.assign((size_t)ncell * 6 * MM, 0.0);
  // cell volumes |T| (the penalty's min(|T-|, |T+|)); constant |det J| unless the cells are multilinear
  std::vector<double> vol(ncell, 0.0);
  // orientation of the mesh: every point of every cell must share the sign of det J at the first one
  double orient = 1.0;
  {
    MapGeo g0;
    const double xi0[3] = {x[0], x[0], x[0]};
    if (int rc = point_geometry(h, 0, xi0, &g0)) return rc;
    orient = g0.sdet;
  }
  for (int64_t cell = 0; cell < ncell; ++cell) {
    for (int q = 0; q < M3; ++q) {
      const size_t pt = (size_t)cell * M3 + q;
      const double* t = D_qp + pt * 6;
      if (!spd(t)) {
        set_error("dg_setup: D_qp must be symmetric positive definite at every point (cell " +
                  std::to_string(cell) + ", point " + std::to_string(q) + ")");
        return DG_ERR_INVALID_ARG;
      }
      MapGeo g;
      const double xi[3] = {x[q % M], x[(q / M) % M], x[q / MM]};
      if (int rc = point_geometry(h, cell, xi, &g)) return rc;
      if (h->ml && (g.sdet > 0) != (orient > 0)) {
        set_error("dg_setup: a multilinear cell is inverted or folded (the sign of det J changes; cell " +
                  std::to_string(cell) + ")");
        return DG_ERR_INVALID_ARG;
      }
      const double wq = w[q % M] * w[(q / M) % M] * w[q / MM];
      vol[cell] += wq * g.det;
      double K[3][3];
      metric(g, t, K);
      const double* bq = b_qp ? b_qp + pt * 3 : b;
      const double cq = c_qp ? c_qp[pt] : c_const;
      if (!std::isfinite(bq[0]) || !std::isfinite(bq[1]) || !std::isfinite(bq[2]) || !std::isfinite(cq)) {
        set_error("dg_setup: b_qp and c_qp must be finite (cell " + std::to_string(cell) + ")");
        return DG_ERR_INVALID_ARG;
      }
      double* o = &kq[(size_t)cell * 10 * M3 + q];
      o[0 * M3] = K[0][0];
      o[1 * M3] = K[1][1];
      o[2 * M3] = K[2][2];
      o[3 * M3] = K[0][1];
      o[4 * M3] = K[0][2];
      o[5 * M3] = K[1][2];
      for (int r = 0; r < 3; ++r)
        o[(6 + r) * M3] = -g.det * (g.Jinv[r][0] * bq[0] + g.Jinv[r][1] * bq[1] + g.Jinv[r][2] * bq[2]);
      o[9 * M3] = cq * g.det * wq;
    }
  }
  const int64_t strides[3] = {1, h->n[0], (int64_t)h->n[0] * h->n[1]};
  for (int64_t cell = 0; cell < ncell; ++cell) {
    const int ic[3] = {(int)(cell % h->n[0]), (int)((cell / h->n[0]) % h->n[1]),
                       (int)(cell / ((int64_t)h->n[0] * h->n[1]))};
    for (int dir = 0; dir < 3; ++dir) {
      const int ta = dir == 0 ? 1 : 0, tb = dir == 2 ? 1 : 2;
      for (int side = 0; side < 2; ++side) {
        const int face = 2 * dir + side;
        const bool at_end = side ? ic[dir] == h->n[dir] - 1 : ic[dir] == 0;
        const bool boundary = at_end && !h->periodic[dir];
        const int64_t wrap = (int64_t)(h->n[dir] - 1) * strides[dir];
        const int64_t nbr = boundary ? -1
                                     : (side ? (at_end ? cell - wrap : cell + strides[dir])
                                             : (at_end ? cell + wrap : cell - strides[dir]));
        const int oface = 2 * dir + 1 - side;
        // |F| / min(|T-|, |T+|): the face area by the face rule
        double areaF = 0.0;
        std::vector<MapGeo> pg(MM);
        for (int p = 0; p < MM; ++p) {
          double xi[3], nu[3];
          face_xi(h, face, p, xi);
          if (int rc = point_geometry(h, cell, xi, &pg[p])) return rc;
          if (h->ml && (pg[p].sdet > 0) != (orient > 0)) {
            set_error("dg_setup: a multilinear cell is inverted or folded at a face (cell " + std::to_string(cell) +
                      ")");
            return DG_ERR_INVALID_ARG;
          }
          areaF += w[p % M] * w[p / M] * face_frame(pg[p], dir, nu);
        }
        const double vmin = boundary ? vol[cell] : std::min(vol[cell], vol[nbr]);
        const double fscale = areaF / vmin;
        for (int p = 0; p < MM; ++p) {
          const double* to = D_face + (((size_t)cell * 6 + face) * MM + p) * 6;
          if (!spd(to)) {
            set_error("dg_setup: D_face must be symmetric positive definite at every point (cell " +
                      std::to_string(cell) + ", face " + std::to_string(face) + ")");
            return DG_ERR_INVALID_ARG;
          }
          double nu[3];
          const double dA = face_frame(pg[p], dir, nu);  // area element |det J| |J^{-T} e_dir|
          double Ko[3][3];
          metric(pg[p], to, Ko);
          const double dlo = along(nu, to);
          double wo = 1.0, wn = 0.0, gam = dlo * h->sigma * fscale;
          if (!boundary) {
            const double* tn = D_face + (((size_t)nbr * 6 + oface) * MM + p) * 6;
            const double dln = along(nu, tn);
            wo = dln / (dlo + dln);
            wn = dlo / (dlo + dln);
            gam = (2.0 * dlo * dln / (dlo + dln)) * h->sigma * fscale;
          }
          // with a unit face measure in the kernels (multilinear cells) every coefficient carries dA
          const double s = h->ml ? dA : 1.0;
          double* c6 = &fc[((size_t)cell * 6 + face) * 6 * MM + p];
          c6[0 * MM] = s * wo;
          c6[1 * MM] = s * wn;
          c6[2 * MM] = s * gam;
          c6[3 * MM] = s * wo * Ko[dir][dir] / dA;
          c6[4 * MM] = s * wo * Ko[dir][ta] / dA;
          c6[5 * MM] = s * wo * Ko[dir][tb] / dA;
          if (boundary) {
            // the second coefficient multiplies the upwind flux on a boundary face; outflow and Neumann faces
            // have no diffusion or penalty term
            const int bt = h->bc_type[face];
            c6[1 * MM] = bt == DG_BC_NEUMANN ? 0.0 : 1.0;
            if (bt != DG_BC_DIRICHLET) c6[0] = c6[2 * MM] = c6[3 * MM] = c6[4 * MM] = c6[5 * MM] = 0.0;
          }
          for (int c = 0; c < 3; ++c) kf[(((size_t)cell * 6 + face) * 3 + c) * MM + p] = Ko[dir][c] / dA;
          const size_t fi = ((size_t)cell * 6 + face) * MM + p;
          const double bnu = nu[0] * b[0] + nu[1] * b[1] + nu[2] * b[2];
          bface[fi] = s * (b_face ? b_face[fi] : bnu);
          if (!std::isfinite(bface[fi])) {
            set_error("dg_setup: b_face must be finite");
            return DG_ERR_INVALID_ARG;
          }
        }
      }
    }
  }
  return DG_OK;
}

}  // namespace dgi
