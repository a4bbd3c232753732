// dg_pointwise.cu -- coefficient tables for Problem B of Sec. 5.1: affine cells with a diffusion tensor,
// velocity and reaction given at the quadrature points (the paper's "coefficients that are polynomials in
// the coordinates", integrated with q = 2p+4).
//
// Everything is moved to reference coordinates once, at set-up (Sec. 3.2: S_T = J^{-T}, Delta_T = |det J|):
//   volume point:  K = |det J| J^{-1} D(x) J^{-T},  beta = -|det J| J^{-1} b(x),  c |det J| w
//   face point of a face normal to reference axis r, with |F_r| = |det J| |J^{-T} e_r| and the unit normal
//   nu along +e_r:  nu . D grad u = (K grad u)_r / |F_r|,  delta = nu^T D nu = K_rr / (|det J| |J^{-T} e_r|^2).
// On an interior face the weights w+- = delta-+/(delta- + delta+) and the penalty
// gamma = <delta-, delta+> sigma |F| / |T| come from the two cells' tensors at the same face point (Sec. 2).
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

// K = |det J| J^{-1} D J^{-T}
void metric(const dg_handle* h, const double* t, double K[3][3]) {
  double D[3][3];
  unpack6(t, D);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double acc = 0.0;
      for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) acc += h->Jinv[a][p] * D[p][q] * h->Jinv[b][q];
      K[a][b] = h->detJ * acc;
    }
}

}  // namespace

namespace dgi {

int build_pointwise_tables(const dg_handle* h, const double* D_qp, const double* D_face, const double* c_qp,
                           double c_const, const double b[3], const double* b_qp, const double* b_face,
                           std::vector<double>& kq, std::vector<double>& kf, std::vector<double>& fc,
                           std::vector<double>& bface) {
  const int M = h->M, MM = M * M, M3 = MM * M;
  const int64_t ncell = h->ncell;
  const double* w = h->tab.w;
  kq.assign((size_t)ncell * 10 * M3, 0.0);
  kf.assign((size_t)ncell * 18 * MM, 0.0);
  fc.assign((size_t)ncell * 36 * MM, 0.0);
  bface.assign((size_t)ncell * 6 * MM, 0.0);
  for (int64_t cell = 0; cell < ncell; ++cell) {
    for (int q = 0; q < M3; ++q) {
      const size_t pt = (size_t)cell * M3 + q;
      const double* t = D_qp + pt * 6;
      if (!spd(t)) {
        set_error("dg_setup: D_qp must be symmetric positive definite at every point (cell " +
                  std::to_string(cell) + ", point " + std::to_string(q) + ")");
        return DG_ERR_INVALID_ARG;
      }
      double K[3][3];
      metric(h, t, K);
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
        o[(6 + r) * M3] = -h->detJ * (h->Jinv[r][0] * bq[0] + h->Jinv[r][1] * bq[1] + h->Jinv[r][2] * bq[2]);
      o[9 * M3] = cq * h->detJ * w[q % M] * w[(q / M) % M] * w[q / MM];
    }
  }
  const int64_t strides[3] = {1, h->n[0], (int64_t)h->n[0] * h->n[1]};
  for (int64_t cell = 0; cell < ncell; ++cell) {
    const int ic[3] = {(int)(cell % h->n[0]), (int)((cell / h->n[0]) % h->n[1]),
                       (int)(cell / ((int64_t)h->n[0] * h->n[1]))};
    for (int dir = 0; dir < 3; ++dir) {
      const int ta = dir == 0 ? 1 : 0, tb = dir == 2 ? 1 : 2;
      const double area = h->detJ * h->fscale[dir];
      const double dscale = 1.0 / (h->detJ * h->fscale[dir] * h->fscale[dir]);
      const double bnu = (h->Jinv[dir][0] * b[0] + h->Jinv[dir][1] * b[1] + h->Jinv[dir][2] * b[2]) / h->fscale[dir];
      for (int side = 0; side < 2; ++side) {
        const int face = 2 * dir + side;
        const bool at_end = side ? ic[dir] == h->n[dir] - 1 : ic[dir] == 0;
        const bool boundary = at_end && !h->periodic[dir];
        const int64_t wrap = (int64_t)(h->n[dir] - 1) * strides[dir];
        const int64_t nbr = boundary ? -1
                                     : (side ? (at_end ? cell - wrap : cell + strides[dir])
                                             : (at_end ? cell + wrap : cell - strides[dir]));
        const int oface = 2 * dir + 1 - side;
        for (int p = 0; p < MM; ++p) {
          const double* to = D_face + (((size_t)cell * 6 + face) * MM + p) * 6;
          if (!spd(to)) {
            set_error("dg_setup: D_face must be symmetric positive definite at every point (cell " +
                      std::to_string(cell) + ", face " + std::to_string(face) + ")");
            return DG_ERR_INVALID_ARG;
          }
          double Ko[3][3];
          metric(h, to, Ko);
          const double dlo = Ko[dir][dir] * dscale;
          double wo = 1.0, wn = 0.0, gam = dlo * h->sigma * h->fscale[dir];
          if (!boundary) {
            double Kn[3][3];
            metric(h, D_face + (((size_t)nbr * 6 + oface) * MM + p) * 6, Kn);
            const double dln = Kn[dir][dir] * dscale;
            wo = dln / (dlo + dln);
            wn = dlo / (dlo + dln);
            gam = (2.0 * dlo * dln / (dlo + dln)) * h->sigma * h->fscale[dir];
          }
          double* c6 = &fc[((size_t)cell * 6 + face) * 6 * MM + p];
          c6[0 * MM] = wo;
          c6[1 * MM] = wn;
          c6[2 * MM] = gam;
          c6[3 * MM] = wo * Ko[dir][dir] / area;
          c6[4 * MM] = wo * Ko[dir][ta] / area;
          c6[5 * MM] = wo * Ko[dir][tb] / area;
          if (boundary) {
            // the second coefficient multiplies the upwind flux on a boundary face; outflow and Neumann faces
            // have no diffusion or penalty term
            const int bt = h->bc_type[face];
            c6[1 * MM] = bt == DG_BC_NEUMANN ? 0.0 : 1.0;
            if (bt != DG_BC_DIRICHLET) c6[0] = c6[2 * MM] = c6[3 * MM] = c6[4 * MM] = c6[5 * MM] = 0.0;
          }
          for (int c = 0; c < 3; ++c) kf[(((size_t)cell * 6 + face) * 3 + c) * MM + p] = Ko[dir][c] / area;
          const size_t fi = ((size_t)cell * 6 + face) * MM + p;
          bface[fi] = b_face ? b_face[fi] : bnu;
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
