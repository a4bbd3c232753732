"""GPU parity of the multilinear-cell path (Problem C of Sec. 5.1: every cell the trilinear image of the reference
cube through its 8 corner vertices, the cell map's Jacobian taken at every quadrature point) against the FP64
oracle, which evaluates eq. blf and l_h by direct quadrature with the same per-point geometry.

Bar: FP64 and double-float results within 1e-12 of the oracle (relative infinity norm).
"""

import numpy as np
import pytest

import oracle
from paper_1711_10885_gb300 import inputs
from tests.test_oracle_tensor_pins import spd_tensors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def dg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_10885_gb300 import dg as _dg
    return _dg


def relerr(y, ref):
    return float(np.max(np.abs(np.asarray(y) - ref)) / max(np.max(np.abs(ref)), 1e-300))


BC = ("dirichlet", "outflow", "neumann", "dirichlet", "dirichlet", "neumann")

# (n, k, m - k, coefficient kind, boundary types)
CASES = [
    ((3, 2, 2), 1, 3, "scalar", None),
    ((2, 3, 2), 2, 1, "tensor", BC),
    ((2, 2, 3), 3, 3, "points", BC),
    ((2, 2, 2), 4, 3, "scalar", BC),
    ((3, 1, 2), 5, 1, "tensor", None),
    ((2, 2, 2), 6, 3, "points", None),
    ((3, 1, 3), 7, 3, "tensor", BC),
    ((1, 3, 1), 8, 3, "points", BC),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"n{c[0]}k{c[1]}m{c[1] + c[2]}{c[3]}{'bc' if c[4] else ''}")
def test_multilinear_operator_and_residual_match_oracle(dg, case):
    n, k, dm, kind, bc = case
    m = k + dm
    nc = int(np.prod(n))
    verts = inputs.multilinear_vertices(n, lo=(0.1, -0.2, 0.3), hi=(1.2, 0.9, 1.1), seed=500 + k, amplitude=0.2)
    sigma = oracle.penalty_sigma(k)
    base = dict(b=(0.6, -0.35, 0.25), c=0.7, sigma=sigma, m=m, bc=bc)
    geo = oracle.Problem(n, k, np.ones(nc), m=m, vertices=verts)
    xv, xf = oracle.volume_points(geo), oracle.cell_face_points(geo)
    lib_kw, ora_kw = {}, {}
    if kind == "scalar":
        D = np.exp(np.random.default_rng(510 + k).standard_normal(nc))
    else:
        D = np.ones(nc)
    if kind == "tensor":
        Dt = spd_tensors(nc, 520 + k)
        lib_kw["D_tensor"] = ora_kw["D_tensor"] = Dt
    if kind == "points":
        fields = inputs.PolynomialFields(530 + k, (0.1, -0.2, 0.3), (1.2, 0.9, 1.1))
        bv = fields.b(xv)
        # b . nu at the face points, nu the per-point normal of the multilinear cells
        bf = oracle_face_normal_velocity(geo, fields.b, xf)
        lib_kw.update(D_qp=fields.D(xv), D_face=fields.D(xf), c_qp=fields.c(xv), velocity="points", b_qp=bv,
                      b_face=bf)
        ora_kw.update(D_vol=fields.D(xv), D_face=fields.D(xf), c_vol=fields.c(xv), b_vol=bv, b_face=bf)
    pr = oracle.Problem(n, k, D, vertices=verts, **base, **ora_kw)
    f = np.cos(xv.sum(axis=-1))
    bcs = bc or ("dirichlet",) * 6
    data = [None if bcs[s] == "outflow" else np.sin(0.5 + oracle.face_points(pr, s) @ np.array([1.0, -0.7, 0.4])).ravel()
            for s in range(6)]
    u = inputs.uniform_u(pr.ndof, 540 + k)
    y_ref = oracle.apply(pr, u)
    r_ref = y_ref - oracle.rhs(pr, f, data)
    op = dg.Operator(n, k, D, vertices=verts, f_qp=f, g_qp=data, **base, **lib_kw)
    assert np.max(np.abs(op.quadrature_points(0) - xv)) < 1e-14
    assert np.max(np.abs(op.quadrature_points(7) - xf)) < 1e-14
    for s in range(6):
        assert np.max(np.abs(op.quadrature_points(1 + s) - oracle.face_points(pr, s))) < 1e-14
    ut = torch.tensor(u, device="cuda")
    assert relerr(op.apply_jacobian(ut).cpu().numpy(), y_ref) <= TOL
    assert relerr(op.apply_residual(ut).cpu().numpy(), r_ref) <= TOL
    assert relerr(op.apply_jacobian(ut, precision=dg.DG_F64X).cpu().numpy(), y_ref) <= TOL
    assert relerr(op.apply_residual(ut, precision=dg.DG_F64X).cpu().numpy(), r_ref) <= TOL
    op.close()


def oracle_face_normal_velocity(geo, bfun, xf):
    """b . nu at every cell's face points, nu the unit normal along +reference axis of the multilinear cell at that
    point, from the tangential derivatives of the trilinear map (nu is parallel to dx/da x dx/db)."""
    n = [int(v) for v in geo.n]
    V = geo.vertices.reshape(n[2] + 1, n[1] + 1, n[0] + 1, 3)
    m = geo.m
    xq, _ = oracle.gauss_legendre(m)
    out = np.empty(xf.shape[:3])
    bval = bfun(xf)
    for cell in range(geo.ncell):
        ix, iy, iz = cell % n[0], (cell // n[0]) % n[1], cell // (n[0] * n[1])
        C = V[iz:iz + 2, iy:iy + 2, ix:ix + 2]  # [c][b][a][xyz]
        for s in range(6):
            d, side = s // 2, s % 2
            ta, tb = (1, 2) if d == 0 else ((0, 2) if d == 1 else (0, 1))
            for p in range(m * m):
                xi = np.empty(3)
                xi[d], xi[ta], xi[tb] = side, xq[p % m], xq[p // m]
                J = np.zeros((3, 3))
                for c in range(2):
                    for b in range(2):
                        for a in range(2):
                            N = [(1 - xi[0], xi[0])[a], (1 - xi[1], xi[1])[b], (1 - xi[2], xi[2])[c]]
                            dN = [(-1.0, 1.0)[a], (-1.0, 1.0)[b], (-1.0, 1.0)[c]]
                            J[:, 0] += C[c, b, a] * dN[0] * N[1] * N[2]
                            J[:, 1] += C[c, b, a] * N[0] * dN[1] * N[2]
                            J[:, 2] += C[c, b, a] * N[0] * N[1] * dN[2]
                nu = np.linalg.inv(J)[d]
                nu /= np.linalg.norm(nu)
                out[cell, s, p] = bval[cell, s, p] @ nu
    return out


def test_multilinear_handles_reject_unsupported_options(dg):
    n, k = (2, 2, 2), 2
    verts = inputs.multilinear_vertices(n, seed=560)
    with pytest.raises(dg.DGError):
        dg.Operator(n, k, 1.0, vertices=verts, periodic=(1, 0, 0))
    with pytest.raises(dg.DGError):
        dg.Operator(n, k, 1.0, vertices=verts, jacobian=np.eye(3) * 0.5)
    bad = verts.copy()
    bad[13] = bad[0]  # the centre vertex moved onto a corner: the first cell folds (det J changes sign)
    with pytest.raises(dg.DGError):
        dg.Operator(n, k, 1.0, vertices=bad)
    op = dg.Operator(n, k, 1.0, vertices=verts, m=k + 3)
    with pytest.raises(dg.DGError):
        op.precond_setup()  # block-Jacobi is built for the scalar axis-parallel kernels only
    with pytest.raises(dg.DGError):
        op.project(torch.zeros(8 * (k + 3) ** 3, dtype=torch.float64, device="cuda"))
    z = torch.zeros(op.ndof, dtype=torch.float64, device="cuda")
    with pytest.raises(dg.DGError):
        op.ssprk2(z, 0.01, 1)
    op.close()


def test_multilinear_sampled_cells_at_bench_size(dg):
    """The benchmark's Problem C launch configuration: 32^3 multilinear cells, k = 7, m = 10, polynomial D(x) and
    c(x), constant b; sampled cells (corners included) against the oracle in FP64 and double-float."""
    n, k, m = (32, 32, 32), 7, 10
    seed = 80
    verts = inputs.multilinear_vertices(n, seed=seed, amplitude=0.2)
    fields = inputs.PolynomialFields(seed, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    nc = 32 ** 3
    geo = oracle.Problem(n, k, np.ones(nc), m=m, vertices=verts)
    xv, xf = oracle.volume_points(geo), oracle.cell_face_points(geo)
    Dv, Df, cv = fields.D(xv), fields.D(xf), fields.c(xv)
    del xv, xf
    b = tuple(fields.b0)
    pr = oracle.Problem(n, k, np.ones(nc), b=b, c=0.0, m=m, vertices=verts, D_vol=Dv, D_face=Df, c_vol=cv)
    op = dg.Operator(n, k, 1.0, b=b, c=0.0, m=m, vertices=verts, D_qp=Dv, D_face=Df, c_qp=cv)
    u = inputs.uniform_u(pr.ndof, seed + 1)
    ut = torch.tensor(u, device="cuda")
    y = op.apply_jacobian(ut).cpu().numpy().reshape(nc, -1)
    yx = op.apply_jacobian(ut, precision=dg.DG_F64X).cpu().numpy().reshape(nc, -1)
    op.close()
    cells = np.concatenate([np.random.default_rng(seed + 2).choice(nc, 8, replace=False),
                            [0, 31, 32 * 31, 32 * 32 - 1, nc - 32 * 32, nc - 1]])
    yref = oracle.apply(pr, u, cells=cells).reshape(len(cells), -1)
    assert relerr(y[cells], yref) <= TOL
    assert relerr(yx[cells], yref) <= TOL
