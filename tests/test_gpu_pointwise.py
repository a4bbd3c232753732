"""GPU parity of the point-wise coefficient kernels (Problem B of Sec. 5.1: affine cells, coefficients that are
polynomials in the coordinates, q = 2p+4) against the FP64 oracle, which evaluates eq. blf by direct quadrature
with D, b and c taken at every quadrature point.

Bar: FP64 and double-float results within 1e-12 of the oracle (relative infinity norm), as for the other
operator paths.  Inputs: the seeded polynomial fields of inputs.PolynomialFields, evaluated at the oracle's
quadrature points (the library's agree with them to rounding, which is checked).
"""

import numpy as np
import pytest

import oracle
from paper_1711_10885_gb300 import inputs

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


def problem_b(n, k, m, periodic, affine, seed, velocity_points, lo=(0.1, -0.2, 0.3), hi=(1.1, 1.3, 1.0)):
    """Oracle problem and library arguments for Problem B on an n-cell grid (affine: sheared cells)."""
    nc = int(np.prod(n))
    h = (np.asarray(hi) - np.asarray(lo)) / np.asarray(n)
    J = inputs.sheared_jacobian(h, seed) if affine else np.diag(h)
    fields = inputs.PolynomialFields(seed, lo, np.asarray(lo) + J @ np.asarray(n, dtype=np.float64))
    sigma = oracle.penalty_sigma(k)
    geo = oracle.Problem(n, k, np.ones(nc), b=(0, 0, 0), c=0.0, sigma=sigma, lo=lo, hi=hi, m=m,
                         periodic=periodic, J=J.ravel() if affine else None)
    xv = oracle.volume_points(geo)
    xf = oracle.cell_face_points(geo)
    Dv, Df, cv = fields.D(xv), fields.D(xf), fields.c(xv)
    b_const = fields.b0
    if velocity_points:
        bv, bf = fields.b(xv), inputs.face_normal_velocity_affine(fields.b, xf, J)
    else:
        bv = np.broadcast_to(b_const, xv.shape).copy()
        bf = inputs.face_normal_velocity_affine(lambda x: np.broadcast_to(b_const, x.shape), xf, J)
    pr = oracle.Problem(n, k, np.ones(nc), b=(0, 0, 0), c=0.0, sigma=sigma, lo=lo, hi=hi, m=m, periodic=periodic,
                        J=J.ravel() if affine else None, D_vol=Dv, D_face=Df, c_vol=cv, b_vol=bv, b_face=bf)
    kw = dict(b=tuple(b_const), c=0.0, sigma=sigma, lo=lo, hi=hi, m=m, periodic=periodic,
              jacobian=J if affine else None, D_qp=Dv, D_face=Df, c_qp=cv)
    if velocity_points:
        kw.update(velocity="points", b_qp=fields.b(xv), b_face=bf)
    return pr, kw, xv, xf


# (n, k, m - k, periodic, affine, velocity given at the points)
CASES = [
    ((3, 2, 2), 1, 3, (0, 0, 0), True, True),
    ((2, 3, 2), 2, 3, (1, 0, 0), True, False),
    ((2, 2, 3), 3, 1, (0, 1, 1), False, False),
    ((2, 2, 2), 4, 3, (0, 0, 0), True, True),
    ((3, 2, 2), 5, 3, (1, 1, 1), True, False),
    ((2, 2, 2), 6, 1, (0, 0, 1), True, False),
    ((3, 1, 3), 7, 3, (0, 0, 0), True, True),
    ((3, 1, 3), 8, 3, (1, 0, 0), False, False),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"n{c[0]}k{c[1]}m{c[1] + c[2]}p{c[3]}{'aff' if c[4] else ''}"
                                                      f"{'bx' if c[5] else ''}")
def test_pointwise_operator_and_residual_match_oracle(dg, case):
    n, k, dm, per, affine, vpts = case
    m = k + dm
    pr, kw, xv, xf = problem_b(n, k, m, per, affine, 100 + k, vpts)
    f = np.cos(xv.sum(axis=-1))
    g = [None if per[s // 2] else np.sin(2 * oracle.face_points(pr, s).sum(axis=-1)).ravel() for s in range(6)]
    u = inputs.uniform_u(pr.ndof, 130 + k)
    y_ref = oracle.apply(pr, u)
    r_ref = y_ref - oracle.rhs(pr, f, g)
    op = dg.Operator(n, k, 1.0, f_qp=f, g_qp=g, **kw)
    # the library's quadrature points (volume and every cell face) follow the map like the oracle's
    assert np.max(np.abs(op.quadrature_points(0) - xv)) < 1e-13
    assert np.max(np.abs(op.quadrature_points(7) - xf)) < 1e-13
    u64 = torch.tensor(u, device="cuda")
    assert relerr(op.apply_jacobian(u64).cpu().numpy(), y_ref) <= TOL
    assert relerr(op.apply_residual(u64).cpu().numpy(), r_ref) <= TOL
    assert relerr(op.apply_jacobian(u64, precision=dg.DG_F64X).cpu().numpy(), y_ref) <= TOL
    assert relerr(op.apply_residual(u64, precision=dg.DG_F64X).cpu().numpy(), r_ref) <= TOL
    op.close()


def test_constant_point_tables_equal_tensor_handle(dg):
    """Point tables that repeat one tensor per cell give the per-cell tensor operator (q = 2p)."""
    from tests.test_oracle_tensor_pins import spd_tensors
    n, k = (3, 2, 3), 3
    nc, m = 18, 4
    Dt = spd_tensors(nc, 140)
    J = inputs.sheared_jacobian((0.3, 0.4, 0.35), 141)
    b, c = (0.6, -0.3, 0.2), 0.8
    Dv = np.repeat(Dt[:, None, :], m ** 3, axis=1)
    Df = np.repeat(Dt[:, None, None, :], 6 * m ** 2, axis=1).reshape(nc, 6, m ** 2, 6)
    op_t = dg.Operator(n, k, 1.0, b=b, c=c, D_tensor=Dt, jacobian=J, f_qp=np.ones(nc * m ** 3))
    op_p = dg.Operator(n, k, 1.0, b=b, c=0.0, D_qp=Dv, D_face=Df, c_qp=np.full((nc, m ** 3), c), jacobian=J,
                       f_qp=np.ones(nc * m ** 3))
    u = torch.tensor(inputs.uniform_u(nc * (k + 1) ** 3, 142), device="cuda")
    for prec in (dg.DG_F64, dg.DG_F64X):
        assert relerr(op_p.apply_residual(u, precision=prec).cpu().numpy(),
                      op_t.apply_residual(u, precision=prec).cpu().numpy()) <= TOL
    op_t.close()
    op_p.close()


def test_pointwise_stage_and_projection(dg):
    n, k, m = (2, 3, 2), 3, 6
    pr, kw, xv, _ = problem_b(n, k, m, (1, 1, 1), True, 150, False)
    op = dg.Operator(n, k, 1.0, **kw)
    u0 = np.exp(-np.sum((xv - xv.mean(axis=(0, 1))) ** 2, axis=-1))
    detJ = abs(np.linalg.det(kw["jacobian"]))
    z_ref = oracle.rhs(pr, u0, None) / detJ
    z = op.project(torch.tensor(u0, device="cuda"))
    assert relerr(z.cpu().numpy(), z_ref) <= TOL
    dt = 0.01
    y = torch.empty_like(z)
    for prec in (dg.DG_F64, dg.DG_F64X):
        op.rk_stage(z, z, y, 0.5, 0.5, dt, precision=prec)
        ref = z_ref - dt / detJ * oracle.apply(pr, z_ref)  # 0.5 z + 0.5 z - dt M^{-1} A z, F = 0
        assert relerr(y.cpu().numpy(), ref) <= TOL
    op.close()


def test_pointwise_sampled_cells_at_bench_size(dg):
    """32^3 sheared cells, k = 7, q = 2p+4 (m = 10), polynomial D(x), b(x), c(x): the benchmark's Problem B
    launch configuration, sampled cells (corners included) against the oracle in FP64 and double-float."""
    n, k, m = (32, 32, 32), 7, 10
    pr, kw, _, _ = problem_b(n, k, m, (0, 0, 0), True, 160, True, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0))
    u = inputs.uniform_u(pr.ndof, 161)
    op = dg.Operator(n, k, 1.0, **kw)
    u64 = torch.tensor(u, device="cuda")
    y = op.apply_jacobian(u64).cpu().numpy().reshape(pr.ncell, -1)
    yx = op.apply_jacobian(u64, precision=dg.DG_F64X).cpu().numpy().reshape(pr.ncell, -1)
    op.close()
    nc = pr.ncell
    cells = np.concatenate([np.random.default_rng(162).choice(nc, 8, replace=False),
                            [0, 31, 32 * 31, 32 * 32 - 1, nc - 32 * 32, nc - 1]])
    yref = oracle.apply(pr, u, cells=cells).reshape(len(cells), -1)
    assert relerr(y[cells], yref) <= TOL
    assert relerr(yx[cells], yref) <= TOL


def test_pointwise_handles_reject_bad_input(dg):
    n, k, m = (2, 2, 2), 2, 5
    pr, kw, xv, xf = problem_b(n, k, m, (0, 0, 0), True, 170, False)
    op = dg.Operator(n, k, 1.0, **kw)
    with pytest.raises(dg.DGError):
        op.apply_jacobian(torch.zeros(op.ndof, device="cuda", dtype=torch.float32))
    with pytest.raises(dg.DGError):
        op.precond_setup()
    op.close()
    bad = dict(kw)
    bad["D_face"] = None
    with pytest.raises(dg.DGError):
        dg.Operator(n, k, 1.0, **bad)
    Dv = kw["D_qp"].copy()
    Dv[3, 7] = [1.0, 1.0, 1.0, 2.0, 0.0, 0.0]  # not positive definite at one point
    bad = dict(kw, D_qp=Dv)
    with pytest.raises(dg.DGError):
        dg.Operator(n, k, 1.0, **bad)
    bad = dict(kw, velocity="taylor_green")
    with pytest.raises(dg.DGError):
        dg.Operator(n, k, 1.0, **bad)
