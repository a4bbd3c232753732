"""GPU parity of the tensor-diffusion / affine-geometry kernels against the FP64 oracle: a symmetric
positive definite diffusion tensor per cell (Sec. 5.1, "tensor-valued diffusion coefficients", the paper's
Problem A) on the axis-parallel grid and on affine cells (the geometry of Problem B).

Bar: FP64 and double-float results within 1e-12 of the oracle (relative infinity norm).
"""

import numpy as np
import pytest

import oracle
from paper_1711_10885_gb300 import inputs
from tests.test_oracle_tensor_pins import full, packed, spd_tensors

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


def shear_rotation():
    th = 0.35
    R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1]])
    S = np.array([[1.0, 0.25, -0.15], [0.0, 1.1, 0.3], [0.05, 0.0, 0.9]])
    return R @ S


# (n, k, periodic, affine)
CASES = [
    ((3, 2, 4), 1, (0, 0, 0), False),
    ((3, 2, 2), 2, (1, 0, 0), False),
    ((2, 3, 2), 3, (0, 1, 1), True),
    ((2, 2, 3), 4, (0, 0, 0), True),
    ((3, 2, 2), 5, (1, 1, 1), False),
    ((2, 2, 2), 6, (0, 0, 0), True),
    ((2, 3, 2), 7, (0, 0, 1), False),
    ((2, 2, 2), 8, (1, 0, 0), True),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"n{c[0]}k{c[1]}p{c[2]}{'aff' if c[3] else ''}")
def test_tensor_operator_and_residual_match_oracle(dg, case):
    n, k, per, affine = case
    nc = int(np.prod(n))
    Dt = spd_tensors(nc, 20 + k)
    b = np.array([0.7, -0.4, 0.3])
    c = 0.6
    lo = (0.1, -0.2, 0.3)
    hi = (1.1, 1.3, 1.0)
    h = (np.asarray(hi) - np.asarray(lo)) / np.asarray(n)
    J = shear_rotation() @ np.diag(h) if affine else None
    sigma = dg.dg_penalty_sigma(k, 0)
    pr = oracle.Problem(n, k, np.ones(nc), b=b, c=c, sigma=sigma, lo=lo, hi=hi, periodic=per, D_tensor=Dt,
                        J=None if J is None else J.ravel())
    xv = oracle.volume_points(pr)
    f = np.cos(xv.sum(axis=-1))
    g = [None if per[s // 2] else np.sin(2 * oracle.face_points(pr, s).sum(axis=-1)).ravel() for s in range(6)]
    u = inputs.uniform_u(pr.ndof, 30 + k)
    y_ref = oracle.apply(pr, u)
    r_ref = y_ref - oracle.rhs(pr, f, g)
    op = dg.Operator(n, k, 1.0, b=b, c=c, sigma=sigma, lo=lo, hi=hi, periodic=per, D_tensor=Dt, jacobian=J,
                     f_qp=f, g_qp=g)
    # the library's quadrature points follow the affine map like the oracle's
    assert np.max(np.abs(op.quadrature_points(0) - xv)) < 1e-13
    u64 = torch.tensor(u, device="cuda")
    assert relerr(op.apply_jacobian(u64).cpu().numpy(), y_ref) <= TOL
    assert relerr(op.apply_residual(u64).cpu().numpy(), r_ref) <= TOL
    assert relerr(op.apply_jacobian(u64, precision=dg.DG_F64X).cpu().numpy(), y_ref) <= TOL
    assert relerr(op.apply_residual(u64, precision=dg.DG_F64X).cpu().numpy(), r_ref) <= TOL
    op.close()


def test_isotropic_tensor_handle_equals_scalar_handle(dg):
    w = inputs.small_case(n=(4, 3, 3), k=3, seed=41)
    Dt = np.stack([w.D, w.D, w.D, 0 * w.D, 0 * w.D, 0 * w.D], axis=1)
    op0 = dg.operator_for(w)
    op1 = dg.Operator(w.n, w.k, 1.0, b=w.b, c=w.c, D_tensor=Dt, f_qp=np.ones(w.ncell * (w.k + 1) ** 3))
    u = torch.tensor(w.u, device="cuda")
    assert relerr(op1.apply_residual(u).cpu().numpy(), op0.apply_residual(u).cpu().numpy()) <= TOL
    op0.close()
    op1.close()


def test_tensor_stage_and_projection_on_affine_mesh(dg):
    n, k = (3, 2, 2), 3
    nc = 12
    J = shear_rotation() @ np.diag([0.4, 0.5, 0.45])
    Dt = spd_tensors(nc, 50)
    b = np.array([0.5, 0.2, -0.3])
    pr = oracle.Problem(n, k, np.ones(nc), b=b, c=0.0, D_tensor=Dt, J=J.ravel(), periodic=(1, 1, 1))
    op = dg.Operator(n, k, 1.0, b=b, c=0.0, D_tensor=Dt, jacobian=J, periodic=(1, 1, 1))
    xv = oracle.volume_points(pr)
    u0 = np.exp(-np.sum((xv - xv.mean(axis=(0, 1))) ** 2, axis=-1))
    detJ = abs(np.linalg.det(J))
    z_ref = oracle.rhs(pr, u0, None) / detJ
    z = op.project(torch.tensor(u0, device="cuda"))
    assert relerr(z.cpu().numpy(), z_ref) <= TOL
    dt = 0.01
    y = torch.empty_like(z)
    op.rk_stage(z, z, y, 0.5, 0.5, dt)
    ref = z_ref - dt / detJ * oracle.apply(pr, z_ref)  # 0.5 z + 0.5 z - dt M^{-1} A z, F = 0
    assert relerr(y.cpu().numpy(), ref) <= TOL
    op.close()


def test_tensor_sampled_cells_at_bench_size(dg):
    """32^3 cells, k = 7 (the q = 2p workload size) with per-cell tensors: sampled cells against the oracle."""
    w = inputs.unit_cube_q7_32()
    Dt = inputs.log_normal_tensors(w.ncell, 1.0, 60)
    op = dg.Operator(w.n, w.k, 1.0, b=w.b, c=w.c, D_tensor=Dt)
    y = op.apply_jacobian(torch.tensor(w.u, device="cuda")).cpu().numpy().reshape(w.ncell, -1)
    pr = oracle.Problem(w.n, w.k, np.ones(w.ncell), b=w.b, c=w.c, D_tensor=Dt)
    cells = np.concatenate([np.random.default_rng(8).choice(w.ncell, 6, replace=False), [0, w.ncell - 1, 1023]])
    yref = oracle.apply(pr, w.u, cells=cells).reshape(len(cells), -1)
    assert relerr(y[cells], yref) <= TOL
    op.close()


def test_tensor_handles_reject_unsupported_calls(dg):
    op = dg.Operator((2, 2, 2), 2, 1.0, D_tensor=spd_tensors(8, 70))
    with pytest.raises(dg.DGError):
        op.apply_jacobian(torch.zeros(op.ndof, device="cuda", dtype=torch.float32))
    with pytest.raises(dg.DGError):
        op.precond_setup()
    with pytest.raises(dg.DGError):
        dg.Batch([op])
    op.close()
