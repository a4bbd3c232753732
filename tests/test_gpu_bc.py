"""GPU parity of the Neumann and outflow boundary sides (Sec. 2, eq. modelproblem: Gamma_N with the total flux
j, Gamma_O with (D grad u) . nu = 0) against the FP64 oracle, on every operator path: the scalar kernels in
FP64, FP32 and double-float, the tensor-diffusion kernels on affine cells, the point-wise coefficient kernels
(Problem B) and the velocity field kernels with m = k+3; plus block-Jacobi, FGMRES and the batched apply.

Bars: FP64 and double-float <= 1e-12, FP32 <= 1e-5 (relative infinity norm), as for the Dirichlet-only tests.
"""

import numpy as np
import pytest

import oracle
from paper_1711_10885_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


@pytest.fixture(scope="module")
def dg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_10885_gb300 import dg as _dg
    return _dg


def relerr(y, ref):
    return float(np.max(np.abs(np.asarray(y, dtype=np.float64) - ref)) / max(np.max(np.abs(ref)), 1e-300))


def side_data(pr, bc, seed):
    """Seeded smooth data per side: g on Dirichlet sides, j on Neumann sides, none on outflow sides."""
    out = []
    for s in range(6):
        if bc[s] == "outflow" or pr.periodic[s // 2]:
            out.append(None)
            continue
        x = oracle.face_points(pr, s)
        out.append(np.sin((seed + s) * 0.7 + x @ np.array([1.1, -0.6, 0.8])).ravel())
    return out


BCS = [
    ("dirichlet", "outflow", "neumann", "dirichlet", "neumann", "outflow"),
    ("neumann",) * 6,
    ("outflow", "neumann", "dirichlet", "outflow", "outflow", "dirichlet"),
]

# (n, k, bc index)
SCALAR_CASES = [((3, 2, 2), 1, 0), ((2, 3, 2), 3, 1), ((2, 2, 3), 4, 2), ((3, 2, 2), 7, 0), ((1, 2, 2), 9, 2)]


@pytest.mark.parametrize("case", SCALAR_CASES, ids=lambda c: f"n{c[0]}k{c[1]}bc{c[2]}")
def test_scalar_kernels_with_mixed_sides_match_oracle(dg, case):
    n, k, bi = case
    bc = BCS[bi]
    w = inputs.small_case(n=n, k=k, sigma_D=1.0, seed=300 + k, b=(0.8, -0.5, 0.35), c=0.6)
    pr = oracle.Problem(w.n, w.k, w.D, b=w.b, c=w.c, bc=bc)
    xv = oracle.volume_points(pr)
    f = np.cos(xv.sum(axis=-1))
    data = side_data(pr, bc, k)
    y_ref = oracle.apply(pr, w.u)
    r_ref = y_ref - oracle.rhs(pr, f, data)
    op = dg.Operator(w.n, w.k, w.D, b=w.b, c=w.c, f_qp=f, g_qp=data, bc=bc)
    u = torch.tensor(w.u, device="cuda")
    assert relerr(op.apply_jacobian(u).cpu().numpy(), y_ref) <= TOL64
    assert relerr(op.apply_residual(u).cpu().numpy(), r_ref) <= TOL64
    assert relerr(op.apply_residual(u, precision=dg.DG_F64X).cpu().numpy(), r_ref) <= TOL64
    assert relerr(op.apply_residual(u.float()).cpu().numpy(), r_ref) <= TOL32
    op.close()


def test_tensor_kernels_on_affine_cells_with_mixed_sides(dg):
    from tests.test_oracle_tensor_pins import spd_tensors
    n, k, bc = (2, 3, 2), 4, BCS[2]
    nc = 12
    Dt = spd_tensors(nc, 310)
    J = inputs.sheared_jacobian((0.4, 0.3, 0.45), 311)
    b, c = (0.6, 0.4, -0.3), 0.5
    pr = oracle.Problem(n, k, np.ones(nc), b=b, c=c, D_tensor=Dt, J=J.ravel(), bc=bc)
    xv = oracle.volume_points(pr)
    f = np.exp(-xv[..., 0]) * np.cos(xv[..., 1])
    data = side_data(pr, bc, 5)
    u = inputs.uniform_u(pr.ndof, 312)
    r_ref = oracle.apply(pr, u) - oracle.rhs(pr, f, data)
    op = dg.Operator(n, k, 1.0, b=b, c=c, D_tensor=Dt, jacobian=J, f_qp=f, g_qp=data, bc=bc)
    ut = torch.tensor(u, device="cuda")
    assert relerr(op.apply_residual(ut).cpu().numpy(), r_ref) <= TOL64
    assert relerr(op.apply_residual(ut, precision=dg.DG_F64X).cpu().numpy(), r_ref) <= TOL64
    op.close()


def test_pointwise_kernels_with_mixed_sides(dg):
    from tests.test_gpu_pointwise import problem_b
    n, k, m, bc = (2, 2, 3), 3, 6, BCS[0]
    pr, kw, xv, _ = problem_b(n, k, m, (0, 0, 0), True, 320, True)
    prb = oracle.Problem(n, k, np.ones(pr.ncell), b=(0, 0, 0), c=0.0, sigma=pr.sigma, lo=pr.lo, hi=pr.hi, m=m,
                         J=pr.J, D_vol=pr.D_vol, D_face=pr.D_face, c_vol=pr.c_vol, b_vol=pr.b_vol,
                         b_face=pr.b_face, bc=bc)
    f = np.cos(xv.sum(axis=-1))
    data = side_data(prb, bc, 7)
    u = inputs.uniform_u(prb.ndof, 321)
    r_ref = oracle.apply(prb, u) - oracle.rhs(prb, f, data)
    op = dg.Operator(n, k, 1.0, f_qp=f, g_qp=data, bc=bc, **kw)
    ut = torch.tensor(u, device="cuda")
    assert relerr(op.apply_residual(ut).cpu().numpy(), r_ref) <= TOL64
    assert relerr(op.apply_residual(ut, precision=dg.DG_F64X).cpu().numpy(), r_ref) <= TOL64
    op.close()


def test_velocity_field_kernels_with_outflow_side(dg):
    """m = k+3 and b(x) given at the points, outflow on the downstream x side (b_x > 0 there)."""
    n, k, m = (3, 2, 2), 3, 6
    bc = ("dirichlet", "outflow", "neumann", "neumann", "dirichlet", "dirichlet")
    w = inputs.small_case(n=n, k=k, sigma_D=0.5, seed=330)
    base = oracle.Problem(n, k, w.D, b=(0, 0, 0), c=0.4, m=m)

    def bfun(x):
        return np.stack([1.0 + 0.3 * x[..., 1], 0.2 * np.sin(x[..., 0]), -0.3 + 0.1 * x[..., 2]], axis=-1)

    bv = bfun(oracle.volume_points(base))
    bf = inputs.face_normal_velocity(bfun, oracle.cell_face_points(base))
    pr = oracle.Problem(n, k, w.D, b=(0, 0, 0), c=0.4, m=m, b_vol=bv, b_face=bf, bc=bc)
    data = side_data(pr, bc, 9)
    r_ref = oracle.apply(pr, w.u) - oracle.rhs(pr, None, data)
    op = dg.Operator(n, k, w.D, b=(0, 0, 0), c=0.4, m=m, velocity="points", b_qp=bv, b_face=bf, g_qp=data, bc=bc)
    u = torch.tensor(w.u, device="cuda")
    assert relerr(op.apply_residual(u).cpu().numpy(), r_ref) <= TOL64
    assert relerr(op.apply_residual(u, precision=dg.DG_F64X).cpu().numpy(), r_ref) <= TOL64
    op.close()


def oracle_matrix(pr):
    N = pr.ndof
    A = np.empty((N, N))
    e = np.zeros(N)
    for j in range(N):
        e[j] = 1.0
        A[:, j] = oracle.apply(pr, e)
        e[j] = 0.0
    return A


def test_block_jacobi_and_solve_with_mixed_sides(dg):
    n, k, bc = (3, 2, 2), 2, BCS[0]
    w = inputs.small_case(n=n, k=k, seed=340, b=(0.7, -0.4, 0.2), c=0.8)
    pr = oracle.Problem(w.n, w.k, w.D, b=w.b, c=w.c, bc=bc)
    A = oracle_matrix(pr)
    xv = oracle.volume_points(pr)
    f = np.cos(xv.sum(axis=-1))
    data = side_data(pr, bc, 11)
    F = oracle.rhs(pr, f, data)
    op = dg.Operator(w.n, w.k, w.D, b=w.b, c=w.c, f_qp=f, g_qp=data, bc=bc)
    op.precond_setup()
    r = np.random.default_rng(341).uniform(-1, 1, w.ndof)
    z = op.precond_apply(torch.tensor(r, device="cuda")).cpu().numpy()
    nb = w.nb
    z_ref = np.concatenate([np.linalg.solve(A[c * nb:(c + 1) * nb, c * nb:(c + 1) * nb], r[c * nb:(c + 1) * nb])
                            for c in range(w.ncell)])
    assert np.max(np.abs(z - z_ref)) <= 1e-10 * np.max(np.abs(z_ref))
    x = torch.zeros(w.ndof, dtype=torch.float64, device="cuda")
    st = op.solve(x, mode=dg.DG_SOLVE_FP64, preconditioner=dg.DG_PRECOND_BLOCK_JACOBI, rtol=1e-12, restart=30)
    assert st["rc"] == 0
    x_ref = np.linalg.solve(A, F)
    assert np.max(np.abs(x.cpu().numpy() - x_ref)) <= 1e-9 * np.max(np.abs(x_ref))
    op.close()


def test_batch_with_mixed_sides_equals_standalone(dg):
    ws = inputs.batch_problems(count=6, seed=350, nmin=1, nmax=4, kmin=1, kmax=6)
    ops = [dg.Operator(w.n, w.k, w.D, b=w.b, c=w.c, f_qp=np.ones(w.ncell * (w.k + 1) ** 3), bc=BCS[i % 3])
           for i, w in enumerate(ws)]
    batch = dg.Batch(ops)
    xs = [torch.tensor(w.u, device="cuda") for w in ws]
    ys = [torch.empty_like(x) for x in xs]
    batch.apply(xs, ys, residual=True)
    torch.cuda.synchronize()
    for i, (w, op, x, y) in enumerate(zip(ws, ops, xs, ys)):
        assert torch.equal(y, op.apply_residual(x))
        pr = oracle.Problem(w.n, w.k, w.D, b=w.b, c=w.c, bc=BCS[i % 3])
        ref = oracle.apply(pr, w.u) - oracle.rhs(pr, np.ones(w.ncell * (w.k + 1) ** 3), None)
        assert relerr(y.cpu().numpy(), ref) <= TOL64
    batch.close()
    for op in ops:
        op.close()


def test_bad_boundary_type_is_rejected(dg):
    with pytest.raises(dg.DGError):
        dg.Operator((2, 2, 2), 2, 1.0, bc=(0, 0, 3, 0, 0, 0))
