"""GPU parity of the transport extension (Sec. 5.3) against the FP64 oracle: periodic axes, a velocity field
at the quadrature points (given point-wise, or the Taylor-Green field evaluated by the library), the
q = 2p+4 rule (m = k+3), the L2 projection of the initial value, Runge-Kutta stages and Heun's method.

Bars (written here): FP64 results within ||y - y_oracle||_inf / ||y_oracle||_inf <= 1e-12 (the library's
Taylor-Green field comes from CUDA's sin/cos and the oracle's from numpy's, a difference of a few units in
the last place of b); FP32 and double-float applies as in test_gpu_operator (the velocity field kernels also run in
double-float and meet the FP64 bar); Heun steps within 1e-11 of
the same steps taken with oracle applies; mass (sum of the cell means) conserved to 1e-13 relative.
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


def smooth_field(seed, lo, hi):
    """A seeded smooth non-polynomial velocity field (not divergence-free) for the point-wise path, periodic
    on the box [lo, hi] so that it is one field across the end faces of a periodic axis (the library takes
    an interior face's normal velocity from its lower cell, the oracle from each cell's own values)."""
    rng = np.random.default_rng(seed)
    A = rng.uniform(0.3, 1.2, 3)
    K = rng.integers(1, 3, (3, 3)) * 2 * np.pi / (np.asarray(hi, float) - np.asarray(lo, float))
    P = rng.uniform(0, 2 * np.pi, 3)

    def b(xyz):
        return np.stack([A[r] * np.sin((xyz - np.asarray(lo, float)) @ K[r] + P[r]) for r in range(3)], axis=-1)
    return b


def oracle_with_field(n, k, D, c, sigma, lo, hi, periodic, m, bfun):
    base = oracle.Problem(n, k, D, b=(0, 0, 0), c=c, sigma=sigma, lo=lo, hi=hi, m=m, periodic=periodic)
    bvol = bfun(oracle.volume_points(base))
    bface = inputs.face_normal_velocity(bfun, oracle.cell_face_points(base))
    return oracle.Problem(n, k, D, b=(0, 0, 0), c=c, sigma=sigma, lo=lo, hi=hi, m=m, periodic=periodic,
                          b_vol=bvol, b_face=bface)


# periodic axes with a constant velocity on the m = k+1 kernels (every precision)
PERIODIC_CONST = [
    ((3, 2, 4), 2, (1, 0, 1), (1.0, -0.5, 0.25)),
    ((5, 4, 3), 3, (1, 1, 1), (-0.7, 0.4, 1.1)),
    ((1, 3, 2), 4, (1, 1, 0), (0.3, 0.9, -0.6)),  # one cell along x: the cell is its own neighbour
    ((4, 3, 3), 7, (0, 0, 1), (1.0, 0.5, 0.25)),
]


@pytest.mark.parametrize("case", PERIODIC_CONST, ids=lambda c: f"n{c[0]}k{c[1]}p{c[2]}")
def test_periodic_constant_velocity_all_precisions(dg, case):
    n, k, per, b = case
    w = inputs.small_case(n=n, k=k, sigma_D=1.0, seed=40 + k, b=b, c=0.7)
    w.periodic = per
    pr = oracle.Problem(w.n, w.k, w.D, b=w.b, c=w.c, periodic=per)
    y_ref = oracle.apply(pr, w.u)
    F_ref = oracle.rhs(pr, np.ones(pr.ncell * pr.m ** 3), None)
    op = dg.operator_for(w)
    u64 = torch.tensor(w.u, device="cuda")
    assert relerr(op.apply_jacobian(u64).cpu().numpy(), y_ref) <= TOL64
    assert relerr(op.apply_residual(u64).cpu().numpy(), y_ref - F_ref) <= TOL64
    assert relerr(op.apply_jacobian(u64.float()).cpu().numpy(), y_ref) <= TOL32
    assert relerr(op.apply_jacobian(u64, precision=dg.DG_F64X).cpu().numpy(), y_ref) <= TOL64
    op.close()


# (n, k, m - k, periodic, lo, hi): velocity given point-wise, both quadrature rules, Dirichlet and periodic axes
FIELD_CASES = [
    ((3, 2, 4), 1, 1, (0, 0, 0), (0, 0, 0), (1, 1, 1)),
    ((3, 2, 4), 2, 3, (1, 0, 0), (0, -1, 0), (1, 1, 2)),
    ((2, 3, 2), 3, 1, (0, 1, 1), (0, 0, 0), (1, 1, 1)),
    ((3, 3, 2), 4, 3, (1, 1, 1), (0, 0, 0), (2, 1, 1)),
    ((2, 2, 3), 5, 3, (0, 0, 0), (0, 0, 0), (1, 1, 1)),
    ((2, 2, 2), 6, 1, (1, 0, 1), (0, 0, 0), (1, 1, 1)),
    ((2, 3, 2), 7, 3, (0, 1, 0), (0, 0, 0), (1, 1, 1)),
    ((2, 2, 2), 8, 3, (1, 1, 1), (0, 0, 0), (1, 1, 1)),
]


@pytest.mark.parametrize("case", FIELD_CASES, ids=lambda c: f"n{c[0]}k{c[1]}m+{c[2]}p{c[3]}")
def test_velocity_field_given_at_points(dg, case):
    n, k, dm, per, lo, hi = case
    m = k + dm
    ncell = int(np.prod(n))
    D = inputs.log_normal_D(ncell, 1.0, 60 + k)
    u = inputs.uniform_u(ncell * (k + 1) ** 3, 61 + k)
    bfun = smooth_field(62 + k, lo, hi)
    sigma = 2.0 * k * (k + 1)
    pr = oracle_with_field(n, k, D, 0.4, sigma, lo, hi, per, m, bfun)
    # right hand side with a source and Dirichlet data on the non-periodic sides (inflow reads b . nu)
    f = np.cos(oracle.volume_points(pr).sum(axis=-1))
    g = [None if per[s // 2] else np.sin(3 * oracle.face_points(pr, s).sum(axis=-1)).ravel() for s in range(6)]
    y_ref = oracle.apply(pr, u)
    r_ref = y_ref - oracle.rhs(pr, f, g)
    op = dg.Operator(n, k, D, b=(0, 0, 0), c=0.4, sigma=sigma, lo=lo, hi=hi, periodic=per, m=m, velocity="points",
                     b_qp=pr.b_vol, b_face=pr.b_face, f_qp=f, g_qp=g)
    # the library's quadrature points are the oracle's (same rule, independently computed)
    assert np.max(np.abs(op.quadrature_points(0) - oracle.volume_points(pr))) < 1e-13
    u64 = torch.tensor(u, device="cuda")
    assert relerr(op.apply_jacobian(u64).cpu().numpy(), y_ref) <= TOL64
    assert relerr(op.apply_residual(u64).cpu().numpy(), r_ref) <= TOL64
    assert relerr(op.apply_residual(u64, precision=dg.DG_F64X).cpu().numpy(), r_ref) <= TOL64
    op.close()


def tg_oracle(w):
    return oracle_with_field(w.n, w.k, w.D, w.c, 2.0 * w.k * (w.k + 1), w.lo, w.hi, w.periodic, w.m,
                             inputs.taylor_green_velocity)


@pytest.mark.parametrize("n,k,m", [(3, 2, 5), (4, 3, 6), (3, 5, 8), (2, 4, 5), (3, 1, 4)])
def test_taylor_green_field_evaluated_on_device(dg, n, k, m):
    w = inputs.taylor_green(n, k, m=m)
    pr = tg_oracle(w)
    u = inputs.uniform_u(w.ndof, 70 + k)
    op = dg.operator_for(w)
    u64 = torch.tensor(u, device="cuda")
    y_ref = oracle.apply(pr, u)
    assert relerr(op.apply_jacobian(u64).cpu().numpy(), y_ref) <= TOL64
    # the same velocity field kernels in double-float arithmetic meet the FP64 bar
    assert relerr(op.apply_jacobian(u64, precision=dg.DG_F64X).cpu().numpy(), y_ref) <= TOL64
    op.close()


def test_projection_of_initial_value(dg):
    w = inputs.taylor_green(3, 4)
    op = dg.operator_for(w)
    pr = tg_oracle(w)
    u0 = inputs.gaussian_bump(oracle.volume_points(pr))
    z = op.project(torch.tensor(u0, device="cuda").contiguous()).cpu().numpy()
    # (u0, phi_i)_T / |T| from the oracle's right hand side functional with f = u0 and no boundary data
    vol = np.prod((np.asarray(w.hi) - np.asarray(w.lo)) / np.asarray(w.n))
    ref = oracle.rhs(pr, u0, None) / vol
    assert relerr(z, ref) <= TOL64
    # a polynomial of degree <= k is reproduced exactly: project the oracle's own evaluation of a DG field
    zc = inputs.uniform_u(w.ndof, 80)
    vals = oracle_field_values(pr, zc)
    zp = op.project(torch.tensor(vals, device="cuda")).cpu().numpy()
    assert relerr(zp, zc) <= 1e-12
    op.close()


def oracle_field_values(pr, z):
    """Values of the DG field z at the oracle's volume points, from its 1D basis (sum over the tensor basis)."""
    x, _ = oracle.gauss_legendre(pr.m)
    th = np.array([oracle.basis_1d(pr.k, xi)[0] for xi in x])  # [m][k+1]
    zc = z.reshape(pr.ncell, pr.k + 1, pr.k + 1, pr.k + 1)      # [cell][j3][j2][j1]
    v = np.einsum("cfed,ad,be,gf->cgba", zc, th, th, th)          # [cell][i3][i2][i1]
    return np.ascontiguousarray(v.reshape(pr.ncell, pr.m ** 3))


def oracle_heun(pr, z, F, dt, vol, steps):
    for _ in range(steps):
        z1 = z - dt / vol * (oracle.apply(pr, z) - F)
        z = 0.5 * (z + z1 - dt / vol * (oracle.apply(pr, z1) - F))
    return z


def test_rk_stage_and_heun_match_oracle_steps(dg):
    w = inputs.taylor_green(3, 3)
    pr = tg_oracle(w)
    op = dg.operator_for(w)
    vol = np.prod((np.asarray(w.hi) - np.asarray(w.lo)) / np.asarray(w.n))
    z0 = oracle.rhs(pr, inputs.gaussian_bump(oracle.volume_points(pr)), None) / vol
    F = np.zeros(w.ndof)
    dt = 0.05
    zt = torch.tensor(z0, device="cuda")
    u = torch.tensor(inputs.uniform_u(w.ndof, 90), device="cuda")
    y = torch.empty_like(zt)
    op.rk_stage(u, zt, y, 0.25, 0.75, dt)
    ref = 0.25 * z0 + 0.75 * u.cpu().numpy() - dt / vol * (oracle.apply(pr, u.cpu().numpy()) - F)
    assert relerr(y.cpu().numpy(), ref) <= TOL64
    yx = torch.empty_like(zt)
    op.rk_stage(u, zt, yx, 0.25, 0.75, dt, precision=dg.DG_F64X)
    assert relerr(yx.cpu().numpy(), ref) <= TOL64
    zx = zt.clone()
    op.ssprk2(zt, dt, 3)
    ref3 = oracle_heun(pr, z0, F, dt, vol, 3)
    assert relerr(zt.cpu().numpy(), ref3) <= 1e-11
    op.ssprk2(zx, dt, 3, precision=dg.DG_F64X)
    assert relerr(zx.cpu().numpy(), ref3) <= 1e-11
    op.close()


def test_heun_with_source_and_dirichlet_data(dg):
    """A non-periodic problem with f and g: the stage subtracts F (M dz/dt + A z = F, Sec. 2)."""
    n, k = (3, 2, 2), 2
    w = inputs.small_case(n=n, k=k, seed=95, b=(0.6, -0.3, 0.2), c=0.5)
    pr = oracle.Problem(w.n, w.k, w.D, b=w.b, c=w.c)
    g = [np.full(pr.n[[1, 0, 0][s // 2]] * pr.n[[2, 2, 1][s // 2]] * pr.m ** 2, 0.3 * (s + 1)) for s in range(6)]
    F = oracle.rhs(pr, np.ones(pr.ncell * pr.m ** 3), g)
    op = dg.Operator(w.n, w.k, w.D, b=w.b, c=w.c, f_qp=np.ones(pr.ncell * pr.m ** 3), g_qp=g)
    vol = 1.0 / np.prod(n)
    zt = torch.tensor(w.u, device="cuda")
    op.ssprk2(zt, 1e-3, 2)
    assert relerr(zt.cpu().numpy(), oracle_heun(pr, w.u, F, 1e-3, vol, 2)) <= 1e-11
    op.close()


def test_mass_is_conserved_by_periodic_transport(dg):
    w = inputs.taylor_green(6, 3)
    op = dg.operator_for(w)
    u0 = inputs.gaussian_bump(op.quadrature_points(0))
    z = op.project(torch.tensor(u0, device="cuda"))
    zx = z.clone()
    mass0 = z.view(w.ncell, -1)[:, 0].sum().item()
    op.ssprk2(z, 0.02, 20)
    op.ssprk2(zx, 0.02, 20, precision=dg.DG_F64X)
    for zz in (z, zx):
        zc = zz.view(w.ncell, -1)[:, 0]
        assert abs(zc.sum().item() - mass0) <= 1e-13 * zc.abs().sum().item()
        assert torch.isfinite(zz).all()
    # 20 steps in double-float stay within FP64-level distance of the FP64 steps
    assert relerr(zx.cpu().numpy(), z.cpu().numpy()) <= 1e-11
    op.close()


def test_velocity_field_handles_reject_unsupported_calls(dg):
    w = inputs.taylor_green(2, 2)
    op = dg.operator_for(w)
    z = torch.zeros(w.ndof, device="cuda", dtype=torch.float32)
    with pytest.raises(dg.DGError):
        op.apply_jacobian(z)
    with pytest.raises(dg.DGError):
        op.precond_setup()
    with pytest.raises(dg.DGError):
        dg.Batch([op])
    x = torch.zeros(w.ndof, device="cuda", dtype=torch.float64)
    with pytest.raises(dg.DGError):
        op.solve(x, mode=dg.DG_SOLVE_MIXED, preconditioner=dg.DG_PRECOND_NONE)
    op.close()
    # block-Jacobi on a periodic axis needs two cells along it
    p1 = dg.Operator((1, 2, 2), 2, periodic=(1, 0, 0))
    with pytest.raises(dg.DGError):
        p1.precond_setup()
    p1.close()


def test_taylor_green_sampled_cells_at_bench_size(dg):
    """The benchmark's launch configuration (k = 5, m = 8, 32^3 cells here to keep the setup short): sampled
    cells against the oracle, which evaluates only those cells' rows."""
    w = inputs.taylor_green(32, 5)
    op = dg.operator_for(w)
    u = inputs.uniform_u(w.ndof, 99)
    y = op.apply_jacobian(torch.tensor(u, device="cuda")).cpu().numpy().reshape(w.ncell, -1)
    pr = tg_oracle(w)
    cells = np.random.default_rng(7).choice(w.ncell, 12, replace=False)
    cells = np.concatenate([cells, [0, w.ncell - 1, 31, 32 * 32 - 1]])
    yref = oracle.apply(pr, u, cells=cells).reshape(len(cells), -1)
    assert relerr(y[cells], yref) <= TOL64
    op.close()
