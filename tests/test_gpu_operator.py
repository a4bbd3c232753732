"""GPU parity of the CUDA operator (through the C ABI) against the FP64 oracle.

Bars (written here, used by every case):
  FP64 apply:  ||y - y_oracle||_inf / ||y_oracle||_inf <= 1e-12
  FP32 apply:  ||y - y_oracle||_inf / ||y_oracle||_inf <= 1e-5
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


def oracle_problem(w, sigma=None):
    return oracle.Problem(w.n, w.k, w.D, b=w.b, c=w.c, sigma=sigma, lo=w.lo, hi=w.hi)


def oracle_F(w, pr):
    f = inputs.f_at(w, oracle.volume_points(pr)) if w.f_kind != "zero" else None
    return oracle.rhs(pr, f, None)


# (n, k, b, c, D sigma, lo, hi): several CTAs with a ragged last CTA, 1-cell meshes, both upwind branches
SMALL = [
    ((3, 5, 3), 1, (1.0, 0.5, 0.25), 1.0, 1.0, (0, 0, 0), (1, 1, 1)),
    ((3, 2, 4), 2, (-1.0, 0.5, -0.25), 0.5, 1.0, (0, 0, 0), (1, 2, 1)),
    ((5, 3, 3), 3, (1.0, 0.5, 0.25), 1.0, 2.0, (0, -1, 0), (1, 1, 3)),
    ((3, 3, 2), 4, (0.3, -0.7, 1.1), 0.0, 1.0, (0, 0, 0), (1, 1, 1)),
    ((2, 3, 3), 5, (1.0, 0.5, 0.25), 1.0, 1.0, (0, 0, 0), (1, 1, 1)),
    ((3, 2, 2), 6, (-0.2, 0.0, 0.9), 2.0, 1.5, (0, 0, 0), (2, 1, 1)),
    ((3, 3, 3), 7, (1.0, 0.5, 0.25), 1.0, 1.0, (0, 0, 0), (1, 1, 1)),
    ((2, 2, 3), 8, (1.0, -0.5, 0.25), 1.0, 1.0, (0, 0, 0), (1, 1, 1)),
    ((2, 3, 2), 9, (0.5, 0.5, -0.5), 0.3, 1.0, (0, 0, 0), (1, 1, 1)),
    ((2, 2, 2), 10, (1.0, 0.5, 0.25), 1.0, 1.0, (0, 0, 0), (1, 1, 1)),
    ((1, 1, 1), 3, (1.0, -0.5, 0.25), 1.0, 1.0, (0, 0, 0), (1, 1, 1)),
    ((1, 1, 6), 2, (0.0, 0.0, -1.0), 0.0, 3.0, (0, 0, 0), (0.5, 0.25, 3)),
]


@pytest.mark.parametrize("case", SMALL, ids=lambda c: f"n{c[0]}k{c[1]}")
def test_small_meshes_all_degrees(dg, case):
    n, k, b, c, sD, lo, hi = case
    w = inputs.small_case(n=n, k=k, sigma_D=sD, seed=17 + k, b=b, c=c)
    w.lo, w.hi = lo, hi
    pr = oracle_problem(w)
    y_ref = oracle.apply(pr, w.u)
    r_ref = y_ref - oracle_F(w, pr)
    op = dg.operator_for(w)
    u64 = torch.tensor(w.u, device="cuda")
    y = op.apply_jacobian(u64).cpu().numpy()
    r = op.apply_residual(u64).cpu().numpy()
    assert relerr(y, y_ref) <= TOL64
    assert relerr(r, r_ref) <= TOL64
    u32 = u64.float()
    y32 = op.apply_jacobian(u32).cpu().numpy()
    r32 = op.apply_residual(u32).cpu().numpy()
    assert relerr(y32, y_ref) <= TOL32
    assert relerr(r32, r_ref) <= TOL32
    # FP64 vectors evaluated in double-float arithmetic meet the FP64 bar
    yx = op.apply_jacobian(u64, precision=dg.DG_F64X).cpu().numpy()
    rx = op.apply_residual(u64, precision=dg.DG_F64X).cpu().numpy()
    assert relerr(yx, y_ref) <= TOL64
    assert relerr(rx, r_ref) <= TOL64
    op.close()


def test_unit_cube_q3_8_full_vector(dg):
    """8^3 cells, Q_3, D = 1, b = (1,.5,.25), c = 1, penalty 2k(k+1)/h, g = 0, f = 1: whole residual."""
    w = inputs.unit_cube_q3_8()
    pr = oracle_problem(w)
    F_ref = oracle_F(w, pr)
    r_ref = oracle.apply(pr, w.u) - F_ref
    op = dg.operator_for(w)
    assert relerr(op.rhs().cpu().numpy(), F_ref) <= TOL64
    u = torch.tensor(w.u, device="cuda")
    assert relerr(op.apply_residual(u).cpu().numpy(), r_ref) <= TOL64
    assert relerr(op.apply_residual(u.float()).cpu().numpy(), r_ref) <= TOL32
    assert relerr(op.apply_residual(u, precision=dg.DG_F64X).cpu().numpy(), r_ref) <= TOL64
    op.close()


def _sample_cells(n, count, seed):
    nx, ny, nz = n
    corners = [ix + nx * (iy + ny * iz) for ix in (0, nx - 1) for iy in (0, ny - 1) for iz in (0, nz - 1)]
    rng = np.random.default_rng(seed)
    rest = rng.choice(nx * ny * nz, size=count, replace=False).tolist()
    return sorted(set(corners + rest))


def test_unit_cube_q7_32_sampled_cells(dg):
    """32^3 cells, Q_7, log-normal D: residual and Jacobian on sampled cells (the full-size launch)."""
    w = inputs.unit_cube_q7_32()
    pr = oracle_problem(w)
    cells = _sample_cells(w.n, 40, 123)
    y_ref = oracle.apply(pr, w.u, cells=cells).reshape(len(cells), w.nb)
    # F restricted to the sampled cells: f = 1, g = 0 gives |T| on mode 0
    F_ref = np.zeros_like(y_ref)
    F_ref[:, 0] = 1.0 / 32 ** 3
    op = dg.operator_for(w)
    u = torch.tensor(w.u, device="cuda")
    y = op.apply_jacobian(u).view(-1, w.nb)[cells].cpu().numpy()
    r = op.apply_residual(u).view(-1, w.nb)[cells].cpu().numpy()
    assert relerr(y, y_ref) <= TOL64
    assert relerr(r, y_ref - F_ref) <= TOL64
    y32 = op.apply_jacobian(u.float()).view(-1, w.nb)[cells].cpu().numpy()
    assert relerr(y32, y_ref) <= TOL32
    rx = op.apply_residual(u, precision=dg.DG_F64X).view(-1, w.nb)[cells].cpu().numpy()
    assert relerr(rx, y_ref - F_ref) <= TOL64
    op.close()


def test_unit_cube_q7_32_full_vector(dg):
    """32^3 cells, Q_7, log-normal D, in the launch configuration that bench.py times: the WHOLE residual and
    Jacobian (16.8 M entries) against the matrix-free Kronecker form of the same operator (exact 1D integrals,
    pinned to the dense form and to the oracle in tests/test_kron_matfree_cpu.py); FP64 and double-float at
    1e-12, FP32 at 1e-5."""
    from tests import kron_reference as kr
    w = inputs.unit_cube_q7_32()
    sigma = dg.dg_penalty_sigma(w.k, 0)
    y_ref = kr.apply_matfree(w.n, w.k, w.D, w.b, w.c, sigma, w.u, w.lo, w.hi)
    r_ref = y_ref.copy()
    r_ref[::w.nb] -= 1.0 / 32 ** 3  # f = 1, g = 0: F = |T| on mode 0
    op = dg.operator_for(w)
    u = torch.tensor(w.u, device="cuda")
    assert relerr(op.apply_jacobian(u).cpu().numpy(), y_ref) <= TOL64
    assert relerr(op.apply_residual(u).cpu().numpy(), r_ref) <= TOL64
    assert relerr(op.apply_residual(u, precision=dg.DG_F64X).cpu().numpy(), r_ref) <= TOL64
    assert relerr(op.apply_jacobian(u, precision=dg.DG_F64X).cpu().numpy(), y_ref) <= TOL64
    assert relerr(op.apply_residual(u.float()).cpu().numpy(), r_ref) <= TOL32
    op.close()


def test_sine_source_and_dirichlet_data(dg):
    """Right hand side with a sine-mode f and non-zero Dirichlet g on every side."""
    w = inputs.small_case(n=(3, 4, 2), k=4, seed=5, f_kind="sines")
    w.f_params = inputs.sine_modes(44)
    pr = oracle_problem(w)
    gfun = lambda x: np.cos(x[..., 0] + 2 * x[..., 1]) * np.exp(x[..., 2])
    g_or = [gfun(oracle.face_points(pr, s)) for s in range(6)]
    F_ref = oracle.rhs(pr, inputs.f_at(w, oracle.volume_points(pr)), g_or)
    op0 = dg.Operator(w.n, w.k, w.D, b=w.b, c=w.c)
    f_lib = inputs.f_at(w, op0.quadrature_points(0))
    g_lib = [gfun(op0.quadrature_points(1 + s)) for s in range(6)]
    op0.close()
    op = dg.Operator(w.n, w.k, w.D, b=w.b, c=w.c, f_qp=f_lib, g_qp=g_lib)
    assert relerr(op.rhs().cpu().numpy(), F_ref) <= TOL64
    u = torch.tensor(w.u, device="cuda")
    assert relerr(op.apply_residual(u).cpu().numpy(), oracle.apply(pr, w.u) - F_ref) <= TOL64
    op.close()


def test_quadrature_points_match_oracle(dg):
    w = inputs.small_case(n=(2, 3, 2), k=5)
    w.lo, w.hi = (0.0, -1.0, 0.5), (1.0, 2.0, 1.0)
    pr = oracle_problem(w)
    op = dg.Operator(w.n, w.k, w.D, lo=w.lo, hi=w.hi)
    assert np.max(np.abs(op.quadrature_points(0) - oracle.volume_points(pr))) < 1e-14
    for s in range(6):
        assert np.max(np.abs(op.quadrature_points(1 + s) - oracle.face_points(pr, s))) < 1e-14
    op.close()


def test_linearity_and_determinism(dg):
    w = inputs.small_case(n=(4, 4, 4), k=3, seed=3)
    op = dg.operator_for(w)
    rng = np.random.default_rng(1)
    a = torch.tensor(rng.uniform(-1, 1, w.ndof), device="cuda")
    b = torch.tensor(rng.uniform(-1, 1, w.ndof), device="cuda")
    ya, yb = op.apply_jacobian(a), op.apply_jacobian(b)
    yab = op.apply_jacobian(2.0 * a - 3.0 * b)
    assert torch.max(torch.abs(yab - (2.0 * ya - 3.0 * yb))).item() <= 1e-12 * torch.max(torch.abs(yab)).item()
    # bitwise reproducible (no atomics, fixed reduction order)
    assert torch.equal(op.apply_jacobian(a), ya)
    op.close()


def test_api_errors(dg):
    w = inputs.small_case(n=(2, 2, 2), k=2)
    op = dg.operator_for(w)
    u = torch.zeros(w.ndof, dtype=torch.float64, device="cuda")
    with pytest.raises(dg.DGError):
        dg.check(dg.lib.dg_apply_jacobian(op.h, dg.ctypes.c_void_p(u.data_ptr()), dg.ctypes.c_void_p(u.data_ptr()),
                                          0, None))
    with pytest.raises(dg.DGError):
        dg.check(dg.lib.dg_apply_jacobian(op.h, dg.ctypes.c_void_p(u.data_ptr()), None, 0, None))
    with pytest.raises(dg.DGError):
        dg.check(dg.lib.dg_apply_jacobian(op.h, dg.ctypes.c_void_p(u.data_ptr()), dg.ctypes.c_void_p(1024), 7,
                                          None))
    op.close()


@pytest.mark.parametrize("which", ["unit_cube_q5_48", "q4_64_sigma15"])
def test_other_full_size_workloads_sampled_cells(dg, which):
    """48^3 Q5 (sine source, log-normal D) and 64^3 Q4 (sigma 1.5): residual on sampled cells, all precisions."""
    if which == "unit_cube_q5_48":
        w = inputs.unit_cube_q5_48()
    else:
        w = inputs.Workload("q4_64", (64, 64, 64), 4, inputs.log_normal_D(64 ** 3, 1.5, 20), f_kind="one")
        w.u = inputs.uniform_u(w.ndof, 21)
    pr = oracle_problem(w)
    cells = _sample_cells(w.n, 30, 7)
    y_ref = oracle.apply(pr, w.u, cells=cells).reshape(len(cells), w.nb)
    # right hand side on the sampled cells: (f, phi_i)_T from the oracle's own quadrature points
    F_full = oracle_F(w, pr).reshape(w.ncell, w.nb)[cells] if w.ncell <= 48 ** 3 else None
    op = dg.operator_for(w)
    u = torch.tensor(w.u, device="cuda")
    y = op.apply_jacobian(u).view(-1, w.nb)[cells].cpu().numpy()
    assert relerr(y, y_ref) <= TOL64
    yx = op.apply_jacobian(u, precision=dg.DG_F64X).view(-1, w.nb)[cells].cpu().numpy()
    assert relerr(yx, y_ref) <= TOL64
    y32 = op.apply_jacobian(u.float()).view(-1, w.nb)[cells].cpu().numpy()
    assert relerr(y32, y_ref) <= TOL32
    if F_full is not None:
        r = op.apply_residual(u).view(-1, w.nb)[cells].cpu().numpy()
        assert relerr(r, y_ref - F_full) <= TOL64
    op.close()
