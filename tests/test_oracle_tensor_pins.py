"""Pins of the oracle's tensor diffusion coefficient and affine geometry (Problems A and B of Sec. 5.1:
"tensor-valued diffusion coefficients", "affine geometries")."""

import numpy as np
import pytest

import oracle
from tests import kron_reference as kr


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def spd_tensors(ncell, seed, off=0.5):
    rng = np.random.default_rng(seed)
    out = np.empty((ncell, 6))
    for c in range(ncell):
        L = rng.uniform(-off, off, (3, 3)) + np.diag(rng.uniform(0.8, 1.5, 3))
        M = L @ L.T
        out[c] = [M[0, 0], M[1, 1], M[2, 2], M[0, 1], M[0, 2], M[1, 2]]
    return out


def full(t):
    return np.array([[t[0], t[3], t[4]], [t[3], t[1], t[5]], [t[4], t[5], t[2]]])


def packed(M):
    return [M[0, 0], M[1, 1], M[2, 2], M[0, 1], M[0, 2], M[1, 2]]


@pytest.mark.parametrize("n,k,per", [((2, 3, 2), 2, (0, 0, 0)), ((3, 2, 2), 1, (1, 0, 1)), ((2, 2, 3), 3, (0, 1, 0))])
def test_tensor_diffusion_matches_kronecker_closed_form(n, k, per):
    nc = int(np.prod(n))
    Dt = spd_tensors(nc, 1 + k)
    b = (0.6, -0.4, 0.3)
    sigma = 6.0 * k * (k + 1)
    pr = oracle.Problem(n, k, np.ones(nc), b=b, c=0.7, sigma=sigma, periodic=per, D_tensor=Dt, hi=(1, 1.5, 2))
    A = kr.assemble_tensor(n, k, Dt, b, 0.7, sigma, (0, 0, 0), (1, 1.5, 2), periodic=per)
    u = np.random.default_rng(k).uniform(-1, 1, pr.ndof)
    assert rel(oracle.apply(pr, u), A @ u) < 1e-13


def test_isotropic_tensor_equals_scalar_diffusion():
    n, k = (3, 2, 2), 3
    nc = int(np.prod(n))
    D = np.exp(np.random.default_rng(3).standard_normal(nc))
    Dt = np.stack([D, D, D, 0 * D, 0 * D, 0 * D], axis=1)
    p0 = oracle.Problem(n, k, D, b=(1, -0.5, 0.25))
    p1 = oracle.Problem(n, k, np.ones(nc), b=(1, -0.5, 0.25), D_tensor=Dt)
    u = np.random.default_rng(4).uniform(-1, 1, p0.ndof)
    assert rel(oracle.apply(p1, u), oracle.apply(p0, u)) < 1e-14


def linear_maps():
    th = 0.4
    R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1]])
    Sh = np.array([[1.0, 0.3, -0.2], [0.0, 1.2, 0.4], [0.1, 0.0, 0.8]])
    return [R, Sh, R @ Sh]


@pytest.mark.parametrize("which", [0, 1, 2])
def test_linear_map_scales_the_operator_by_its_determinant(which):
    """x' = S x with D' = S D S^T, b' = S b (and the same penalty factor): every integral of eq. blf changes by
    |det S| -- gradients map as S^{-T}, volumes by |det S|, face normals as S^{-T} nu, areas by |det S| |S^{-T} nu|,
    so the operator matrix is |det S| times the original one."""
    S = linear_maps()[which]
    n, k = (2, 3, 2), 2
    nc = int(np.prod(n))
    hi = (1.0, 1.5, 0.8)
    h = np.asarray(hi) / np.asarray(n)
    Dt = spd_tensors(nc, 7)
    b = np.array([0.7, -0.3, 0.5])
    base = oracle.Problem(n, k, np.ones(nc), b=b, c=0.9, D_tensor=Dt, hi=hi, periodic=(1, 0, 0))
    Dm = np.array([packed(S @ full(t) @ S.T) for t in Dt])
    J = S @ np.diag(h)
    mapped = oracle.Problem(n, k, np.ones(nc), b=S @ b, c=0.9, D_tensor=Dm, J=J.ravel(), lo=(0.3, -0.2, 0.1),
                            periodic=(1, 0, 0), sigma=base.sigma)
    u = np.random.default_rng(which).uniform(-1, 1, base.ndof)
    assert rel(oracle.apply(mapped, u), abs(np.linalg.det(S)) * oracle.apply(base, u)) < 1e-13


def test_affine_diffusion_part_is_symmetric_positive_definite():
    S = linear_maps()[2]
    n, k = (2, 2, 2), 2
    nc = 8
    pr = oracle.Problem(n, k, np.ones(nc), b=(0, 0, 0), c=0.0, D_tensor=spd_tensors(nc, 9),
                        J=(S @ np.diag([0.5, 0.5, 0.5])).ravel(), sigma=12.0 * 3)
    A = np.stack([oracle.apply(pr, e) for e in np.eye(pr.ndof)], axis=1)
    assert rel(A, A.T) < 1e-13
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0


@pytest.mark.parametrize("k", [2, 3])
def test_polynomial_solution_on_affine_mesh_has_zero_residual(k):
    """u(x) = 1 + a.x + x^T B x (total degree 2 <= k) is in the DG space on an affine mesh; with
    f = -div(D grad u) + div(b u) + c u and g = u, consistency of eq. blf gives A u_h - F = 0."""
    S = linear_maps()[2]
    n = (2, 2, 3)
    nc = 12
    D = full(spd_tensors(1, 11)[0])
    a = np.array([0.3, -0.7, 0.5])
    B = np.array([[0.4, 0.1, -0.2], [0.1, -0.3, 0.25], [-0.2, 0.25, 0.6]])
    b = np.array([0.8, -0.4, 0.3])
    c = 0.6
    lo = np.array([0.2, -0.1, 0.05])
    J = S @ np.diag([0.5, 0.4, 0.3])
    pr = oracle.Problem(n, k, np.ones(nc), b=b, c=c, D_tensor=np.tile(packed(D), (nc, 1)), J=J.ravel(), lo=lo)

    def u(x):
        return 1.0 + x @ a + np.einsum("...i,ij,...j->...", x, B, x)

    def f(x):
        return -2.0 * np.trace(D @ B) + (a + 2.0 * x @ B) @ b + c * u(x)

    xv = oracle.volume_points(pr)
    g = [u(oracle.face_points(pr, s)).ravel() for s in range(6)]
    F = oracle.rhs(pr, f(xv), g)
    # u_h: the L2 projection of u (exact, u is in the space); the mass matrix is |det J| I
    z = oracle.rhs(oracle.Problem(n, k, np.ones(nc), b=(0, 0, 0), c=0.0, J=J.ravel(), lo=lo), u(xv), None)
    z /= abs(np.linalg.det(J))
    r = oracle.apply(pr, z) - F
    assert np.max(np.abs(r)) < 1e-11 * np.max(np.abs(F))


def face_normals(J):
    """Unit normals along +reference axis r of affine cells with Jacobian J: rows of J^{-1}, normalised."""
    Ji = np.linalg.inv(J)
    return Ji / np.linalg.norm(Ji, axis=1)[:, None]


def test_constant_point_tables_equal_per_cell_coefficients():
    n, k = (2, 3, 2), 2
    nc = 12
    Dt = spd_tensors(nc, 31)
    S = linear_maps()[1] @ np.diag([0.5, 0.3, 0.5])
    base = oracle.Problem(n, k, np.ones(nc), b=(0.4, -0.2, 0.3), c=0.8, D_tensor=Dt, J=S.ravel(), m=k + 3)
    Dv = np.repeat(Dt[:, None, :], base.m ** 3, axis=1)
    Df = np.repeat(Dt[:, None, None, :], 6 * base.m ** 2, axis=1).reshape(nc, 6, base.m ** 2, 6)
    cv = np.full((nc, base.m ** 3), 0.8)
    pw = oracle.Problem(n, k, np.ones(nc), b=(0.4, -0.2, 0.3), c=0.0, D_tensor=Dt, J=S.ravel(), m=k + 3,
                        D_vol=Dv, D_face=Df, c_vol=cv)
    u = np.random.default_rng(32).uniform(-1, 1, base.ndof)
    assert rel(oracle.apply(pw, u), oracle.apply(base, u)) < 1e-14
    g = [np.cos(oracle.face_points(base, s).sum(axis=-1)).ravel() for s in range(6)]
    assert rel(oracle.rhs(pw, None, g), oracle.rhs(base, None, g)) < 1e-14


@pytest.mark.parametrize("k", [2, 3])
def test_polynomial_solution_with_polynomial_coefficients_has_zero_residual(k):
    """Problem B (Sec. 5.1): affine cells, D(x), b(x), c(x) polynomials in x, q = 2p+4 (m = k+3).  For the
    quadratic u(x) = 1 + a.x + x^T B x, f = -div(D grad u) + div(b u) + c u and g = u, the integrands are
    integrated exactly and consistency of eq. blf gives A u_h - F = 0."""
    S = linear_maps()[2]
    n = (2, 2, 2)
    nc = 8
    lo = np.array([0.1, 0.2, -0.1])
    J = S @ np.diag([0.5, 0.45, 0.4])
    m = k + 3
    D0 = full(spd_tensors(1, 40, off=0.3)[0]) + 2.0 * np.eye(3)
    Dk = [0.3 * (M + M.T) / 2 for M in np.random.default_rng(41).uniform(-1, 1, (3, 3, 3))]
    b0 = np.array([0.5, -0.3, 0.2])
    B1 = np.random.default_rng(42).uniform(-0.4, 0.4, (3, 3))
    c0, c1 = 0.7, np.array([0.2, -0.1, 0.3])
    a = np.array([0.3, -0.7, 0.5])
    B = np.array([[0.4, 0.1, -0.2], [0.1, -0.3, 0.25], [-0.2, 0.25, 0.6]])

    def Dfield(x):
        return D0 + np.einsum("...k,kij->...ij", x, np.asarray(Dk))

    def bfield(x):
        return b0 + x @ B1.T

    def cfield(x):
        return c0 + x @ c1

    def u(x):
        return 1.0 + x @ a + np.einsum("...i,ij,...j->...", x, B, x)

    def f(x):
        gu = a + 2.0 * x @ B                                     # grad u (B symmetric)
        divD = np.einsum("iij->j", np.asarray(Dk))                # sum_i d_i D_ij (D_ij linear in x)
        div_flux = gu @ divD + 2.0 * np.einsum("...ij,ji->...", Dfield(x), B)
        return -div_flux + np.trace(B1) * u(x) + np.einsum("...i,...i->...", bfield(x), gu) + cfield(x) * u(x)

    geo = oracle.Problem(n, k, np.ones(nc), J=J.ravel(), lo=lo, m=m)
    xv = oracle.volume_points(geo)
    xf = oracle.cell_face_points(geo)
    packD = lambda M: np.stack([M[..., 0, 0], M[..., 1, 1], M[..., 2, 2], M[..., 0, 1], M[..., 0, 2], M[..., 1, 2]],
                               axis=-1)
    nrm = face_normals(J)
    bface = np.einsum("cspi,si->csp", bfield(xf), np.repeat(nrm, 2, axis=0))
    pr = oracle.Problem(n, k, np.ones(nc), b=(0, 0, 0), c=0.0, J=J.ravel(), lo=lo, m=m,
                        D_tensor=np.tile(packD(D0), (nc, 1)), D_vol=packD(Dfield(xv)), D_face=packD(Dfield(xf)),
                        c_vol=cfield(xv), b_vol=bfield(xv), b_face=bface)
    g = [u(oracle.face_points(pr, s)).ravel() for s in range(6)]
    F = oracle.rhs(pr, f(xv), g)
    z = oracle.rhs(oracle.Problem(n, k, np.ones(nc), b=(0, 0, 0), c=0.0, J=J.ravel(), lo=lo, m=m), u(xv), None)
    z /= abs(np.linalg.det(J))
    r = oracle.apply(pr, z) - F
    assert np.max(np.abs(r)) < 1e-11 * np.max(np.abs(F))
    # the point tables are used: cell-constant coefficients do not reproduce the solution
    pc = oracle.Problem(n, k, np.ones(nc), b=b0, c=c0, J=J.ravel(), lo=lo, m=m, D_tensor=np.tile(packD(D0), (nc, 1)))
    assert np.max(np.abs(oracle.apply(pc, z) - F)) > 1e-3 * np.max(np.abs(F))
