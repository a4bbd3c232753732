"""Pins of the oracle on multilinear cells (Problem C of Sec. 5.1: "multilinear geometries"; CPU only).

Each cell is the trilinear image of the reference cube through its 8 corner vertices; gradients map with
J(x)^{-T}, the volume element is |det J(x)| and a face across reference axis r has the unit normal
J^{-T} e_r / |J^{-T} e_r| and the area element |det J| |J^{-T} e_r|, all taken at each quadrature point.
Pinned by:

* affine vertices reproduce the affine-map oracle (itself pinned in test_oracle_tensor_pins.py);
* consistency: zero residual for a quadratic solution with constant coefficients.  On trilinear cells every
  integrand of eq. blf and l_h that does not multiply a vanishing jump is a polynomial in the reference
  coordinates (the cofactor matrix of J is polynomial), so q = 2p+5 (m = k+3) integrates it exactly;
* the volume element: sum over cells of (1, phi_0) = |Omega| for a perturbed grid of the unit cube;
* symmetry and coercivity of the diffusion part, conservation and A 1 = 0 with Neumann sides;
* invariance under a rigid motion of the mesh with D -> R D R^T, b -> R b.
"""

import numpy as np
import pytest

import oracle
from paper_1711_10885_gb300 import inputs
from tests.test_oracle_tensor_pins import spd_tensors


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def affine_vertices(n, lo, J):
    k, j, i = np.meshgrid(np.arange(n[2] + 1), np.arange(n[1] + 1), np.arange(n[0] + 1), indexing="ij")
    idx = np.stack([i, j, k], axis=-1).reshape(-1, 3).astype(np.float64)
    return np.asarray(lo) + idx @ np.asarray(J).T


@pytest.mark.parametrize("k,m", [(2, 3), (3, 6)])
def test_affine_vertices_reproduce_the_affine_map(k, m):
    n = (2, 3, 2)
    nc = 12
    lo = np.array([0.1, -0.2, 0.3])
    J = np.array([[0.4, 0.1, -0.05], [0.0, 0.35, 0.08], [0.06, 0.0, 0.5]])
    Dt = spd_tensors(nc, 400)
    bc = ("dirichlet", "outflow", "neumann", "dirichlet", "dirichlet", "neumann")
    kw = dict(b=(0.6, -0.3, 0.2), c=0.7, m=m, D_tensor=Dt, bc=bc)
    pa = oracle.Problem(n, k, np.ones(nc), lo=lo, J=J.ravel(), **kw)
    pv = oracle.Problem(n, k, np.ones(nc), vertices=affine_vertices(n, lo, J), **kw)
    assert np.max(np.abs(oracle.volume_points(pv) - oracle.volume_points(pa))) < 1e-14
    assert np.max(np.abs(oracle.cell_face_points(pv) - oracle.cell_face_points(pa))) < 1e-14
    u = np.random.default_rng(401).uniform(-1, 1, pa.ndof)
    assert rel(oracle.apply(pv, u), oracle.apply(pa, u)) < 1e-13
    f = np.cos(oracle.volume_points(pa).sum(axis=-1))
    g = [None if bc[s] == "outflow" else np.sin(oracle.face_points(pa, s).sum(axis=-1)).ravel() for s in range(6)]
    assert rel(oracle.rhs(pv, f, g), oracle.rhs(pa, f, g)) < 1e-13


def interpolate(pr, values):
    """DG coefficients whose function equals `values` at the volume points (exact for mapped polynomials of
    degree <= k per reference direction): a least-squares solve with the 3D basis table."""
    xq, _ = oracle.gauss_legendre(pr.m)
    B1 = np.array([oracle.basis_1d(pr.k, x)[0] for x in xq])  # [point, j]
    B = np.kron(B1, np.kron(B1, B1))  # point q = i1 + m (i2 + m i3), J = j1 + n (j2 + n j3)
    z = np.linalg.lstsq(B, values.reshape(pr.ncell, -1).T, rcond=None)[0]
    return z.T.ravel()


@pytest.mark.parametrize("k", [2, 3])
def test_quadratic_solution_on_multilinear_mesh_has_zero_residual(k):
    n = (2, 3, 2)
    m = k + 3
    verts = inputs.multilinear_vertices(n, seed=410 + k, amplitude=0.2)
    d, b, c = 1.4, np.array([0.7, -0.4, 0.3]), 0.6
    a = np.array([0.3, -0.6, 0.45])
    Bq = np.array([[0.5, 0.2, -0.1], [0.2, -0.4, 0.3], [-0.1, 0.3, 0.6]])

    def u(x):
        return 1.0 + x @ a + np.einsum("...i,ij,...j->...", x, Bq, x)

    def grad(x):
        return a + 2.0 * x @ Bq

    def f(x):
        return -d * 2.0 * np.trace(Bq) + grad(x) @ b + c * u(x)

    bc = ("dirichlet", "dirichlet", "neumann", "dirichlet", "dirichlet", "neumann")
    pr = oracle.Problem(n, k, d, b=tuple(b), c=c, m=m, vertices=verts, bc=bc)
    normals = {2: np.array([0.0, -1.0, 0.0]), 5: np.array([0.0, 0.0, 1.0])}
    data = []
    for s in range(6):
        xs = oracle.face_points(pr, s)
        data.append(u(xs).ravel() if bc[s] == "dirichlet" else
                    (u(xs) * (b @ normals[s]) - d * grad(xs) @ normals[s]).ravel())
    xv = oracle.volume_points(pr)
    F = oracle.rhs(pr, f(xv), data)
    z = interpolate(pr, u(xv))
    r = oracle.apply(pr, z) - F
    assert np.max(np.abs(r)) < 1e-11 * np.max(np.abs(F))
    # the geometry is used point by point: the same data on the unperturbed grid leave a residual
    flat = oracle.Problem(n, k, d, b=tuple(b), c=c, m=m, bc=bc)
    assert np.max(np.abs(oracle.apply(flat, z) - F)) > 1e-4 * np.max(np.abs(F))


def test_volume_element_integrates_the_domain():
    n, k = (3, 2, 2), 2
    verts = inputs.multilinear_vertices(n, seed=420, amplitude=0.22)
    pr = oracle.Problem(n, k, 1.0, m=k + 3, vertices=verts)
    F = oracle.rhs(pr, np.ones(pr.ncell * pr.m ** 3), None).reshape(pr.ncell, -1)
    assert abs(F[:, 0].sum() - 1.0) < 1e-14  # (1, phi_0)_T = |T|, phi_0 = 1
    assert np.ptp(F[:, 0]) > 1e-3  # the cells really differ in volume


def test_multilinear_diffusion_is_symmetric_coercive_and_conservative():
    n, k = (2, 2, 3), 2
    verts = inputs.multilinear_vertices(n, seed=430, amplitude=0.2)
    rng = np.random.default_rng(431)
    D = np.exp(rng.standard_normal(12))
    pr = oracle.Problem(n, k, D, b=(0, 0, 0), c=0.0, m=k + 3, vertices=verts)
    for _ in range(2):
        u = rng.uniform(-1, 1, pr.ndof)
        v = rng.uniform(-1, 1, pr.ndof)
        vau, uav = v @ oracle.apply(pr, u), u @ oracle.apply(pr, v)
        assert abs(vau - uav) <= 1e-12 * (abs(vau) + abs(uav))
        assert u @ oracle.apply(pr, u) > 0
    prn = oracle.Problem(n, k, D, b=(0.5, -0.2, 0.3), c=0.0, m=k + 3, vertices=verts, bc=("neumann",) * 6)
    y = oracle.apply(prn, rng.uniform(-1, 1, pr.ndof)).reshape(12, -1)
    assert abs(y[:, 0].sum()) < 1e-12 * np.max(np.abs(y))
    pr0 = oracle.Problem(n, k, D, b=(0, 0, 0), c=0.0, m=k + 3, vertices=verts, bc=("neumann",) * 6)
    one = np.zeros((12, (k + 1) ** 3))
    one[:, 0] = 1.0
    assert np.max(np.abs(oracle.apply(pr0, one.ravel()))) < 1e-12


def test_rigid_motion_invariance():
    n, k = (2, 2, 2), 2
    verts = inputs.multilinear_vertices(n, seed=440, amplitude=0.2)
    th = 0.7
    R = np.array([[np.cos(th), 0, np.sin(th)], [0, 1, 0], [-np.sin(th), 0, np.cos(th)]]) @ \
        np.array([[1, 0, 0], [0, np.cos(0.3), -np.sin(0.3)], [0, np.sin(0.3), np.cos(0.3)]])
    t = np.array([0.5, -1.0, 2.0])
    Dt = spd_tensors(8, 441)
    full = lambda p: np.array([[p[0], p[3], p[4]], [p[3], p[1], p[5]], [p[4], p[5], p[2]]])
    Dr = inputs.pack_sym(np.stack([R @ full(p) @ R.T for p in Dt]))
    b = np.array([0.4, 0.3, -0.5])
    pr = oracle.Problem(n, k, np.ones(8), b=tuple(b), c=0.5, m=k + 3, vertices=verts, D_tensor=Dt)
    pm = oracle.Problem(n, k, np.ones(8), b=tuple(R @ b), c=0.5, m=k + 3, vertices=verts @ R.T + t, D_tensor=Dr)
    u = np.random.default_rng(442).uniform(-1, 1, pr.ndof)
    assert rel(oracle.apply(pm, u), oracle.apply(pr, u)) < 1e-12


def test_interior_penalty_on_multilinear_cells():
    """Two trilinear cells with Neumann sides, D = I, b = 0, c = 0 and u = v = 1 on the first cell: every term of
    eq. blf vanishes except the penalty, so a_h(u, u) = gamma_F |F| = sigma |F|^2 / min(|T-|, |T+|) (Sec. 2;
    <delta-, delta+> = 1).  |F| and |T| are computed here independently with numpy: the volume from det of the
    trilinear Jacobian, the face area from the cross product of its tangential derivatives (20-point rule)."""
    n, k = (2, 1, 1), 1
    verts = inputs.multilinear_vertices(n, seed=450, amplitude=0.24)
    # move the shared face's interior-free vertices too, so the two cells differ clearly in volume
    X = verts.reshape(2, 2, 3, 3).copy()  # [k][j][i][xyz]
    X[:, :, 1, 0] += np.array([[0.08, -0.05], [0.11, 0.02]])
    verts = X.reshape(-1, 3)
    sigma = 3.0
    pr = oracle.Problem(n, k, 1.0, b=(0, 0, 0), c=0.0, sigma=sigma, m=k + 3, vertices=verts, bc=("neumann",) * 6)
    u = np.zeros(pr.ndof)
    u[0] = 1.0
    val = u @ oracle.apply(pr, u)
    t, w = np.polynomial.legendre.leggauss(20)
    t, w = (t + 1) / 2, w / 2

    def corners(cell):
        return np.array([[[X[c, b, cell + a] for a in range(2)] for b in range(2)] for c in range(2)])  # [c][b][a]

    def jac(C, x0, x1, x2):
        """d x / d xi of the trilinear map with corners C[c][b][a] at the points (x0, x1, x2) (arrays): [..., 3, 3]."""
        N = [lambda x: 1 - x, lambda x: x]
        dN = [-1.0, 1.0]
        Jm = np.zeros(np.broadcast(x0, x1, x2).shape + (3, 3))
        for c in range(2):
            for b in range(2):
                for a in range(2):
                    X_ = C[c, b, a]
                    Jm[..., :, 0] += np.multiply.outer(dN[a] * N[b](x1) * N[c](x2), X_)
                    Jm[..., :, 1] += np.multiply.outer(N[a](x0) * dN[b] * N[c](x2), X_)
                    Jm[..., :, 2] += np.multiply.outer(N[a](x0) * N[b](x1) * dN[c], X_)
        return Jm

    g0, g1, g2 = np.meshgrid(t, t, t, indexing="ij")
    w3 = np.einsum("i,j,l->ijl", w, w, w)
    vols = [float(np.sum(w3 * np.abs(np.linalg.det(jac(corners(cell), g0, g1, g2))))) for cell in range(2)]
    f1, f2 = np.meshgrid(t, t, indexing="ij")
    Jf = jac(corners(0), np.ones_like(f1), f1, f2)
    area = float(np.sum(np.outer(w, w) * np.linalg.norm(np.cross(Jf[..., :, 1], Jf[..., :, 2]), axis=-1)))
    assert abs(vols[0] - vols[1]) > 1e-3
    expect = sigma * area ** 2 / min(vols)
    assert abs(val - expect) < 1e-10 * expect
