"""Pins of the oracle's Neumann and outflow boundary conditions (CPU only).

The model problem (Sec. 2, eq. modelproblem) splits the boundary into Dirichlet (u = g), Neumann (total flux
(b u - D grad u) . nu = j) and outflow ((D grad u) . nu = 0, on the part where b . nu >= 0) sides.  In eq. blf
a Neumann face contributes nothing to a_h and -(j, v) to l_h; an outflow face contributes only the upwind
flux Phi(u, 0, b_nu).  Pinned by:

* an independent Kronecker closed form with exact 1D integrals (tests/kron_reference.py) for mixed types;
* consistency: zero residual for a global polynomial solution whose data g, j fit its boundary values and
  whose normal derivative vanishes on the outflow side;
* conservation: with Neumann data on every side and c = 0, sum over cells of a_h(u, 1_T) = 0 for every u,
  and A 1 = 0 when b = 0 (constants are in the kernel);
* the Neumann right hand side in closed form: l_h(phi) = -(j, phi)_F on the boundary cells.
"""

import numpy as np
import pytest

import oracle
from tests import kron_reference as kr


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


BC_CASES = [
    # n, k, b, c, bc per side
    ((2, 2, 2), 2, (1.0, 0.5, 0.25), 1.0, ("dirichlet", "outflow", "neumann", "dirichlet", "neumann", "outflow")),
    ((2, 3, 2), 3, (-0.7, 0.4, -1.3), 0.3, ("outflow", "neumann", "dirichlet", "outflow", "outflow", "dirichlet")),
    ((3, 1, 2), 1, (0.0, -2.0, 0.5), 0.0, ("neumann",) * 6),
    ((1, 2, 2), 2, (0.6, 0.0, -0.4), 0.5, ("neumann", "outflow") * 3),
]


@pytest.mark.parametrize("case", BC_CASES, ids=lambda c: "".join(t[0] for t in c[4]))
def test_mixed_boundary_types_match_kronecker_closed_form(case):
    n, k, b, c, bc = case
    ncell = int(np.prod(n))
    rng = np.random.default_rng(21)
    D = np.exp(rng.standard_normal(ncell))
    sigma = oracle.penalty_sigma(k)
    lo, hi = (0.0, -0.5, 0.25), (1.0, 1.0, 1.0)
    pr = oracle.Problem(n, k, D, b=b, c=c, sigma=sigma, lo=lo, hi=hi, bc=bc)
    A = kr.assemble(n, k, D, b, c, sigma, lo, hi, bc=bc)
    for _ in range(3):
        u = rng.uniform(-1, 1, pr.ndof)
        assert rel(oracle.apply(pr, u), A @ u) < 1e-12
    # the boundary types are used: the all-Dirichlet operator differs
    A0 = kr.assemble(n, k, D, b, c, sigma, lo, hi)
    assert np.max(np.abs(A - A0)) > 1e-3 * np.max(np.abs(A0))


@pytest.mark.parametrize("k", [2, 3])
def test_polynomial_solution_with_mixed_boundary_types_has_zero_residual(k):
    """u*(x) = 1 + a (x - 1)^2 + p(y, z) with D = d I, constant b (b_x > 0) and c on [0,1]^3: outflow at x = 1
    (d u*/dx = 0 there, b . nu > 0), Neumann j = (b u* - d grad u*) . nu on y = 0 and z = 1, Dirichlet g = u*
    elsewhere; f = -d lap u* + b . grad u* + c u*.  Consistency of eq. blf and l_h gives A u_h - F = 0."""
    n = (2, 3, 2)
    d, b, c = 1.3, np.array([0.9, -0.4, 0.3]), 0.7
    a = 0.6
    pc = np.array([0.2, -0.5, 0.35, 0.25, -0.3])  # 1, y, z, y z, y^2 coefficients of p

    def u(x):
        X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
        return 1.0 + a * (X - 1.0) ** 2 + pc[0] + pc[1] * Y + pc[2] * Z + pc[3] * Y * Z + pc[4] * Y ** 2

    def grad(x):
        X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
        return np.stack([2 * a * (X - 1.0), pc[1] + pc[3] * Z + 2 * pc[4] * Y, pc[2] + pc[3] * Y], axis=-1)

    def f(x):
        lap = 2 * a + 2 * pc[4]
        return -d * lap + grad(x) @ b + c * u(x)

    bc = ("dirichlet", "outflow", "neumann", "dirichlet", "dirichlet", "neumann")
    pr = oracle.Problem(n, k, d, b=tuple(b), c=c, bc=bc)
    normals = {2: np.array([0.0, -1.0, 0.0]), 5: np.array([0.0, 0.0, 1.0])}
    data = []
    for s in range(6):
        xs = oracle.face_points(pr, s)
        if bc[s] == "dirichlet":
            data.append(u(xs).ravel())
        elif bc[s] == "neumann":
            nu = normals[s]
            data.append((u(xs) * (b @ nu) - d * grad(xs) @ nu).ravel())
        else:
            data.append(None)
    F = oracle.rhs(pr, f(oracle.volume_points(pr)), data)
    proj = oracle.Problem(n, k, 1.0, b=(0, 0, 0), c=0.0)
    z = oracle.rhs(proj, u(oracle.volume_points(proj)), None) / (0.5 * (1 / 3) * 0.5)  # L2 projection, M = |T| I
    r = oracle.apply(pr, z) - F
    assert np.max(np.abs(r)) < 1e-11 * np.max(np.abs(F))
    # the Neumann data enter with the right sign: flipping j leaves a residual
    flipped = [(-g if bc[s] == "neumann" else g) for s, g in enumerate(data)]
    r2 = oracle.apply(pr, z) - oracle.rhs(pr, f(oracle.volume_points(pr)), flipped)
    assert np.max(np.abs(r2)) > 1e-3 * np.max(np.abs(F))


def test_all_neumann_operator_conserves_and_has_constants_in_its_kernel():
    rng = np.random.default_rng(23)
    n, k = (3, 2, 2), 2
    D = np.exp(rng.standard_normal(12))
    vol = (1.0 / 3) * (1.0 / 2) * (1.0 / 2)
    # c = 0, any b: the sum over cells of a_h(u, 1_T) vanishes (interior fluxes cancel, no boundary term)
    pr = oracle.Problem(n, k, D, b=(0.8, -0.5, 0.3), c=0.0, bc=("neumann",) * 6)
    for _ in range(3):
        y = oracle.apply(pr, rng.uniform(-1, 1, pr.ndof)).reshape(12, -1)
        assert abs(np.sum(y[:, 0]) * np.sqrt(vol)) < 1e-12 * np.max(np.abs(y))
    # b = 0, c = 0: A 1 = 0
    pr0 = oracle.Problem(n, k, D, b=(0, 0, 0), c=0.0, bc=("neumann",) * 6)
    one = np.zeros((12, (k + 1) ** 3))
    one[:, 0] = 1.0
    assert np.max(np.abs(oracle.apply(pr0, one.ravel()))) < 1e-12
    # with a Dirichlet side the constant is no longer in the kernel
    pr1 = oracle.Problem(n, k, D, b=(0, 0, 0), c=0.0, bc=("dirichlet",) + ("neumann",) * 5)
    assert np.max(np.abs(oracle.apply(pr1, one.ravel()))) > 1e-2


def test_neumann_rhs_closed_form():
    """f = 0, j = j0 on the lower x side: F_(T, (j1, 0, 0)) = -j0 |F| theta_j1(0) on the cells at x = 0."""
    n, k = (2, 2, 3), 3
    lo, hi = (0.0, 0.0, 0.0), (1.0, 0.5, 1.5)
    j0 = 0.7
    pr = oracle.Problem(n, k, 1.0, lo=lo, hi=hi, bc=("neumann",) + ("dirichlet",) * 5)
    nf = n[1] * n[2]
    data = [np.full(nf * (k + 1) ** 2, j0)] + [None] * 5
    F = oracle.rhs(pr, None, data).reshape(n[2], n[1], n[0], k + 1, k + 1, k + 1)
    area = (0.5 / n[1]) * (1.5 / n[2])
    expect = np.zeros_like(F)
    th0 = np.array([np.sqrt(2 * j + 1) * (-1) ** j for j in range(k + 1)])
    expect[:, :, 0, 0, 0, :] = -j0 * area * th0
    assert rel(F, expect) < 1e-13
