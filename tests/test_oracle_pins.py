"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test names the property it pins and the passage that fixes it:

* Gauss-Legendre rule (Sec. 3.1) -> numpy's leggauss (library special case).
* 1D basis (Sec. 3.1, "L2-orthogonal Legendre", Sec. 2) -> numpy Legendre series; orthonormality.
* whole operator (eq. blf) -> an independent Kronecker closed form with exact 1D integrals.
* consistency of eq. blf with l_h (Sec. 2) -> zero residual for global polynomials of degree <= k.
* symmetry of the diffusion part of WSIPG (Sec. 2) -> v^T A u = u^T A v, u^T A u > 0.
* local conservation (Sec. 2) -> global balance with test function 1.
* reaction term / diagonal mass matrix (Sec. 2, eq. ODE_system) -> A(c1) - A(c2) = (c1-c2)|T| I.
* exactness of the m = k+1 Gauss rule for Problem A (q = 2p, Sec. 5.1) -> m = k+1 equals m = k+3.
* right hand side (Sec. 2) with f = 1, g = 0 -> F = |T| on mode 0.
* the discretisation as a whole -> L2 convergence of order k+1 for a smooth manufactured solution.
"""

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

import oracle
from tests import kron_reference as kr


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("m", list(range(1, 13)))
def test_gauss_legendre_matches_numpy(m):
    x, w = oracle.gauss_legendre(m)
    t, wt = npleg.leggauss(m)
    assert np.max(np.abs(x - 0.5 * (t + 1.0))) < 2e-15
    assert np.max(np.abs(w - 0.5 * wt)) < 2e-15
    # exact on monomials up to degree 2m-1
    for e in range(2 * m):
        assert abs(np.dot(w, x ** e) - 1.0 / (e + 1)) < 1e-14


@pytest.mark.parametrize("k", [0, 1, 3, 7, 10])
def test_basis_matches_numpy_and_is_orthonormal(k):
    th = kr.theta(k)
    for x in [0.0, 0.13, 0.5, 0.77, 1.0]:
        v, d = oracle.basis_1d(k, x)
        assert np.allclose(v, [t(x) for t in th], rtol=1e-13, atol=1e-13)
        assert np.allclose(d, [t.deriv()(x) for t in th], rtol=1e-12, atol=1e-12)
    xq, wq = oracle.gauss_legendre(k + 1)
    B = np.array([oracle.basis_1d(k, x)[0] for x in xq])  # [point, j]
    assert np.max(np.abs(B.T @ np.diag(wq) @ B - np.eye(k + 1))) < 1e-13
    mt = kr.matrices_1d(k)
    assert np.max(np.abs(mt["M"] - np.eye(k + 1))) < 1e-12


KRON_CASES = [
    # n, k, b, c, penalty mode, lo, hi
    ((1, 1, 1), 1, (1.0, 0.5, 0.25), 1.0, "workload", (0, 0, 0), (1, 1, 1)),
    ((2, 2, 2), 2, (1.0, 0.5, 0.25), 1.0, "workload", (0, 0, 0), (1, 1, 1)),
    ((2, 3, 2), 3, (-0.7, 0.4, -1.3), 0.3, "paper", (0, -1, 0.5), (1, 2, 1.25)),
    ((3, 1, 2), 2, (0.0, -2.0, 0.5), 0.0, "workload", (-1, -1, -1), (2, 0, 1)),
]


@pytest.mark.parametrize("case", KRON_CASES)
def test_oracle_matches_kronecker_closed_form(case):
    n, k, b, c, mode, lo, hi = case
    ncell = int(np.prod(n))
    rng = np.random.default_rng(11)
    D = np.exp(rng.standard_normal(ncell))
    sigma = oracle.penalty_sigma(k, mode)
    pr = oracle.Problem(n, k, D, b=b, c=c, sigma=sigma, lo=lo, hi=hi)
    A = kr.assemble(n, k, D, b, c, sigma, lo, hi)
    for trial in range(3):
        u = rng.uniform(-1, 1, pr.ndof)
        y = oracle.apply(pr, u)
        assert rel(y, A @ u) < 1e-12
    # sampled cells path agrees with the full path
    cells = [ncell - 1, 0]
    ys = oracle.apply(pr, u, cells=cells).reshape(2, pr.nb)
    yf = oracle.apply(pr, u).reshape(ncell, pr.nb)
    assert np.array_equal(ys, yf[cells])


def _proj_poly(pr, coeffs):
    """DG coefficients of the global polynomial u*(x) = sum_t prod_r poly_t_r(x_r) (exact L2 projection).

    Uses numpy Gauss points (independent of the oracle), (k+2) per direction: exact for degree 2k+2.
    """
    k = pr.k
    n1 = k + 1
    th = kr.theta(k)
    t, wt = npleg.leggauss(k + 2)
    xs, ws = 0.5 * (t + 1.0), 0.5 * wt
    Bv = np.array([[th[j](x) for j in range(n1)] for x in xs])  # [pt, j]
    h = (pr.hi - pr.lo) / pr.n
    z = np.zeros((pr.ncell, n1, n1, n1))  # [cell, j3, j2, j1]
    for iz in range(pr.n[2]):
        for iy in range(pr.n[1]):
            for ix in range(pr.n[0]):
                cell = ix + pr.n[0] * (iy + pr.n[1] * iz)
                for polys in coeffs:
                    f1 = polys[0](pr.lo[0] + h[0] * (ix + xs)) * ws
                    f2 = polys[1](pr.lo[1] + h[1] * (iy + xs)) * ws
                    f3 = polys[2](pr.lo[2] + h[2] * (iz + xs)) * ws
                    z[cell] += np.einsum("a,b,c->abc", Bv.T @ f3, Bv.T @ f2, Bv.T @ f1)
    return z.reshape(-1)


def _poly_terms(k, rng):
    P = np.polynomial.Polynomial
    terms = []
    for _ in range(3):
        terms.append([P(rng.standard_normal(k + 1)) for _ in range(3)])
    return terms


def _eval_terms(terms, xyz, op):
    out = np.zeros(xyz.shape[:-1])
    for polys in terms:
        vals = [polys[r](xyz[..., r]) for r in range(3)]
        ders = [polys[r].deriv()(xyz[..., r]) for r in range(3)]
        sec = [polys[r].deriv(2)(xyz[..., r]) for r in range(3)]
        out += op(vals, ders, sec)
    return out


@pytest.mark.parametrize("k,n", [(1, (2, 2, 2)), (2, (3, 2, 2)), (3, (2, 2, 3)), (4, (1, 2, 1))])
def test_polynomial_solution_has_zero_residual(k, n):
    """Consistency: for u* in Q_k globally, f = -D lap u* + b.grad u* + c u*, g = u*: A Pi u* = F exactly."""
    rng = np.random.default_rng(3 + k)
    D0, b, c = 1.7, (0.8, -0.6, 0.35), 0.9
    pr = oracle.Problem(n, k, D0, b=b, c=c, sigma=oracle.penalty_sigma(k, "workload"), lo=(0.1, -0.2, 0.0),
                        hi=(1.3, 0.7, 0.8))
    terms = _poly_terms(k, rng)
    z = _proj_poly(pr, terms)

    def src(v, d, s):
        lap = s[0] * v[1] * v[2] + v[0] * s[1] * v[2] + v[0] * v[1] * s[2]
        grad = [d[0] * v[1] * v[2], v[0] * d[1] * v[2], v[0] * v[1] * d[2]]
        return -D0 * lap + sum(b[r] * grad[r] for r in range(3)) + c * v[0] * v[1] * v[2]

    f = _eval_terms(terms, oracle.volume_points(pr), src)
    g = [_eval_terms(terms, oracle.face_points(pr, s), lambda v, d, s_: v[0] * v[1] * v[2]) for s in range(6)]
    F = oracle.rhs(pr, f, g)
    r = oracle.residual(pr, z, F)
    assert np.max(np.abs(r)) / np.max(np.abs(F)) < 1e-11


def test_diffusion_part_is_symmetric_and_coercive():
    rng = np.random.default_rng(5)
    n, k = (3, 2, 2), 3
    D = np.exp(2.0 * rng.standard_normal(12))
    pr = oracle.Problem(n, k, D, b=(0, 0, 0), c=0.0, lo=(0, 0, 0), hi=(1, 2, 0.5))
    for _ in range(3):
        u = rng.uniform(-1, 1, pr.ndof)
        v = rng.uniform(-1, 1, pr.ndof)
        vau = v @ oracle.apply(pr, u)
        uav = u @ oracle.apply(pr, v)
        assert abs(vau - uav) <= 1e-12 * (abs(vau) + abs(uav))
        assert u @ oracle.apply(pr, u) > 0
    # convection breaks the symmetry (the test would notice a dropped convection term)
    prb = oracle.Problem(n, k, D, b=(1.0, 0.3, -0.2), c=0.0, lo=(0, 0, 0), hi=(1, 2, 0.5))
    u = rng.uniform(-1, 1, pr.ndof)
    v = rng.uniform(-1, 1, pr.ndof)
    assert abs(v @ oracle.apply(prb, u) - u @ oracle.apply(prb, v)) > 1e-3


@pytest.mark.parametrize("b", [(1.0, 0.5, 0.25), (-0.4, 1.1, -0.9)])
def test_global_conservation(b):
    """sum_T (A u)_{T,0} = a_h(u, 1) = (c u, 1) + boundary fluxes (interior fluxes cancel, grad 1 = 0)."""
    rng = np.random.default_rng(9)
    n, k, c = (2, 3, 2), 2, 0.7
    D = np.exp(rng.standard_normal(12))
    lo, hi = np.array([0.0, -1.0, 0.5]), np.array([1.0, 0.5, 1.5])
    sigma = oracle.penalty_sigma(k)
    pr = oracle.Problem(n, k, D, b=b, c=c, sigma=sigma, lo=lo, hi=hi)
    u = rng.uniform(-1, 1, pr.ndof)
    y = oracle.apply(pr, u).reshape(pr.ncell, pr.nb)
    lhs = y[:, 0].sum()
    # independent evaluation with numpy polynomials and numpy Gauss points
    h = (hi - lo) / np.array(n)
    volT = np.prod(h)
    th = kr.theta(k)
    dth = [t.deriv() for t in th]
    t, wt = npleg.leggauss(k + 2)
    xs, ws = 0.5 * (t + 1), 0.5 * wt
    U = u.reshape(pr.ncell, k + 1, k + 1, k + 1)  # [cell, j3, j2, j1]
    total = c * volT * u.reshape(pr.ncell, pr.nb)[:, 0].sum()  # int_T u = |T| z_0
    Bv = np.array([[th[j](x) for j in range(k + 1)] for x in xs])
    for q in range(3):
        area = volT / h[q]
        for side in (0, 1):
            e = np.array([tj(float(side)) for tj in th])
            dd = np.array([dj(float(side)) for dj in dth])
            sgn = 1.0 if side else -1.0
            bnu = sgn * b[q]
            for cell in range(pr.ncell):
                ic = [cell % n[0], (cell // n[0]) % n[1], cell // (n[0] * n[1])]
                if ic[q] != (n[q] - 1 if side else 0):
                    continue
                # contract the normal index with the end-point values, tangential with Gauss points
                axes = {0: 3, 1: 2, 2: 1}  # array axis of j_q in U[cell]
                val = np.tensordot(U[cell], e, axes=([axes[q] - 1], [0]))
                der = np.tensordot(U[cell], dd, axes=([axes[q] - 1], [0]))
                uf = Bv @ val @ Bv.T
                dnu = sgn * (Bv @ der @ Bv.T) / h[q]
                wf = np.outer(ws, ws) * area
                gam = D[cell] * sigma * area / volT
                flux = (np.where(bnu >= 0, bnu * uf, 0.0) - D[cell] * dnu + gam * uf)
                total += np.sum(wf * flux)
    assert abs(lhs - total) < 1e-12 * max(1.0, abs(total))


def test_reaction_term_is_mass_matrix():
    rng = np.random.default_rng(2)
    n, k = (2, 2, 3), 3
    D = np.exp(rng.standard_normal(12))
    lo, hi = (0, 0, 0), (0.5, 1.0, 3.0)
    p1 = oracle.Problem(n, k, D, c=2.5, lo=lo, hi=hi)
    p0 = oracle.Problem(n, k, D, c=-0.5, lo=lo, hi=hi)
    u = rng.uniform(-1, 1, p1.ndof)
    volT = 0.25 * 0.5 * 1.0
    y1, y0 = oracle.apply(p1, u), oracle.apply(p0, u)
    # the difference cancels the large diffusion/face terms: measure against their size
    assert np.max(np.abs((y1 - y0) - 3.0 * volT * u)) < 1e-13 * np.max(np.abs(y1))


@pytest.mark.parametrize("k", [1, 3, 5])
def test_quadrature_order_independence(k):
    rng = np.random.default_rng(4)
    n = (2, 2, 2)
    D = np.exp(rng.standard_normal(8))
    pa = oracle.Problem(n, k, D)
    pb = oracle.Problem(n, k, D, m=k + 3)
    u = rng.uniform(-1, 1, pa.ndof)
    assert rel(oracle.apply(pa, u), oracle.apply(pb, u)) < 1e-12


def test_rhs_constant_source():
    """f = 1, g = 0: (1, phi_i)_T = |T| delta_{i,0} for the orthonormal basis with theta_0 = 1."""
    pr = oracle.Problem((8, 8, 8), 3, 1.0)
    F = oracle.rhs(pr, np.ones(pr.ncell * pr.m ** 3), None).reshape(pr.ncell, pr.nb)
    assert np.max(np.abs(F[:, 0] - 1.0 / 512)) < 1e-17
    assert np.max(np.abs(F[:, 1:])) < 1e-17


def _l2_error(pr, z, exact):
    k = pr.k
    th = kr.theta(k)
    t, wt = npleg.leggauss(k + 4)
    xs, ws = 0.5 * (t + 1), 0.5 * wt
    Bv = np.array([[th[j](x) for j in range(k + 1)] for x in xs])
    h = (pr.hi - pr.lo) / pr.n
    err2 = 0.0
    Z = z.reshape(pr.ncell, k + 1, k + 1, k + 1)
    for cell in range(pr.ncell):
        ic = [cell % pr.n[0], (cell // pr.n[0]) % pr.n[1], cell // (pr.n[0] * pr.n[1])]
        uh = np.einsum("ai,bj,ck,kji->abc", Bv, Bv, Bv, Z[cell])  # [x, y, z]
        X = pr.lo[0] + h[0] * (ic[0] + xs)
        Y = pr.lo[1] + h[1] * (ic[1] + xs)
        W = pr.lo[2] + h[2] * (ic[2] + xs)
        ue = exact(X[:, None, None], Y[None, :, None], W[None, None, :])
        err2 += np.sum(np.einsum("a,b,c->abc", ws, ws, ws) * (uh - ue) ** 2) * np.prod(h)
    return np.sqrt(err2)


@pytest.mark.parametrize("k", [1, 2])
def test_convergence_rate(k):
    """Smooth manufactured solution: the L2 error decays like h^(k+1) (standard DG estimate)."""
    D0, b, c = 1.0, (1.0, 0.5, 0.25), 1.0

    def ue(x, y, z):
        return np.exp(0.5 * x) * np.sin(1.3 * y + 0.2) * np.cos(0.9 * z)

    def f(x, y, z):
        u = ue(x, y, z)
        lap = (0.25 - 1.69 - 0.81) * u
        ux = 0.5 * u
        uy = np.exp(0.5 * x) * 1.3 * np.cos(1.3 * y + 0.2) * np.cos(0.9 * z)
        uz = -np.exp(0.5 * x) * np.sin(1.3 * y + 0.2) * 0.9 * np.sin(0.9 * z)
        return -D0 * lap + b[0] * ux + b[1] * uy + b[2] * uz + c * u

    errs = []
    for nn in (2, 4):
        pr = oracle.Problem((nn, nn, nn), k, D0, b=b, c=c)
        vp = oracle.volume_points(pr)
        fq = f(vp[..., 0], vp[..., 1], vp[..., 2])
        g = []
        for s in range(6):
            fp = oracle.face_points(pr, s)
            g.append(ue(fp[..., 0], fp[..., 1], fp[..., 2]))
        F = oracle.rhs(pr, fq, g)
        N = pr.ndof
        A = np.empty((N, N))
        eye = np.zeros(N)
        for j in range(N):
            eye[j] = 1.0
            A[:, j] = oracle.apply(pr, eye)
            eye[j] = 0.0
        z = np.linalg.solve(A, F)
        errs.append(_l2_error(pr, z, ue))
    rate = np.log2(errs[0] / errs[1])
    assert rate > k + 0.6, (errs, rate)
