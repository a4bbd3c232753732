"""Pins of the oracle's periodic axes and point-wise velocity field (the transport example of Sec. 5.3)."""

import numpy as np
import pytest

import oracle
from paper_1711_10885_gb300 import inputs
from tests import kron_reference as kr


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("periodic", [(1, 0, 0), (0, 1, 1), (1, 1, 1)])
def test_periodic_matches_kronecker_closed_form(periodic):
    n, k = (3, 2, 3), 2
    rng = np.random.default_rng(1)
    D = np.exp(rng.standard_normal(18))
    b = (0.7, -0.4, 0.3)
    pr = oracle.Problem(n, k, D, b=b, c=0.6, periodic=periodic, lo=(0, 0, 0), hi=(1, 2, 1.5))
    A = kr.assemble(n, k, D, b, 0.6, pr.sigma, (0, 0, 0), (1, 2, 1.5), periodic=periodic)
    u = rng.uniform(-1, 1, pr.ndof)
    assert rel(oracle.apply(pr, u), A @ u) < 1e-12


def test_constant_field_given_at_points_equals_constant_velocity():
    n, k = (2, 3, 2), 3
    rng = np.random.default_rng(2)
    D = np.exp(rng.standard_normal(12))
    b = np.array([0.9, -0.2, 0.5])
    p0 = oracle.Problem(n, k, D, b=b, c=0.3)
    vol = np.broadcast_to(b, (p0.ncell, p0.m ** 3, 3)).copy()
    fxyz = oracle.cell_face_points(p0)
    bface = inputs.face_normal_velocity(lambda x: np.broadcast_to(b, x.shape).copy(), fxyz)
    p1 = oracle.Problem(n, k, D, b=(0, 0, 0), c=0.3, b_vol=vol, b_face=bface)
    u = rng.uniform(-1, 1, p0.ndof)
    assert rel(oracle.apply(p1, u), oracle.apply(p0, u)) < 1e-14
    # the inflow part of l_h reads b . nu from the face field too
    g = [np.sin(oracle.face_points(p0, s).sum(axis=-1)).ravel() for s in range(6)]
    assert rel(oracle.rhs(p1, None, g), oracle.rhs(p0, None, g)) < 1e-14


def test_constant_velocity_transport_annihilates_constants_and_is_dissipative():
    """D -> 0 (the weights need D > 0), c = 0, constant b, all axes periodic: A 1 = 0 (the upwind flux of a
    continuous field cancels the volume term, div b = 0), and u^T A u = 1/2 sum_F |b.nu| ||[u]||^2 >= 0."""
    n, k = (3, 2, 2), 3
    pr = oracle.Problem(n, k, 1e-12, b=(0.8, -0.5, 0.3), c=0.0, periodic=(1, 1, 1))
    one = np.zeros((pr.ncell, pr.nb))
    one[:, 0] = 1.0
    y = oracle.apply(pr, one.ravel())
    assert np.max(np.abs(y)) < 1e-13
    rng = np.random.default_rng(5)
    for _ in range(4):
        u = rng.uniform(-1, 1, pr.ndof)
        e = u @ oracle.apply(pr, u)
        assert e > 0
    # without periodicity the same field has inflow boundaries and the constant is no longer annihilated
    pd = oracle.Problem(n, k, 1e-12, b=(0.8, -0.5, 0.3), c=0.0)
    assert np.max(np.abs(oracle.apply(pd, one.ravel()))) > 1e-2


def _tg_problem(n=3, k=2):
    w = inputs.taylor_green(n, k)
    pr = oracle.Problem(w.n, w.k, w.D, b=(0, 0, 0), c=0.0, lo=w.lo, hi=w.hi, periodic=w.periodic)
    vol = inputs.taylor_green_velocity(oracle.volume_points(pr))
    bface = inputs.face_normal_velocity(inputs.taylor_green_velocity, oracle.cell_face_points(pr))
    return oracle.Problem(w.n, w.k, w.D, b=(0, 0, 0), c=0.0, lo=w.lo, hi=w.hi, periodic=w.periodic, b_vol=vol,
                          b_face=bface)


def test_periodic_transport_conserves_mass_exactly():
    """With every axis periodic and c = 0, sum_T a_h(u, 1_T) = 0 for any u: each face flux enters its two
    cells with opposite signs (including the faces across the periodic seam) and grad 1 = 0."""
    pr = _tg_problem(3, 2)
    rng = np.random.default_rng(3)
    for _ in range(3):
        u = rng.uniform(-1, 1, pr.ndof)
        y = oracle.apply(pr, u).reshape(pr.ncell, pr.nb)
        scale = np.abs(y[:, 0]).sum()
        assert abs(y[:, 0].sum()) <= 1e-13 * scale


def test_periodic_translation_invariance():
    """Constant coefficients on a periodic mesh: shifting u by one cell along an axis shifts A u."""
    n, k = (4, 3, 3), 2
    pr = oracle.Problem(n, k, 1.3, b=(0.5, -0.8, 0.2), c=0.4, periodic=(1, 1, 1))
    rng = np.random.default_rng(4)
    u = rng.uniform(-1, 1, pr.ndof).reshape(n[2], n[1], n[0], pr.nb)
    y = oracle.apply(pr, u.ravel()).reshape(n[2], n[1], n[0], pr.nb)
    for axis in (0, 1, 2):
        ys = oracle.apply(pr, np.roll(u, 1, axis=axis).ravel()).reshape(y.shape)
        assert rel(ys, np.roll(y, 1, axis=axis)) < 1e-13


def test_rhs_volume_term_reproduces_a_dg_field():
    """(u_h, phi_i)_T / |T| = z_i for u_h = sum_j z_j phi_j: the m >= k+1 point rule integrates the
    degree-2k product exactly and the basis is orthonormal (mass matrix |T| I, Sec. 2)."""
    from tests.test_gpu_transport import oracle_field_values
    for k, m in ((2, 3), (3, 6)):
        pr = oracle.Problem((2, 3, 2), k, 1.0, b=(0, 0, 0), c=0.0, m=m, lo=(0, 0, 0), hi=(1, 2, 0.5))
        z = np.random.default_rng(k).uniform(-1, 1, pr.ndof)
        vol = 1.0 / 2 * 2.0 / 3 * 0.5 / 2
        F = oracle.rhs(pr, oracle_field_values(pr, z), None)
        assert rel(F / vol, z) < 1e-13
