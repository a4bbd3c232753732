"""Independent closed form of the WSIPG operator for the oracle pins (test helper).

On an axis-parallel uniform mesh with a per-cell constant scalar D, constant b
and c, every integrand of eq. blf (Sec. 2) is a tensor product of 1D
polynomials.  With the orthonormal 1D basis the tangential factors are
identities, so the whole operator is a sum of Kronecker products of small 1D
matrices.  The 1D entries here are EXACT polynomial integrals and end-point
values from ``numpy.polynomial`` -- no quadrature rule and none of the oracle's
tables -- and the matrix is assembled densely cell by cell and face by face.
It is a second, structurally different computation of a_h(phi_j, phi_i); it
shares nothing with the oracle except the documented layouts.
"""

from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as npleg


def theta(k: int):
    """Orthonormal shifted Legendre polynomials on [0,1] as numpy Legendre series objects."""
    return [np.sqrt(2 * j + 1) * npleg.Legendre.basis(j, domain=[0.0, 1.0]) for j in range(k + 1)]


def _integral01(p):
    P = p.integ()
    return P(1.0) - P(0.0)


def matrices_1d(k: int):
    th = theta(k)
    dth = [t.deriv() for t in th]
    n = k + 1
    M = np.array([[_integral01(th[i] * th[j]) for j in range(n)] for i in range(n)])
    S = np.array([[_integral01(dth[i] * dth[j]) for j in range(n)] for i in range(n)])
    C = np.array([[_integral01(dth[i] * th[j]) for j in range(n)] for i in range(n)])  # test' * trial
    e0 = np.array([t(0.0) for t in th])
    e1 = np.array([t(1.0) for t in th])
    d0 = np.array([t(0.0) for t in dth])
    d1 = np.array([t(1.0) for t in dth])
    return dict(M=M, S=S, C=C, e0=e0, e1=e1, d0=d0, d1=d1)


def _embed(mat1d, q, n):
    """Kronecker product acting on index j_q of J = j1 + n j2 + n^2 j3, identity on the others."""
    eye = np.eye(n)
    mats = [eye, eye, eye]
    mats[q] = mat1d
    # J = j1 + n*(j2 + n*j3): j3 slowest, so kron(order z, y, x)
    return np.kron(mats[2], np.kron(mats[1], mats[0]))


def assemble(n, k, D, b, c, sigma, lo=(0, 0, 0), hi=(1, 1, 1), periodic=(0, 0, 0), bc=None):
    """Dense A with A[(T,I),(S,J)] = a_h(phi_{S,J}, phi_{T,I}) (row = test function).

    On a periodic axis the face after the last cell couples it to the first cell (an interior face).  bc: the
    type of each boundary side 2*dir + (0 lower | 1 upper), 0 Dirichlet (default), 1 Neumann (no term in
    a_h), 2 outflow (only the upwind flux Phi(u, 0, b_nu))."""
    bc = [0] * 6 if bc is None else [{"dirichlet": 0, "neumann": 1, "outflow": 2}.get(t, t) for t in bc]
    n = tuple(int(v) for v in n)
    nb1 = k + 1
    nb = nb1 ** 3
    ncell = n[0] * n[1] * n[2]
    h = [(hi[r] - lo[r]) / n[r] for r in range(3)]
    volT = h[0] * h[1] * h[2]
    mt = matrices_1d(k)
    A = np.zeros((ncell * nb, ncell * nb))

    def cid(ix, iy, iz):
        return ix + n[0] * (iy + n[1] * iz)

    def blk(t, s):
        return (slice(t * nb, (t + 1) * nb), slice(s * nb, (s + 1) * nb))

    for iz in range(n[2]):
        for iy in range(n[1]):
            for ix in range(n[0]):
                T = cid(ix, iy, iz)
                DT = D[T]
                V = c * volT * np.eye(nb)
                for r in range(3):
                    V += DT * volT / h[r] ** 2 * _embed(mt["S"], r, nb1)
                    V -= b[r] * volT / h[r] * _embed(mt["C"], r, nb1)
                A[blk(T, T)] += V

    e0, e1, d0, d1 = mt["e0"], mt["e1"], mt["d0"], mt["d1"]
    for q in range(3):
        area = volT / h[q]
        hq = h[q]
        for iz in range(n[2]):
            for iy in range(n[1]):
                for ix in range(n[0]):
                    ic = [ix, iy, iz]
                    T = cid(*ic)
                    # interior face to the upper neighbour along q: T- = T, T+ = neighbour
                    if ic[q] + 1 < n[q] or periodic[q]:
                        jc = list(ic)
                        jc[q] = (jc[q] + 1) % n[q]
                        P = cid(*jc)
                        Dm, Dp = D[T], D[P]
                        wm, wp = Dp / (Dm + Dp), Dm / (Dm + Dp)
                        gam = 2 * Dm * Dp / (Dm + Dp) * sigma / hq
                        bq = b[q]
                        # trace functionals (rows: test index, cols: trial index), 1D along q
                        up_m = np.outer(e1, e1) * bq if bq >= 0 else np.zeros((nb1, nb1))
                        up_p = np.outer(e1, e0) * bq if bq < 0 else np.zeros((nb1, nb1))
                        # test in T-: jump(phi) = e1_i
                        mm = up_m - wm * Dm / hq * np.outer(e1, d1) - wm * Dm / hq * np.outer(d1, e1) \
                            + gam * np.outer(e1, e1)
                        mp = up_p - wp * Dp / hq * np.outer(e1, d0) + wm * Dm / hq * np.outer(d1, e0) \
                            - gam * np.outer(e1, e0)
                        # test in T+: jump(phi) = -e0_i
                        up_m2 = -np.outer(e0, e1) * bq if bq >= 0 else np.zeros((nb1, nb1))
                        up_p2 = -np.outer(e0, e0) * bq if bq < 0 else np.zeros((nb1, nb1))
                        pm = up_m2 + wm * Dm / hq * np.outer(e0, d1) - wp * Dp / hq * np.outer(d0, e1) \
                            - gam * np.outer(e0, e1)
                        pp = up_p2 + wp * Dp / hq * np.outer(e0, d0) + wp * Dp / hq * np.outer(d0, e0) \
                            + gam * np.outer(e0, e0)
                        A[blk(T, T)] += area * _embed(mm, q, nb1)
                        A[blk(T, P)] += area * _embed(mp, q, nb1)
                        A[blk(P, T)] += area * _embed(pm, q, nb1)
                        A[blk(P, P)] += area * _embed(pp, q, nb1)
                    # Dirichlet faces
                    for side in (0, 1):
                        on_b = not periodic[q] and ((ic[q] == 0) if side == 0 else (ic[q] == n[q] - 1))
                        if not on_b:
                            continue
                        DT = D[T]
                        gam = DT * sigma / hq
                        sgn = 1.0 if side else -1.0
                        ev = e1 if side else e0
                        dv = sgn * (d1 if side else d0) / hq  # nu . grad of the 1D factor
                        bnu = sgn * b[q]
                        kind = bc[2 * q + side]
                        if kind == 1:
                            continue
                        mat = bnu * np.outer(ev, ev) if bnu >= 0 else np.zeros((nb1, nb1))
                        if kind == 0:
                            mat = mat - DT * np.outer(ev, dv) - DT * np.outer(dv, ev) + gam * np.outer(ev, ev)
                        A[blk(T, T)] += area * _embed(mat, q, nb1)
    return A


def _kron3(mats):
    """Kronecker product of per-axis 1D matrices (mats[0] acts on j1, the fastest index)."""
    return np.kron(mats[2], np.kron(mats[1], mats[0]))


def assemble_tensor(n, k, Dten, b, c, sigma, lo=(0, 0, 0), hi=(1, 1, 1), periodic=(0, 0, 0)):
    """Dense A for a per-cell constant symmetric diffusion tensor Dten[cell] = (xx, yy, zz, xy, xz, yz) on the
    axis-parallel grid.  Off-diagonal entries couple a derivative along one axis with a derivative (volume) or
    a tangential derivative (faces) along another; each term is a Kronecker product of exact 1D integrals."""
    n = tuple(int(v) for v in n)
    nb1 = k + 1
    nb = nb1 ** 3
    ncell = n[0] * n[1] * n[2]
    h = [(hi[r] - lo[r]) / n[r] for r in range(3)]
    volT = h[0] * h[1] * h[2]
    mt = matrices_1d(k)
    I1 = np.eye(nb1)
    C = mt["C"]  # C[i][j] = int theta_i' theta_j (test derivative, trial value)
    A = np.zeros((ncell * nb, ncell * nb))

    def tensor(cell):
        t = Dten[cell]
        return np.array([[t[0], t[3], t[4]], [t[3], t[1], t[5]], [t[4], t[5], t[2]]])

    def cid(ix, iy, iz):
        return ix + n[0] * (iy + n[1] * iz)

    def blk(t, s):
        return (slice(t * nb, (t + 1) * nb), slice(s * nb, (s + 1) * nb))

    for iz in range(n[2]):
        for iy in range(n[1]):
            for ix in range(n[0]):
                T = cid(ix, iy, iz)
                D = tensor(T)
                V = c * volT * np.eye(nb)
                for r in range(3):  # test derivative axis
                    V -= b[r] * volT / h[r] * _embed(C, r, nb1)
                    for s in range(3):  # trial derivative axis
                        mats = [I1, I1, I1]
                        if r == s:
                            mats[r] = mt["S"]
                        else:
                            mats[r] = C
                            mats[s] = C.T
                        V += D[r, s] * volT / (h[r] * h[s]) * _kron3(mats)
                A[blk(T, T)] += V

    e = {0: mt["e0"], 1: mt["e1"]}
    d = {0: mt["d0"], 1: mt["d1"]}

    def flux_trial(D, q, end, sgn):
        """sgn * nu . D grad(trial) at the face across axis q at reference end `end`, as per-axis factors to be
        paired with the test factors: list of (coefficient, q-column vector, {axis: matrix})."""
        out = []
        for s in range(3):
            if s == q:
                out.append((sgn * D[q, s] / h[q], d[end], {}))
            else:
                out.append((sgn * D[q, s] / h[s], e[end], {s: C.T}))
        return out

    def flux_test(D, q, end, sgn):
        out = []
        for s in range(3):
            if s == q:
                out.append((sgn * D[q, s] / h[q], d[end], {}))
            else:
                out.append((sgn * D[q, s] / h[s], e[end], {s: C}))
        return out

    def term(test_vec, trial_vec, q, extra):
        mats = [I1, I1, I1]
        mats[q] = np.outer(test_vec, trial_vec)
        for ax, mtx in extra.items():
            mats[ax] = mtx
        return _kron3(mats)

    for q in range(3):
        area = volT / h[q]
        for iz in range(n[2]):
            for iy in range(n[1]):
                for ix in range(n[0]):
                    ic = [ix, iy, iz]
                    T = cid(*ic)
                    if ic[q] + 1 < n[q] or periodic[q]:
                        jc = list(ic)
                        jc[q] = (jc[q] + 1) % n[q]
                        P = cid(*jc)
                        Dm, Dp = tensor(T), tensor(P)
                        dm, dp = Dm[q, q], Dp[q, q]
                        wm, wp = dp / (dm + dp), dm / (dm + dp)
                        gam = 2 * dm * dp / (dm + dp) * sigma / h[q]
                        bq = b[q]
                        # cells: minus T (face at its end 1), plus P (face at its end 0); nu = +e_q
                        sides = {0: (T, 1, Dm, wm, +1.0), 1: (P, 0, Dp, wp, -1.0)}  # (cell, end, D, w, jump sign)
                        for xs in (0, 1):
                            X, ex_, DX, wX, jX = sides[xs]
                            for ys in (0, 1):
                                Y, ey_, DY, wY, jY = sides[ys]
                                M = np.zeros((nb, nb))
                                # upwind: Phi(u-, u+, b) [[v]] with the upwind side's trace of the trial function
                                up = 0 if bq >= 0 else 1
                                if ys == up:
                                    M += jX * bq * term(e[ex_], e[ey_], q, {})
                                # -{nu.D grad u}_w [[v]]
                                for coef, tv, extra in flux_trial(DY, q, ey_, 1.0):
                                    M -= jX * wY * coef * term(e[ex_], tv, q, extra)
                                # -{nu.D grad v}_w [[u]]
                                for coef, tv, extra in flux_test(DX, q, ex_, 1.0):
                                    M -= jY * wX * coef * term(tv, e[ey_], q, extra)
                                # penalty
                                M += gam * jX * jY * term(e[ex_], e[ey_], q, {})
                                A[blk(X, Y)] += area * M
                    for side in (0, 1):
                        on_b = not periodic[q] and ((ic[q] == 0) if side == 0 else (ic[q] == n[q] - 1))
                        if not on_b:
                            continue
                        D = tensor(T)
                        sgn = 1.0 if side else -1.0
                        gam = D[q, q] * sigma / h[q]
                        M = np.zeros((nb, nb))
                        if sgn * b[q] >= 0:
                            M += sgn * b[q] * term(e[side], e[side], q, {})
                        for coef, tv, extra in flux_trial(D, q, side, sgn):
                            M -= coef * term(e[side], tv, q, extra)
                        for coef, tv, extra in flux_test(D, q, side, sgn):
                            M -= coef * term(tv, e[side], q, extra)
                        M += gam * term(e[side], e[side], q, {})
                        A[blk(T, T)] += area * M
    return A
