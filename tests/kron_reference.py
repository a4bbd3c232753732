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


def _along(mat, X, r):
    """Apply the 1D matrix mat (out i = sum_j mat[i, j] x_j) along reference axis r of every cell block of X,
    X shaped (nz, ny, nx, n, n, n) with the last three axes (j3, j2, j1)."""
    ax = 5 - r
    return np.moveaxis(np.tensordot(X, mat, axes=([ax], [1])), -1, ax)


def _trace(X, vec, r):
    """The 1D functional vec applied along reference axis r: removes that axis."""
    return np.tensordot(X, vec, axes=([5 - r], [0]))


def _outer_add(Y, idx, vec, F, r):
    """Y[idx] += vec (along reference axis r) times the face array F (the two tangential axes)."""
    shp = [1] * 6
    shp[5 - r] = vec.size
    Y[idx] += np.expand_dims(F, 5 - r) * vec.reshape(shp)


def apply_matfree(n, k, D, b, c, sigma, u, lo=(0, 0, 0), hi=(1, 1, 1), periodic=(0, 0, 0), bc=None):
    """y = A u for the operator that ``assemble`` writes out, without forming A: the same exact 1D integrals
    and end-point values, applied block by block.

    The volume term of every cell is c|T| u + sum_r |T| (D_T / h_r^2 S - b_r / h_r C) along axis r.  On a face
    across axis q the four trace functionals (values e0, e1 and reference derivatives d0, d1 at the two ends of
    the 1D factor) of both cells give, with the orthonormal tangential factors, the face quantities
      jump = u- - u+,  avg = w- D- u-' + w+ D+ u+',  Phi = b_q u_upwind,  H = Phi - avg + gamma jump,
    and the face adds |F| (e1 H - d1 w- D- / h jump) to the lower cell and |F| (-e0 H - d0 w+ D+ / h jump) to
    the upper one (the physical derivative is the reference one over h).  Cost O(N k) for N unknowns, so it
    checks whole vectors of meshes with tens of millions of unknowns.  u and the result are in the documented
    layout [cell][j1 + n (j2 + n j3)], cells x fastest."""
    bc = [0] * 6 if bc is None else [{"dirichlet": 0, "neumann": 1, "outflow": 2}.get(t, t) for t in bc]
    nx, ny, nz = (int(v) for v in n)
    nb1 = k + 1
    U = np.asarray(u, dtype=np.float64).reshape(nz, ny, nx, nb1, nb1, nb1)
    Dg = np.asarray(D, dtype=np.float64).reshape(nz, ny, nx)
    h = [(hi[r] - lo[r]) / (nx, ny, nz)[r] for r in range(3)]
    volT = h[0] * h[1] * h[2]
    mt = matrices_1d(k)
    e0, e1, d0, d1 = mt["e0"], mt["e1"], mt["d0"], mt["d1"]
    Dc = Dg[..., None, None, None]
    Y = c * volT * U
    for r in range(3):
        Y = Y + (volT / h[r] ** 2) * Dc * _along(mt["S"], U, r) - (b[r] * volT / h[r]) * _along(mt["C"], U, r)
    for q in range(3):
        cax = 2 - q  # cell axis of direction q in (nz, ny, nx)
        nq = (nx, ny, nz)[q]
        hq, area, bq = h[q], volT / h[q], b[q]
        tv0, tv1 = _trace(U, e0, q), _trace(U, e1, q)
        td0, td1 = _trace(U, d0, q) / hq, _trace(U, d1, q) / hq
        Df = Dg[..., None, None]

        def cells(sl):
            idx = [slice(None)] * 3
            idx[cax] = sl
            return tuple(idx)

        # interior faces: lower cell T- (index i) and upper cell T+ (index i+1, wrapping on a periodic axis)
        if periodic[q]:
            lo_idx = cells(slice(None))
            roll = lambda a: np.roll(a, -1, axis=cax)
            um, dm, Dm = tv1, td1, Df
            up, dp, Dp = roll(tv0), roll(td0), roll(Df)
        else:
            lo_idx, hi_idx = cells(slice(0, nq - 1)), cells(slice(1, nq))
            um, dm, Dm = tv1[lo_idx], td1[lo_idx], Df[lo_idx]
            up, dp, Dp = tv0[hi_idx], td0[hi_idx], Df[hi_idx]
        if um.size:
            wm, wp = Dp / (Dm + Dp), Dm / (Dm + Dp)
            gam = 2 * Dm * Dp / (Dm + Dp) * sigma / hq
            jump = um - up
            avg = wm * Dm * dm + wp * Dp * dp
            phi = bq * (um if bq >= 0 else up)
            H = phi - avg + gam * jump
            Wm, Wp = -wm * Dm * jump, -wp * Dp * jump
            lower = np.zeros_like(Y)
            upper = np.zeros_like(Y)
            if periodic[q]:
                _outer_add(lower, Ellipsis, e1, area * H, q)
                _outer_add(lower, Ellipsis, d1 / hq, area * Wm, q)
                _outer_add(upper, Ellipsis, e0, -area * H, q)
                _outer_add(upper, Ellipsis, d0 / hq, area * Wp, q)
                Y = Y + lower + np.roll(upper, 1, axis=cax)
            else:
                _outer_add(lower, lo_idx, e1, area * H, q)
                _outer_add(lower, lo_idx, d1 / hq, area * Wm, q)
                _outer_add(upper, hi_idx, e0, -area * H, q)
                _outer_add(upper, hi_idx, d0 / hq, area * Wp, q)
                Y = Y + lower + upper
        if periodic[q]:
            continue
        # boundary sides: Dirichlet (all terms), outflow (upwind flux only), Neumann (nothing in a_h)
        for side in (0, 1):
            kind = bc[2 * q + side]
            if kind == 1:
                continue
            idx = cells(slice(0, 1) if side == 0 else slice(nq - 1, nq))
            sgn = 1.0 if side else -1.0
            ev, dv = (e1, d1) if side else (e0, d0)
            tv = (tv1 if side else tv0)[idx]
            tdv = sgn * (td1 if side else td0)[idx]  # nu . grad u
            DT = Df[idx]
            bnu = sgn * bq
            Hs = bnu * tv if bnu >= 0 else np.zeros_like(tv)
            add = np.zeros_like(Y)
            if kind == 0:
                Hs = Hs - DT * tdv + DT * sigma / hq * tv
                _outer_add(add, idx, sgn * dv / hq, -area * DT * tv, q)
            _outer_add(add, idx, ev, area * Hs, q)
            Y = Y + add
    return Y.reshape(-1)
