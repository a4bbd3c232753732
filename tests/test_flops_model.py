"""The executed-flop model (flops.py), which every reported fraction of peak divides by, against an
instrumented CPU sum factorisation.

The even-odd building blocks of the kernels are written out below in plain numpy with an operation counter
(FMA = 2, MUL and ADD = 1, as in flops.py).  They run on the real 1D tables (orthonormal Legendre modes,
Gauss-Legendre points on [0, 1], collocation derivative; Sec. 3.3 and 3.4), so each block is checked twice:
its result against the plain matrix product it replaces, and its count against the formula in flops.py.
"""

import numpy as np
import pytest
from numpy.polynomial import legendre as L

from paper_1711_10885_gb300 import flops


class Count:
    def __init__(self):
        self.n = 0

    def mul(self, a, b):
        self.n += 1
        return a * b

    def add(self, a, b):
        self.n += 1
        return a + b

    def sub(self, a, b):
        self.n += 1
        return a - b

    def fma(self, a, b, c):
        self.n += 2
        return a * b + c


def tables(N, M):
    """Phi[i][j] = theta_j(xi_i) (M points, N modes), the collocation derivative D (M x M) and weights w."""
    x, w = L.leggauss(M)
    xi, w = (x + 1) / 2, w / 2
    Phi = np.stack([np.sqrt(2 * j + 1) * L.legval(2 * xi - 1, np.eye(N)[j]) for j in range(N)], axis=1)
    # derivative of the Lagrange basis at the points: D = V' V^{-1} with the full M-mode Legendre Vandermonde
    V = np.stack([L.legval(2 * xi - 1, np.eye(M)[j]) for j in range(M)], axis=1)
    Vd = np.stack([2 * L.legval(2 * xi - 1, L.legder(np.eye(M)[j])) for j in range(M)], axis=1)
    return Phi, Vd @ np.linalg.inv(V), w


def dot(c, coefs, vals):
    acc = c.mul(coefs[0], vals[0])
    for a, v in zip(coefs[1:], vals[1:]):
        acc = c.fma(a, v, acc)
    return acc


def split(c, x):
    n = len(x)
    h = n // 2
    s = [c.add(x[i], x[n - 1 - i]) for i in range(h)] + ([x[h]] if n % 2 else [])
    d = [c.sub(x[i], x[n - 1 - i]) for i in range(h)]
    return s, d


def eo_fwd(c, Phi, x):
    M, N = Phi.shape
    HM, CM, HN, CN = M // 2, (M + 1) // 2, N // 2, (N + 1) // 2
    e = [dot(c, [Phi[i][2 * k] for k in range(CN)], [x[2 * k] for k in range(CN)]) for i in range(CM)]
    o = [dot(c, [Phi[i][2 * k + 1] for k in range(HN)], [x[2 * k + 1] for k in range(HN)]) for i in range(HM)]
    y = [0.0] * M
    for i in range(HM):
        y[i] = c.add(e[i], o[i])
        y[M - 1 - i] = c.sub(e[i], o[i])
    if M % 2:
        y[HM] = e[HM]
    return np.array(y)


def eo_bwd(c, Phi, x):
    M, N = Phi.shape
    HM, CM, HN, CN = M // 2, (M + 1) // 2, N // 2, (N + 1) // 2
    s, d = split(c, x)
    y = [0.0] * N
    for k in range(CN):
        y[2 * k] = dot(c, [Phi[i][2 * k] for i in range(CM)], s)
    for k in range(HN):
        y[2 * k + 1] = dot(c, [Phi[i][2 * k + 1] for i in range(HM)], d)
    return np.array(y)


def eo_anti(c, D, s, d):
    """out = D x for a centro-antisymmetric D, from the split parts (s, d) of x."""
    N = D.shape[0]
    H, C = N // 2, (N + 1) // 2
    Hm = [[(D[i][l] - D[i][N - 1 - l]) / 2 for l in range(H)] for i in range(C)]
    Hp = [[(D[i][l] + D[i][N - 1 - l]) / 2 for l in range(H)] + ([D[i][H]] if N % 2 else []) for i in range(H)]
    gp = [dot(c, Hm[i], d) for i in range(C)]
    gm = [dot(c, Hp[i], s) for i in range(H)]
    out = [0.0] * N
    for i in range(H):
        out[i] = c.add(gp[i], gm[i])
        out[N - 1 - i] = c.sub(gp[i], gm[i])
    if N % 2:
        out[H] = gp[H]
    return np.array(out)


def deriv_line(c, D, w, u, v, sa, sb, sc, first):
    """One derivative pass on a line: v (+)= B [sa d u + sb u] (+ sc w u on the first pass), B = D^T diag(w),
    and the value and derivative traces at both ends (the kernels' deriv_line)."""
    M = len(u)
    H, C = M // 2, (M + 1) // 2
    s, d = split(c, u)
    gr = eo_anti(c, D, s, d)
    X = [c.fma(sa, gr[i], c.mul(sb, u[i])) for i in range(M)]
    xs, xd = split(c, X)
    B = D.T * w[None, :]
    cc = eo_anti(c, B, xs, xd)
    if first:
        v = np.array([c.fma(c.mul(sc, w[l]), u[l], cc[l]) for l in range(M)])
    else:
        v = np.array([c.add(v[l], cc[l]) for l in range(M)])
    # traces: value and derivative at xi = 0 and 1 from the split parts (fma chains, then 4 add/sub); only
    # their count matters here (their values are part of the operator parity tests)
    e1 = np.array([1.0] * M)
    t1 = t2 = q1 = q2 = 0.0
    for l in range(C):
        t1 = c.fma(e1[l], s[l], t1)
        q1 = c.fma(e1[l], s[l], q1)
    for l in range(H):
        t2 = c.fma(e1[l], d[l], t2)
        q2 = c.fma(e1[l], d[l], q2)
    c.sub(t1, t2), c.sub(q2, q1), c.add(t1, t2), c.add(q1, q2)
    return v, gr, np.array(X)


@pytest.mark.parametrize("N", range(2, 12))
def test_even_odd_blocks_reproduce_the_products_and_the_counts(N):
    rng = np.random.default_rng(N)
    for M in (N, N + 2):
        Phi, _, _ = tables(N, M)
        x = rng.standard_normal(N)
        c = Count()
        assert np.allclose(eo_fwd(c, Phi, x), Phi @ x, atol=1e-12)
        assert c.n == flops.eo_fwd_flops(N, M)
        y = rng.standard_normal(M)
        c = Count()
        assert np.allclose(eo_bwd(c, Phi, y), Phi.T @ y, atol=1e-12)
        assert c.n == flops.eo_bwd_flops(N, M)
    _, D, w = tables(N, N)
    assert np.allclose(D[::-1, ::-1], -D, atol=1e-9)  # centro-antisymmetric at symmetric points
    x = rng.standard_normal(N)
    c = Count()
    s, d = split(c, x)
    c0 = c.n
    assert np.allclose(eo_anti(c, D, s, d), D @ x, atol=1e-9)
    assert c.n - c0 == flops.eo_anti_flops(N)


@pytest.mark.parametrize("N", range(2, 12))
def test_derivative_pass_reproduces_the_volume_term_and_the_count(N):
    rng = np.random.default_rng(100 + N)
    _, D, w = tables(N, N)
    u = rng.standard_normal(N)
    v0 = rng.standard_normal(N)
    sa, sb, sc = 1.3, -0.4, 0.7
    for first in (True, False):
        c = Count()
        v, gr, X = deriv_line(c, D, w, u, v0, sa, sb, sc, first)
        assert np.allclose(gr, D @ u, atol=1e-9)
        ref = D.T @ (w * (sa * (D @ u) + sb * u)) + (sc * w * u if first else v0)
        assert np.allclose(v, ref, atol=1e-8)
        assert c.n == flops.deriv_line_flops(N, first)
