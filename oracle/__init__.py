"""FP64 CPU oracle for the WSIPG DG operator (arXiv 1711.10885, Sec. 2, eq. blf).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU-baseline
leg of the benchmark may import this package; the product path (the CUDA
library and its Python binding) never does.

The arithmetic lives in ``dg_oracle.c`` (plain C, direct quadrature over all
basis functions and points, no sum factorisation).  This module compiles it
with gcc on first use (or via :func:`build`) and wraps it with ctypes.

Every function here cites the passage of the paper it follows:

* :func:`gauss_legendre` -- the tensor Gauss rule of Sec. 3.1, one axis on [0,1].
* :func:`basis_1d` -- the 1D shape functions theta_j of Sec. 3.1, read as the
  orthonormal shifted Legendre polynomials ("L2-orthogonal Legendre", Sec. 2).
* :func:`apply` -- (A u)_i = a_h(u, phi_i), eq. blf (scalar or tensor D, axis-parallel or affine cells).
* :func:`rhs` -- F_i = l_h(phi_i), the right hand side functional of Sec. 2.
* :func:`residual` -- r = A u - F (the residual evaluation of Sec. 1).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libdg_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile dg_oracle.c into oracle/_build/libdg_oracle.so (gcc, -O2, portable flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"],
                       check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _configure(lib):
    lib.oracle_gauss_legendre.argtypes = [ctypes.c_int, _dp, _dp]
    lib.oracle_basis_1d.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp]
    lib.oracle_basis_1d.restype = None
    lib.oracle_apply.argtypes = [_ip, _dp, _dp, ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_double,
                                 ctypes.c_double, _dp, _dp, _ip, ctypes.c_int]
    lib.oracle_rhs.argtypes = [_ip, _dp, _dp, ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_double,
                               ctypes.c_double, _dp, ctypes.POINTER(_dp), _dp]
    lib.oracle_apply_ex.argtypes = [_ip, _dp, _dp, ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_double,
                                    ctypes.c_double, _ip, _ip, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp,
                                    _ip, ctypes.c_int]
    lib.oracle_rhs_ex.argtypes = [_ip, _dp, _dp, ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_double,
                                  ctypes.c_double, _ip, _ip, _dp, _dp, _dp, _dp, _dp, _dp, ctypes.POINTER(_dp), _dp]
    lib.oracle_cell_face_points.argtypes = [_ip, _dp, _dp, ctypes.c_int, _dp]
    lib.oracle_volume_points_ex.argtypes = [_ip, _dp, _dp, _dp, _dp, ctypes.c_int, _dp]
    lib.oracle_face_points_ex.argtypes = [_ip, _dp, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int, _dp]
    lib.oracle_cell_face_points_ex.argtypes = [_ip, _dp, _dp, _dp, _dp, ctypes.c_int, _dp]
    lib.oracle_volume_points.argtypes = [_ip, _dp, _dp, ctypes.c_int, _dp]
    lib.oracle_face_points.argtypes = [_ip, _dp, _dp, ctypes.c_int, ctypes.c_int, _dp]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(ctypes.CDLL(build()))
    return _lib


class use_library:
    """Context manager that routes this module's calls to another build of the oracle source (the
    mutation tests compile copies of dg_oracle.c with one planted mistake)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        _load()
        with _lock:
            self.saved = _lib
            _lib = _configure(ctypes.CDLL(self.path))
        return self

    def __exit__(self, *exc):
        global _lib
        with _lock:
            _lib = self.saved
        return False


def _d(a):
    return a.ctypes.data_as(_dp)


def _arr(x, n=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def gauss_legendre(m: int):
    """m-point Gauss-Legendre nodes (ascending) and weights on [0,1] (Sec. 3.1)."""
    x = np.empty(m)
    w = np.empty(m)
    if _load().oracle_gauss_legendre(m, _d(x), _d(w)) != 0:
        raise ValueError("bad m")
    return x, w


def basis_1d(k: int, x: float):
    """theta_j(x), theta_j'(x) for j = 0..k: sqrt(2j+1) P_j(2x-1) (Sec. 3.1 / Sec. 2)."""
    v = np.empty(k + 1)
    d = np.empty(k + 1)
    _load().oracle_basis_1d(k, float(x), _d(v), _d(d))
    return v, d


class Problem:
    """Axis-parallel uniform cuboid mesh with per-cell scalar D, constant b, c (Problem A, Sec. 5.1).

    ``sigma`` is the penalty factor of gamma_F = <delta-,delta+> sigma |F| / min(|T-|,|T+|) (Sec. 2);
    ``penalty_sigma`` gives the two readings.  ``m`` defaults to k+1 Gauss points (q = 2p, Sec. 5.1).
    Options: ``periodic`` axes and a velocity field ``b_vol``/``b_face`` (Sec. 5.3); a per-cell diffusion
    tensor ``D_tensor`` [ncell, 6] = (xx, yy, zz, xy, xz, yz) (Sec. 5.1); an affine geometry ``J`` (3x3 cell
    Jacobian, cells lo + J (ic + [0,1]^3); ``hi`` is then unused).  ``bc``: the boundary type of each side
    2*dir + (0 lower | 1 upper), "dirichlet", "neumann" or "outflow" (eq. modelproblem: Gamma_D, Gamma_N,
    Gamma_O); rhs() then reads g on Dirichlet sides and the total flux j = (b u - D grad u) . nu on Neumann
    sides from its per-side arrays.  ``vertices`` [(n0+1)(n1+1)(n2+1), 3] (x fastest): multilinear cells,
    each the trilinear image of [0,1]^3 through its 8 corner vertices (Problem C of Sec. 5.1); ``lo``, ``hi``
    and ``J`` are then unused.
    """

    def __init__(self, n, k, D, b=(1.0, 0.5, 0.25), c=1.0, sigma=None, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0),
                 m=None, periodic=(0, 0, 0), b_vol=None, b_face=None, D_tensor=None, J=None, D_vol=None,
                 D_face=None, c_vol=None, bc=None, vertices=None):
        self.n = np.ascontiguousarray(np.asarray(n, dtype=np.int32).reshape(3))
        self.lo = _arr(lo, 3)
        self.hi = _arr(hi, 3)
        self.k = int(k)
        self.m = int(m) if m is not None else self.k + 1
        self.ncell = int(np.prod(self.n))
        D = np.asarray(D, dtype=np.float64)
        self.D = _arr(np.full(self.ncell, float(D)) if D.ndim == 0 else D, self.ncell)
        self.b = _arr(b, 3)
        self.c = float(c)
        self.sigma = float(sigma) if sigma is not None else penalty_sigma(self.k, "workload")
        self.nb = (self.k + 1) ** 3
        # periodic axes and a velocity field at the quadrature points (Sec. 5.3); see oracle_apply_ex
        self.periodic = np.ascontiguousarray(np.asarray(periodic, dtype=np.int32).reshape(3))
        self.b_vol = None if b_vol is None else _arr(b_vol, self.ncell * self.m ** 3 * 3)
        self.b_face = None if b_face is None else _arr(b_face, self.ncell * 6 * self.m ** 2)
        self.D_tensor = None if D_tensor is None else _arr(D_tensor, self.ncell * 6)
        self.J = None if J is None else _arr(J, 9)
        # coefficients at the quadrature points (Problem B): D_vol [ncell, m^3, 6], D_face [ncell, 6, m^2, 6],
        # c_vol [ncell, m^3]
        self.D_vol = None if D_vol is None else _arr(D_vol, self.ncell * self.m ** 3 * 6)
        self.D_face = None if D_face is None else _arr(D_face, self.ncell * 6 * self.m ** 2 * 6)
        self.c_vol = None if c_vol is None else _arr(c_vol, self.ncell * self.m ** 3)
        # multilinear cells (Problem C): vertex coordinates [(n0+1)(n1+1)(n2+1), 3], x fastest
        nv = int(np.prod(self.n + 1))
        self.vertices = None if vertices is None else _arr(vertices, nv * 3)
        kinds = {"dirichlet": 0, "neumann": 1, "outflow": 2}
        self.bc = np.ascontiguousarray(np.asarray([kinds[t] if isinstance(t, str) else int(t)
                                                   for t in (bc if bc is not None else ["dirichlet"] * 6)],
                                                  dtype=np.int32).reshape(6))

    def _general(self):
        return (_d(self.D_tensor) if self.D_tensor is not None else None, _d(self.J) if self.J is not None else None,
                _d(self.vertices) if self.vertices is not None else None)

    def _pointwise(self):
        return tuple(_d(a) if a is not None else None for a in (self.D_vol, self.D_face, self.c_vol))

    @property
    def ndof(self):
        return self.ncell * self.nb

    def _args(self):
        return (self.n.ctypes.data_as(_ip), _d(self.lo), _d(self.hi), self.k, self.m, _d(self.D), _d(self.b),
                self.c, self.sigma)


def penalty_sigma(k: int, mode: str = "workload", alpha: float = 2.0, d: int = 3) -> float:
    """sigma in gamma_F = <delta-,delta+> sigma |F|/min|T| (Sec. 2).

    'paper': alpha * p (p + d - 1) as printed with alpha = 2; 'workload': 2 k (k+1), the value that the
    benchmark workloads prescribe as "2k(k+1)/h" for D = I.
    """
    if mode == "paper":
        return alpha * k * (k + d - 1)
    if mode == "workload":
        return 2.0 * k * (k + 1)
    raise ValueError(mode)


def apply(pr: Problem, u, cells=None) -> np.ndarray:
    """y = A u with (A u)_i = a_h(u, phi_i) (eq. blf); if ``cells`` is given only those cells' blocks."""
    u = _arr(u, pr.ndof)
    ex = (pr.periodic.ctypes.data_as(_ip), pr.bc.ctypes.data_as(_ip), _d(pr.b_vol) if pr.b_vol is not None else None,
          _d(pr.b_face) if pr.b_face is not None else None, *pr._general(), *pr._pointwise())
    if cells is None:
        y = np.empty(pr.ndof)
        rc = _load().oracle_apply_ex(*pr._args(), *ex, _d(u), _d(y), None, 0)
    else:
        cl = np.ascontiguousarray(np.asarray(cells, dtype=np.int32).reshape(-1))
        y = np.empty(cl.size * pr.nb)
        rc = _load().oracle_apply_ex(*pr._args(), *ex, _d(u), _d(y), cl.ctypes.data_as(_ip), int(cl.size))
    if rc != 0:
        raise RuntimeError(f"oracle_apply failed ({rc})")
    return y


def rhs(pr: Problem, f_qp=None, g_qp=None) -> np.ndarray:
    """F_i = l_h(phi_i) (Sec. 2): f at volume points [ncell, m^3]; g_qp: list of 6 side arrays (g on Dirichlet
    sides, j on Neumann sides) or None."""
    F = np.empty(pr.ndof)
    fa = None if f_qp is None else _arr(f_qp, pr.ncell * pr.m ** 3)
    keep = []
    garr = None
    if g_qp is not None:
        garr = (_dp * 6)()
        for s in range(6):
            if g_qp[s] is None:
                garr[s] = _dp()
            else:
                a = _arr(g_qp[s])
                keep.append(a)
                garr[s] = _d(a)
    rc = _load().oracle_rhs_ex(*pr._args(), pr.periodic.ctypes.data_as(_ip), pr.bc.ctypes.data_as(_ip),
                               _d(pr.b_face) if pr.b_face is not None else None, *pr._general(),
                               pr._pointwise()[1], _d(fa) if fa is not None else None, garr, _d(F))
    if rc != 0:
        raise RuntimeError(f"oracle_rhs failed ({rc})")
    return F


def residual(pr: Problem, u, F) -> np.ndarray:
    """r = A u - F (residual evaluation, Sec. 1)."""
    return apply(pr, u) - F


def volume_points(pr: Problem) -> np.ndarray:
    """Physical coordinates [ncell, m^3, 3] of the volume quadrature points (oracle's own nodes)."""
    xyz = np.empty(pr.ncell * pr.m ** 3 * 3)
    if _load().oracle_volume_points_ex(pr.n.ctypes.data_as(_ip), _d(pr.lo), _d(pr.hi), *pr._general()[1:],
                                       pr.m, _d(xyz)) != 0:
        raise RuntimeError("oracle_volume_points failed")
    return xyz.reshape(pr.ncell, pr.m ** 3, 3)


def cell_face_points(pr: Problem) -> np.ndarray:
    """Physical coordinates [ncell, 6, m^2, 3] of the face points of every face of every cell."""
    xyz = np.empty(pr.ncell * 6 * pr.m ** 2 * 3)
    if _load().oracle_cell_face_points_ex(pr.n.ctypes.data_as(_ip), _d(pr.lo), _d(pr.hi), *pr._general()[1:],
                                          pr.m, _d(xyz)) != 0:
        raise RuntimeError("oracle_cell_face_points failed")
    return xyz.reshape(pr.ncell, 6, pr.m ** 2, 3)


def face_points(pr: Problem, s: int) -> np.ndarray:
    """Physical coordinates [nfaces, m^2, 3] of the boundary face points of side s = 2*dir + (0 lo | 1 hi)."""
    d = s // 2
    ta, tb = (1, 2) if d == 0 else ((0, 2) if d == 1 else (0, 1))
    nf = int(pr.n[ta] * pr.n[tb])
    xyz = np.empty(nf * pr.m ** 2 * 3)
    if _load().oracle_face_points_ex(pr.n.ctypes.data_as(_ip), _d(pr.lo), _d(pr.hi), *pr._general()[1:],
                                     pr.m, s, _d(xyz)) != 0:
        raise RuntimeError("oracle_face_points failed")
    return xyz.reshape(nf, pr.m ** 2, 3)
