"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module only draws random numbers and describes workloads; it holds none of
the method's arithmetic.  Everything is generated with
``numpy.random.default_rng(seed)`` and handed to both the CUDA library and the
oracle as plain arrays, so the two sides never need a common generator.

Workloads (Problem A of Sec. 5.1: axis-parallel cells, per-cell constant
coefficients, q = 2p i.e. m = k+1 Gauss points per direction):

* ``unit_cube_q3_8``  -- 8^3 cells on [0,1]^3, k = 3, D = 1, b = (1, .5, .25),
  c = 1, penalty 2k(k+1)/h, Dirichlet g = 0, f = 1, u ~ U[-1,1] (seed 0).
* ``unit_cube_q7_32`` -- 32^3 cells, k = 7, D_T = exp(N(0,1)) per cell (seed 1),
  same b, c, f, g, u ~ U[-1,1] (seed 2).
* ``unit_cube_q5_48`` -- 48^3 cells, k = 5, log-normal D (sigma 1, seed 3),
  f = a sum of 8 seeded sine modes (seed 4).
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

B_DEFAULT = (1.0, 0.5, 0.25)
C_DEFAULT = 1.0


@dataclass
class Workload:
    name: str
    n: tuple
    k: int
    D: np.ndarray
    b: tuple = B_DEFAULT
    c: float = C_DEFAULT
    u: np.ndarray | None = None
    f_kind: str = "one"          # "one" (f = 1), "zero" or "sines"
    f_params: dict = field(default_factory=dict)
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)
    periodic: tuple = (0, 0, 0)     # 1 on an axis whose two end faces are identified
    velocity: str = "constant"      # "constant" (b) or "taylor_green" (the flow field of Sec. 5.3)
    m: int | None = None            # Gauss points per direction (None: k+1)

    @property
    def ncell(self):
        return int(np.prod(self.n))

    @property
    def nb(self):
        return (self.k + 1) ** 3

    @property
    def ndof(self):
        return self.ncell * self.nb


def log_normal_D(ncell: int, sigma: float, seed: int) -> np.ndarray:
    """Per-cell diffusion D_T = exp(sigma * N(0,1)), i.i.d."""
    return np.exp(sigma * np.random.default_rng(seed).standard_normal(ncell))


def uniform_u(ndof: int, seed: int) -> np.ndarray:
    """DG coefficient vector with i.i.d. U[-1,1] entries."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, ndof)


def sine_modes(seed: int, count: int = 8) -> dict:
    """Parameters of f(x) = sum_l a_l sin(2 pi n_l . x + phi_l): a ~ N(0,1), n in {1..4}^3, phi ~ U[0, 2pi)."""
    rng = np.random.default_rng(seed)
    return {"a": rng.standard_normal(count), "n": rng.integers(1, 5, size=(count, 3)),
            "phi": rng.uniform(0.0, 2.0 * np.pi, count)}


def eval_sines(params: dict, xyz: np.ndarray) -> np.ndarray:
    """Evaluate the sine-mode source at points xyz[..., 3]."""
    arg = 2.0 * np.pi * (xyz @ params["n"].T.astype(np.float64)) + params["phi"]
    return np.sin(arg) @ params["a"]


def f_at(w: Workload, xyz: np.ndarray) -> np.ndarray:
    """Source term f at the given quadrature point coordinates xyz[..., 3]."""
    if w.f_kind == "one":
        return np.ones(xyz.shape[:-1])
    if w.f_kind == "zero":
        return np.zeros(xyz.shape[:-1])
    if w.f_kind == "sines":
        return eval_sines(w.f_params, xyz)
    raise ValueError(w.f_kind)


def unit_cube_q3_8() -> Workload:
    w = Workload("unit_cube_q3_8", (8, 8, 8), 3, np.ones(512))
    w.u = uniform_u(w.ndof, 0)
    return w


def unit_cube_q7_32() -> Workload:
    n = (32, 32, 32)
    w = Workload("unit_cube_q7_32", n, 7, log_normal_D(32 ** 3, 1.0, 1))
    w.u = uniform_u(w.ndof, 2)
    return w


def unit_cube_q5_48(with_u: bool = True) -> Workload:
    w = Workload("unit_cube_q5_48", (48, 48, 48), 5, log_normal_D(48 ** 3, 1.0, 3), f_kind="sines",
                 f_params=sine_modes(4))
    if with_u:
        w.u = uniform_u(w.ndof, 5)
    return w


def small_case(n=(3, 2, 4), k=2, sigma_D=1.0, seed=7, b=B_DEFAULT, c=C_DEFAULT, f_kind="one") -> Workload:
    """Small anisotropic-count mesh for fast parity checks: seeded D and u."""
    ncell = int(np.prod(n))
    w = Workload(f"small_{n}_{k}", tuple(n), k, log_normal_D(ncell, sigma_D, seed), b=tuple(b), c=c, f_kind=f_kind)
    w.u = uniform_u(w.ndof, seed + 1)
    return w


def batch_problems(count: int = 64, seed: int = 5, nmin: int = 4, nmax: int = 24, kmin: int = 2, kmax: int = 8):
    """Many uneven problems: n ~ U{nmin..nmax}, k ~ U{kmin..kmax} per problem, log-normal D, U[-1,1] u."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(nmin, nmax + 1, size=count)
    ks = rng.integers(kmin, kmax + 1, size=count)
    out = []
    for i in range(count):
        n = int(ns[i])
        k = int(ks[i])
        w = Workload(f"batch{i}", (n, n, n), k, log_normal_D(n ** 3, 1.0, 1000 + i))
        w.u = uniform_u(w.ndof, 2000 + i)
        out.append(w)
    return out


def taylor_green_velocity(xyz: np.ndarray) -> np.ndarray:
    """The fixed Taylor-Green type flow field of the transport example (Sec. 5.3) at points xyz[..., 3]:
    b = (cos x1 sin(-x2) sin(-x3), 1/2 sin x1 cos(-x2) sin(-x3), 1/2 sin x1 sin(-x2) cos(-x3))."""
    x1, x2, x3 = xyz[..., 0], xyz[..., 1], xyz[..., 2]
    return np.stack([np.cos(x1) * np.sin(-x2) * np.sin(-x3),
                     0.5 * np.sin(x1) * np.cos(-x2) * np.sin(-x3),
                     0.5 * np.sin(x1) * np.sin(-x2) * np.cos(-x3)], axis=-1)


def gaussian_bump(xyz: np.ndarray, x0=(0.5, 0.0, 0.0)) -> np.ndarray:
    """Initial concentration of the transport example: exp(-2 |x - x0|^2)."""
    d = xyz - np.asarray(x0)
    return np.exp(-2.0 * np.sum(d * d, axis=-1))


def gaussian_bump_grid(w: Workload, xi, x0=(0.5, 0.0, 0.0), xp=np, **kw):
    """exp(-2 |x - x0|^2) at the volume points [ncell, m^3] of the workload's mesh, built from its three
    one-dimensional factors (the bump is separable), so no [ncell, m^3, 3] coordinate array is formed.
    xi: the m Gauss points on [0,1]; xp: numpy or torch (kw, e.g. device=, go to xp.asarray)."""
    m = len(xi)
    xi = xp.asarray(np.asarray(xi, dtype=np.float64), **kw)
    g = []
    for r in range(3):
        h = (w.hi[r] - w.lo[r]) / w.n[r]
        ic = xp.asarray(np.arange(w.n[r], dtype=np.float64), **kw)
        x = w.lo[r] + h * (ic[:, None] + xi[None, :])          # [n_r, m]
        g.append(xp.exp(-2.0 * (x - x0[r]) ** 2))
    gx, gy, gz = g
    # axes (iz, iy, ix, i3, i2, i1): cell = ix + nx (iy + ny iz), point q = i1 + m (i2 + m i3)
    v = gz[:, None, None, :, None, None] * gy[None, :, None, None, :, None] * gx[None, None, :, None, None, :]
    return v.reshape(w.ncell, m ** 3)


def face_normal_velocity(bfun, face_xyz: np.ndarray) -> np.ndarray:
    """b . e_dir at the face points of every face of every cell, face_xyz[ncell, 6, m^2, 3] (face s = 2 dir + side)."""
    b = bfun(face_xyz)
    out = np.empty(face_xyz.shape[:3])
    for s in range(6):
        out[:, s] = b[:, s, :, s // 2]
    return out


def taylor_green(n=16, k=5, m=None) -> Workload:
    """Transport on the periodic cube (-pi, pi)^3: D = 5e-6, c = 0, f = 0, Taylor-Green velocity and
    q = 2p+4, i.e. m = k+3 Gauss points per direction (Sec. 5.3).  The initial value is the Gaussian bump
    exp(-2 |x - (1/2, 0, 0)|^2), projected onto the DG space by the caller."""
    w = Workload(f"taylor_green_q{k}_{n}", (n, n, n), k, np.full(n ** 3, 5e-6), b=(0.0, 0.0, 0.0), c=0.0,
                 f_kind="zero", lo=(-np.pi,) * 3, hi=(np.pi,) * 3, periodic=(1, 1, 1), velocity="taylor_green",
                 m=m if m is not None else k + 3)
    return w


def log_normal_tensors(ncell: int, sigma: float, seed: int, anisotropy: float = 0.5) -> np.ndarray:
    """Per-cell symmetric positive definite diffusion tensors (xx, yy, zz, xy, xz, yz): R diag(l) R^T with
    log-normal eigenvalues l = exp(sigma N(0,1)) and a random rotation R per cell, the eigenvalues spread by
    a further factor exp(anisotropy N(0,1)) each."""
    rng = np.random.default_rng(seed)
    base = np.exp(sigma * rng.standard_normal(ncell))
    lam = base[:, None] * np.exp(anisotropy * rng.standard_normal((ncell, 3)))
    Q, R = np.linalg.qr(rng.standard_normal((ncell, 3, 3)))
    Q = Q * np.sign(np.diagonal(R, axis1=1, axis2=2))[:, None, :]
    M = np.einsum("cij,cj,ckj->cik", Q, lam, Q)
    return np.stack([M[:, 0, 0], M[:, 1, 1], M[:, 2, 2], M[:, 0, 1], M[:, 0, 2], M[:, 1, 2]], axis=1)


def pack_sym(Mx: np.ndarray) -> np.ndarray:
    """Symmetric 3x3 matrices [..., 3, 3] as (xx, yy, zz, xy, xz, yz) [..., 6], the layout of the tensor inputs."""
    return np.stack([Mx[..., 0, 0], Mx[..., 1, 1], Mx[..., 2, 2], Mx[..., 0, 1], Mx[..., 0, 2], Mx[..., 1, 2]],
                    axis=-1)


class PolynomialFields:
    """Seeded coefficients that are polynomials in the coordinates (Problem B of Sec. 5.1).

    With s = (x - lo) / (hi - lo) the position normalised to the domain's bounding box:
      D(x) = A(s) A(s)^T + d0 I,  A(s) = A0 + s_0 A1 + s_1 A2 + s_2 A3   (quadratic, symmetric positive definite),
      b(x) = b0 + B1 s,   c(x) = c0 + c1 . s  (c0 > |c1|_1, so c > 0 on the box).
    ``spread`` scales the random parts of A relative to the identity part.
    """

    def __init__(self, seed: int, lo, hi, spread: float = 0.4, d0: float = 0.2):
        rng = np.random.default_rng(seed)
        self.lo = np.asarray(lo, dtype=np.float64)
        self.scale = 1.0 / (np.asarray(hi, dtype=np.float64) - self.lo)
        self.A = np.concatenate([np.eye(3)[None] + spread * rng.uniform(-1, 1, (1, 3, 3)),
                                 spread * rng.uniform(-1, 1, (3, 3, 3))])
        self.d0 = d0
        self.b0 = rng.uniform(-1, 1, 3)
        self.B1 = rng.uniform(-0.5, 0.5, (3, 3))
        self.c1 = rng.uniform(-0.3, 0.3, 3)
        self.c0 = 1.0 + np.abs(self.c1).sum()

    def _s(self, xyz):
        return (np.asarray(xyz, dtype=np.float64) - self.lo) * self.scale

    def D(self, xyz) -> np.ndarray:
        """D at the points xyz [..., 3] as [..., 6] (pack_sym layout)."""
        s = self._s(xyz)
        A = self.A[0] + np.einsum("...k,kij->...ij", s, self.A[1:])
        return pack_sym(np.einsum("...ik,...jk->...ij", A, A) + self.d0 * np.eye(3))

    def b(self, xyz) -> np.ndarray:
        return self.b0 + self._s(xyz) @ self.B1.T

    def c(self, xyz) -> np.ndarray:
        return self.c0 + self._s(xyz) @ self.c1


def face_unit_normals(J) -> np.ndarray:
    """Unit normals along +reference axis r of the cells lo + J (ic + [0,1]^3): the rows of J^{-1}, normalised
    (the axis-parallel grid has J = diag(h) and e_r)."""
    Ji = np.linalg.inv(np.asarray(J, dtype=np.float64).reshape(3, 3))
    return Ji / np.linalg.norm(Ji, axis=1)[:, None]


def face_normal_velocity_affine(bfun, face_xyz: np.ndarray, J) -> np.ndarray:
    """b . nu at the points of every face of every cell, face_xyz [ncell, 6, m^2, 3] (face s = 2 dir + side, nu
    the unit normal along +reference axis dir)."""
    nrm = face_unit_normals(J)
    return np.einsum("cspi,si->csp", bfun(face_xyz), np.repeat(nrm, 2, axis=0))


def sheared_jacobian(h, seed: int = 0, shear: float = 0.25) -> np.ndarray:
    """A seeded affine cell map J = (I + shear * U) diag(h), U with entries in [-1, 1] above the diagonal (an
    invertible sheared version of the axis-parallel cell of size h)."""
    rng = np.random.default_rng(seed)
    U = np.triu(rng.uniform(-1, 1, (3, 3)), 1)
    return (np.eye(3) + shear * U) @ np.diag(np.asarray(h, dtype=np.float64))


def multilinear_vertices(n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), seed: int = 0, amplitude: float = 0.2):
    """Vertices [(n0+1)(n1+1)(n2+1), 3] (x fastest) of a structured grid of [lo, hi] whose vertices are moved by
    seeded offsets of up to amplitude * h per component, so that the cells are general trilinear hexahedra
    (Problem C of Sec. 5.1).  A vertex on the boundary moves only within its boundary face, so the domain stays
    the box [lo, hi]; amplitude < 0.25 keeps every cell's map invertible."""
    n = [int(v) for v in n]
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    h = (hi - lo) / np.asarray(n)
    k, j, i = np.meshgrid(np.arange(n[2] + 1), np.arange(n[1] + 1), np.arange(n[0] + 1), indexing="ij")
    idx = np.stack([i, j, k], axis=-1).reshape(-1, 3)
    X = lo + idx * h
    rng = np.random.default_rng(seed)
    d = rng.uniform(-amplitude, amplitude, X.shape) * h
    on_bnd = (idx == 0) | (idx == np.asarray(n))
    d[on_bnd] = 0.0
    return X + d
