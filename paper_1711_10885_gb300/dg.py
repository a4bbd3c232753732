"""Thin Python binding of libdg.so (argument marshalling only).

Every step of the operator runs in the CUDA library; this module turns torch
tensors into device pointers and a stream into a ``cudaStream_t`` and calls the
C ABI declared in ``include/dg.h`` under the same names.  There is no CPU or
PyTorch fallback: if the compiled library is missing, importing fails loudly.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libdg.so")

DG_OK = 0
DG_ERR_INVALID_ARG, DG_ERR_CUDA, DG_ERR_OOM, DG_ERR_NOT_CONVERGED, DG_ERR_TIMEOUT, DG_ERR_NAN = -1, -2, -3, -4, -5, -6
DG_F64 = 0
DG_F32 = 1
DG_F64X = 2  # FP64 vectors, double-float arithmetic on the FP32 pipes
DG_PROBE_DFMA, DG_PROBE_DMMA, DG_PROBE_FFMA = 0, 1, 2
DG_BATCH_CANDIDATES = 4
DG_MAX_DEGREE = 10

_dp = ctypes.POINTER(ctypes.c_double)


class DGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"dg error {code}: {msg}")
        self.code = code


class dg_mesh(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3), ("n", ctypes.c_int32 * 3)]


class dg_coeffs(ctypes.Structure):
    _fields_ = [("D_cell", _dp), ("D_const", ctypes.c_double), ("b", ctypes.c_double * 3),
                ("c", ctypes.c_double), ("sigma", ctypes.c_double)]


class dg_bc(ctypes.Structure):
    _fields_ = [("g_qp", _dp * 6)]


DG_BC_DIRICHLET = 0
DG_BC_NEUMANN = 1
DG_BC_OUTFLOW = 2
DG_VELOCITY_CONSTANT = 0
DG_VELOCITY_POINTS = 1
DG_VELOCITY_TAYLOR_GREEN = 2
_VELOCITY = {"constant": DG_VELOCITY_CONSTANT, "points": DG_VELOCITY_POINTS, "taylor_green": DG_VELOCITY_TAYLOR_GREEN}


class dg_setup_ext(ctypes.Structure):
    _fields_ = [("periodic", ctypes.c_int32 * 3), ("m", ctypes.c_int32), ("velocity", ctypes.c_int32),
                ("b_qp", _dp), ("b_face", _dp), ("D_tensor", _dp), ("jacobian", _dp), ("D_qp", _dp),
                ("D_face", _dp), ("c_qp", _dp), ("bc_type", ctypes.c_int32 * 6), ("vertices", _dp)]


DG_SOLVE_FP64 = 0
DG_SOLVE_MIXED = 1
DG_PRECOND_NONE = 0
DG_PRECOND_BLOCK_JACOBI = 1
DG_PRECOND_MLP = 2
DG_PRECOND_BJ_MLP = 3
DG_PRECOND_RB_GS = 4
DG_BJ_DENSE = 1
DG_BJ_FAST_DIAG = 2
DG_PRECOND_HAS_DENSE = 1
DG_PRECOND_HAS_FAST_DIAG = 2
DG_PRECOND_FAST_DIAG_REAL = 4


class dg_solve_opts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("preconditioner", ctypes.c_int32), ("restart", ctypes.c_int32),
                ("outer_restart", ctypes.c_int32), ("max_iterations", ctypes.c_int32), ("rtol", ctypes.c_double),
                ("inner_rtol", ctypes.c_double), ("mlp", ctypes.c_void_p), ("mlp_placement", ctypes.c_int32),
                ("fallback_ratio", ctypes.c_double), ("inner_block_precision", ctypes.c_int32),
                ("outer_precision", ctypes.c_int32), ("inner_basis_precision", ctypes.c_int32)]


class dg_mlp_train_opts(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_double)]


class dg_mlp_train_stats(ctypes.Structure):
    _fields_ = [("first_epoch_loss", ctypes.c_double), ("last_epoch_loss", ctypes.c_double),
                ("steps", ctypes.c_int64)]


class dg_solve_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32), ("inner_iterations", ctypes.c_int32),
                ("applies_f64", ctypes.c_int32), ("applies_f32", ctypes.c_int32), ("rel_residual", ctypes.c_double),
                ("seconds", ctypes.c_double), ("fallback", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libdg.so not built ({LIB_PATH}); run __graft_entry__.build() first")
    lib = ctypes.CDLL(LIB_PATH)
    vp = ctypes.c_void_p
    lib.dg_last_error.restype = ctypes.c_char_p
    lib.dg_penalty_sigma.restype = ctypes.c_double
    lib.dg_penalty_sigma.argtypes = [ctypes.c_int32, ctypes.c_int32]
    lib.dg_setup.argtypes = [ctypes.POINTER(dg_mesh), ctypes.c_int32, ctypes.POINTER(dg_coeffs),
                             ctypes.POINTER(dg_bc), _dp, vp, ctypes.POINTER(vp)]
    lib.dg_setup_ex.argtypes = [ctypes.POINTER(dg_mesh), ctypes.c_int32, ctypes.POINTER(dg_coeffs),
                                ctypes.POINTER(dg_bc), _dp, ctypes.POINTER(dg_setup_ext), vp, ctypes.POINTER(vp)]
    lib.dg_project.argtypes = [vp, vp, vp, vp]
    lib.dg_rk_stage.argtypes = [vp, vp, vp, vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int32, vp]
    lib.dg_ssprk2.argtypes = [vp, vp, ctypes.c_double, ctypes.c_int32, ctypes.c_int32, vp]
    lib.dg_assemble.argtypes = [vp, vp, ctypes.POINTER(vp)]
    lib.dg_matrix_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                   ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)]
    lib.dg_matrix_export.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32), _dp]
    lib.dg_spmv.argtypes = [vp, vp, vp, vp]
    lib.dg_matrix_destroy.argtypes = [vp]
    lib.dg_destroy.argtypes = [vp]
    lib.dg_sizes.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32),
                             ctypes.POINTER(ctypes.c_int64)]
    lib.dg_quadrature_points.argtypes = [vp, ctypes.c_int32, _dp]
    lib.dg_apply_jacobian.argtypes = [vp, vp, vp, ctypes.c_int32, vp]
    lib.dg_apply_residual.argtypes = [vp, vp, vp, ctypes.c_int32, vp]
    lib.dg_rhs.argtypes = [vp, vp, ctypes.c_int32, vp]
    lib.dg_apply_stage.argtypes = [vp, ctypes.c_int32, vp, vp, ctypes.c_int32, ctypes.c_int32, vp]
    lib.dg_precond_setup.argtypes = [vp, ctypes.c_int32, vp]
    lib.dg_precond_apply.argtypes = [vp, vp, vp, ctypes.c_int32, vp]
    lib.dg_precond_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)]
    lib.dg_precond_apply_rbgs.argtypes = [vp, vp, vp, vp, ctypes.c_int32, vp]
    lib.dg_solve.argtypes = [vp, vp, vp, ctypes.POINTER(dg_solve_opts), ctypes.POINTER(dg_solve_stats), vp]
    lib.dg_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int32, vp, ctypes.POINTER(vp)]
    lib.dg_batch_apply.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.c_int32, vp]
    lib.dg_batch_tuning.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                    ctypes.POINTER(ctypes.c_float)]
    lib.dg_batch_destroy.argtypes = [vp]
    lib.dg_mlp_create.argtypes = [ctypes.c_int32, ctypes.c_uint64, ctypes.POINTER(vp)]
    lib.dg_mlp_destroy.argtypes = [vp]
    lib.dg_mlp_dims.argtypes = [vp] + [ctypes.POINTER(ctypes.c_int32)] * 4 + [ctypes.POINTER(ctypes.c_int64)]
    lib.dg_mlp_params.argtypes = [vp, ctypes.POINTER(ctypes.c_float), ctypes.c_int32, ctypes.POINTER(ctypes.c_float)]
    lib.dg_mlp_param_offsets.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
    lib.dg_mlp_set_target_scale.argtypes = [vp, ctypes.c_float]
    lib.dg_mlp_features.argtypes = [vp, vp, vp, ctypes.c_int32, vp, ctypes.c_int64, vp, vp, vp]
    lib.dg_mlp_forward.argtypes = [vp, vp, ctypes.c_int64, vp, vp]
    lib.dg_mlp_pairs.argtypes = [vp, vp, vp, vp, vp, vp, ctypes.c_int64, ctypes.c_int32, vp, vp, vp]
    lib.dg_mlp_normalize_targets.argtypes = [vp, vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_float), vp]
    lib.dg_mlp_loss_grad.argtypes = [vp, vp, vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_double), vp]
    lib.dg_mlp_train.argtypes = [vp, vp, vp, ctypes.c_int64, ctypes.POINTER(dg_mlp_train_opts),
                                 ctypes.POINTER(dg_mlp_train_stats), vp]
    lib.dg_mlp_apply.argtypes = [vp, vp, vp, vp, ctypes.c_int32, vp]
    lib.dg_mlp_apply_add.argtypes = [vp, vp, vp, vp, ctypes.c_int32, vp]
    lib.dg_peak_probe.argtypes = [ctypes.c_int32, ctypes.c_int64, vp, _dp, vp]
    lib.dg_mlp_save.argtypes = [vp, ctypes.c_char_p]
    lib.dg_mlp_load.argtypes = [ctypes.c_char_p, ctypes.POINTER(vp)]
    return lib


lib = _load()

# C-ABI symbols declared in include/dg.h (checked by the CPU test suite)
EXPORTED = ["dg_penalty_sigma", "dg_setup", "dg_destroy", "dg_sizes", "dg_quadrature_points", "dg_apply_jacobian",
            "dg_apply_residual", "dg_rhs", "dg_last_error", "dg_apply_stage", "dg_precond_setup",
            "dg_precond_apply", "dg_precond_info", "dg_precond_apply_rbgs", "dg_solve", "dg_batch_create", "dg_batch_apply", "dg_batch_tuning",
            "dg_batch_destroy", "dg_mlp_create", "dg_mlp_destroy", "dg_mlp_dims", "dg_mlp_params",
            "dg_mlp_param_offsets", "dg_mlp_set_target_scale", "dg_mlp_features", "dg_mlp_forward", "dg_mlp_loss_grad",
            "dg_mlp_train", "dg_mlp_apply", "dg_mlp_apply_add", "dg_mlp_save", "dg_mlp_load",
            "dg_apply_jacobian_static", "dg_setup_ex", "dg_project", "dg_rk_stage", "dg_ssprk2", "dg_assemble",
            "dg_matrix_info", "dg_matrix_export", "dg_spmv", "dg_matrix_destroy", "dg_peak_probe", "dg_mlp_pairs",
            "dg_mlp_normalize_targets"]


def peak_probe(kind, iterations, sink, stream=None):
    """Launch one arithmetic throughput probe (dg_peak_probe) on the stream; returns its floating-point
    operation count.  sink: a float64 device tensor of at least one element."""
    fl = ctypes.c_double()
    check(lib.dg_peak_probe(int(kind), int(iterations), ctypes.c_void_p(sink.data_ptr()), ctypes.byref(fl),
                            _stream_ptr(stream)))
    return fl.value


def check(rc):
    if rc != DG_OK:
        raise DGError(rc, lib.dg_last_error().decode())
    return rc


def dg_penalty_sigma(k: int, mode: int = 0) -> float:
    return lib.dg_penalty_sigma(k, mode)


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _prec(t):
    import torch
    if t.dtype == torch.float64:
        return DG_F64
    if t.dtype == torch.float32:
        return DG_F32
    raise TypeError("vectors must be float64 or float32")


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class Operator:
    """A dg_handle: mesh, degree, coefficients and right hand side (dg_setup / dg_setup_ex), freed by close().

    Transport options (dg_setup_ext): ``periodic`` flags per axis, ``m`` Gauss points per direction (k+1 or
    k+3), ``velocity`` "constant" (b), "points" (b_qp [ncell, m^3, 3] and b_face [ncell, 6, m^2]) or
    "taylor_green" (the flow field of Sec. 5.3, evaluated by the library); ``D_tensor`` [ncell, 6] per-cell
    diffusion tensors and ``jacobian`` (3x3) affine cells lo + J (ic + [0,1]^3) (Sec. 5.1).  Problem B's
    coefficients at the quadrature points: ``D_qp`` [ncell, m^3, 6] and ``D_face`` [ncell, 6, m^2, 6] (both, at
    quadrature_points(0) and quadrature_points(7)), ``c_qp`` [ncell, m^3] optional.  ``bc``: the type of each
    boundary side 2*dir + side, "dirichlet" (default), "neumann" (g_qp then holds the total flux j) or
    "outflow" (Sec. 2, eq. modelproblem).  ``vertices`` [(n0+1)(n1+1)(n2+1), 3] (x fastest): multilinear cells
    (Problem C of Sec. 5.1)."""

    def __init__(self, n, k, D=1.0, b=(1.0, 0.5, 0.25), c=1.0, sigma=None, lo=(0.0, 0.0, 0.0),
                 hi=(1.0, 1.0, 1.0), f_qp=None, g_qp=None, stream=None, periodic=(0, 0, 0), m=None,
                 velocity="constant", b_qp=None, b_face=None, D_tensor=None, jacobian=None, D_qp=None,
                 D_face=None, c_qp=None, bc=None, vertices=None):
        mesh = dg_mesh()
        for r in range(3):
            mesh.lo[r], mesh.hi[r], mesh.n[r] = float(lo[r]), float(hi[r]), int(n[r])
        co = dg_coeffs()
        self.ncell = int(np.prod([int(v) for v in n]))
        Darr = np.asarray(D, dtype=np.float64)
        self._D = None
        if Darr.ndim == 0:
            co.D_cell = _dp()
            co.D_const = float(Darr)
        else:
            self._D = _f64(Darr).reshape(-1)
            if self._D.size != self.ncell:
                raise ValueError("D must have one value per cell")
            co.D_cell = self._D.ctypes.data_as(_dp)
            co.D_const = 0.0
        for r in range(3):
            co.b[r] = float(b[r])
        co.c = float(c)
        co.sigma = float(sigma) if sigma is not None else dg_penalty_sigma(int(k), 0)
        keep = []
        bcp = None
        if g_qp is not None:
            bdata = dg_bc()
            for s in range(6):
                if g_qp[s] is None:
                    bdata.g_qp[s] = _dp()
                else:
                    a = _f64(g_qp[s]).reshape(-1)
                    keep.append(a)
                    bdata.g_qp[s] = a.ctypes.data_as(_dp)
            bcp = ctypes.byref(bdata)
        fptr = None
        if f_qp is not None:
            fa = _f64(f_qp).reshape(-1)
            keep.append(fa)
            fptr = fa.ctypes.data_as(_dp)
        ext = dg_setup_ext()
        for r in range(3):
            ext.periodic[r] = int(periodic[r])
        ext.m = int(m) if m is not None else 0
        ext.velocity = _VELOCITY[velocity]
        if velocity == "points":
            bq = _f64(b_qp).reshape(-1)
            bf = _f64(b_face).reshape(-1)
            keep += [bq, bf]
            ext.b_qp = bq.ctypes.data_as(_dp)
            ext.b_face = bf.ctypes.data_as(_dp)
        if D_tensor is not None:
            dt = _f64(D_tensor).reshape(-1)
            if dt.size != 6 * self.ncell:
                raise ValueError("D_tensor must have 6 values per cell")
            keep.append(dt)
            ext.D_tensor = dt.ctypes.data_as(_dp)
        if jacobian is not None:
            jm = _f64(jacobian).reshape(-1)
            if jm.size != 9:
                raise ValueError("jacobian must be 3x3")
            keep.append(jm)
            ext.jacobian = jm.ctypes.data_as(_dp)
        if bc is not None:
            kinds = {"dirichlet": DG_BC_DIRICHLET, "neumann": DG_BC_NEUMANN, "outflow": DG_BC_OUTFLOW}
            for f in range(6):
                ext.bc_type[f] = kinds[bc[f]] if isinstance(bc[f], str) else int(bc[f])
        for name, arr in (("D_qp", D_qp), ("D_face", D_face), ("c_qp", c_qp), ("vertices", vertices)):
            if arr is not None:
                a = _f64(arr).reshape(-1)
                keep.append(a)
                setattr(ext, name, a.ctypes.data_as(_dp))
        h = ctypes.c_void_p()
        check(lib.dg_setup_ex(ctypes.byref(mesh), int(k), ctypes.byref(co), bcp, fptr, ctypes.byref(ext),
                              _stream_ptr(stream), ctypes.byref(h)))
        self.h = h
        self.k = int(k)
        self.m = int(m) if m else int(k) + 1
        self.periodic = tuple(int(v) for v in periodic)
        self.n = tuple(int(v) for v in n)
        nc, dpc, nd = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64()
        check(lib.dg_sizes(h, ctypes.byref(nc), ctypes.byref(dpc), ctypes.byref(nd)))
        self.dofs_per_cell = dpc.value
        self.ndof = nd.value

    def close(self):
        if getattr(self, "h", None):
            lib.dg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def quadrature_points(self, which: int = 0) -> np.ndarray:
        m = self.m
        if which == 0:
            shape = (self.ncell, m ** 3, 3)
        elif which == 7:
            shape = (self.ncell, 6, m ** 2, 3)
        else:
            d = (which - 1) // 2
            ta, tb = (1, 2) if d == 0 else ((0, 2) if d == 1 else (0, 1))
            shape = (self.n[ta] * self.n[tb], m ** 2, 3)
        out = np.empty(shape, dtype=np.float64)
        check(lib.dg_quadrature_points(self.h, int(which), out.ctypes.data_as(_dp)))
        return out

    def _vec_check(self, *ts):
        for t in ts:
            if not t.is_cuda or not t.is_contiguous() or t.numel() != self.ndof:
                raise ValueError("vectors must be contiguous CUDA tensors with ndof entries")

    def _precision(self, t, precision):
        p = _prec(t)
        if precision is None:
            return p
        if precision == DG_F64X and p != DG_F64:
            raise TypeError("DG_F64X takes float64 vectors")
        return int(precision)

    def apply_jacobian(self, z, y=None, stream=None, precision=None):
        """y = A z (dg_apply_jacobian); precision DG_F64X evaluates FP64 vectors in double-float."""
        import torch
        if y is None:
            y = torch.empty_like(z)
        self._vec_check(z, y)
        if z.dtype != y.dtype:
            raise TypeError("z and y must have the same dtype")
        check(lib.dg_apply_jacobian(self.h, ctypes.c_void_p(z.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                    self._precision(z, precision), _stream_ptr(stream)))
        return y

    def apply_residual(self, u, r=None, stream=None, precision=None):
        """r = A u - F (dg_apply_residual)."""
        import torch
        if r is None:
            r = torch.empty_like(u)
        self._vec_check(u, r)
        if u.dtype != r.dtype:
            raise TypeError("u and r must have the same dtype")
        check(lib.dg_apply_residual(self.h, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(r.data_ptr()),
                                    self._precision(u, precision), _stream_ptr(stream)))
        return r

    def apply_stage(self, stage, x, y, residual=False, stream=None, precision=None):
        """One kernel of an apply (dg_apply_stage): stage 0 cell kernel from x, stage 1 face kernel into y."""
        self._vec_check(x, y)
        check(lib.dg_apply_stage(self.h, int(stage), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                 self._precision(x, precision), int(bool(residual)), _stream_ptr(stream)))
        return y

    def precond_setup(self, kind=DG_BJ_DENSE, stream=None):
        """Block-Jacobi set-up (dg_precond_setup): DG_BJ_DENSE (default) assembles and inverts the dense per-cell
        blocks and builds the fast-diagonalisation tables; DG_BJ_FAST_DIAG builds only the latter."""
        check(lib.dg_precond_setup(self.h, int(kind), _stream_ptr(stream)))

    def precond_info(self):
        """(bits of what dg_precond_setup built: DG_PRECOND_HAS_DENSE, _HAS_FAST_DIAG, _FAST_DIAG_REAL; the
        number of cells with complex fast-diagonalisation tables)."""
        v, n = ctypes.c_int32(), ctypes.c_int64()
        check(lib.dg_precond_info(self.h, ctypes.byref(v), ctypes.byref(n)))
        return v.value, n.value

    def precond_apply_rbgs(self, r, z=None, work=None, stream=None):
        """z = M^{-1} r with red-black block Gauss-Seidel (dg_precond_apply_rbgs); work: scratch like r."""
        import torch
        if z is None:
            z = torch.empty_like(r)
        if work is None:
            work = torch.empty_like(r)
        self._vec_check(r, z, work)
        check(lib.dg_precond_apply_rbgs(self.h, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(z.data_ptr()),
                                        ctypes.c_void_p(work.data_ptr()), _prec(r), _stream_ptr(stream)))
        return z

    def precond_apply(self, r, z=None, stream=None):
        """z = M^{-1} r with the block-Jacobi preconditioner (dg_precond_apply)."""
        import torch
        if z is None:
            z = torch.empty_like(r)
        self._vec_check(r, z)
        check(lib.dg_precond_apply(self.h, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(z.data_ptr()), _prec(r),
                                   _stream_ptr(stream)))
        return z

    def solve(self, x, b=None, mode=DG_SOLVE_FP64, preconditioner=DG_PRECOND_BLOCK_JACOBI, restart=30,
              outer_restart=20, max_iterations=0, rtol=1e-10, inner_rtol=1e-3, stream=None, raise_on_error=True,
              mlp=None, fallback_ratio=0.0, mlp_placement=0, inner_block_precision=0, outer_precision=0,
              inner_basis_precision=0):
        """Solve A x = b (b = F when None) in place on the FP64 tensor x (dg_solve); returns the stats dict.

        DG_SOLVE_MIXED: inner_block_precision picks the inner FP32 solve's block inverse (0 fast
        diagonalisation, 1 FP32 dense blocks, 2 scaled FP16 blocks); outer_precision picks the outer operator
        (0 double-float with an FP64-confirmed stop, 1 FP64); inner_basis_precision the storage of the inner
        Krylov basis (0 FP32, 1 scaled FP16)."""
        import torch
        if x.dtype != torch.float64:
            raise TypeError("x must be float64")
        self._vec_check(x)
        if b is not None:
            self._vec_check(b)
        o = dg_solve_opts(mode, preconditioner, restart, outer_restart, max_iterations, rtol, inner_rtol,
                          mlp.m.value if mlp is not None else None, int(mlp_placement), fallback_ratio,
                          int(inner_block_precision), int(outer_precision), int(inner_basis_precision))
        st = dg_solve_stats()
        rc = lib.dg_solve(self.h, ctypes.c_void_p(b.data_ptr()) if b is not None else None,
                          ctypes.c_void_p(x.data_ptr()), ctypes.byref(o), ctypes.byref(st), _stream_ptr(stream))
        if raise_on_error:
            check(rc)
        d = st.as_dict()
        d["rc"] = rc
        return d

    def project(self, u_qp, z=None, stream=None):
        """z = L2 projection of u given at the volume points [ncell, m^3] (dg_project, FP64 CUDA tensors)."""
        import torch
        if z is None:
            z = torch.empty(self.ndof, dtype=torch.float64, device=u_qp.device)
        self._vec_check(z)
        if not u_qp.is_cuda or u_qp.dtype != torch.float64 or not u_qp.is_contiguous() or \
                u_qp.numel() != self.ncell * self.m ** 3:
            raise ValueError("u_qp must be a contiguous float64 CUDA tensor with ncell * m^3 entries")
        check(lib.dg_project(self.h, ctypes.c_void_p(u_qp.data_ptr()), ctypes.c_void_p(z.data_ptr()),
                             _stream_ptr(stream)))
        return z

    def rk_stage(self, u, z0, y, cz, cu, cdt, stream=None, precision=DG_F64):
        """y = cz z0 + cu u - cdt M^{-1}(A u - F) (dg_rk_stage, FP64 CUDA tensors; y may alias u or z0)."""
        self._vec_check(u, z0, y)
        check(lib.dg_rk_stage(self.h, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(z0.data_ptr()),
                              ctypes.c_void_p(y.data_ptr()), float(cz), float(cu), float(cdt), int(precision),
                              _stream_ptr(stream)))
        return y

    def ssprk2(self, z, dt, nsteps=1, stream=None, precision=DG_F64):
        """nsteps Heun steps on the FP64 CUDA tensor z in place (dg_ssprk2); precision DG_F64 or DG_F64X."""
        self._vec_check(z)
        check(lib.dg_ssprk2(self.h, ctypes.c_void_p(z.data_ptr()), float(dt), int(nsteps), int(precision),
                            _stream_ptr(stream)))
        return z

    def rhs(self, dtype=None, stream=None):
        """F = l_h(phi_i) (dg_rhs)."""
        import torch
        dtype = dtype or torch.float64
        F = torch.empty(self.ndof, dtype=dtype, device="cuda")
        check(lib.dg_rhs(self.h, ctypes.c_void_p(F.data_ptr()), _prec(F), _stream_ptr(stream)))
        return F


class Matrix:
    """The operator's assembled block-sparse matrix (dg_assemble), its product (dg_spmv) and export."""

    def __init__(self, op, stream=None):
        m = ctypes.c_void_p()
        check(lib.dg_assemble(op.h, _stream_ptr(stream), ctypes.byref(m)))
        self.m = m
        nr, nz, nb, secs = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_double()
        check(lib.dg_matrix_info(m, ctypes.byref(nr), ctypes.byref(nz), ctypes.byref(nb), ctypes.byref(secs)))
        self.nrows, self.nnzb, self.block, self.assemble_seconds = nr.value, nz.value, nb.value, secs.value

    def spmv(self, x, y=None, stream=None):
        import torch
        if y is None:
            y = torch.empty_like(x)
        if x.dtype != torch.float64 or y.dtype != torch.float64 or not x.is_cuda:
            raise TypeError("dg_spmv takes FP64 CUDA vectors")
        check(lib.dg_spmv(self.m, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), _stream_ptr(stream)))
        return y

    def export(self):
        """(rowptr, colidx, vals[nnzb, nb, nb] with vals[b, i, j] = entry (i, j) of block b)."""
        rp = np.empty(self.nrows + 1, dtype=np.int32)
        ci = np.empty(self.nnzb, dtype=np.int32)
        v = np.empty((self.nnzb, self.block, self.block))
        check(lib.dg_matrix_export(self.m, rp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   ci.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), v.ctypes.data_as(_dp)))
        return rp, ci, np.ascontiguousarray(v.transpose(0, 2, 1))  # stored column-major

    def dense(self):
        rp, ci, v = self.export()
        nb = self.block
        A = np.zeros((self.nrows * nb, self.nrows * nb))
        for t in range(self.nrows):
            for b in range(rp[t], rp[t + 1]):
                s = ci[b]
                A[t * nb:(t + 1) * nb, s * nb:(s + 1) * nb] = v[b]
        return A

    def close(self):
        if getattr(self, "m", None):
            lib.dg_matrix_destroy(self.m)
            self.m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MLP:
    """Learned per-element preconditioner network (dg_mlp_*)."""

    def __init__(self, k=None, seed=0, path=None):
        m = ctypes.c_void_p()
        if path is not None:
            check(lib.dg_mlp_load(str(path).encode(), ctypes.byref(m)))
        else:
            check(lib.dg_mlp_create(int(k), int(seed), ctypes.byref(m)))
        self.m = m
        k_, kin, kinp, outp = (ctypes.c_int32() for _ in range(4))
        npar = ctypes.c_int64()
        check(lib.dg_mlp_dims(m, ctypes.byref(k_), ctypes.byref(kin), ctypes.byref(kinp), ctypes.byref(outp),
                              ctypes.byref(npar)))
        self.k, self.kin, self.kinp, self.outp, self.nparam = k_.value, kin.value, kinp.value, outp.value, npar.value
        self.nb = (self.k + 1) ** 3
        offs = (ctypes.c_int64 * 6)()
        check(lib.dg_mlp_param_offsets(m, offs))
        self.offsets = list(offs)

    def close(self):
        if getattr(self, "m", None):
            lib.dg_mlp_destroy(self.m)
            self.m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        out = np.empty(self.nparam, dtype=np.float32)
        ts = ctypes.c_float()
        check(lib.dg_mlp_params(self.m, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), 0, ctypes.byref(ts)))
        return out, ts.value

    def set_params(self, p, t_scale=None):
        p = np.ascontiguousarray(p, dtype=np.float32)
        ts = ctypes.c_float(t_scale) if t_scale is not None else None
        check(lib.dg_mlp_params(self.m, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), 1,
                                ctypes.byref(ts) if ts is not None else None))

    def grad(self):
        out = np.empty(self.nparam, dtype=np.float32)
        check(lib.dg_mlp_params(self.m, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), 2, None))
        return out

    def set_target_scale(self, t):
        check(lib.dg_mlp_set_target_scale(self.m, float(t)))

    def features(self, op, r, cells=None, stream=None):
        import torch
        rows = op.ncell if cells is None else cells.numel()
        X = torch.empty((rows, self.kinp), dtype=torch.bfloat16, device=r.device)
        sc = torch.empty(rows, dtype=torch.float32, device=r.device)
        cp = ctypes.c_void_p(cells.data_ptr()) if cells is not None else None
        check(lib.dg_mlp_features(self.m, op.h, ctypes.c_void_p(r.data_ptr()), _prec(r), cp, rows,
                                  ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(sc.data_ptr()), _stream_ptr(stream)))
        return X, sc

    def pairs(self, op, x, xstar, cells, rows, X, E, subtract_block_jacobi=False, stream=None):
        """Training pairs from a solver state (dg_mlp_pairs): cells and rows are int32 device tensors; X (BF16
        [*, kin_padded]) and E (FP32 [*, (k+1)^3]) are written at the given rows."""
        check(lib.dg_mlp_pairs(self.m, op.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(xstar.data_ptr()),
                               ctypes.c_void_p(cells.data_ptr()), ctypes.c_void_p(rows.data_ptr()), cells.numel(),
                               int(bool(subtract_block_jacobi)), ctypes.c_void_p(X.data_ptr()),
                               ctypes.c_void_p(E.data_ptr()), _stream_ptr(stream)))

    def normalize_targets(self, E, stream=None):
        """E /= RMS(E) in place; the RMS becomes the network's target scale and is returned."""
        t = ctypes.c_float()
        check(lib.dg_mlp_normalize_targets(self.m, ctypes.c_void_p(E.data_ptr()), E.shape[0], ctypes.byref(t),
                                           _stream_ptr(stream)))
        return t.value

    def forward(self, X, stream=None):
        import torch
        Y = torch.empty((X.shape[0], self.outp), dtype=torch.float32, device=X.device)
        check(lib.dg_mlp_forward(self.m, ctypes.c_void_p(X.data_ptr()), X.shape[0], ctypes.c_void_p(Y.data_ptr()),
                                 _stream_ptr(stream)))
        return Y

    def loss_grad(self, X, T, stream=None):
        loss = ctypes.c_double()
        check(lib.dg_mlp_loss_grad(self.m, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(T.data_ptr()), X.shape[0],
                                   ctypes.byref(loss), _stream_ptr(stream)))
        return loss.value

    def train(self, X, T, epochs=10, batch=256, lr=1e-3, stream=None):
        o = dg_mlp_train_opts(int(epochs), int(batch), float(lr))
        st = dg_mlp_train_stats()
        check(lib.dg_mlp_train(self.m, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(T.data_ptr()), X.shape[0],
                               ctypes.byref(o), ctypes.byref(st), _stream_ptr(stream)))
        return {"first_epoch_loss": st.first_epoch_loss, "last_epoch_loss": st.last_epoch_loss, "steps": st.steps}

    def apply(self, op, r, z=None, stream=None):
        import torch
        if z is None:
            z = torch.empty_like(r)
        check(lib.dg_mlp_apply(self.m, op.h, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(z.data_ptr()), _prec(r),
                               _stream_ptr(stream)))
        return z

    def apply_add(self, op, r, z, stream=None):
        check(lib.dg_mlp_apply_add(self.m, op.h, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(z.data_ptr()),
                                   _prec(r), _stream_ptr(stream)))
        return z

    def save(self, path):
        check(lib.dg_mlp_save(self.m, str(path).encode()))


class Batch:
    """Many Operators applied in one graph launch (dg_batch_create / dg_batch_apply)."""

    def __init__(self, ops, stream=None):
        self.ops = list(ops)
        arr = (ctypes.c_void_p * len(self.ops))(*[o.h.value for o in self.ops])
        b = ctypes.c_void_p()
        check(lib.dg_batch_create(arr, len(self.ops), _stream_ptr(stream), ctypes.byref(b)))
        self.b = b

    def apply(self, xs, ys, residual=False, stream=None):
        n = len(self.ops)
        for op, x, y in zip(self.ops, xs, ys):
            op._vec_check(x, y)
        ins = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
        outs = (ctypes.c_void_p * n)(*[y.data_ptr() for y in ys])
        check(lib.dg_batch_apply(self.b, ins, outs, int(bool(residual)), _stream_ptr(stream)))
        return ys

    def tuning(self, k):
        """Autotuner result for degree k: chosen cells per CTA and lines per thread, and the time (ms) of every
        candidate layout (see dg_batch_tuning)."""
        cpb, lpt = ctypes.c_int32(), ctypes.c_int32()
        ms = (ctypes.c_float * DG_BATCH_CANDIDATES)()
        check(lib.dg_batch_tuning(self.b, int(k), ctypes.byref(cpb), ctypes.byref(lpt), ms))
        return {"cells_per_cta": cpb.value, "lines_per_thread": lpt.value, "ms_candidates": list(ms)}

    def close(self):
        if getattr(self, "b", None):
            lib.dg_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def operator_for(w, stream=None, sigma=None):
    """Build an Operator for an inputs.Workload, with f sampled at the library's own quadrature points."""
    import numpy as np
    from . import inputs
    m = getattr(w, "m", None) or w.k + 1
    ext = dict(periodic=getattr(w, "periodic", (0, 0, 0)), m=m, velocity=getattr(w, "velocity", "constant"))
    if w.f_kind == "zero":
        f = None
    elif w.f_kind == "one":
        f = np.ones(w.ncell * m ** 3)
    else:
        probe = Operator(w.n, w.k, w.D, b=w.b, c=w.c, sigma=sigma, lo=w.lo, hi=w.hi, stream=stream, **ext)
        f = inputs.f_at(w, probe.quadrature_points(0))
        probe.close()
    return Operator(w.n, w.k, w.D, b=w.b, c=w.c, sigma=sigma, lo=w.lo, hi=w.hi, f_qp=f, stream=stream, **ext)
