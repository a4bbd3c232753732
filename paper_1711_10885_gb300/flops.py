"""Operation counts of the operator kernels and of the paper's cost model.

``cell_kernel_flops`` / ``face_kernel_flops`` count the floating point
operations the two CUDA kernels execute per cell (FMA = 2, MUL/ADD = 1), read
off the kernel code line by line; they are cross-checked against the hardware
instruction counters of a profiled launch.  ``paper_flopdof`` is the paper's
lower bound FLOPDOF_vol + FLOPDOF_face (Sec. 3.6) for n = m = p+1.
"""

from __future__ import annotations


def paper_flopdof(p: int, d: int = 3) -> float:
    """FLOPDOF_vol(d,p) + FLOPDOF_face(d,p) of Sec. 3.6 (constant full tensor D, affine geometry)."""
    vol = 4 * (d + 1) * d * (p + 1) + 2 * d * d + 5 * d + 3
    face = 8 * (d + 1) * d * d + d * (2 * d * d + 8 * d + 18) / (p + 1)
    return vol + face


def _halves(N):
    return N // 2, (N + 1) // 2


def eo_fwd_flops(N, M=None):
    """Modal (N) -> points (M) on one line in even-odd form (mul + fma chains, then the +/- recombination)."""
    M = M or N
    HN, CN = _halves(N)
    HM, CM = _halves(M)
    return CM * (2 * CN - 1) + HM * (2 * HN - 1) + 2 * HM


def eo_bwd_flops(N, M=None):
    """Points (M) -> modal (N): split of the line, then the two half-size products."""
    M = M or N
    HN, CN = _halves(N)
    HM, CM = _halves(M)
    return 2 * HM + CN * (2 * CM - 1) + HN * (2 * HM - 1)


def eo_anti_flops(N):
    """Centro-antisymmetric N x N point operator from the split parts of its input."""
    H, C = _halves(N)
    return C * (2 * H - 1) + H * (2 * C - 1) + 2 * H


def deriv_line_flops(N, first):
    """One derivative pass on a line of N points (the point count, M in the kernels)."""
    H, C = _halves(N)
    split = 2 * H
    flux = 3 * N  # sa * grad + sb * u (or the point-wise b * u)
    acc = 3 * N if first else N  # reaction (mul + fma) on the first pass, else add
    traces = 4 * N + 4
    return split + eo_anti_flops(N) + flux + split + eo_anti_flops(N) + acc + traces


def cell_kernel_flops(N: int, M: int | None = None, vb: bool = False) -> float:
    """Executed FP operations of dg_cell_kernel for one cell: N = k+1 modes, M Gauss points per direction
    (default N); vb: the velocity field kernels (the constant convection weight is not formed)."""
    M = M or N
    MM = M * M
    fwd = (N * N + M * N + M * M) * eo_fwd_flops(N, M)  # x, y and z modal passes
    deriv = MM * (deriv_line_flops(M, True) + 2 * deriv_line_flops(M, False))
    scalars = MM * (1 + 3 * (2 if vb else 3) + 1)  # wperp; sa (2) [and sb (1)] per pass; sc once
    return fwd + deriv + scalars


def face_kernel_flops(N: int, n=(1, 1, 1), residual: bool = True, M: int | None = None,
                      stage: bool = False) -> float:
    """Executed FP operations of dg_face_kernel per cell; stage: the Runge-Kutta epilogue (mode 3)."""
    M = M or N
    MM = M * M
    per_point = 11  # face weights: jump, average (mul+fma), upwind, H (sub+fma), V, W (2 mul), sign
    lift = 3 * MM * (1 + 2 * (per_point + 4 * M))  # wf, then per side the weights and 2 fma per point
    back = (M * M + M * N + N * N) * eo_bwd_flops(N, M)
    epilogue = 6 * N ** 3 if stage else (N ** 3 if residual else 0)
    return MM + lift + back + epilogue


def cell_kernel_flops_td(N: int) -> float:
    """Executed FP operations of dg_cell_kernel_td (tensor diffusion / affine cells, M = N) per cell."""
    H, C = _halves(N)
    NN = N * N
    fwd = 3 * NN * eo_fwd_flops(N)
    traces_u = 2 * C + 2 * H + 2
    deriv = 3 * NN * (2 * H + eo_anti_flops(N) + traces_u)
    pointwise = NN * (1 + N * (3 * 7 + 3))  # wab; per point 3 rows (3 fma + beta mul) and the reaction
    traces_x = 2 * C + 2 * H + 2 + 8
    transposed = 3 * NN * (2 * H + traces_x + 1 + N + eo_anti_flops(N) + N)
    return fwd + deriv + pointwise + transposed


def face_kernel_flops_td(N: int, residual: bool = True) -> float:
    """Executed FP operations of the tensor-diffusion face kernel per cell: the face weights with the two
    tangential weights, their transposed tangential derivatives (2 N fma per point and side), the lift and
    the backward contractions."""
    NN = N * N
    per_point = 11 + 4 + 4 * N  # weights, tangential weights, tangential derivative sums
    lift = 3 * NN * (1 + 2 * (per_point + 4 * N))
    back = 3 * NN * eo_bwd_flops(N)
    return NN + lift + back + (N ** 3 if residual else 0)


def cell_kernel_flops_pw(N: int, M: int | None = None) -> float:
    """Executed FP operations per cell of dg_cell_kernel_td with coefficients at the quadrature points (Problem B):
    modal passes N -> M, three derivative passes with value traces, the conormal traces from the three
    gradient components extrapolated to both faces of each line, the point-wise flux (3 rows of 3 fma and a
    beta mul, plus the reaction mul) and the three weighted transposed passes."""
    M = M or N
    H, C = _halves(M)
    MM = M * M
    fwd = (N * N + M * N + MM) * eo_fwd_flops(N, M)
    deriv = 3 * MM * (2 * H + eo_anti_flops(M) + 2 * C + 2 * H + 2)
    conormal = 3 * MM * 3 * (2 * H + 2 * C + 2 * H + 2 + 4)
    pointwise = MM * M * 22
    transposed = 3 * MM * (2 * H + 1 + M + eo_anti_flops(M) + M)
    return fwd + deriv + conormal + pointwise + transposed


def face_kernel_flops_pw(N: int, M: int | None = None, residual: bool = True) -> float:
    """Executed FP operations per cell of the point-wise tensor face kernel (the tensor-diffusion face kernel on
    M-point faces, contracted back to N modes)."""
    M = M or N
    MM = M * M
    per_point = 11 + 4 + 4 * M
    lift = 3 * MM * (1 + 2 * (per_point + 4 * M))
    back = (MM + M * N + N * N) * eo_bwd_flops(N, M)
    return MM + lift + back + (N ** 3 if residual else 0)


def bytes_per_cell_pw(N: int, M: int, elt: int = 8, residual: bool = True) -> dict:
    """Algorithmic DRAM bytes per cell of the point-wise coefficient kernels.  Cell kernel: read z, the ten
    point fields (K, beta, c w) at M^3 points and the 3 conormal rows at 6 M^2 face points; write V and the
    6 x 2 traces.  Face kernel: read V, the traces (once, as for the other kernels), the 6 face coefficients
    at 6 M^2 points, the normal velocity (one value per interior face point, 3 M^2), write y (and read F)."""
    n3, m3, mm = N ** 3, M ** 3, M * M
    cell = elt * (n3 + 10 * m3 + 18 * mm + m3 + 12 * mm)
    face = elt * (m3 + 12 * mm + 36 * mm + 3 * mm + n3 + (n3 if residual else 0))
    return {"cell": cell, "face": face}


def apply_flops_per_dof(k: int, n=(1, 1, 1), residual: bool = True) -> float:
    N = k + 1
    return (cell_kernel_flops(N) + face_kernel_flops(N, n, residual)) / N ** 3


def bytes_per_cell(N: int, elt: int = 8, residual: bool = True, M: int | None = None, vb: bool = False,
                   stage: bool = False) -> dict:
    """Algorithmic DRAM bytes per cell of each kernel: its compulsory reads and writes.  The face kernel
    reads every cell's traces twice (as its own and as a neighbour's); the second read is an L2 hit, so
    the traces count once.  vb adds the velocity tables (3 M^3 volume values; 3 M^2 face values, one per
    interior face point); stage the Runge-Kutta epilogue's reads of u and z0 next to F."""
    M = M or N
    n3, m3, mm = N ** 3, M ** 3, M * M
    cell = elt * (n3 + 1 + m3 + 12 * mm + (3 * m3 if vb else 0))  # read z, D (, b); write V and 6x2 traces
    face = elt * (m3 + 12 * mm + 18 + n3 + (n3 if residual or stage else 0) + (2 * n3 if stage else 0)
                  + (3 * mm if vb else 0))  # V, traces, fc, y, F (, u, z0, b . nu)
    return {"cell": cell, "face": face}
