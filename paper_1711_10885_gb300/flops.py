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


def eo_fwd_flops(N):
    """Modal -> points on one line in even-odd form (mul + fma chains, then the +/- recombination)."""
    H, C = _halves(N)
    return C * (2 * C - 1) + H * (2 * H - 1) + 2 * H


def eo_bwd_flops(N):
    H, C = _halves(N)
    return 2 * H + C * (2 * C - 1) + H * (2 * H - 1)


def eo_anti_flops(N):
    """Centro-antisymmetric N x N point operator from the split parts of its input."""
    H, C = _halves(N)
    return C * (2 * H - 1) + H * (2 * C - 1) + 2 * H


def deriv_line_flops(N, first):
    H, C = _halves(N)
    split = 2 * H
    flux = 3 * N  # sa * grad + sb * u
    acc = 3 * N if first else N  # reaction (mul + fma) on the first pass, else add
    traces = 4 * N + 4
    return split + eo_anti_flops(N) + flux + split + eo_anti_flops(N) + acc + traces


def cell_kernel_flops(N: int) -> float:
    """Executed FP operations of dg_cell_kernel for one cell (n = m = N)."""
    NN = N * N
    fwd = 3 * NN * eo_fwd_flops(N)
    deriv = NN * (deriv_line_flops(N, True) + 2 * deriv_line_flops(N, False))
    scalars = NN * (1 + 3 * 3 + 1)  # wperp; sa (2) and sb (1) per pass; sc once
    return fwd + deriv + scalars


def face_kernel_flops(N: int, n=(1, 1, 1), residual: bool = True) -> float:
    """Executed FP operations of dg_face_kernel, averaged per cell for an n[0] x n[1] x n[2] mesh."""
    NN = N * N
    per_point = 11  # face weights: jump, average (mul+fma), upwind, H (sub+fma), V, W (2 mul), sign
    lift = 3 * NN * (1 + 2 * (per_point + 4 * N))  # wf, then per side the weights and 2 fma per point
    back = 3 * NN * eo_bwd_flops(N)
    return NN + lift + back + (N ** 3 if residual else 0)


def apply_flops_per_dof(k: int, n=(1, 1, 1), residual: bool = True) -> float:
    N = k + 1
    return (cell_kernel_flops(N) + face_kernel_flops(N, n, residual)) / N ** 3


def bytes_per_cell(N: int, elt: int = 8, residual: bool = True) -> dict:
    """Algorithmic DRAM bytes per cell of each kernel: its compulsory reads and writes."""
    n3, nn = N ** 3, N * N
    cell = elt * (n3 + 1 + n3 + 12 * nn)  # read z, D; write V and 6x2 traces
    face = elt * (n3 + 2 * 12 * nn + 18 + n3 + (n3 if residual else 0))  # V, own+nbr traces, fc, y, F
    return {"cell": cell, "face": face}
