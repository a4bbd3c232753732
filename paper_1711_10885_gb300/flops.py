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


def _mv(N):
    return N * (2 * N - 1)  # one mul and N-1 fma per output


def cell_kernel_flops(N: int) -> float:
    """Executed FP operations of dg_cell_kernel for one cell (n = m = N)."""
    NN = N * N
    fwd = 3 * NN * _mv(N)
    per_dir_line = _mv(N) + 3 * N + 2 * N * N + 8 * N + 3  # Dt u, flux, Dt^T acc, 4 traces, scalars
    deriv = 3 * NN * per_dir_line + NN * (2 * N + 1)  # + reaction init on the x pass
    return fwd + deriv + NN  # wperp


def face_kernel_flops(N: int, n=(1, 1, 1), residual: bool = True) -> float:
    """Executed FP operations of dg_face_kernel, averaged per cell for an n[0] x n[1] x n[2] mesh."""
    NN = N * N
    ncell = n[0] * n[1] * n[2]
    nbound = 2 * (n[1] * n[2] + n[0] * n[2] + n[0] * n[1])  # boundary face-sides
    face_sides = 6 * ncell
    interior_pt = 11  # jump, avg (mul+fma), upwind, H (sub+fma), V, W (2 mul), sign
    boundary_pt = 10
    pointwise = NN * (interior_pt * (face_sides - nbound) + boundary_pt * nbound) / ncell
    lift = 3 * NN * (2 + 2 * 4 * N)  # wf, and 2 fma per point per side
    back = 3 * NN * _mv(N)
    return pointwise + lift + back + (N ** 3 if residual else 0)


def apply_flops_per_dof(k: int, n=(1, 1, 1), residual: bool = True) -> float:
    N = k + 1
    return (cell_kernel_flops(N) + face_kernel_flops(N, n, residual)) / N ** 3


def bytes_per_cell(N: int, elt: int = 8, residual: bool = True) -> dict:
    """Algorithmic DRAM bytes per cell of each kernel: its compulsory reads and writes."""
    n3, nn = N ** 3, N * N
    cell = elt * (n3 + 1 + n3 + 12 * nn)  # read z, D; write V and 6x2 traces
    face = elt * (n3 + 2 * 12 * nn + 18 + n3 + (n3 if residual else 0))  # V, own+nbr traces, fc, y, F
    return {"cell": cell, "face": face}
