"""GPU tests of the block-Jacobi preconditioner and the FGMRES solvers against the FP64 oracle.

The diagonal blocks are pinned to the oracle (A e_j restricted to the cell, with e_j supported on
that cell); solutions are pinned to a dense LU solve of the oracle-assembled matrix.
"""

import numpy as np
import pytest

import oracle
from paper_1711_10885_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_10885_gb300 import dg as _dg
    return _dg


def oracle_problem(w):
    return oracle.Problem(w.n, w.k, w.D, b=w.b, c=w.c, lo=w.lo, hi=w.hi)


def oracle_matrix(pr):
    N = pr.ndof
    A = np.empty((N, N))
    e = np.zeros(N)
    for j in range(N):
        e[j] = 1.0
        A[:, j] = oracle.apply(pr, e)
        e[j] = 0.0
    return A


@pytest.mark.parametrize("n,k", [((3, 2, 2), 2), ((2, 2, 3), 3), ((1, 1, 2), 4), ((2, 1, 1), 1)])
def test_block_jacobi_matches_oracle_blocks(dg, n, k):
    w = inputs.small_case(n=n, k=k, seed=31 + k, b=(0.7, -0.4, 0.2))
    pr = oracle_problem(w)
    A = oracle_matrix(pr)
    nb = w.nb
    op = dg.operator_for(w)
    op.precond_setup()
    rng = np.random.default_rng(3)
    r = rng.uniform(-1, 1, w.ndof)
    z64 = op.precond_apply(torch.tensor(r, device="cuda")).cpu().numpy()
    z32 = op.precond_apply(torch.tensor(r, device="cuda").float()).cpu().numpy()
    z_ref = np.empty_like(r)
    for c in range(w.ncell):
        sl = slice(c * nb, (c + 1) * nb)
        z_ref[sl] = np.linalg.solve(A[sl, sl], r[sl])
    assert np.max(np.abs(z64 - z_ref)) <= 1e-10 * np.max(np.abs(z_ref))
    # FP32: the exact block inverse by fast diagonalisation (complex FP32 1D contractions)
    assert np.max(np.abs(z32 - z_ref)) <= 1e-4 * np.max(np.abs(z_ref))
    op.close()


@pytest.mark.parametrize("mode", ["fp64", "fp64_bj", "mixed_bj", "mixed_bj32", "mixed_bj16", "mixed",
                                  "mixed_bj_fp64outer"])
def test_fgmres_solution_matches_dense_solve(dg, mode):
    w = inputs.small_case(n=(3, 2, 2), k=2, seed=8, b=(1.0, 0.5, 0.25), f_kind="sines")
    w.f_params = inputs.sine_modes(9)
    pr = oracle_problem(w)
    A = oracle_matrix(pr)
    F = oracle.rhs(pr, inputs.f_at(w, oracle.volume_points(pr)), None)
    x_ref = np.linalg.solve(A, F)
    op = dg.operator_for(w)
    # the block inverse of the inner FP32 solve: mixed_bj by fast diagonalisation (the default), mixed_bj32 the FP32
    # dense blocks, mixed_bj16 the scaled FP16 dense blocks
    pc = dg.DG_PRECOND_BLOCK_JACOBI if "bj" in mode else dg.DG_PRECOND_NONE
    if pc:
        op.precond_setup()
    x = torch.zeros(w.ndof, dtype=torch.float64, device="cuda")
    m = dg.DG_SOLVE_MIXED if mode.startswith("mixed") else dg.DG_SOLVE_FP64
    # mixed modes: the outer operator in double-float with an FP64-confirmed stop (default), or FP64 throughout
    st = op.solve(x, mode=m, preconditioner=pc, rtol=1e-12, restart=20, outer_restart=8, inner_rtol=1e-2,
                  inner_block_precision={"mixed_bj32": 1, "mixed_bj16": 2}.get(mode, 0),
                  outer_precision=1 if mode.endswith("fp64outer") else 0)
    assert st["rc"] == 0 and st["rel_residual"] <= 1e-12
    xs = x.cpu().numpy()
    # field error bound: ||x - x*|| <= cond(A) * rtol * ||x*||; checked directly against the LU solution
    assert np.max(np.abs(xs - x_ref)) <= 1e-9 * np.max(np.abs(x_ref)), st
    # the true residual with the oracle operator
    assert np.linalg.norm(A @ xs - F) <= 1e-11 * np.linalg.norm(F)
    if m == dg.DG_SOLVE_MIXED:
        assert st["applies_f32"] > st["applies_f64"]
    op.close()


@pytest.mark.parametrize("n,k,basis,mixed_cells", [((3, 2, 2), 3, 1, False), ((3, 2, 2), 2, 1, False),
                                                   ((4, 2, 2), 2, 1, False), ((3, 2, 2), 3, 1, True)])
def test_fp16_inner_basis_solution_matches_dense_solve(dg, n, k, basis, mixed_cells):
    """The inner Krylov basis stored in scaled FP16: 768 unknowns (k = 3, the block inverse reads the FP16 rows
    itself), 432 unknowns (k = 2: odd n, the rows are converted to FP32 first); with 324 unknowns (not a multiple
    of 8) the option falls back to the FP32 basis.  mixed_cells: D alternating 100 / 0.01 with strong convection,
    so the block inverse has real and complex cells (the complex ones converted from FP16 first).  Same bounds as
    the FP32-basis solves."""
    w = inputs.small_case(n=n, k=k, seed=18, b=(40.0, -30.0, 20.0) if mixed_cells else (1.0, 0.5, 0.25),
                          f_kind="sines")
    if mixed_cells:
        w.D = np.where(np.arange(w.ncell) % 2 == 0, 100.0, 0.01)
    w.f_params = inputs.sine_modes(10)
    pr = oracle_problem(w)
    A = oracle_matrix(pr)
    F = oracle.rhs(pr, inputs.f_at(w, oracle.volume_points(pr)), None)
    x_ref = np.linalg.solve(A, F)
    op = dg.operator_for(w)
    op.precond_setup()
    if mixed_cells:
        assert 0 < op.precond_info()[1] < w.ncell
    for outer in (0, 1):
        x = torch.zeros(w.ndof, dtype=torch.float64, device="cuda")
        st = op.solve(x, mode=dg.DG_SOLVE_MIXED, rtol=1e-12, restart=20, outer_restart=8, inner_rtol=1e-2,
                      outer_precision=outer, inner_basis_precision=basis)
        assert st["rc"] == 0 and st["rel_residual"] <= 1e-12
        xs = x.cpu().numpy()
        assert np.max(np.abs(xs - x_ref)) <= 1e-9 * np.max(np.abs(x_ref)), st
        assert np.linalg.norm(A @ xs - F) <= 1e-11 * np.linalg.norm(F)
    op.close()


@pytest.mark.parametrize("basis", [0, 1])
def test_mixed_and_fp64_solutions_agree(dg, basis):
    w = inputs.small_case(n=(4, 4, 4), k=3, seed=12, f_kind="sines")
    w.f_params = inputs.sine_modes(13)
    op = dg.operator_for(w)
    op.precond_setup()
    x64 = torch.zeros(w.ndof, dtype=torch.float64, device="cuda")
    xmx = torch.zeros_like(x64)
    s1 = op.solve(x64, mode=dg.DG_SOLVE_FP64, rtol=1e-13)
    s2 = op.solve(xmx, mode=dg.DG_SOLVE_MIXED, rtol=1e-13, inner_rtol=1e-3, inner_basis_precision=basis)
    diff = (torch.max(torch.abs(x64 - xmx)) / torch.max(torch.abs(x64))).item()
    assert diff <= 1e-10, (diff, s1, s2)
    op.close()


def test_solver_errors(dg):
    w = inputs.small_case(n=(2, 2, 2), k=2)
    op = dg.operator_for(w)
    x = torch.zeros(w.ndof, dtype=torch.float64, device="cuda")
    with pytest.raises(dg.DGError):  # block-Jacobi not set up
        op.solve(x, preconditioner=dg.DG_PRECOND_BLOCK_JACOBI)
    with pytest.raises(dg.DGError):  # restart too long
        op.solve(x, preconditioner=dg.DG_PRECOND_NONE, restart=100)
    with pytest.raises(dg.DGError):  # outer operator precision is 0 (double-float) or 1 (FP64)
        op.solve(x, mode=dg.DG_SOLVE_MIXED, preconditioner=dg.DG_PRECOND_NONE, outer_precision=2)
    with pytest.raises(dg.DGError):  # inner basis storage is 0 (FP32) or 1 (FP16)
        op.solve(x, mode=dg.DG_SOLVE_MIXED, preconditioner=dg.DG_PRECOND_NONE, inner_basis_precision=2)
    st = op.solve(x, preconditioner=dg.DG_PRECOND_NONE, max_iterations=2, rtol=1e-14, raise_on_error=False)
    assert st["rc"] == -4 and st["status"] == -4  # DG_ERR_NOT_CONVERGED
    op.close()


FDM_CASES = [
    ((3, 2, 2), 2, (0, 0, 0), None),
    ((2, 3, 2), 3, (1, 0, 0), None),
    ((4, 2, 2), 4, (0, 1, 1), ("dirichlet", "outflow", "neumann", "dirichlet", "neumann", "outflow")),
    ((2, 2, 3), 7, (0, 0, 0), ("neumann",) * 6),
    ((2, 2, 2), 6, (0, 0, 1), None),
    ((3, 2, 3), 5, (1, 0, 1), ("outflow", "dirichlet", "dirichlet", "neumann", "dirichlet", "dirichlet")),
    ((5, 3, 2), 1, (0, 1, 0), None),
]


@pytest.mark.parametrize("case", FDM_CASES, ids=lambda c: f"n{c[0]}k{c[1]}p{c[2]}{'bc' if c[3] else ''}")
def test_fast_diagonalisation_equals_dense_block_inverse(dg, case):
    """The FP32 block-Jacobi application (every diagonal block inverted through the eigen-decompositions of its
    three 1D cell operators) against the FP64 dense inverse blocks, on periodic axes, mixed boundary sides,
    negative velocity components and high degree."""
    n, k, per, bc = case
    w = inputs.small_case(n=n, k=k, seed=60 + k, b=(-0.8, 0.6, -0.3), c=0.5)
    op = dg.Operator(w.n, w.k, w.D, b=w.b, c=w.c, periodic=per, bc=bc)
    op.precond_setup()
    r = torch.tensor(np.random.default_rng(61 + k).uniform(-1, 1, w.ndof), device="cuda")
    z64 = op.precond_apply(r).cpu().numpy()
    z32 = op.precond_apply(r.float()).cpu().numpy()
    assert np.max(np.abs(z32 - z64)) <= 1e-4 * np.max(np.abs(z64))
    # the same inverse in complex FP64 when only the fast diagonalisation is set up
    op2 = dg.Operator(w.n, w.k, w.D, b=w.b, c=w.c, periodic=per, bc=bc)
    op2.precond_setup(dg.DG_BJ_FAST_DIAG)
    z64f = op2.precond_apply(r).cpu().numpy()
    assert np.max(np.abs(z64f - z64)) <= 1e-10 * np.max(np.abs(z64))
    op.close()
    op2.close()


@pytest.mark.parametrize("regime,k", [("diffusion", 5), ("diffusion", 7), ("diffusion", 2), ("convection", 5),
                                      ("convection", 3), ("mixed", 5), ("mixed", 3), ("mixed", 7)])
def test_fast_diagonalisation_real_and_complex_tables(dg, regime, k):
    """Diffusion-dominated cells have real 1D spectra: their tables are real (the real plane kernel at n <= 8 in
    FP32, one thread per line otherwise and in FP64).  Strong convection (|b| h / D of order 1000) gives complex
    pairs: complex tables.  "mixed" alternates D = 100 and D = 0.01 between cells, so both groups run, each through
    its list of cells.  Either way the application equals the dense FP64 block inverse."""
    conv = regime != "diffusion"
    w = inputs.small_case(n=(3, 2, 2), k=k, seed=90 + k, b=(40.0, -30.0, 20.0) if conv else (1.0, 0.5, 0.25), c=0.5)
    if regime == "mixed":
        D = np.where(np.arange(w.ncell) % 2 == 0, 100.0, 0.01)
    else:
        D = w.D * (0.02 if conv else 1.0)
    op = dg.Operator(w.n, w.k, D, b=w.b, c=w.c)
    op.precond_setup()
    info, ncx = op.precond_info()
    assert info & dg.DG_PRECOND_HAS_DENSE and info & dg.DG_PRECOND_HAS_FAST_DIAG
    assert bool(info & dg.DG_PRECOND_FAST_DIAG_REAL) == (not conv), info
    assert (ncx > 0) == conv and ncx <= w.ncell
    if regime == "mixed":
        assert 0 < ncx < w.ncell, ncx
    r = torch.tensor(np.random.default_rng(91 + k).uniform(-1, 1, w.ndof), device="cuda")
    z64 = op.precond_apply(r).cpu().numpy()
    z32 = op.precond_apply(r.float()).cpu().numpy()
    # FP32 rounding is amplified by the conditioning of the eigenvector matrices, which grows with the
    # non-normality of convection-dominated 1D operators: 1e-4 of the cell group's largest entry for real cells,
    # 1e-2 for complex ones (a flexible outer method absorbs it like any inexact preconditioner)
    nb = w.nb
    cells = np.arange(w.ncell)
    groups = [(cells % 2 == 0, 1e-4), (cells % 2 == 1, 1e-2)] if regime == "mixed" else \
        [(cells >= 0, 1e-2 if conv else 1e-4)]
    for sel, tol in groups:
        m = np.repeat(sel, nb)
        assert np.max(np.abs(z32[m] - z64[m])) <= tol * np.max(np.abs(z64[m])), (regime, tol)
    # FP32 vectors one element past a 16-byte boundary take the one-thread-per-line kernel: the same inverse up to
    # FP32 rounding order
    rb = torch.zeros(w.ndof + 1, dtype=torch.float32, device="cuda")
    zb = torch.zeros_like(rb)
    rb[1:] = r.float()
    op.precond_apply(rb[1:], zb[1:])
    zu = zb[1:].cpu().numpy()
    assert np.max(np.abs(zu - z32)) <= 1e-4 * np.max(np.abs(z32))
    op2 = dg.Operator(w.n, w.k, D, b=w.b, c=w.c)
    op2.precond_setup(dg.DG_BJ_FAST_DIAG)
    assert op2.precond_info() == (info & ~dg.DG_PRECOND_HAS_DENSE, ncx)
    z64f = op2.precond_apply(r).cpu().numpy()
    assert np.max(np.abs(z64f - z64)) <= (1e-9 if conv else 1e-10) * np.max(np.abs(z64))
    op.close()
    op2.close()


@pytest.mark.parametrize("k", [8, 10])
def test_fast_diagonalisation_inverts_the_one_cell_operator(dg, k):
    """Degrees whose dense blocks are not built ((k+1)^3 > 512): on a one-cell mesh the operator is its own
    diagonal block, so A M^{-1} r = r (FP64 fast diagonalisation; FP32 to its rounding)."""
    w = inputs.small_case(n=(1, 1, 1), k=k, seed=70 + k, b=(0.9, -0.4, 0.2), c=0.3)
    op = dg.Operator(w.n, w.k, w.D, b=w.b, c=w.c)
    op.precond_setup(dg.DG_BJ_FAST_DIAG)
    r = torch.tensor(np.random.default_rng(71 + k).uniform(-1, 1, w.ndof), device="cuda")
    z = op.precond_apply(r)
    assert torch.max(torch.abs(op.apply_jacobian(z) - r)).item() <= 1e-8
    z32 = op.precond_apply(r.float())
    assert torch.max(torch.abs(op.apply_jacobian(z32.double()) - r)).item() <= 1e-2
    op.close()


def test_solves_with_the_fast_diagonalisation_only(dg):
    w = inputs.small_case(n=(3, 2, 2), k=3, seed=8, b=(1.0, 0.5, 0.25), f_kind="sines")
    w.f_params = inputs.sine_modes(9)
    pr = oracle_problem(w)
    x_ref = np.linalg.solve(oracle_matrix(pr), oracle.rhs(pr, inputs.f_at(w, oracle.volume_points(pr)), None))
    op = dg.operator_for(w)
    op.precond_setup(dg.DG_BJ_FAST_DIAG)
    for mode in (dg.DG_SOLVE_FP64, dg.DG_SOLVE_MIXED):
        x = torch.zeros(w.ndof, dtype=torch.float64, device="cuda")
        st = op.solve(x, mode=mode, preconditioner=dg.DG_PRECOND_BLOCK_JACOBI, rtol=1e-12, restart=20,
                      outer_restart=8, inner_rtol=1e-2)
        assert st["rc"] == 0
        assert np.max(np.abs(x.cpu().numpy() - x_ref)) <= 1e-9 * np.max(np.abs(x_ref))
    op.close()


@pytest.mark.parametrize("case", ["odd_length", "unaligned_x", "restart_60"])
def test_fgmres_basis_passes_off_the_packed_path(dg, case):
    """The basis passes of FGMRES move 16-byte packs only when the vector length and every row start allow it.
    An odd number of DOFs (81) runs them one element per load in FP32 and FP64; a solution vector one element past
    a 16-byte boundary runs the update of x that way; a restart of 60 without a preconditioner takes up to 61 rows
    of per-thread partial sums (more than 48 KB of shared memory in FP64)."""
    n, k = ((3, 1, 1), 2) if case == "odd_length" else ((3, 2, 2), 2)
    w = inputs.small_case(n=n, k=k, seed=8, b=(1.0, 0.5, 0.25), f_kind="sines")
    w.f_params = inputs.sine_modes(9)
    pr = oracle_problem(w)
    A = oracle_matrix(pr)
    F = oracle.rhs(pr, inputs.f_at(w, oracle.volume_points(pr)), None)
    x_ref = np.linalg.solve(A, F)
    op = dg.operator_for(w)
    op.precond_setup()
    long = case == "restart_60"
    pc = dg.DG_PRECOND_NONE if long else dg.DG_PRECOND_BLOCK_JACOBI
    for mode in (dg.DG_SOLVE_FP64, dg.DG_SOLVE_MIXED):
        buf = torch.zeros(w.ndof + 1, dtype=torch.float64, device="cuda")
        x = buf[1:] if case == "unaligned_x" else buf[:w.ndof]
        st = op.solve(x, mode=mode, preconditioner=pc, rtol=1e-12, restart=60 if long else 20,
                      outer_restart=8, inner_rtol=1e-2)
        assert st["rc"] == 0
        if long and mode == dg.DG_SOLVE_FP64:
            assert st["iterations"] > 30  # the restart cycle grew past 30 rows
        assert np.max(np.abs(x.cpu().numpy() - x_ref)) <= 1e-9 * np.max(np.abs(x_ref)), st
    op.close()


def test_fp16_basis_with_restart_60_and_no_preconditioner(dg):
    """The FP16 basis passes at their largest size: an inner FGMRES(60) without a preconditioner takes up to 61
    FP16 rows (the dot pass's 123 rows of per-thread partial sums need more than 48 KB of shared memory) and the
    identity preconditioner copies the converted row; the solution matches a dense LU solve."""
    w = inputs.small_case(n=(4, 2, 2), k=2, seed=8, b=(1.0, 0.5, 0.25), f_kind="sines")
    w.f_params = inputs.sine_modes(9)
    pr = oracle_problem(w)
    A = oracle_matrix(pr)
    F = oracle.rhs(pr, inputs.f_at(w, oracle.volume_points(pr)), None)
    x_ref = np.linalg.solve(A, F)
    op = dg.operator_for(w)
    x = torch.zeros(w.ndof, dtype=torch.float64, device="cuda")
    st = op.solve(x, mode=dg.DG_SOLVE_MIXED, preconditioner=dg.DG_PRECOND_NONE, rtol=1e-12, restart=60,
                  outer_restart=8, inner_rtol=1e-9, inner_basis_precision=1)
    assert st["rc"] == 0 and st["inner_iterations"] >= 60  # inner cycles of the full 60 steps
    assert np.max(np.abs(x.cpu().numpy() - x_ref)) <= 1e-9 * np.max(np.abs(x_ref))
    op.close()


def test_non_finite_right_hand_side_is_reported(dg):
    """A NaN in b: both solvers stop at the first residual norm and return DG_ERR_NAN (-6) with the status set."""
    w = inputs.small_case(n=(2, 2, 2), k=2, seed=21)
    op = dg.operator_for(w)
    op.precond_setup()
    b = torch.ones(w.ndof, dtype=torch.float64, device="cuda")
    b[3] = float("nan")
    for mode, basis in ((dg.DG_SOLVE_FP64, 0), (dg.DG_SOLVE_MIXED, 0), (dg.DG_SOLVE_MIXED, 1)):
        x = torch.zeros(w.ndof, dtype=torch.float64, device="cuda")
        st = op.solve(x, b=b, mode=mode, preconditioner=dg.DG_PRECOND_BLOCK_JACOBI, raise_on_error=False,
                      inner_basis_precision=basis)
        assert st["rc"] == -6 and st["status"] == -6, (mode, basis, st)
    op.close()


def _rbgs_reference(pr, w, A, r):
    """z_red = A_TT^{-1} r on the red cells (ix + iy + iz even), z_black = A_TT^{-1} (r - A z_red) on the black
    ones, with the diagonal blocks of the oracle matrix."""
    nb = w.nb
    n = w.n
    z = np.zeros_like(r)
    cells = np.arange(w.ncell)
    color = (cells % n[0] + (cells // n[0]) % n[1] + cells // (n[0] * n[1])) % 2
    for c in cells[color == 0]:
        sl = slice(c * nb, (c + 1) * nb)
        z[sl] = np.linalg.solve(A[sl, sl], r[sl])
    t = r - A @ z
    for c in cells[color == 1]:
        sl = slice(c * nb, (c + 1) * nb)
        z[sl] = np.linalg.solve(A[sl, sl], t[sl])
    return z


@pytest.mark.parametrize("n,k,per", [((3, 2, 2), 2, (0, 0, 0)), ((2, 3, 2), 3, (0, 0, 0)), ((3, 2, 2), 3, (1, 0, 0)),
                                     ((4, 2, 3), 1, (0, 1, 1)), ((3, 2, 2), 5, (0, 0, 0)), ((3, 2, 2), 5, (1, 1, 0)),
                                     ((3, 3, 1), 5, (1, 1, 0)), ((3, 2, 2), 4, (1, 0, 0)), ((2, 3, 2), 4, (0, 0, 0))])
def test_red_black_gauss_seidel_matches_dense_reference(dg, n, k, per):
    """dg_precond_apply_rbgs in FP64 and FP32 against the sweep written out with the oracle matrix's blocks,
    including periodic axes of three cells (the two cells across the wrap share a colour) and even ones.  At
    k = 4 and 5 the FP32 sweep applies the operator on the red cells only and writes the black ones only (plane
    kernels with a cell list, the listed cells' own terms taken as zero)."""
    w = inputs.small_case(n=n, k=k, seed=40 + k, b=(0.9, -0.5, 0.3), c=0.7)
    pr = oracle.Problem(w.n, w.k, w.D, b=w.b, c=w.c, periodic=per)
    A = oracle_matrix(pr)
    op = dg.Operator(w.n, w.k, w.D, b=w.b, c=w.c, periodic=per)
    op.precond_setup(dg.DG_BJ_FAST_DIAG)
    r = np.random.default_rng(41 + k).uniform(-1, 1, w.ndof)
    z_ref = _rbgs_reference(pr, w, A, r)
    z64 = op.precond_apply_rbgs(torch.tensor(r, device="cuda")).cpu().numpy()
    z32 = op.precond_apply_rbgs(torch.tensor(r, device="cuda").float()).cpu().numpy()
    scale = np.max(np.abs(z_ref))
    assert np.max(np.abs(z64 - z_ref)) <= 1e-10 * scale
    assert np.max(np.abs(z32 - z_ref)) <= 1e-4 * scale
    op.close()


@pytest.mark.parametrize("mode,basis,k,per", [("fp64", 0, 3, 0), ("mixed", 0, 3, 0), ("mixed", 1, 3, 0),
                                              ("mixed", 1, 5, 0), ("mixed", 0, 5, 0), ("mixed", 1, 4, 0),
                                              ("mixed", 1, 5, 1)])
def test_red_black_gauss_seidel_solves(dg, mode, basis, k, per):
    """FGMRES with red-black block Gauss-Seidel reaches the dense LU solution, in fewer iterations than with
    block-Jacobi (plain FP64: inner iterations; mixed: with the FP32 and the FP16 inner basis).  k = 4, 5: the
    operator restricted to one colour, and on the two-cyclic mesh the Krylov step's A z_j formed as u_j + U z_j;
    per = 1: a periodic x axis of three cells (not two-cyclic), which keeps the whole operator application."""
    w = inputs.small_case(n=(4, 4, 3) if k == 3 else (3, 2, 2), k=k, seed=19, b=(1.0, 0.5, 0.25), f_kind="sines")
    w.f_params = inputs.sine_modes(11)
    w.periodic = (per, 0, 0)
    pr = oracle.Problem(w.n, w.k, w.D, b=w.b, c=w.c, lo=w.lo, hi=w.hi, periodic=w.periodic)
    A = oracle_matrix(pr)
    F = oracle.rhs(pr, inputs.f_at(w, oracle.volume_points(pr)), None)
    x_ref = np.linalg.solve(A, F)
    op = dg.operator_for(w)
    op.precond_setup(dg.DG_BJ_FAST_DIAG)
    m = dg.DG_SOLVE_FP64 if mode == "fp64" else dg.DG_SOLVE_MIXED
    its = {}
    for pc in (dg.DG_PRECOND_BLOCK_JACOBI, dg.DG_PRECOND_RB_GS):
        x = torch.zeros(w.ndof, dtype=torch.float64, device="cuda")
        st = op.solve(x, mode=m, preconditioner=pc, rtol=1e-12, restart=20, outer_restart=8, inner_rtol=1e-3,
                      inner_basis_precision=basis)
        assert st["rc"] == 0 and st["rel_residual"] <= 1e-12
        xs = x.cpu().numpy()
        assert np.max(np.abs(xs - x_ref)) <= 1e-9 * np.max(np.abs(x_ref)), (pc, st)
        its[pc] = st["inner_iterations"]
    # the periodic mesh of three cells along x: same-colour neighbours across the wrap (no strict gain required)
    if per:
        assert its[dg.DG_PRECOND_RB_GS] <= its[dg.DG_PRECOND_BLOCK_JACOBI], its
    else:
        assert its[dg.DG_PRECOND_RB_GS] < its[dg.DG_PRECOND_BLOCK_JACOBI], its
    op.close()
