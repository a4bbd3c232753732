"""GPU parity of the matrix-based comparison (Sec. 5.2): the block-sparse matrix assembled by probing the
operator equals the independently assembled Kronecker closed form of eq. blf (tests/kron_reference.py, exact
1D integrals, no quadrature), and its product equals the matrix-free application.

Bars: assembled entries within 1e-12 of the closed form relative to max |A|; products within 1e-12 of the
FP64 matrix-free apply (relative infinity norm).
"""

import numpy as np
import pytest

from paper_1711_10885_gb300 import inputs
from tests import kron_reference as kr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_10885_gb300 import dg as _dg
    return _dg


def relerr(y, ref):
    return float(np.max(np.abs(np.asarray(y) - ref)) / max(np.max(np.abs(ref)), 1e-300))


# (n, k, periodic, b): Dirichlet and periodic meshes, one and two cells along a periodic axis, both upwind signs
CASES = [
    ((2, 3, 2), 1, (0, 0, 0), (1.0, 0.5, 0.25)),
    ((3, 2, 4), 2, (0, 0, 0), (-0.6, 0.5, -0.25)),
    ((4, 2, 3), 2, (1, 0, 1), (0.7, -0.2, 0.4)),
    ((1, 2, 5), 3, (1, 1, 0), (0.3, 0.9, -0.6)),
    ((3, 3, 2), 3, (1, 1, 1), (1.0, 0.5, 0.25)),
    ((2, 2, 2), 4, (0, 0, 0), (0.2, -0.4, 0.9)),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"n{c[0]}k{c[1]}p{c[2]}")
def test_assembled_matrix_equals_closed_form(dg, case):
    n, k, per, b = case
    w = inputs.small_case(n=n, k=k, seed=120 + k, b=b, c=0.8)
    w.periodic = per
    sigma = dg.dg_penalty_sigma(k, 0)
    op = dg.operator_for(w)
    A = dg.Matrix(op)
    ref = kr.assemble(w.n, k, w.D, w.b, w.c, sigma, w.lo, w.hi, periodic=per)
    assert relerr(A.dense(), ref) <= 1e-12
    x = torch.tensor(w.u, device="cuda")
    assert relerr(A.spmv(x).cpu().numpy(), op.apply_jacobian(x).cpu().numpy()) <= 1e-12
    # every block row holds the cell and its distinct face neighbours
    rp, ci, _ = A.export()
    assert rp[0] == 0 and np.all(np.diff(rp) >= 1) and np.all(np.diff(rp) <= 7)
    A.close()
    op.close()


@pytest.mark.parametrize("n,k", [((6, 5, 4), 3), ((4, 3, 3), 5), ((3, 3, 4), 7)])
def test_spmv_matches_matrix_free_apply(dg, n, k):
    """Several CTAs and ragged row groups of the product kernel (rows per CTA = max(1, 256 / (k+1)^3))."""
    w = inputs.small_case(n=n, k=k, seed=130 + k)
    op = dg.operator_for(w)
    A = dg.Matrix(op)
    # one diagonal block per cell and two blocks per interior face
    interior_faces = sum((n[d] - 1) * int(np.prod(n)) // n[d] for d in range(3))
    assert A.nnzb == int(np.prod(n)) + 2 * interior_faces
    x = torch.tensor(w.u, device="cuda")
    assert relerr(A.spmv(x).cpu().numpy(), op.apply_jacobian(x).cpu().numpy()) <= 1e-12
    A.close()
    op.close()


def test_velocity_field_operator_assembles(dg):
    """The probing uses the operator as it is: the Taylor-Green operator (m = k+3, periodic) assembles too."""
    w = inputs.taylor_green(4, 2)
    op = dg.operator_for(w)
    A = dg.Matrix(op)
    x = torch.tensor(inputs.uniform_u(w.ndof, 140), device="cuda")
    assert relerr(A.spmv(x).cpu().numpy(), op.apply_jacobian(x).cpu().numpy()) <= 1e-12
    A.close()
    op.close()


def test_assembly_rejects_large_blocks(dg):
    op = dg.Operator((1, 1, 1), 8)
    with pytest.raises(dg.DGError):
        dg.Matrix(op)
    op.close()
