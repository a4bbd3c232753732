"""CPU pins of the matrix-free Kronecker apply (tests/kron_reference.apply_matfree), the check that covers whole
vectors of the full-size workloads.

It is compared with the dense Kronecker matrix of the same exact 1D integrals (``assemble``, itself pinned
against the oracle and the invariants of eq. blf) on small meshes with every boundary type, periodic axes,
both upwind branches and non-unit cells; and with the oracle's direct quadrature on sampled cells of the
32^3 Q_7 workload (log-normal D, penalty 2k(k+1)/h).
"""

import numpy as np
import pytest

import oracle
from paper_1711_10885_gb300 import inputs
from tests import kron_reference as kr

CASES = [
    ((3, 2, 4), 2, (1.0, 0.5, 0.25), (0, 0, 0), None),
    ((2, 3, 2), 3, (-1.0, 0.5, -0.3), (0, 0, 0), None),
    ((3, 2, 2), 2, (0.3, -0.7, 1.1), (1, 0, 1), None),
    ((1, 2, 3), 1, (1.0, -1.0, 0.5), (1, 1, 0), None),
    ((3, 2, 2), 2, (1.0, -0.5, 0.25), (0, 0, 0), ["dirichlet", "neumann", "outflow", "dirichlet", "neumann",
                                                  "outflow"]),
    ((2, 2, 3), 3, (-1.0, 0.5, 0.25), (0, 0, 0), ["outflow", "outflow", "neumann", "neumann", "dirichlet",
                                                   "dirichlet"]),
    ((1, 1, 1), 4, (0.0, 0.0, 0.0), (0, 0, 0), None),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"n{c[0]}k{c[1]}p{c[3]}")
def test_matfree_equals_dense_kronecker(case):
    n, k, b, per, bc = case
    rng = np.random.default_rng(k + 10 * len(n))
    ncell = int(np.prod(n))
    D = np.exp(rng.standard_normal(ncell))
    u = rng.uniform(-1.0, 1.0, ncell * (k + 1) ** 3)
    lo, hi = (0.0, -1.0, 0.0), (1.0, 1.0, 3.0)
    sigma = 2.0 * k * (k + 1)
    A = kr.assemble(n, k, D, b, 0.7, sigma, lo, hi, periodic=per, bc=bc)
    y = kr.apply_matfree(n, k, D, b, 0.7, sigma, u, lo, hi, periodic=per, bc=bc)
    ref = A @ u
    assert np.max(np.abs(y - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_matfree_equals_oracle_on_sampled_cells_of_q7_32():
    """The full-size check itself, against the oracle's direct quadrature on a few cells (corners included)."""
    w = inputs.unit_cube_q7_32()
    pr = oracle.Problem(w.n, w.k, w.D, b=w.b, c=w.c, lo=w.lo, hi=w.hi)
    y = kr.apply_matfree(w.n, w.k, w.D, w.b, w.c, pr.sigma, w.u, w.lo, w.hi).reshape(-1, w.nb)
    cells = [0, 31, 32 * 31, 32 ** 3 - 1, 12345, 20000]
    yo = oracle.apply(pr, w.u, cells=cells).reshape(len(cells), w.nb)
    assert np.max(np.abs(y[cells] - yo)) <= 1e-13 * np.max(np.abs(yo))
