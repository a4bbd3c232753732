"""GPU tests of the batched persistent apply: every problem's result equals its standalone apply bit
for bit (same per-cell arithmetic and order), for Jacobian and residual, over mixed meshes and degrees."""

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


def test_batch_equals_standalone_bitwise(dg):
    ws = inputs.batch_problems(count=12, seed=3, nmin=1, nmax=6, kmin=1, kmax=8)
    ops = [dg.operator_for(w) for w in ws]
    batch = dg.Batch(ops)
    xs = [torch.tensor(w.u, device="cuda") for w in ws]
    for residual in (False, True, False):
        ys = [torch.full_like(x, float("nan")) for x in xs]
        batch.apply(xs, ys, residual=residual)
        torch.cuda.synchronize()
        for op, x, y in zip(ops, xs, ys):
            ref = op.apply_residual(x) if residual else op.apply_jacobian(x)
            assert torch.equal(y, ref)
    for k in sorted({w.k for w in ws}):
        t = batch.tuning(k)
        assert t["cells_per_cta"] >= 1 and t["lines_per_thread"] in (1, 2)
        assert len(t["ms_candidates"]) == dg.DG_BATCH_CANDIDATES and min(t["ms_candidates"]) > 0
        # the chosen layout is the fastest candidate
        F = 256 // (k + 1) ** 2
        shapes = [(F, 1), (max(1, F // 2), 1), (F, 2), (2 * F, 2)]
        best = min(range(len(shapes)), key=lambda v: t["ms_candidates"][v])
        assert (t["cells_per_cta"], t["lines_per_thread"]) == shapes[best]
    batch.close()
    for op in ops:
        op.close()


def test_batch_against_oracle(dg):
    ws = inputs.batch_problems(count=5, seed=9, nmin=1, nmax=3, kmin=2, kmax=6)
    ops = [dg.operator_for(w) for w in ws]
    batch = dg.Batch(ops)
    xs = [torch.tensor(w.u, device="cuda") for w in ws]
    ys = [torch.empty_like(x) for x in xs]
    batch.apply(xs, ys)
    for w, y in zip(ws, ys):
        pr = oracle.Problem(w.n, w.k, w.D, b=w.b, c=w.c)
        ref = oracle.apply(pr, w.u)
        assert np.max(np.abs(y.cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(ref))
    batch.close()
    for op in ops:
        op.close()


def test_batch_rejects_degree_nine(dg):
    w = inputs.small_case(n=(1, 1, 1), k=9)
    op = dg.operator_for(w)
    with pytest.raises(dg.DGError):
        dg.Batch([op])
    op.close()
