"""Pins of the FP64 MLP reference (CPU): its gradient against central finite differences, and its
BF16 rounding against torch's bfloat16 conversion (a library special case)."""

import numpy as np
import pytest

from oracle import mlp as om


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(10000) * 10.0 ** rng.integers(-6, 6, 10000),
                        [0.0, -0.0, 1.0, 65504.0, 1e-40, 3.0e38]]).astype(np.float32)
    ref = torch.tensor(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(om.bf16_round(x), ref)


def _small_net(rng, kin=13, kinp=16, hid=256, nb=9, outp=16):
    W1 = np.zeros((hid, kinp))
    W1[:, :kin] = rng.standard_normal((hid, kin)) / np.sqrt(kin)
    b1 = rng.standard_normal(hid) * 0.1
    W2 = rng.standard_normal((hid, hid)) / np.sqrt(hid)
    b2 = rng.standard_normal(hid) * 0.1
    W3 = np.zeros((outp, hid))
    W3[:nb] = rng.standard_normal((nb, hid)) / np.sqrt(hid)
    b3 = np.zeros(outp)
    b3[:nb] = rng.standard_normal(nb) * 0.1
    return [W1, b1, W2, b2, W3, b3]


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    nb, kinp = 9, 16
    P = _small_net(rng)
    X = np.zeros((12, kinp))
    X[:, :13] = rng.standard_normal((12, 13))
    T = rng.standard_normal((12, nb))
    loss, grads = om.loss_and_grad(X, T, *P, nb=nb, bf16_hidden=False)
    eps = 1e-6
    for pi, (param, g) in enumerate(zip(P, grads)):
        flat = param.reshape(-1)
        gflat = g.reshape(-1)
        idx = rng.choice(flat.size, size=min(12, flat.size), replace=False)
        for i in idx:
            old = flat[i]
            flat[i] = old + eps
            lp, _ = om.loss_and_grad(X, T, *P, nb=nb, bf16_hidden=False)
            flat[i] = old - eps
            lm, _ = om.loss_and_grad(X, T, *P, nb=nb, bf16_hidden=False)
            flat[i] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - gflat[i]) <= 1e-6 * max(1.0, abs(fd)), (pi, i, fd, gflat[i])


def test_padding_outputs_do_not_enter_the_loss():
    rng = np.random.default_rng(2)
    P = _small_net(rng)
    X = rng.standard_normal((5, 16))
    T = rng.standard_normal((5, 9))
    l1, g1 = om.loss_and_grad(X, T, *P, nb=9, bf16_hidden=False)
    P[4][12] = 100.0  # a padding output row of W3
    l2, g2 = om.loss_and_grad(X, T, *P, nb=9, bf16_hidden=False)
    assert l1 == l2
    assert np.all(g2[4][9:] == 0)


# ---- pins of the element-wise bounds that the GPU parity tests use (tests/mlp_bounds.py) ----

def _dims(k):
    nb = (k + 1) ** 3
    kin = nb + 7
    return nb, kin, (kin + 15) // 16 * 16, (nb + 15) // 16 * 16


def _random_net(rng, k):
    from tests import mlp_bounds as mb
    nb, kin, kinp, outp = _dims(k)
    W1, b1, W2, b2, W3, b3 = _small_net(rng, kin=kin, kinp=kinp, nb=nb, outp=outp)
    f = lambda a: a.astype(np.float32).astype(np.float64)
    X = np.zeros((150, kinp))
    X[:, :kin] = rng.standard_normal((150, kin))
    return [f(W1), f(b1), f(W2), f(b2), f(W3), f(b3)], om.bf16_round(X), rng.standard_normal((150, nb))


@pytest.mark.parametrize("k", [1, 2, 4, 5, 7])
def test_exact_network_is_exact(k):
    """The exact network's precondition holds, and an FP32 evaluation in two different summation orders
    reproduces the FP64 reference bit for bit."""
    from tests import mlp_bounds as mb
    rng = np.random.default_rng(k)
    nb, kin, kinp, outp = _dims(k)
    W1, b1, W2, b2, W3, b3, make_rows = mb.exact_network(kin, kinp, nb, outp, rng)
    X = make_rows(97)
    assert mb.forward_is_exact(X, W1, b1, W2, b2, W3, b3)
    y_ref, _, _ = om.forward(X, W1, b1, W2, b2, W3, b3, bf16_hidden=True)
    y32, _ = mb.emulate_fp32(X, None, W1, b1, W2, b2, W3, b3, nb)
    assert np.array_equal(y32.astype(np.float64), y_ref)
    rev = np.arange(kinp)[::-1]
    y32r, _ = mb.emulate_fp32(X[:, rev], None, W1[:, rev], b1, W2, b2, W3, b3, nb)
    assert np.array_equal(y32r.astype(np.float64), y_ref)
    assert not mb.forward_is_exact(X, W1 * 1.01, b1, W2, b2, W3, b3)


@pytest.mark.parametrize("k", [2, 4])
def test_bounds_hold_for_an_fp32_evaluation(k):
    """An FP32 evaluation with BF16 hidden roundings (numpy's own summation order) stays inside every
    per-element bound: forward and gradients, random and exact networks."""
    from tests import mlp_bounds as mb
    rng = np.random.default_rng(30 + k)
    W, X, T = _random_net(rng, k)
    nb = _dims(k)[0]
    fb = mb.forward_bound(X, *W)
    y32, g32 = mb.emulate_fp32(X, T, *W, nb)
    assert np.all(np.abs(y32[:, :nb] - fb["y"][:, :nb]) <= fb["dy"][:, :nb])
    _, g_ref, bounds = mb.grad_bound(X, T, *W, nb=nb)
    for a, b, bd in zip(g32, g_ref, bounds):
        assert np.all(np.abs(a - b) <= bd)
    nb, kin, kinp, outp = _dims(k)
    W1, b1, W2, b2, W3, b3, make_rows = mb.exact_network(kin, kinp, nb, outp, rng)
    X = make_rows(120)
    T = np.round(rng.standard_normal((120, nb)) * 64) / 64
    _, g32 = mb.emulate_fp32(X, T, W1, b1, W2, b2, W3, b3, nb)
    _, g_ref, bounds = mb.grad_bound(X, T, W1, b1, W2, b2, W3, b3, nb, exact_forward=True)
    for a, b, bd in zip(g32, g_ref, bounds):
        assert np.all(np.abs(a - b) <= bd)
        # tight enough to see a wrong element (a single-term sum can reach the BF16 rounding of its operand)
        assert np.median(bd) <= 5e-2 * np.max(np.abs(b))


def test_bounds_catch_planted_mistakes():
    """A swapped pair of output columns, or one gradient row taken from its neighbour, breaks the bounds."""
    from tests import mlp_bounds as mb
    rng = np.random.default_rng(5)
    k = 2
    nb, kin, kinp, outp = _dims(k)
    W, X, T = _random_net(rng, k)
    fb = mb.forward_bound(X, *W)
    y32, _ = mb.emulate_fp32(X, None, *W, nb)
    y_bad = y32.copy()
    y_bad[:, [3, 4]] = y_bad[:, [4, 3]]
    assert not np.all(np.abs(y_bad[:, :nb] - fb["y"][:, :nb]) <= fb["dy"][:, :nb])
    W1, b1, W2, b2, W3, b3, make_rows = mb.exact_network(kin, kinp, nb, outp, rng)
    X = make_rows(64)
    T = np.round(rng.standard_normal((64, nb)) * 64) / 64
    _, g32 = mb.emulate_fp32(X, T, W1, b1, W2, b2, W3, b3, nb)
    _, g_ref, bounds = mb.grad_bound(X, T, W1, b1, W2, b2, W3, b3, nb, exact_forward=True)
    for blk in (0, 2, 4):  # W1, W2, W3: row 1 replaced by row 0
        bad = g32[blk].copy()
        bad[1] = bad[0]
        assert not np.all(np.abs(bad - g_ref[blk]) <= bounds[blk])
