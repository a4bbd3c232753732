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
