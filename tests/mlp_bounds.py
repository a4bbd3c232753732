"""Element-wise error bounds for the MLP kernels against the FP64 reference network (test helper).

The GPU forward pass multiplies BF16 operands, accumulates in FP32 and rounds each hidden activation to
BF16; the reference (oracle/mlp.py) does the same arithmetic in FP64.  Two effects separate them:

* the FP32 accumulation: a sum of K products (plus the bias) in FP32, in any order, is within
  gamma_K = 2 (K + 2) 2^-24 of the sum of the absolute values of its terms (the usual a-priori bound
  K u / (1 - K u), doubled to cover truncating accumulation);
* a BF16 rounding decided differently: when the FP32 pre-activation lies within that distance of a
  rounding midpoint, the GPU may take the neighbouring BF16 value.  Rounding and ReLU are monotone, so the
  GPU's activation lies between rnd(relu(pre - d)) and rnd(relu(pre + d)); the bound takes the larger of the
  two distances to the reference activation.

Both are propagated through the layers with absolute values (|W| times the deviation of the previous
layer, plus the accumulation term of this layer), which gives a bound for every output element rather
than a norm of the whole tensor.  The backward pass (FP32 GEMMs on the GPU) is bounded the same way from
the forward deviations: |a' b' - a b| <= (|a| + da)(|b| + db) - |a||b| term by term, plus gamma_K of the
absolute sums, with a ReLU mask counted as undecided where the activation's range touches zero.  The backward
GEMMs run on the tensor cores with BF16 operands: their FP32 left operands (dY, dZ2, dZ1) are rounded to BF16
(relative error <= 2^-8 each), which enters each product's bound as a deviation of that operand; the bias
gradients are FP32 column sums of the unrounded operands.
"""

from __future__ import annotations

import numpy as np

from oracle import mlp as om

U32 = 2.0 ** -24
U_BF16 = 2.0 ** -8  # bound on the relative error of rounding to BF16 (half an ulp of an 8-bit significand)


def gam(K: int) -> float:
    return 2.0 * (K + 2) * U32


def _range_dev(pre, d, h):
    lo = om.bf16_round(np.maximum(pre - d, 0.0))
    hi = om.bf16_round(np.maximum(pre + d, 0.0))
    return np.maximum(np.abs(hi - h), np.abs(h - lo))


def forward_bound(X, W1, b1, W2, b2, W3, b3, exact_forward=False):
    """Reference forward pass and per-element bounds.  Returns a dict with y, h1, h2 (reference values), dh1,
    dh2 (bounds on the GPU's hidden activations' deviation) and dy (bound on |y_gpu - y|).  exact_forward:
    every sum of the forward pass is exact in FP32 (``exact_network``), so all three deviations are zero."""
    X = np.asarray(X, dtype=np.float64)
    W1q, W2q, W3q = (om.bf16_round(W) for W in (W1, W2, W3))
    aX, a1, a2, a3 = np.abs(X), np.abs(W1q), np.abs(W2q), np.abs(W3q)
    pre1 = X @ W1q.T + b1
    d1 = gam(W1q.shape[1]) * (aX @ a1.T + np.abs(b1))
    h1 = om.bf16_round(np.maximum(pre1, 0.0))
    dh1 = _range_dev(pre1, d1, h1)
    pre2 = h1 @ W2q.T + b2
    d2 = dh1 @ a2.T + gam(W2q.shape[1]) * ((np.abs(h1) + dh1) @ a2.T + np.abs(b2))
    h2 = om.bf16_round(np.maximum(pre2, 0.0))
    dh2 = _range_dev(pre2, d2, h2)
    y = h2 @ W3q.T + b3
    dy = dh2 @ a3.T + gam(W3q.shape[1]) * ((np.abs(h2) + dh2) @ a3.T + np.abs(b3))
    if exact_forward:
        dh1, dh2, dy = np.zeros_like(h1), np.zeros_like(h2), np.zeros_like(y)
    return dict(y=y, h1=h1, h2=h2, dh1=dh1, dh2=dh2, dy=dy, W2q=W2q, W3q=W3q)


def _prod_dev(A, dA, B, dB, K):
    """Bound on |A'^T B' - A^T B| for |A' - A| <= dA, |B' - B| <= dB, computed in FP32 with K terms."""
    aA, aB = np.abs(A), np.abs(B)
    full = (aA + dA).T @ (aB + dB)
    return full - aA.T @ aB + gam(K) * full


def _mask_dev(dH, ddH, h, dh):
    """dZ = dH * (h > 0): bound on the GPU's deviation, with the mask undecided where h's range touches 0."""
    pos = h > 0
    unsure = (pos & (h <= dh)) | (~pos & (dh > 0))
    return np.where(unsure, np.abs(dH) + ddH, np.where(pos, ddH, 0.0))


def grad_bound(X, T, W1, b1, W2, b2, W3, b3, nb, exact_forward=False):
    """Reference loss and gradients (oracle/mlp.py) and per-element bounds on the GPU's gradients, in the order
    W1, b1, W2, b2, W3, b3 (exact_forward as in forward_bound)."""
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    rows = X.shape[0]
    fb = forward_bound(X, W1, b1, W2, b2, W3, b3, exact_forward)
    loss, g = om.loss_and_grad(X, T, W1, b1, W2, b2, W3, b3, nb=nb, bf16_hidden=True)
    y, h1, h2, dh1, dh2 = fb["y"], fb["h1"], fb["h2"], fb["dh1"], fb["dh2"]
    W2q, W3q = fb["W2q"], fb["W3q"]
    n = rows * nb
    dY = np.zeros_like(y)
    dY[:, :nb] = 2.0 * (y[:, :nb] - T) / n
    ddY = np.zeros_like(y)
    ddY[:, :nb] = 2.0 / n * (fb["dy"][:, :nb] + 2 * U32 * (np.abs(y[:, :nb]) + np.abs(T) + fb["dy"][:, :nb])) \
        + 2 * U32 * np.abs(dY[:, :nb])
    A = np.abs(dY) + ddY
    bf = lambda a, da: da + U_BF16 * (np.abs(a) + da)  # deviation of a GEMM operand after rounding to BF16
    bW3 = _prod_dev(dY, bf(dY, ddY), h2, dh2, rows)
    bb3 = ddY.sum(axis=0) + gam(rows) * A.sum(axis=0)
    dH2 = dY @ W3q
    ddH2 = bf(dY, ddY) @ np.abs(W3q) + gam(W3q.shape[0]) * A @ np.abs(W3q)
    dZ2 = dH2 * (h2 > 0)
    ddZ2 = _mask_dev(dH2, ddH2, h2, dh2)
    bW2 = _prod_dev(dZ2, bf(dZ2, ddZ2), h1, dh1, rows)
    bb2 = ddZ2.sum(axis=0) + gam(rows) * (np.abs(dZ2) + ddZ2).sum(axis=0)
    dH1 = dZ2 @ W2q
    ddH1 = bf(dZ2, ddZ2) @ np.abs(W2q) + gam(W2q.shape[0]) * (np.abs(dZ2) + ddZ2) @ np.abs(W2q)
    dZ1 = dH1 * (h1 > 0)
    ddZ1 = _mask_dev(dH1, ddH1, h1, dh1)
    bW1 = _prod_dev(dZ1, bf(dZ1, ddZ1), X, np.zeros_like(X), rows)
    bb1 = ddZ1.sum(axis=0) + gam(rows) * (np.abs(dZ1) + ddZ1).sum(axis=0)
    return loss, g, (bW1, bb1, bW2, bb2, bW3, bb3)


def emulate_fp32(X, T, W1, b1, W2, b2, W3, b3, nb):
    """The GPU's arithmetic emulated on the CPU: BF16 weights, FP32 sums (numpy's own summation order), BF16
    hidden activations, backward GEMMs on BF16-rounded operands with FP32 sums.  Used only to pin the bounds above
    on the CPU."""
    f = np.float32
    X = np.asarray(X, dtype=f)
    W1q, W2q, W3q = (om.bf16_round(W).astype(f) for W in (W1, W2, W3))
    h1 = om.bf16_round(np.maximum(X @ W1q.T + b1.astype(f), 0)).astype(f)
    h2 = om.bf16_round(np.maximum(h1 @ W2q.T + b2.astype(f), 0)).astype(f)
    y = h2 @ W3q.T + b3.astype(f)
    if T is None:
        return y, None
    rows = X.shape[0]
    dY = np.zeros_like(y)
    dY[:, :nb] = (y[:, :nb] - np.asarray(T, dtype=f)) * f(2.0 / (rows * nb))
    r16 = lambda a: om.bf16_round(a).astype(f)  # the tensor-core GEMMs take BF16 operands
    gW3 = r16(dY).T @ h2
    gb3 = dY.sum(axis=0, dtype=f)
    dZ2 = (r16(dY) @ W3q) * (h2 > 0)
    gW2 = r16(dZ2).T @ h1
    gb2 = dZ2.sum(axis=0, dtype=f)
    dZ1 = (r16(dZ2) @ W2q) * (h1 > 0)
    gW1 = r16(dZ1).T @ X
    gb1 = dZ1.sum(axis=0, dtype=f)
    return y, (gW1, gb1, gW2, gb2, gW3, gb3)


def forward_is_exact(X, W1, b1, W2, b2, W3, b3):
    """The precondition of exact_forward, checked in FP64: every hidden activation a BF16 number, and in every
    layer the operands on grids whose products and the bias share one grid g, with the sum of absolute terms
    below 2^24 g (so every partial sum in FP32 is exact, in any order)."""
    h1 = np.maximum(X @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    if not (np.array_equal(om.bf16_round(h1), h1) and np.array_equal(om.bf16_round(h2), h2)):
        return False
    on = lambda a, g: np.array_equal(np.round(np.asarray(a) / g) * g, a)
    # (input, its grid, weights, their grid, bias): the products and the bias lie on the product grid
    for A, ga, W, gw, b in ((X, 1.0, W1, 2.0 ** -4, b1), (h1, 2.0 ** -4, W2, 2.0 ** -4, b2),
                            (h2, 2.0 ** -8, W3, 2.0 ** -6, b3)):
        g = ga * gw
        if not (on(A, ga) and on(W, gw) and on(b, g)):
            return False
        if not np.all(np.abs(A) @ np.abs(W).T + np.abs(b) < 2.0 ** 24 * g):
            return False
    return True


def exact_network(kin, kinp, nb, outp, rng, hid=256):
    """Parameters and inputs on which the GPU forward pass is EXACT, so it must equal the reference bit for bit.

    X in {-1, 0, 1}; each row of W1 has 16 entries +-2^-4 (so |W1 x + b1| <= 32 * 2^-4 on a 2^-4 grid); each
    row of W2 has 4 entries +-2^-4 (pre-activations on a 2^-8 grid below 256 * 2^-8); W3 is dense on a 2^-6
    grid.  Every hidden pre-activation is then an integer multiple of its grid below 2^8, i.e. a BF16 number,
    and every FP32 sum is exact in any order.  Positions are random, so a transposed operand, a wrong column or
    a wrong K chunk changes the result.  Returns (W1, b1, W2, b2, W3, b3, X_rows_fn)."""
    W1 = np.zeros((hid, kinp))
    for j in range(hid):
        cols = rng.choice(kin, size=min(16, kin), replace=False)
        W1[j, cols] = rng.choice([-1.0, 1.0], size=cols.size) / 16
    b1 = rng.integers(-8, 9, hid) / 16
    W2 = np.zeros((hid, hid))
    for j in range(hid):
        cols = rng.choice(hid, size=4, replace=False)
        W2[j, cols] = rng.choice([-1.0, 1.0], size=4) / 16
    b2 = rng.integers(-16, 17, hid) / 256
    W3 = np.zeros((outp, hid))
    W3[:nb] = rng.integers(-4, 5, (nb, hid)) / 64
    b3 = np.zeros(outp)
    b3[:nb] = rng.integers(-64, 65, nb) / 64

    def rows(n):
        X = np.zeros((n, kinp))
        X[:, :kin] = rng.integers(-1, 2, (n, kin))
        return X

    return W1, b1, W2, b2, W3, b3, rows
