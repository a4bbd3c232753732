"""FP64 CPU reference of the per-element MLP preconditioner network (test infrastructure only).

Only the test suite uses this module.  It restates the network that the library's header documents
(two ReLU layers of 256 units and a linear output layer), written from that definition with plain
numpy in float64:

    h1 = relu(W1 x + b1),  h2 = relu(W2 h1 + b2),  y = W3 h2 + b3,
    loss = mean over rows and real outputs of (y - t)^2.

The GPU forward pass multiplies BF16 inputs and weights and rounds the hidden activations to BF16
before the next layer; ``forward(..., bf16_hidden=True)`` applies the same roundings (BF16 round to
nearest even) so that the two differ only by summation order.  ``loss_and_grad`` is the chain rule
written out and is pinned by central finite differences in the CPU tests.
"""

from __future__ import annotations

import numpy as np


def bf16_round(a) -> np.ndarray:
    """Round float values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if nan.any():
        out[nan] = np.nan
    return out


def unpack(params, offsets, kinp, outp, hid=256):
    """Split the flat FP32 parameter block into (W1, b1, W2, b2, W3, b3)."""
    p = np.asarray(params, dtype=np.float64)
    o = offsets
    W1 = p[o[0]:o[0] + hid * kinp].reshape(hid, kinp)
    b1 = p[o[1]:o[1] + hid]
    W2 = p[o[2]:o[2] + hid * hid].reshape(hid, hid)
    b2 = p[o[3]:o[3] + hid]
    W3 = p[o[4]:o[4] + outp * hid].reshape(outp, hid)
    b3 = p[o[5]:o[5] + outp]
    return W1, b1, W2, b2, W3, b3


def forward(X, W1, b1, W2, b2, W3, b3, bf16_hidden=True):
    """Rows of X through the network; returns (y, h1, h2).  bf16_hidden mirrors the GPU roundings."""
    rnd = bf16_round if bf16_hidden else (lambda a: np.asarray(a, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64)
    W1q, W2q, W3q = (rnd(W) for W in (W1, W2, W3))
    h1 = rnd(np.maximum(X @ W1q.T + b1, 0.0))
    h2 = rnd(np.maximum(h1 @ W2q.T + b2, 0.0))
    y = h2 @ W3q.T + b3
    return y, h1, h2


def loss_and_grad(X, T, W1, b1, W2, b2, W3, b3, nb, bf16_hidden=True):
    """Mean squared error over rows x nb real outputs and its gradient with respect to every parameter.

    With bf16_hidden the backward pass uses the rounded weights and activations of the forward pass
    (what the GPU uses), i.e. it is the gradient of the network as evaluated, rounding steps treated as
    identity.
    """
    rnd = bf16_round if bf16_hidden else (lambda a: np.asarray(a, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64)
    rows = X.shape[0]
    W1q, W2q, W3q = (rnd(W) for W in (W1, W2, W3))
    y, h1, h2 = forward(X, W1, b1, W2, b2, W3, b3, bf16_hidden)
    diff = np.zeros_like(y)
    diff[:, :nb] = y[:, :nb] - T
    loss = float(np.sum(diff[:, :nb] ** 2) / (rows * nb))
    dy = 2.0 * diff / (rows * nb)
    gW3 = dy.T @ h2
    gb3 = dy.sum(axis=0)
    dz2 = (dy @ W3q) * (h2 > 0)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2q) * (h1 > 0)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(axis=0)
    return loss, (gW1, gb1, gW2, gb2, gW3, gb3)


def features(r_cell, logD7, kinp):
    """Input row of one cell: [r / ||r||, log D (own, x-, x+, y-, y+, z-, z+)], zero-padded; and ||r||."""
    r_cell = np.asarray(r_cell, dtype=np.float64)
    s = float(np.linalg.norm(r_cell))
    row = np.zeros(kinp)
    nb = r_cell.size
    if s > 0:
        row[:nb] = r_cell / s
    row[nb:nb + 7] = logD7
    return row, s
