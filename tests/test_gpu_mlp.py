"""GPU tests of the learned preconditioner: feature rows, forward pass and gradients against the FP64
MLP reference (oracle/mlp.py) element by element (bit for bit on a network whose arithmetic is exact,
within propagated per-element bounds on random ones), training, checkpointing, and what the trained
network gains inside FGMRES over block-Jacobi alone, with the block-Jacobi fallback."""

import os
import tempfile

import numpy as np
import pytest

import oracle
from oracle import mlp as om
from paper_1711_10885_gb300 import inputs
from tests import mlp_bounds as mb

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_10885_gb300 import dg as _dg
    return _dg


def _random_params(mlp, rng):
    p = np.zeros(mlp.nparam, dtype=np.float32)
    o, H = mlp.offsets, 256
    W1 = np.zeros((H, mlp.kinp), np.float32)
    W1[:, :mlp.kin] = rng.standard_normal((H, mlp.kin)) / np.sqrt(mlp.kin)
    W3 = np.zeros((mlp.outp, H), np.float32)
    W3[:mlp.nb] = rng.standard_normal((mlp.nb, H)) / np.sqrt(H)
    b3 = np.zeros(mlp.outp, np.float32)
    b3[:mlp.nb] = rng.standard_normal(mlp.nb) * 0.1
    p[o[0]:o[0] + W1.size] = W1.ravel()
    p[o[1]:o[1] + H] = rng.standard_normal(H) * 0.1
    p[o[2]:o[2] + H * H] = (rng.standard_normal((H, H)) / np.sqrt(H)).ravel()
    p[o[3]:o[3] + H] = rng.standard_normal(H) * 0.1
    p[o[4]:o[4] + W3.size] = W3.ravel()
    p[o[5]:o[5] + mlp.outp] = b3
    return p


def _rows(mlp, rng, n):
    X = np.zeros((n, mlp.kinp), np.float32)
    X[:, :mlp.kin] = rng.standard_normal((n, mlp.kin))
    return om.bf16_round(X)


def test_feature_rows(dg):
    w = inputs.small_case(n=(3, 4, 2), k=2, seed=3, sigma_D=1.5)
    op = dg.operator_for(w)
    mlp = dg.MLP(2, seed=1)
    rng = np.random.default_rng(5)
    r = rng.standard_normal(w.ndof)
    r[:w.nb] = 0.0  # a cell with zero residual gives a zero row
    X, s = mlp.features(op, torch.tensor(r, device="cuda"))
    X = X.float().cpu().numpy()
    s = s.cpu().numpy()
    logD = np.log(w.D)
    nx, ny, nz = w.n
    for c in range(w.ncell):
        ic = [c % nx, (c // nx) % ny, c // (nx * ny)]
        nbr = [c]
        for d, st, nn in ((0, 1, nx), (1, nx, ny), (2, nx * ny, nz)):
            nbr.append(c - st if ic[d] > 0 else c)
            nbr.append(c + st if ic[d] < nn - 1 else c)
        row, sr = om.features(r[c * w.nb:(c + 1) * w.nb], logD[nbr], mlp.kinp)
        assert abs(s[c] - sr) <= 1e-6 * max(sr, 1e-30)
        ref = om.bf16_round(row)
        assert np.max(np.abs(X[c] - ref)) <= 2 ** -7 * np.max(np.abs(ref)), c
    op.close()
    mlp.close()


def _pack(mlp, W1, b1, W2, b2, W3, b3):
    p = np.zeros(mlp.nparam, dtype=np.float32)
    o = mlp.offsets
    for off, a in zip(o, (W1, b1, W2, b2, W3, b3)):
        a = np.asarray(a, dtype=np.float32).ravel()
        p[off:off + a.size] = a
    return p


# forward kernels: the tcgen05 kernel serves inference for degrees 1..5; the mma.sync kernel (training, and
# degrees 6..7) is selected for every degree by DG_MLP_NO_TCGEN05
KERNEL_CASES = [(1, 128, "tcgen05"), (2, 77, "tcgen05"), (4, 300, "tcgen05"), (5, 129, "tcgen05"),
                (2, 77, "mma"), (4, 300, "mma"), (7, 65, "mma")]


def _forward(mlp, X, kernel):
    if kernel == "mma":
        os.environ["DG_MLP_NO_TCGEN05"] = "1"
    try:
        return mlp.forward(X).cpu().numpy().astype(np.float64)
    finally:
        os.environ.pop("DG_MLP_NO_TCGEN05", None)


@pytest.mark.parametrize("k,rows,kernel", KERNEL_CASES, ids=lambda c: str(c))
def test_forward_exact_network_bitwise(dg, k, rows, kernel):
    """On a network whose every FP32 sum and BF16 hidden activation is exact (tests/mlp_bounds.exact_network,
    precondition checked here), the forward pass has one correct result: every output element must equal
    the FP64 reference exactly, padding columns included (zero)."""
    rng = np.random.default_rng(100 + k)
    mlp = dg.MLP(k, seed=0)
    W1, b1, W2, b2, W3, b3, make_rows = mb.exact_network(mlp.kin, mlp.kinp, mlp.nb, mlp.outp, rng)
    X = make_rows(rows)
    assert mb.forward_is_exact(X, W1, b1, W2, b2, W3, b3)
    mlp.set_params(_pack(mlp, W1, b1, W2, b2, W3, b3))
    y_ref, _, _ = om.forward(X, W1, b1, W2, b2, W3, b3, bf16_hidden=True)
    Y = _forward(mlp, torch.tensor(X, dtype=torch.bfloat16, device="cuda"), kernel)
    bad = np.argwhere(Y != y_ref)
    assert bad.size == 0, (bad[:5], Y[tuple(bad[0])], y_ref[tuple(bad[0])])
    mlp.close()


@pytest.mark.parametrize("k,rows,kernel", KERNEL_CASES, ids=lambda c: str(c))
def test_forward_random_network_elementwise(dg, k, rows, kernel):
    """Random weights: every output element within its propagated bound (FP32 accumulation and possible BF16
    flips of the hidden activations, tests/mlp_bounds.forward_bound), and in every output column
    max |Y - Y_ref| <= 2^-8 max |Y_ref| (a hidden flip moves one activation by one BF16 step, 2^-7 of it)."""
    rng = np.random.default_rng(k)
    mlp = dg.MLP(k, seed=0)
    p = _random_params(mlp, rng)
    mlp.set_params(p)
    X = _rows(mlp, rng, rows)
    Y = _forward(mlp, torch.tensor(X, dtype=torch.bfloat16, device="cuda"), kernel)
    W = om.unpack(p, mlp.offsets, mlp.kinp, mlp.outp)
    fb = mb.forward_bound(X, *W)
    nb = mlp.nb
    err = np.abs(Y[:, :nb] - fb["y"][:, :nb])
    assert np.all(err <= fb["dy"][:, :nb]), np.max(err / fb["dy"][:, :nb])
    colmax = np.max(np.abs(fb["y"][:, :nb]), axis=0)
    assert np.all(np.max(err, axis=0) <= 2.0 ** -8 * colmax)
    assert np.all(Y[:, nb:] == fb["y"][:, nb:])  # padding rows of W3 and b3 are zero
    mlp.close()


@pytest.mark.parametrize("k,rows,kernel", [(4, 200, "tcgen05"), (4, 200, "mma"), (2, 131, "tcgen05"),
                                           (7, 96, "mma")])
def test_gradient_exact_network_elementwise(dg, k, rows, kernel):
    """Loss and every gradient element on the exact network, with the training forward pass on the tcgen05 or
    the mma.sync kernel: the forward pass is exact, so each gradient element differs from the FP64 reference
    only by the backward arithmetic on the tensor cores (BF16 operands, FP32 accumulation), bounded element by
    element (tests/mlp_bounds.grad_bound)."""
    rng = np.random.default_rng(200 + k)
    mlp = dg.MLP(k, seed=0)
    W1, b1, W2, b2, W3, b3, make_rows = mb.exact_network(mlp.kin, mlp.kinp, mlp.nb, mlp.outp, rng)
    X = make_rows(rows)
    assert mb.forward_is_exact(X, W1, b1, W2, b2, W3, b3)
    T = np.round(rng.standard_normal((rows, mlp.nb)) * 64) / 64
    mlp.set_params(_pack(mlp, W1, b1, W2, b2, W3, b3))
    if kernel == "mma":
        os.environ["DG_MLP_NO_TCGEN05"] = "1"
    try:
        loss = mlp.loss_grad(torch.tensor(X, dtype=torch.bfloat16, device="cuda"),
                             torch.tensor(T, dtype=torch.float32, device="cuda"))
    finally:
        os.environ.pop("DG_MLP_NO_TCGEN05", None)
    loss_ref, g_ref, bounds = mb.grad_bound(X, T, W1, b1, W2, b2, W3, b3, mlp.nb, exact_forward=True)
    assert abs(loss - loss_ref) <= 1e-6 * loss_ref
    g = om.unpack(mlp.grad(), mlp.offsets, mlp.kinp, mlp.outp)
    for name, a, b, bd in zip(["W1", "b1", "W2", "b2", "W3", "b3"], g, g_ref, bounds):
        err = np.abs(a - b)
        assert np.all(err <= bd), (name, np.unravel_index(np.argmax(err - bd), err.shape), np.max(err / (bd + 1e-300)))
    mlp.close()


def test_gradient_random_network_elementwise(dg):
    """Random weights and inputs: every gradient element within its propagated bound, and per block
    max |g - g_ref| <= 2^-6 max |g_ref| (the BF16 operands of the backward GEMMs and a flipped BF16 hidden
    value each change one factor of a term by at most 2^-8 and 2^-7 of it)."""
    rng = np.random.default_rng(7)
    mlp = dg.MLP(4, seed=0)
    p = _random_params(mlp, rng)
    mlp.set_params(p)
    X = _rows(mlp, rng, 200)
    T = rng.standard_normal((200, mlp.nb)).astype(np.float32)
    loss = mlp.loss_grad(torch.tensor(X, dtype=torch.bfloat16, device="cuda"), torch.tensor(T, device="cuda"))
    W = om.unpack(p, mlp.offsets, mlp.kinp, mlp.outp)
    loss_ref, g_ref, bounds = mb.grad_bound(X, T, *W, nb=mlp.nb)
    assert abs(loss - loss_ref) <= 1e-3 * loss_ref
    g = om.unpack(mlp.grad(), mlp.offsets, mlp.kinp, mlp.outp)
    for name, a, b, bd in zip(["W1", "b1", "W2", "b2", "W3", "b3"], g, g_ref, bounds):
        err = np.abs(a - b)
        assert np.all(err <= bd), name
        assert np.max(err) <= 2.0 ** -6 * np.max(np.abs(b)), (name, np.max(err) / np.max(np.abs(b)))
    mlp.close()


def test_training_reduces_loss_and_checkpoint_round_trips(dg):
    rng = np.random.default_rng(11)
    mlp = dg.MLP(3, seed=2)
    X = _rows(mlp, rng, 2048)
    A = rng.standard_normal((mlp.nb, mlp.kin)) / np.sqrt(mlp.kin)
    T = np.tanh(X[:, :mlp.kin] @ A.T).astype(np.float32)
    Xt = torch.tensor(X, dtype=torch.bfloat16, device="cuda")
    st = mlp.train(Xt, torch.tensor(T, device="cuda"), epochs=15, batch=128, lr=2e-3)
    assert st["last_epoch_loss"] < 0.3 * st["first_epoch_loss"], st
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "net.bin")
        mlp.save(path)
        m2 = dg.MLP(path=path)
        p1, t1 = mlp.params()
        p2, t2 = m2.params()
        assert np.array_equal(p1, p2) and t1 == t2
        assert torch.equal(mlp.forward(Xt), m2.forward(Xt))
        m2.close()
    mlp.close()


def test_preconditioner_apply_is_scaled_forward(dg):
    w = inputs.small_case(n=(4, 3, 3), k=4, seed=9)
    op = dg.operator_for(w)
    mlp = dg.MLP(4, seed=3)
    mlp.set_target_scale(2.5)
    r = torch.randn(w.ndof, dtype=torch.float64, device="cuda")
    z = mlp.apply(op, r)
    X, s = mlp.features(op, r)
    Y = mlp.forward(X)
    ref = (Y[:, :w.nb] * s[:, None]).double().reshape(-1)
    assert torch.allclose(z, ref, rtol=1e-6, atol=0)
    z32 = mlp.apply(op, r.float())
    assert torch.max(torch.abs(z32.double() - z)).item() <= 1e-2 * torch.max(torch.abs(z)).item()
    op.close()
    mlp.close()


def test_learned_preconditioner_gain_and_fallback(dg):
    """FGMRES(30) in FP64 with block-Jacobi stalls on this problem; the network trained on the solver's own
    (residual, error) pairs, used on the first direction of every cycle (whose input is a true residual),
    gives a smaller residual after the same 1500 iterations (measured 0.12 to 0.41 against 0.94 over
    training-data variants; after 3000 iterations 1e-5 against 0.94)."""
    from paper_1711_10885_gb300 import learned
    train = [inputs.small_case(n=(16, 16, 16), k=4, seed=s, sigma_D=1.5) for s in (10, 11)]
    mlp, info = learned.train_preconditioner(train, 4, pairs=8000, epochs=40, batch=256, lr=1e-3, seed=0,
                                             minus_block_jacobi=False)
    assert info["last_epoch_loss"] < 0.5 * info["first_epoch_loss"], info
    w = inputs.small_case(n=(16, 16, 16), k=4, seed=20, sigma_D=1.5)
    op = dg.operator_for(w)
    op.precond_setup()
    res = {}
    for name, pc in (("bj", dg.DG_PRECOND_BLOCK_JACOBI), ("learned", dg.DG_PRECOND_BJ_MLP)):
        x = torch.zeros(w.ndof, dtype=torch.float64, device="cuda")
        res[name] = op.solve(x, mode=dg.DG_SOLVE_FP64, preconditioner=pc, mlp=mlp, mlp_placement=1, rtol=1e-8,
                             max_iterations=1500, raise_on_error=False)
    assert res["learned"]["rel_residual"] <= 0.75 * res["bj"]["rel_residual"], res
    # mixed precision with the learned first direction converges to the tolerance
    x = torch.zeros(w.ndof, dtype=torch.float64, device="cuda")
    st = op.solve(x, mode=dg.DG_SOLVE_MIXED, preconditioner=dg.DG_PRECOND_BJ_MLP, mlp=mlp, mlp_placement=1,
                  rtol=1e-8, inner_rtol=1e-2)
    assert st["rel_residual"] <= 1e-8
    # the network alone in every application stagnates; the stagnation test switches to block-Jacobi
    x = torch.zeros(w.ndof, dtype=torch.float64, device="cuda")
    st = op.solve(x, mode=dg.DG_SOLVE_MIXED, preconditioner=dg.DG_PRECOND_MLP, mlp=mlp, rtol=1e-8,
                  inner_rtol=1e-2, fallback_ratio=0.5)
    assert st["fallback"] == 1 and st["rel_residual"] <= 1e-8
    mlp.close()
    op.close()


@pytest.mark.parametrize("k,rows", [(4, 1000), (5, 129), (1, 128)])
def test_tensor_memory_forward_equals_mma_sync_forward(dg, k, rows):
    """The tcgen05 forward kernel (inference, degrees 1..5) and the mma.sync kernel compute the same network in
    the same precisions (BF16 operands and hidden layers, FP32 accumulation); they differ only in summation
    order, and in a rare hidden value rounded to the neighbouring BF16 number."""
    rng = np.random.default_rng(40 + k)
    mlp = dg.MLP(k, seed=4)
    mlp.set_params(_random_params(mlp, rng))
    X = torch.tensor(_rows(mlp, rng, rows), dtype=torch.bfloat16, device="cuda")
    y_tc = mlp.forward(X)
    os.environ["DG_MLP_NO_TCGEN05"] = "1"
    try:
        y_mma = mlp.forward(X)
    finally:
        del os.environ["DG_MLP_NO_TCGEN05"]
    assert torch.isfinite(y_tc).all()
    err = (torch.linalg.norm(y_tc - y_mma) / torch.linalg.norm(y_mma)).item()
    assert err <= 1e-3, err
    mlp.close()


def test_tcgen05_weight_wait_timeout_gives_nan_rows(dg):
    """The tcgen05 forward kernel's bounded wait for its weights, made to give up at once
    (DG_MLP_WEIGHT_WAIT_TRIES=0): the kernel issues no MMA and no further copy, waits for the copy in flight,
    frees its tensor memory and returns NaN rows; a solve using the network reports DG_ERR_NAN; afterwards the
    same call gives the normal result (the context is intact)."""
    rng = np.random.default_rng(61)
    mlp = dg.MLP(4, seed=0)
    mlp.set_params(_random_params(mlp, rng))
    X = torch.tensor(_rows(mlp, rng, 300), dtype=torch.bfloat16, device="cuda")
    y_ok = mlp.forward(X)
    os.environ["DG_MLP_WEIGHT_WAIT_TRIES"] = "0"
    try:
        y_to = mlp.forward(X)
        torch.cuda.synchronize()
        assert torch.isnan(y_to).all()
        w = inputs.small_case(n=(4, 3, 3), k=4, seed=9)
        op = dg.operator_for(w)
        x = torch.zeros(w.ndof, dtype=torch.float64, device="cuda")
        st = op.solve(x, mode=dg.DG_SOLVE_FP64, preconditioner=dg.DG_PRECOND_MLP, mlp=mlp, rtol=1e-8,
                      max_iterations=50, raise_on_error=False)
        assert st["status"] == dg.DG_ERR_NAN, st
        op.close()
    finally:
        del os.environ["DG_MLP_WEIGHT_WAIT_TRIES"]
    assert torch.equal(mlp.forward(X), y_ok)
    mlp.close()


@pytest.mark.parametrize("subtract", [False, True])
def test_training_pairs_match_oracle(dg, subtract):
    """dg_mlp_pairs: the feature rows of r = F - A x and the targets e_T / ||r_T|| (e = x* - x, minus the exact
    block inverse of r when subtract) at shuffled rows, against the FP64 oracle (A and F by direct quadrature,
    the diagonal blocks solved with numpy); dg_mlp_normalize_targets against the RMS of the targets."""
    w = inputs.small_case(n=(3, 4, 2), k=2, seed=19, sigma_D=1.5)
    pr = oracle.Problem(w.n, w.k, w.D, b=w.b, c=w.c, lo=w.lo, hi=w.hi)
    rng = np.random.default_rng(23)
    x = rng.uniform(-1, 1, w.ndof)
    xstar = rng.uniform(-1, 1, w.ndof)
    F = oracle.rhs(pr, np.ones(pr.ncell * pr.m ** 3), None)
    r = F - oracle.apply(pr, x)
    e = xstar - x
    nb = w.nb
    if subtract:
        for c in range(w.ncell):
            sl = slice(c * nb, (c + 1) * nb)
            B = np.empty((nb, nb))
            for j in range(nb):
                ej = np.zeros(w.ndof)
                ej[c * nb + j] = 1.0
                B[:, j] = oracle.apply(pr, ej)[sl]
            e[sl] -= np.linalg.solve(B, r[sl])
    op = dg.operator_for(w)
    op.precond_setup()
    mlp = dg.MLP(2, seed=1)
    cells = np.array([0, 5, 7, 11, 13, 23], dtype=np.int32)
    rows = np.array([3, 0, 5, 1, 4, 2], dtype=np.int32)
    X = torch.zeros((len(cells), mlp.kinp), dtype=torch.bfloat16, device="cuda")
    E = torch.zeros((len(cells), nb), dtype=torch.float32, device="cuda")
    mlp.pairs(op, torch.tensor(x, device="cuda"), torch.tensor(xstar, device="cuda"),
              torch.tensor(cells, device="cuda"), torch.tensor(rows, device="cuda"), X, E,
              subtract_block_jacobi=subtract)
    Xh, Eh = X.float().cpu().numpy(), E.cpu().numpy()
    logD = np.log(w.D)
    nx, ny, nz = w.n
    E_ref = np.zeros_like(Eh, dtype=np.float64)
    for c, row in zip(cells, rows):
        ic = [c % nx, (c // nx) % ny, c // (nx * ny)]
        nbr = [c]
        for d, st, nn in ((0, 1, nx), (1, nx, ny), (2, nx * ny, nz)):
            nbr.append(c - st if ic[d] > 0 else c)
            nbr.append(c + st if ic[d] < nn - 1 else c)
        feat, s = om.features(r[c * nb:(c + 1) * nb], logD[nbr], mlp.kinp)
        ref = om.bf16_round(feat)
        assert np.max(np.abs(Xh[row] - ref)) <= 2 ** -7 * np.max(np.abs(ref)), (c, row)
        E_ref[row] = e[c * nb:(c + 1) * nb] / s
        assert np.max(np.abs(Eh[row] - E_ref[row])) <= 1e-6 * np.max(np.abs(E_ref[row])), (c, row)
    t = mlp.normalize_targets(E)
    rms = np.sqrt(np.mean(E_ref ** 2))
    assert abs(t - rms) <= 1e-6 * rms
    assert np.max(np.abs(E.cpu().numpy() - E_ref / rms)) <= 1e-6 * np.max(np.abs(E_ref / rms))
    assert mlp.params()[1] == pytest.approx(t)
    op.close()
    mlp.close()
