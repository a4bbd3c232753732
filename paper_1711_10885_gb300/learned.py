"""Training of the learned per-element preconditioner on pairs produced by the solver itself.

Only orchestration lives here: every numerical step is a call into libdg.so (solves, the residual and the
feature and target rows of the sampled cells, their normalisation, forward/backward/Adam kernels); torch only
provides the device buffers and numpy the seeded sampling.  The pairs are (cell residual, cell error) taken
from FGMRES iterates x_i of the plain FP64 block-Jacobi solve:
    r_i = F - A x_i,   e_i = x* - x_i   (x* from a tight solve),
restricted to uniformly sampled cells.  With the network input normalised by s = ||r_T|| the target of a cell
is e_T / (s * t_scale), t_scale being the RMS of e_T / s over the training set.
"""

from __future__ import annotations

import numpy as np

from . import dg


def solver_pairs(workloads, mlp, pairs_per_problem, snapshots=(0, 3, 8, 16, 32, 64), seed=0, restart=30,
                 verbose=False, minus_block_jacobi=False):
    """(X, E) with X the BF16 feature rows and E = e_T / s (FP32), over all workloads and snapshots, in a
    seeded random row order (each sample is written straight to its shuffled row).

    minus_block_jacobi: the target is the part of the error that block-Jacobi misses, e - BJ(r)
    (for the block-Jacobi + network preconditioner)."""
    import torch
    rng = np.random.default_rng(seed)
    per_snap = max(1, pairs_per_problem // len(snapshots))
    counts = [min(per_snap, w.ncell) for w in workloads for _ in snapshots]
    total = int(sum(counts))
    X = torch.empty((total, mlp.kinp), dtype=torch.bfloat16, device="cuda")
    E = torch.empty((total, mlp.nb), dtype=torch.float32, device="cuda")
    dest = rng.permutation(total).astype(np.int32)
    pos = 0
    for w in workloads:
        op = dg.operator_for(w)
        op.precond_setup()
        xstar = torch.zeros(w.ndof, dtype=torch.float64, device="cuda")
        # the reference solution only has to be accurate relative to the errors of the early iterates;
        # 1e-9 stays above the attainable FP64 residual of high-contrast problems
        op.solve(xstar, mode=dg.DG_SOLVE_MIXED, preconditioner=dg.DG_PRECOND_BLOCK_JACOBI, rtol=1e-9,
                 inner_rtol=1e-3, max_iterations=2000, raise_on_error=False)
        x = torch.zeros_like(xstar)
        done = 0
        for target in snapshots:
            if target > done:
                op.solve(x, mode=dg.DG_SOLVE_FP64, preconditioner=dg.DG_PRECOND_BLOCK_JACOBI, restart=restart,
                         max_iterations=target - done, rtol=1e-14, raise_on_error=False)
                done = target
            k = min(per_snap, w.ncell)
            cells = torch.tensor(np.sort(rng.choice(w.ncell, k, replace=False)).astype(np.int32), device="cuda")
            rows = torch.tensor(dest[pos:pos + k], device="cuda")
            mlp.pairs(op, x, xstar, cells, rows, X, E, subtract_block_jacobi=minus_block_jacobi)
            pos += k
            if verbose:
                print(f"{w.name}: snapshot {target}: {k} pairs")
        op.close()
    return X, E


def train_preconditioner(workloads, k, pairs=20000, epochs=60, batch=256, lr=1e-3, seed=0, verbose=False,
                         minus_block_jacobi=True, snapshots=(0, 3, 8, 16, 32, 64)):
    """New MLP for degree k trained on solver pairs of the given workloads; returns (mlp, info)."""
    mlp = dg.MLP(k, seed=seed)
    X, E = solver_pairs(workloads, mlp, max(1, pairs // max(1, len(workloads))), seed=seed, verbose=verbose,
                        minus_block_jacobi=minus_block_jacobi, snapshots=snapshots)
    t_scale = mlp.normalize_targets(E)
    st = mlp.train(X, E, epochs=epochs, batch=min(batch, X.shape[0]), lr=lr)
    info = {"pairs": int(X.shape[0]), "t_scale": t_scale, **st}
    return mlp, info
