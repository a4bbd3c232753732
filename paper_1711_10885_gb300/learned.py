"""Training of the learned per-element preconditioner on pairs produced by the solver itself.

Only orchestration lives here: every numerical step is a call into libdg.so (solves, residual
applications, feature gathering, forward/backward/Adam kernels).  The pairs are (cell residual,
cell error) taken from FGMRES iterates x_i of the plain FP64 block-Jacobi solve:
    r_i = b - A x_i,   e_i = x* - x_i   (x* from a tight solve),
restricted to uniformly sampled cells.  With the network input normalised by s = ||r_T|| the target
of a cell is e_T / (s * t_scale), t_scale being the RMS of e_T / s over the training set.
"""

from __future__ import annotations

import numpy as np

from . import dg


def solver_pairs(workloads, mlp, pairs_per_problem, snapshots=(0, 3, 8, 16, 32, 64), seed=0, restart=30,
                 verbose=False, minus_block_jacobi=False):
    """(X, E) with X the BF16 feature rows and E = e_T / s (FP32), over all workloads and snapshots.

    minus_block_jacobi: the target is the part of the error that block-Jacobi misses, e - BJ(r)
    (for the block-Jacobi + network preconditioner)."""
    import torch
    rng = np.random.default_rng(seed)
    Xs, Es = [], []
    per_snap = max(1, pairs_per_problem // len(snapshots))
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
            r = -op.apply_residual(x)  # b - A x
            e = xstar - x
            if minus_block_jacobi:
                e = e - op.precond_apply(r)
            cells = torch.tensor(np.sort(rng.choice(w.ncell, min(per_snap, w.ncell), replace=False)),
                                 dtype=torch.int32, device="cuda")
            X, s = mlp.features(op, r, cells)
            E = e.view(w.ncell, w.nb)[cells.long()].float()
            keep = s > 0
            Xs.append(X[keep])
            Es.append(E[keep] / s[keep, None])
            if verbose:
                print(f"{w.name}: snapshot {target}: |r| {float(r.norm()):.3e}")
        op.close()
    return torch.cat(Xs), torch.cat(Es)


def train_preconditioner(workloads, k, pairs=20000, epochs=60, batch=256, lr=1e-3, seed=0, verbose=False,
                         minus_block_jacobi=True, snapshots=(0, 3, 8, 16, 32, 64)):
    """New MLP for degree k trained on solver pairs of the given workloads; returns (mlp, info)."""
    import torch
    mlp = dg.MLP(k, seed=seed)
    X, E = solver_pairs(workloads, mlp, max(1, pairs // max(1, len(workloads))), seed=seed, verbose=verbose,
                        minus_block_jacobi=minus_block_jacobi, snapshots=snapshots)
    t_scale = float(torch.sqrt(torch.mean(E.double() ** 2)))
    T = (E / t_scale).contiguous()
    mlp.set_target_scale(t_scale)
    perm = torch.randperm(X.shape[0], generator=torch.Generator().manual_seed(seed)).to(X.device)
    X = X[perm].contiguous()
    T = T[perm].contiguous()
    st = mlp.train(X, T, epochs=epochs, batch=min(batch, X.shape[0]), lr=lr)
    info = {"pairs": int(X.shape[0]), "t_scale": t_scale, **st}
    return mlp, info
