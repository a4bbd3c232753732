"""The recurrences of the FGMRES Arnoldi step with the reorthogonalisation delayed by one step (the host logic of
csrc/dg_solve.cu), written out in plain FP64 numpy on small dense systems.  The library runs them on the GPU; this
model checks the algebra they rest on:

* A Z = V Hbar with V orthonormal, where z_j = M_j(u_j) is the preconditioned *provisional* row and column j of H
  is completed one step later (c + beta a', beta alpha');
* the least-squares residual estimate |g_m| equals the true residual of x0 + Z y (FGMRES with a preconditioner
  that changes at every step);
* the solve converges to the dense solution.
"""

import numpy as np


def delayed_fgmres_cycle(A, b, x0, m, precs, contaminate=0.0, mutant=None):
    """One FGMRES(m) cycle; precs[j] is the preconditioner of step j (a matrix, different at every step).
    contaminate is added to every coefficient c_0 = v_0 . w before pass 2 (an error of known size in a dot
    product, which leaves the provisional row that much off orthogonal to v_0);
    mutant plants a mistake: "no_lag" completes column j-1 without the term beta a', "no_reorth" keeps the
    provisional row as the final one."""
    n = len(b)
    r0 = b - A @ x0
    beta = np.linalg.norm(r0)
    V = np.zeros((m + 1, n))
    Z = np.zeros((m, n))
    H = np.zeros((m + 1, m))
    V[0] = r0 / beta
    cprev = None
    btil = 0.0
    for j in range(m):
        u = V[j]
        Z[j] = precs[j] @ u                      # precondition the provisional row
        w = A @ Z[j]
        # pass 1: dots of rows 0..j with u_j and with w, and w . w
        pu = V[: j + 1] @ u
        qw = V[: j + 1] @ w
        ww = w @ w
        if j > 0:
            a = pu[:j]
            alpha = np.sqrt(pu[j] - a @ a)
            if mutant == "no_reorth":
                a, alpha = np.zeros(j), np.sqrt(pu[j])
            H[:j, j - 1] = cprev + (0.0 if mutant == "no_lag" else btil) * a  # column j-1, one step late
            H[j, j - 1] = btil * alpha
        else:
            a, alpha = np.zeros(0), 1.0
        c = np.empty(j + 1)
        c[:j] = qw[:j]
        c[j] = (qw[j] - a @ qw[:j]) / alpha
        c[0] += contaminate
        btil = np.sqrt(ww - c @ c)
        # pass 2: final v_j and the next provisional row
        e = c[j] / alpha
        d = c[:j] - e * a
        vj = (u - a @ V[:j]) / alpha
        V[j + 1] = (w - d @ V[:j] - e * u) / btil
        V[j] = vj
        cprev = c
    # finalise the last column: reorthogonalisation of u_m against rows 0..m-1
    pu = V[:m] @ V[m]
    alpha = np.sqrt(V[m] @ V[m] - pu @ pu)
    H[:m, m - 1] = cprev + btil * pu
    H[m, m - 1] = btil * alpha
    Vfin = V.copy()
    Vfin[m] = (V[m] - pu @ V[:m]) / alpha
    g = np.zeros(m + 1)
    g[0] = beta
    y, *_ = np.linalg.lstsq(H, g, rcond=None)
    est = np.linalg.norm(g - H @ y)
    return Vfin, Z, H, x0 + y @ Z, est


def test_delayed_reorthogonalisation_keeps_the_arnoldi_relation():
    rng = np.random.default_rng(11)
    for n, m in ((40, 12), (80, 30)):
        A = np.eye(n) * 2.0 + rng.standard_normal((n, n)) / np.sqrt(n)
        b = rng.standard_normal(n)
        precs = [np.eye(n) + 0.2 * rng.standard_normal((n, n)) / np.sqrt(n) for _ in range(m)]
        V, Z, H, x, est = delayed_fgmres_cycle(A, b, np.zeros(n), m, precs)
        assert np.max(np.abs(V @ V.T - np.eye(m + 1))) <= 1e-12
        assert np.max(np.abs(A @ Z.T - V.T @ H)) <= 1e-12 * np.max(np.abs(A @ Z.T))
        true = np.linalg.norm(b - A @ x)
        assert abs(est - true) <= 1e-10 * np.linalg.norm(b)


def test_delayed_fgmres_converges_to_the_dense_solution():
    rng = np.random.default_rng(12)
    n, m = 60, 20
    A = np.eye(n) * 3.0 + rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    x = np.zeros(n)
    for cycle in range(6):
        precs = [np.eye(n) + 0.1 * rng.standard_normal((n, n)) / np.sqrt(n) for _ in range(m)]
        *_, x, est = delayed_fgmres_cycle(A, b, x, m, precs)
    xs = np.linalg.solve(A, b)
    assert np.linalg.norm(x - xs) <= 1e-10 * np.linalg.norm(xs)


def test_the_lagged_column_absorbs_the_reorthogonalisation():
    """A planted error of 1e-6 in every coefficient v_0 . w (the size of an FP32 dot-product error) leaves each
    provisional row that much off orthogonal to v_0.  The next step measures it (a'), removes it from the final
    row and returns beta a' to the lagged column, so A Z = V Hbar and V^T V = I hold to rounding.  Dropping beta
    a' breaks the relation; keeping the provisional row breaks the orthogonality."""
    rng = np.random.default_rng(13)
    n, m = 50, 15
    A = np.eye(n) * 2.0 + rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    precs = [np.eye(n) + 0.2 * rng.standard_normal((n, n)) / np.sqrt(n) for _ in range(m)]

    def errors(mutant):
        V, Z, H, x, est = delayed_fgmres_cycle(A, b, np.zeros(n), m, precs, contaminate=1e-6, mutant=mutant)
        return (np.max(np.abs(V @ V.T - np.eye(m + 1))),
                np.max(np.abs(A @ Z.T - V.T @ H)) / np.max(np.abs(A @ Z.T)))

    orth, rel = errors(None)
    assert orth <= 1e-12 and rel <= 1e-12
    assert errors("no_lag")[1] > 1e-8
    assert errors("no_reorth")[0] > 1e-8
