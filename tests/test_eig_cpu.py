"""The small non-symmetric eigen-solver of the fast-diagonalisation block-Jacobi preconditioner
(paper_1711_10885_gb300/csrc/dg_eig.h, host code) against numpy's LAPACK eigen-solver (CPU only).

A host driver compiled with g++ decomposes seeded matrices: real non-symmetric ones with complex pairs, the
1D DG operators it is used for (diffusion, upwind convection, penalty) and nearly symmetric ones.  Checked:
the eigenvalues match numpy's as a multiset, A V = V diag(lambda) and V V^{-1} = I to round-off."""

import os
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1711_10885_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <vector>
#include "dg_eig.h"
int main() {
  int count;
  if (std::scanf("%d", &count) != 1) return 2;
  for (int c = 0; c < count; ++c) {
    int n;
    if (std::scanf("%d", &n) != 1) return 2;
    std::vector<double> A(n * n);
    for (auto& a : A) if (std::scanf("%lf", &a) != 1) return 2;
    std::vector<dge::cd> V(n * n), W(n * n), lam(n);
    const bool ok = dge::eig_general(n, A.data(), V.data(), W.data(), lam.data());
    std::vector<double> Vr(n * n), Wr(n * n), lr(n);
    const bool real = ok && dge::real_decomposition(n, V.data(), lam.data(), Vr.data(), Wr.data(), lr.data());
    std::printf("%d %d\n", ok ? 1 : 0, real ? 1 : 0);
    for (int i = 0; i < n; ++i) std::printf("%.17g %.17g\n", lam[i].real(), lam[i].imag());
    for (int i = 0; i < n * n; ++i) std::printf("%.17g %.17g\n", V[i].real(), V[i].imag());
    for (int i = 0; i < n * n; ++i) std::printf("%.17g %.17g\n", W[i].real(), W[i].imag());
    for (int i = 0; i < n; ++i) std::printf("%.17g\n", real ? lr[i] : 0.0);
    for (int i = 0; i < n * n; ++i) std::printf("%.17g\n", real ? Vr[i] : 0.0);
    for (int i = 0; i < n * n; ++i) std::printf("%.17g\n", real ? Wr[i] : 0.0);
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    d = tmp_path_factory.mktemp("eig")
    src = d / "drv.cpp"
    src.write_text(DRIVER)
    exe = d / "drv"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    return str(exe)


def dg_1d_operator(k, rng):
    """A 1D DG cell operator of the kind the preconditioner decomposes: stiffness and convection of the
    orthonormal Legendre basis on [0,1] plus interior-face penalty / consistency / upwind terms."""
    from tests import kron_reference as kr
    mt = kr.matrices_1d(k)
    D, b, h, sigma = np.exp(rng.standard_normal()), rng.uniform(-2, 2), 0.05, 2.0 * k * (k + 1)
    e0, e1, d0, d1 = mt["e0"], mt["e1"], mt["d0"], mt["d1"]
    A = D / h ** 2 * mt["S"] - b / h * mt["C"]
    w, gam = 0.5, D * sigma / h
    A += (max(b, 0) * np.outer(e1, e1) - w * D / h * (np.outer(e1, d1) + np.outer(d1, e1)) + gam * np.outer(e1, e1)) / h
    A += (max(-b, 0) * np.outer(e0, e0) + w * D / h * (np.outer(e0, d0) + np.outer(d0, e0)) + gam * np.outer(e0, e0)) / h
    return A


def run(driver, mats):
    inp = [str(len(mats))]
    for A in mats:
        inp.append(str(A.shape[0]))
        inp.append(" ".join(repr(float(v)) for v in A.ravel()))
    out = subprocess.run([driver], input="\n".join(inp), capture_output=True, text=True, check=True).stdout.split()
    pos, res, reals = 0, [], []
    for A in mats:
        n = A.shape[0]
        ok, real = int(out[pos]), int(out[pos + 1])
        pos += 2
        vals = np.array([float(x) for x in out[pos:pos + 2 * (n + 2 * n * n)]])
        pos += 2 * (n + 2 * n * n)
        c = vals[0::2] + 1j * vals[1::2]
        res.append((ok, c[:n], c[n:n + n * n].reshape(n, n), c[n + n * n:].reshape(n, n)))
        r = np.array([float(x) for x in out[pos:pos + n + 2 * n * n]])
        pos += n + 2 * n * n
        reals.append((real, r[:n], r[n:n + n * n].reshape(n, n), r[n + n * n:].reshape(n, n)))
    return res, reals


def test_eigen_decomposition_matches_lapack(driver):
    rng = np.random.default_rng(0)
    mats = [rng.standard_normal((n, n)) for n in (1, 2, 3, 5, 8, 11, 12)]
    mats += [dg_1d_operator(k, rng) for k in (1, 2, 4, 7, 10)]
    S = rng.standard_normal((9, 9))
    mats.append(S + S.T + 1e-3 * rng.standard_normal((9, 9)))  # nearly symmetric, real spectrum
    for A, (ok, lam, V, W) in zip(mats, run(driver, mats)[0]):
        n = A.shape[0]
        assert ok, n
        ref = np.linalg.eigvals(A)
        scale = max(np.max(np.abs(ref)), 1e-300)
        # eigenvalues as multisets: greedy matching
        left = list(ref)
        for l in lam:
            j = int(np.argmin([abs(l - r) for r in left]))
            assert abs(l - left[j]) <= 1e-9 * scale, (n, l, left[j])
            left.pop(j)
        assert np.max(np.abs(A @ V - V * lam[None, :])) <= 1e-11 * scale * np.max(np.abs(V))
        assert np.max(np.abs(V @ W - np.eye(n))) <= 1e-9


def test_real_decomposition_of_real_spectra(driver):
    """The real form of the decomposition: produced exactly when the spectrum is real (diffusion-dominated 1D DG
    operators, symmetric matrices), with A Vr = Vr diag(lr) and Vr Wr = I to round-off; refused for matrices
    with complex pairs (a rotation, a convection-dominated operator)."""
    rng = np.random.default_rng(4)
    real_mats = [dg_1d_operator(k, rng) for k in (1, 3, 5, 7)]
    S = rng.standard_normal((6, 6))
    real_mats.append(S + S.T)
    T = np.triu(rng.standard_normal((5, 5)), 1) + np.diag([1.0, 2.0, 3.0, 4.0, 5.0])
    real_mats.append(T)  # distinct real eigenvalues, non-normal
    rot = np.array([[0.0, -1.0], [1.0, 0.0]])
    from tests import kron_reference as kr
    mt = kr.matrices_1d(5)
    conv = 1.0 * mt["S"] - 400.0 * mt["C"] + 50.0 * np.outer(mt["e1"], mt["e1"])  # convection-dominated
    skew = np.eye(7) + np.diag(np.ones(6), 1) - np.diag(np.ones(6), -1)  # I + skew-symmetric: 1 +- i t pairs
    complex_mats = [rot, skew, conv]
    mats = real_mats + complex_mats
    res, reals = run(driver, mats)
    for i, A in enumerate(mats):
        ok, lam = res[i][0], res[i][1]
        real, lr, Vr, Wr = reals[i]
        assert ok
        has_complex = np.max(np.abs(lam.imag)) > 1e-13 * np.max(np.abs(lam))
        assert real == (0 if has_complex else 1), (i, lam)
        if real:
            scale = np.max(np.abs(lr))
            assert np.max(np.abs(A @ Vr - Vr * lr[None, :])) <= 1e-11 * scale * np.max(np.abs(Vr))
            assert np.max(np.abs(Vr @ Wr - np.eye(A.shape[0]))) <= 1e-9
            assert np.allclose(np.linalg.norm(Vr, axis=0), 1.0, atol=1e-14)
            assert np.allclose(np.sort(lr), np.sort(np.linalg.eigvals(A).real), rtol=1e-9, atol=1e-9 * scale)
    assert sum(r[0] for r in reals) == len(real_mats)
