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
    std::printf("%d\n", ok ? 1 : 0);
    for (int i = 0; i < n; ++i) std::printf("%.17g %.17g\n", lam[i].real(), lam[i].imag());
    for (int i = 0; i < n * n; ++i) std::printf("%.17g %.17g\n", V[i].real(), V[i].imag());
    for (int i = 0; i < n * n; ++i) std::printf("%.17g %.17g\n", W[i].real(), W[i].imag());
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
    pos, res = 0, []
    for A in mats:
        n = A.shape[0]
        ok = int(out[pos])
        pos += 1
        vals = np.array([float(x) for x in out[pos:pos + 2 * (n + 2 * n * n)]])
        pos += 2 * (n + 2 * n * n)
        c = vals[0::2] + 1j * vals[1::2]
        res.append((ok, c[:n], c[n:n + n * n].reshape(n, n), c[n + n * n:].reshape(n, n)))
    return res


def test_eigen_decomposition_matches_lapack(driver):
    rng = np.random.default_rng(0)
    mats = [rng.standard_normal((n, n)) for n in (1, 2, 3, 5, 8, 11, 12)]
    mats += [dg_1d_operator(k, rng) for k in (1, 2, 4, 7, 10)]
    S = rng.standard_normal((9, 9))
    mats.append(S + S.T + 1e-3 * rng.standard_normal((9, 9)))  # nearly symmetric, real spectrum
    for A, (ok, lam, V, W) in zip(mats, run(driver, mats)):
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
