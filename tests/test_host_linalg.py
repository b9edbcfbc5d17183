"""Host dense linear algebra of the library (csrc/host_linalg.h: Cholesky inverse of an overlap and
the Jacobi eigen-decomposition of a Hermitian matrix), compiled into a small harness with the host
C++ compiler and checked against numpy on random matrices (CPU only)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_1804_01404_gb300", "csrc", "host_linalg.h")

HARNESS = r"""
#include <cstdio>
#include "host_linalg.h"
// stdin: mode n, then n*n (re, im) row-major.  mode 0: herm_eig -> w[n], then Y (re, im);
// mode 1: cholesky_inverse_h -> ok, then C (re, im).
int main() {
  int mode, n;
  if (std::scanf("%d %d", &mode, &n) != 2) return 2;
  std::vector<std::complex<double>> A((size_t)n * n);
  for (auto& a : A) { double re, im; if (std::scanf("%lf %lf", &re, &im) != 2) return 2; a = {re, im}; }
  if (mode == 0) {
    std::vector<double> w;
    std::vector<std::complex<double>> Y;
    tdks::herm_eig(A, n, w, Y);
    for (double x : w) std::printf("%.17g\n", x);
    for (auto& y : Y) std::printf("%.17g %.17g\n", y.real(), y.imag());
  } else {
    std::vector<std::complex<double>> C((size_t)n * n);
    std::printf("%d\n", tdks::cholesky_inverse_h(A.data(), n, C.data()) ? 1 : 0);
    for (auto& c : C) std::printf("%.17g %.17g\n", c.real(), c.imag());
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("linalg")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    exe = d / "h"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    return str(exe)


def _run(exe, mode, A):
    n = A.shape[0]
    text = f"{mode} {n}\n" + "\n".join(f"{z.real:.17g} {z.imag:.17g}" for z in A.ravel()) + "\n"
    out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout.split()
    return [float(x) for x in out]


def _random_hermitian(rng, n):
    B = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    return 0.5 * (B + B.conj().T)


@pytest.mark.parametrize("n", [1, 2, 5, 17, 64])
def test_herm_eig_against_numpy(harness, n):
    rng = np.random.default_rng(n)
    A = _random_hermitian(rng, n)
    v = _run(harness, 0, A)
    w = np.array(v[:n])
    Y = (np.array(v[n::2]) + 1j * np.array(v[n + 1::2])).reshape(n, n)
    scale = np.max(np.abs(np.linalg.eigvalsh(A)))
    assert np.all(np.diff(w) >= 0)
    assert np.max(np.abs(w - np.linalg.eigvalsh(A))) < 1e-12 * scale
    assert np.max(np.abs(A @ Y - Y * w[None, :])) < 1e-12 * scale
    assert np.max(np.abs(Y.conj().T @ Y - np.eye(n))) < 1e-12


def test_herm_eig_degenerate(harness):
    """A fourfold and a twofold eigenvalue, hidden by a random unitary: the eigenvectors of each
    eigenspace come out orthonormal."""
    rng = np.random.default_rng(7)
    Q, _ = np.linalg.qr(rng.normal(size=(6, 6)) + 1j * rng.normal(size=(6, 6)))
    A = Q @ np.diag([1.0, 1.0, 1.0, 1.0, 2.5, 2.5]) @ Q.conj().T
    A = 0.5 * (A + A.conj().T)
    v = _run(harness, 0, A)
    w = np.array(v[:6])
    Y = (np.array(v[6::2]) + 1j * np.array(v[7::2])).reshape(6, 6)
    assert np.allclose(w, [1, 1, 1, 1, 2.5, 2.5], atol=1e-13)
    assert np.max(np.abs(Y.conj().T @ Y - np.eye(6))) < 1e-13
    assert np.max(np.abs(A @ Y - Y * w[None, :])) < 1e-13


@pytest.mark.parametrize("n", [1, 3, 16, 64])
def test_cholesky_inverse(harness, n):
    """C = L^{-H} of S = L L^H: upper triangular, C^H S C = I; a singular S is refused."""
    rng = np.random.default_rng(100 + n)
    B = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    S = B.conj().T @ B + 0.5 * np.eye(n)
    v = _run(harness, 1, S)
    assert v[0] == 1.0
    C = (np.array(v[1::2]) + 1j * np.array(v[2::2])).reshape(n, n)
    assert np.max(np.abs(np.tril(C, -1))) == 0.0
    assert np.max(np.abs(C.conj().T @ S @ C - np.eye(n))) < 1e-10
    L = np.linalg.cholesky(S)
    assert np.max(np.abs(C - np.linalg.inv(L).conj().T)) < 1e-10 * np.max(np.abs(C))
    if n > 1:
        Sz = S.copy()
        Sz[:, 0] = Sz[:, 1]
        Sz[0, :] = Sz[1, :]                         # two equal rows and columns: singular
        assert _run(harness, 1, Sz)[0] == 0.0
