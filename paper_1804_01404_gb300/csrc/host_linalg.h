// Dense linear algebra of the small norb x norb matrices, on the host (the overlaps and projected
// Hamiltonians of the ground-state iteration and of the Ritz rotation).  Row-major, complex.
//
// cholesky_inverse_h: Cholesky S = L L^H of a Hermitian positive definite n x n matrix and
// C = L^{-H} (upper triangular), so that the combinations W C of vectors with overlap S are
// orthonormal (C^H S C = I).  False if S is not positive definite.
//
// herm_eig: eigen-decomposition of a Hermitian matrix by cyclic Jacobi rotations,
// A = Y diag(w) Y^H with w ascending and Y unitary.  Each rotation zeroes one off-diagonal pair
// (p, q): the phase of a_pq is moved into column q (D = diag(1, e^{-i phi}) turns the 2 x 2 block
// into the real symmetric [[a, r], [r, b]], r = |a_pq|), then the real Jacobi rotation with
// cot(2 theta) = (b - a) / (2 r) zeroes it.  Sweeps over all pairs until the off-diagonal norm is
// below 1e-15 of the matrix norm (at most 100 sweeps).
#pragma once

#include <algorithm>
#include <cmath>
#include <complex>
#include <numeric>
#include <vector>

namespace tdks {

inline bool cholesky_inverse_h(const std::complex<double>* S, int n, std::complex<double>* Cout) {
  std::vector<double> Lr((size_t)n * n, 0.0), Li((size_t)n * n, 0.0), Xr((size_t)n * n, 0.0), Xi((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double d = S[j * n + j].real();
    for (int k = 0; k < j; ++k) d -= Lr[j * n + k] * Lr[j * n + k] + Li[j * n + k] * Li[j * n + k];
    if (!(d > 0.0)) return false;
    const double ljj = std::sqrt(d);
    Lr[j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double re = S[i * n + j].real(), im = S[i * n + j].imag();
      for (int k = 0; k < j; ++k) {   // - L_ik conj(L_jk)
        re -= Lr[i * n + k] * Lr[j * n + k] + Li[i * n + k] * Li[j * n + k];
        im -= Li[i * n + k] * Lr[j * n + k] - Lr[i * n + k] * Li[j * n + k];
      }
      Lr[i * n + j] = re / ljj;
      Li[i * n + j] = im / ljj;
    }
  }
  for (int j = 0; j < n; ++j) {          // X = L^{-1} by forward substitution, column by column
    Xr[j * n + j] = 1.0 / Lr[j * n + j];
    for (int i = j + 1; i < n; ++i) {
      double re = 0.0, im = 0.0;
      for (int k = j; k < i; ++k) {
        re += Lr[i * n + k] * Xr[k * n + j] - Li[i * n + k] * Xi[k * n + j];
        im += Lr[i * n + k] * Xi[k * n + j] + Li[i * n + k] * Xr[k * n + j];
      }
      Xr[i * n + j] = -re / Lr[i * n + i];
      Xi[i * n + j] = -im / Lr[i * n + i];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Cout[i * n + j] = std::complex<double>(Xr[j * n + i], -Xi[j * n + i]);   // C = X^H
  return true;
}

inline void herm_eig(std::vector<std::complex<double>> A, int n, std::vector<double>& w,
                     std::vector<std::complex<double>>& Y) {
  using Z = std::complex<double>;
  Y.assign((size_t)n * n, Z(0.0, 0.0));
  for (int i = 0; i < n; ++i) Y[(size_t)i * n + i] = 1.0;
  auto at = [&](int i, int j) -> Z& { return A[(size_t)i * n + j]; };
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const double m = std::norm(at(i, j));
        tot += m;
        if (i != j) off += m;
      }
    if (off <= 1e-30 * tot || off == 0.0) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double r = std::abs(at(p, q));
        if (r == 0.0) continue;
        const Z ph = at(p, q) / r;                                  // e^{i phi}
        const double a = at(p, p).real(), b = at(q, q).real();
        const double tau = (b - a) / (2.0 * r);
        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        // U on columns p, q: [[c, s], [-s e^{-i phi}, c e^{-i phi}]]
        const Z upp = c, upq = s, uqp = -s * std::conj(ph), uqq = c * std::conj(ph);
        for (int k = 0; k < n; ++k) {                               // A <- A U
          const Z akp = at(k, p), akq = at(k, q);
          at(k, p) = akp * upp + akq * uqp;
          at(k, q) = akp * upq + akq * uqq;
        }
        for (int k = 0; k < n; ++k) {                               // A <- U^H A
          const Z apk = at(p, k), aqk = at(q, k);
          at(p, k) = std::conj(upp) * apk + std::conj(uqp) * aqk;
          at(q, k) = std::conj(upq) * apk + std::conj(uqq) * aqk;
        }
        at(p, q) = at(q, p) = 0.0;
        at(p, p) = at(p, p).real();
        at(q, q) = at(q, q).real();
        for (int k = 0; k < n; ++k) {                               // Y <- Y U
          const Z ykp = Y[(size_t)k * n + p], ykq = Y[(size_t)k * n + q];
          Y[(size_t)k * n + p] = ykp * upp + ykq * uqp;
          Y[(size_t)k * n + q] = ykp * upq + ykq * uqq;
        }
      }
  }
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int i, int j) { return at(i, i).real() < at(j, j).real(); });
  w.resize(n);
  std::vector<Z> Ys((size_t)n * n);
  for (int jn = 0; jn < n; ++jn) {
    w[jn] = at(order[jn], order[jn]).real();
    for (int k = 0; k < n; ++k) Ys[(size_t)k * n + jn] = Y[(size_t)k * n + order[jn]];
  }
  Y.swap(Ys);
}

}  // namespace tdks
