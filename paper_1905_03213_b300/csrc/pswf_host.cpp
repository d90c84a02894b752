// Prolate spheroidal wave function psi_0(c, x) by its Legendre expansion (host side).
//
// psi_0 is the even eigenfunction of the prolate operator
//     L psi = -((1 - x^2) psi')' + c^2 x^2 psi
// with the smallest eigenvalue. In the orthonormal Legendre basis Pn_k = sqrt(k + 1/2) P_k
// the operator is tridiagonal and splits into even and odd degrees:
//     <Pn_k, L Pn_k>     = k (k + 1) + c^2 (2k^2 + 2k - 1) / ((2k + 3)(2k - 1))
//     <Pn_{k+2}, L Pn_k> = c^2 (k + 1)(k + 2) / ((2k + 3) sqrt((2k + 1)(2k + 5)))
// (from x P_k = ((k+1) P_{k+1} + k P_{k-1}) / (2k+1) and the Legendre equation), the
// method of Xiao, Rokhlin & Yarvin (2001). The even block is diagonalised by cyclic
// Jacobi rotations; the eigenvector of the smallest eigenvalue gives the coefficients.
// The W-projection taper is t(x) = psi_0(c, x) / psi_0(c, 0) with c = pi S_min / 2.
#include <cmath>
#include <vector>

#include "internal.h"

namespace wp {

static void jacobi_eigen(std::vector<double>& a, int n, std::vector<double>& v) {
  v.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) v[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < n; ++i) {
      diag += a[(size_t)i * n + i] * a[(size_t)i * n + i];
      for (int j = i + 1; j < n; ++j) off += a[(size_t)i * n + j] * a[(size_t)i * n + j];
    }
    if (off <= 1e-34 * diag) break;
    for (int p = 0; p < n; ++p) {
      for (int q = p + 1; q < n; ++q) {
        const double apq = a[(size_t)p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double app = a[(size_t)p * n + p], aqq = a[(size_t)q * n + q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          const double akp = a[(size_t)k * n + p], akq = a[(size_t)k * n + q];
          a[(size_t)k * n + p] = c * akp - s * akq;
          a[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          const double apk = a[(size_t)p * n + k], aqk = a[(size_t)q * n + k];
          a[(size_t)p * n + k] = c * apk - s * aqk;
          a[(size_t)q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = v[(size_t)k * n + p], vkq = v[(size_t)k * n + q];
          v[(size_t)k * n + p] = c * vkp - s * vkq;
          v[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
    }
  }
}

std::vector<double> pswf_legendre_coefficients(double c) {
  const int n = 30 + (int)std::ceil(c);  // even degrees 0, 2, .., 2(n-1)
  std::vector<double> a((size_t)n * n, 0.0);
  const double c2 = c * c;
  for (int i = 0; i < n; ++i) {
    const double k = 2.0 * i;
    a[(size_t)i * n + i] = k * (k + 1.0) + c2 * (2.0 * k * k + 2.0 * k - 1.0) / ((2.0 * k + 3.0) * (2.0 * k - 1.0));
    if (i + 1 < n) {
      const double off = c2 * (k + 1.0) * (k + 2.0) / ((2.0 * k + 3.0) * std::sqrt((2.0 * k + 1.0) * (2.0 * k + 5.0)));
      a[(size_t)i * n + i + 1] = off;
      a[(size_t)(i + 1) * n + i] = off;
    }
  }
  std::vector<double> vec;
  jacobi_eigen(a, n, vec);
  int best = 0;
  for (int i = 1; i < n; ++i)
    if (a[(size_t)i * n + i] < a[(size_t)best * n + best]) best = i;
  std::vector<double> g(n);
  for (int i = 0; i < n; ++i) g[i] = vec[(size_t)i * n + best] * std::sqrt(2.0 * i + 0.5);  // sqrt(k + 1/2), k = 2i
  const double at0 = legendre_even_series(g.data(), n, 0.0);
  for (int i = 0; i < n; ++i) g[i] /= at0;
  return g;
}

}  // namespace wp
