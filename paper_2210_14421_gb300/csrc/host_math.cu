// Host-side numerics of the set-up: quadrature rules, Lagrange tables and a
// symmetric eigensolver (Sec. "Spectral finite elements", Eq. MSquareRoot).
#include <cmath>
#include <vector>

#include "efe_internal.h"

namespace efe {

// Legendre P_n(x) and P_{n-1}(x) by the three-term recurrence.
static void legendre_pair(int n, double x, double& pn, double& pnm1) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { pn = 1.0; pnm1 = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  pn = p1;
  pnm1 = p0;
}

// n-point Gauss-Legendre rule: Newton iteration on P_n from the classical
// cosine guesses; w_i = 2 / ((1 - x_i^2) P_n'(x_i)^2).
void gauss_legendre(int n, double* x, double* w) {
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = -std::cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double pn, pnm1;
      legendre_pair(n, z, pn, pnm1);
      dp = n * (z * pn - pnm1) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double pn, pnm1;
    legendre_pair(n, z, pn, pnm1);
    dp = n * (z * pn - pnm1) / (z * z - 1.0);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// (p+1)-point Gauss-Lobatto-Legendre rule: end points and the zeros of P_p',
// found by Newton with P_p'' from the Legendre equation; w = 2 / (p(p+1) P_p^2).
void gauss_lobatto(int p, double* x, double* w) {
  const double pi = 3.14159265358979323846;
  x[0] = -1.0;
  x[p] = 1.0;
  for (int i = 1; i < p; ++i) {
    double z = -std::cos(pi * i / p);
    for (int it = 0; it < 100; ++it) {
      double pn, pnm1;
      legendre_pair(p, z, pn, pnm1);
      double d1 = p * (pnm1 - z * pn) / (1.0 - z * z);
      double d2 = (2.0 * z * d1 - p * (p + 1.0) * pn) / (1.0 - z * z);
      double dz = d1 / d2;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
  }
  for (int i = 0; i <= p; ++i) {
    double pn, pnm1;
    legendre_pair(p, x[i], pn, pnm1);
    w[i] = 2.0 / (p * (p + 1.0) * pn * pn);
  }
}

// L[k * n + i] = l_i(pts_k), dL likewise for l_i'.
void lagrange_tables(int n, const double* nodes, int m, const double* pts, double* L, double* dL) {
  for (int k = 0; k < m; ++k) {
    double x = pts[k];
    for (int i = 0; i < n; ++i) {
      double v = 1.0;
      for (int j = 0; j < n; ++j)
        if (j != i) v *= (x - nodes[j]) / (nodes[i] - nodes[j]);
      double d = 0.0;
      for (int a = 0; a < n; ++a) {
        if (a == i) continue;
        double t = 1.0 / (nodes[i] - nodes[a]);
        for (int j = 0; j < n; ++j)
          if (j != i && j != a) t *= (x - nodes[j]) / (nodes[i] - nodes[j]);
        d += t;
      }
      L[k * n + i] = v;
      dL[k * n + i] = d;
    }
  }
}

// Cyclic Jacobi eigensolver for a symmetric n x n matrix (row-major).  On
// return A is destroyed, V holds the eigenvectors in its columns and lam the
// eigenvalues.  Returns false if the sweep limit is reached.
bool jacobi_eigen(int n, std::vector<double>& A, std::vector<double>& V, std::vector<double>& lam) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  lam.assign(n, 0.0);
  double total = 0.0;
  for (double v : A) total += v * v;
  bool ok = false;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += A[(size_t)i * n + j] * A[(size_t)i * n + j];
    if (off <= 1e-32 * total || off == 0.0) { ok = true; break; }
    for (int pp = 0; pp < n; ++pp) {
      for (int q = pp + 1; q < n; ++q) {
        double apq = A[(size_t)pp * n + q];
        if (apq == 0.0) continue;
        double app = A[(size_t)pp * n + pp], aqq = A[(size_t)q * n + q];
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {   // columns p, q of A
          double akp = A[(size_t)k * n + pp], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + pp] = c * akp - s * akq;
          A[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {   // rows p, q
          double apk = A[(size_t)pp * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)pp * n + k] = c * apk - s * aqk;
          A[(size_t)q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = V[(size_t)k * n + pp], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + pp] = c * vkp - s * vkq;
          V[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
    }
  }
  for (int i = 0; i < n; ++i) lam[i] = A[(size_t)i * n + i];
  return ok;
}

}  // namespace efe
