// Reference-element tables for LGL collocation, computed on the host in FP64.
//
// The paper evaluates its DG integrals with Legendre-Gauss-Lobatto
// quadrature (Sec. 4).  On p+1 LGL nodes r_0 = -1 < ... < r_p = 1 (the
// endpoints and the zeros of P_p'), the quadrature weights are
// w_i = 2 / (p (p+1) P_p(r_i)^2) and the derivative of the Lagrange basis
// l_j at r_i is
//     D_ij = P_p(r_i) / (P_p(r_j) (r_i - r_j))   (i != j),
//     D_00 = -p(p+1)/4,  D_pp = p(p+1)/4,  D_ii = 0 otherwise.
#include "tables.h"

#include <cmath>

namespace expdg {

namespace {

// Evaluate P_n(x) and P_n'(x) by the Bonnet recurrence.
void legendre_and_derivative(int n, double x, double* pn, double* dpn) {
  double p0 = 1.0, p1 = x;
  if (n == 0) {
    *pn = 1.0;
    *dpn = 0.0;
    return;
  }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  *pn = p1;
  // P_n'(x) = n (x P_n - P_{n-1}) / (x^2 - 1), valid for |x| < 1
  *dpn = (std::fabs(x) < 1.0) ? n * (x * p1 - p0) / (x * x - 1.0) : 0.5 * n * (n + 1) * (x > 0 ? 1.0 : (n % 2 ? 1.0 : -1.0));
}

}  // namespace

void build_lgl(int p, double* r, double* w, double* D) {
  const int n = p + 1;
  r[0] = -1.0;
  r[p] = 1.0;
  // interior nodes: zeros of P_p'.  Newton on g(x) = P_p'(x) with
  // g'(x) = (2 x P_p' - p (p+1) P_p) / (1 - x^2)  (Legendre's equation).
  for (int i = 1; i < p; ++i) {
    double x = -std::cos(M_PI * i / p);
    for (int it = 0; it < 100; ++it) {
      double pn, dpn;
      legendre_and_derivative(p, x, &pn, &dpn);
      double d2 = (2.0 * x * dpn - p * (p + 1.0) * pn) / (1.0 - x * x);
      double dx = dpn / d2;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    r[i] = x;
  }
  // enforce the exact symmetry r_i = -r_{p-i}
  for (int i = 0; i < n; ++i) {
    double a = 0.5 * (r[i] - r[p - i]);
    r[i] = a;
  }
  r[0] = -1.0;
  r[p] = 1.0;
  double P[EXPDG_MAX_ORDER + 1];
  for (int i = 0; i < n; ++i) {
    double pn, dpn;
    legendre_and_derivative(p, r[i], &pn, &dpn);
    P[i] = pn;
    w[i] = 2.0 / (p * (p + 1.0) * pn * pn);
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      D[i * n + j] = (i == j) ? 0.0 : P[i] / (P[j] * (r[i] - r[j]));
  D[0] = -0.25 * p * (p + 1.0);
  D[p * n + p] = 0.25 * p * (p + 1.0);
}

}  // namespace expdg
