// Wigner's small d^J_(m'm)(beta) through a Jacobi polynomial, for host and device code.
//
// With k = min(J+m, J-m, J+m', J-m') the matrix element is
//   d = (-1)^lam sqrt(C(2J-k, k+a) / C(k+b, b)) sin(beta/2)^a cos(beta/2)^b P_k^(a,b)(cos beta),
// where (a, lam) = (m'-m, m'-m) if k = J+m or k = J-m', and (m-m', 0) otherwise, and
// b = 2J - 2k - a (the standard Jacobi-polynomial form of the rotation matrix; see e.g.
// Biedenharn and Louck). P_k^(a,b) comes from its three-term recurrence in k, which stays
// accurate where Wigner's explicit alternating sum loses digits (about 1e-7 at J = 40).
#pragma once

#include <cmath>

#ifdef __CUDACC__
#define MW3_HD __host__ __device__
#else
#define MW3_HD
#endif

namespace mw3 {

struct WignerIdx {
  int k, a, b;
  int sign;   // (-1)^lam
};

MW3_HD inline WignerIdx wigner_index(int J, int mp, int m) {
  int k = J + m;
  if (J - m < k) k = J - m;
  if (J + mp < k) k = J + mp;
  if (J - mp < k) k = J - mp;
  int a, lam;
  if (k == J + m) {
    a = mp - m;
    lam = mp - m;
  } else if (k == J - m) {
    a = m - mp;
    lam = 0;
  } else if (k == J + mp) {
    a = m - mp;
    lam = 0;
  } else {
    a = mp - m;
    lam = mp - m;
  }
  WignerIdx w;
  w.k = k;
  w.a = a;
  w.b = 2 * J - 2 * k - a;
  w.sign = (lam & 1) ? -1 : 1;
  return w;
}

// sqrt(C(2J-k, k+a) / C(k+b, b)) (host: lgamma of the C library).
inline double wigner_prefactor(int J, const WignerIdx& w) {
  const double l = std::lgamma(2.0 * J - w.k + 1) - std::lgamma(w.k + w.a + 1.0) -
                   std::lgamma(2.0 * J - 2 * w.k - w.a + 1) -
                   (std::lgamma(w.k + w.b + 1.0) - std::lgamma(w.k + 1.0) - std::lgamma(w.b + 1.0));
  return std::exp(0.5 * l);
}

// P_n^(a,b)(x) by the three-term recurrence in n.
MW3_HD inline double jacobi_p(int n, int a, int b, double x) {
  if (n == 0) return 1.0;
  double p0 = 1.0, p1 = (a + 1) + 0.5 * (a + b + 2) * (x - 1.0);
  for (int j = 2; j <= n; ++j) {
    const double c = 2.0 * j + a + b;
    const double A = 2.0 * j * (j + a + b) * (c - 2.0);
    const double B = (c - 1.0) * (c * (c - 2.0) * x + (double)a * a - (double)b * b);
    const double C = 2.0 * (j + a - 1.0) * (j + b - 1.0) * c;
    const double p2 = (B * p1 - C * p0) / A;
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

// d from its index data and prefactor, given sin(beta/2), cos(beta/2) and cos(beta).
MW3_HD inline double wigner_d_eval(const WignerIdx& w, double pref, double sh, double ch,
                                   double cb) {
  double v = pref * jacobi_p(w.k, w.a, w.b, cb);
  for (int i = 0; i < w.a; ++i) v *= sh;
  for (int i = 0; i < w.b; ++i) v *= ch;
  return w.sign * v;
}

inline double wigner_small_d_jacobi(int J, int mp, int m, double beta) {
  const WignerIdx w = wigner_index(J, mp, m);
  return wigner_d_eval(w, wigner_prefactor(J, w), std::sin(0.5 * beta), std::cos(0.5 * beta),
                       std::cos(beta));
}

}  // namespace mw3
