// Host-side set-up mathematics of libmw3 (FP64): quadratures, bases, the
// symmetric eigensolver for the diatomic states, and the built-in LEPS surface.
// These run once per set-up call; the propagation itself runs on the device.
#include "mw3_host.h"
#include "mw3_wigner.h"

#include <algorithm>
#include <cmath>

namespace mw3 {

// Gauss-Legendre nodes (ascending) and weights by Newton iteration on P_n.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));  // i-th largest root estimate
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      if (n == 1) p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      const double pn = (n == 0) ? 1.0 : p1;
      const double pnm1 = (n == 1) ? 1.0 : p0;
      dp = n * (z * pn - pnm1) / (z * z - 1.0);
      const double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16 && it > 2) break;
    }
    // final derivative at the converged root
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    const double pnm1 = (n == 1) ? 1.0 : p0;
    dp = n * (z * p1 - pnm1) / (z * z - 1.0);
    const double wi = 2.0 / ((1.0 - z * z) * dp * dp);
    x[n - 1 - i] = z;
    x[i] = -z;
    w[i] = w[n - 1 - i] = wi;
  }
  if (n % 2 == 1) x[n / 2] = 0.0;
}

// Normalised associated Legendre functions (Condon-Shortley phase), j = om..jmax,
// at points x: out[(j - om) * npts + p].
void norm_assoc_legendre(int jmax, int om, const std::vector<double>& x,
                         std::vector<double>& out) {
  const int np = (int)x.size();
  const int nj = jmax - om + 1;
  out.assign((size_t)nj * np, 0.0);
  double c = 1.0 / std::sqrt(2.0);
  for (int m = 1; m <= om; ++m) c *= -std::sqrt((2.0 * m + 1.0) / (2.0 * m));
  for (int p = 0; p < np; ++p) {
    const double xx = x[p];
    const double s2 = 1.0 - xx * xx;
    double pm2 = c * std::pow(s2, 0.5 * om);
    out[p] = pm2;
    if (nj == 1) continue;
    double pm1 = std::sqrt(2.0 * om + 3.0) * xx * pm2;
    out[(size_t)np + p] = pm1;
    double a_prev = std::sqrt((4.0 * (om + 1.0) * (om + 1.0) - 1.0) /
                              ((om + 1.0) * (om + 1.0) - (double)om * om));
    for (int j = om + 2; j <= jmax; ++j) {
      const double a = std::sqrt((4.0 * j * j - 1.0) / ((double)j * j - (double)om * om));
      const double pj = a * (xx * pm1 - pm2 / a_prev);
      out[(size_t)(j - om) * np + p] = pj;
      pm2 = pm1;
      pm1 = pj;
      a_prev = a;
    }
  }
}

// T^Omega: rows P-bar_j^Omega(x_k) sqrt(w_k), j = om..n-1 (n - om rows), zero-padded to
// n x n, row-major. With n Gauss-Legendre points these rows are exactly orthonormal:
// every product of two of them integrates a polynomial of degree <= 2n - 2.
void fbr_matrix(int om, int n, const std::vector<double>& x, const std::vector<double>& w,
                std::vector<double>& T) {
  T.assign((size_t)n * n, 0.0);
  if (om > n - 1) return;
  std::vector<double> P;
  norm_assoc_legendre(n - 1, om, x, P);
  for (int i = 0; i < n - om; ++i)
    for (int k = 0; k < n; ++k) T[(size_t)i * n + k] = P[(size_t)i * n + k] * std::sqrt(w[k]);
}

// Implicit QL with shifts on a symmetric tridiagonal matrix (diagonal d, e[i] coupling
// d[i] and d[i+1]; e is destroyed), eigenvalues left in d (unsorted). With Z != nullptr the
// plane rotations are accumulated into the n x n row-major Z (eigenvectors in its columns).
static void ql_implicit(int n, std::vector<double>& d, std::vector<double>& e, double* Z) {
  for (int l = 0; l < n; ++l) {
    int iter = 0;
    int m;
    do {
      for (m = l; m + 1 < n; ++m) {
        const double dd = std::fabs(d[m]) + std::fabs(d[m + 1]);
        if (std::fabs(e[m]) + dd == dd) break;  // negligible at working precision
      }
      if (m != l) {
        if (++iter > 200) break;
        double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
        double r = std::hypot(g, 1.0);
        g = d[m] - d[l] + e[l] / (g + (g >= 0 ? std::fabs(r) : -std::fabs(r)));
        double s = 1.0, c = 1.0, pp = 0.0;
        int i;
        bool deflated = false;
        for (i = m - 1; i >= l; --i) {
          double f = s * e[i];
          const double b = c * e[i];
          r = std::hypot(f, g);
          e[i + 1] = r;
          if (r == 0.0) {
            d[i + 1] -= pp;
            e[m] = 0.0;
            deflated = true;
            break;
          }
          s = f / r;
          c = g / r;
          g = d[i + 1] - pp;
          r = (d[i] - g) * s + 2.0 * c * b;
          pp = s * r;
          d[i + 1] = g + pp;
          g = c * r - b;
          if (Z) {
            for (int kk = 0; kk < n; ++kk) {
              f = Z[(size_t)kk * n + i + 1];
              Z[(size_t)kk * n + i + 1] = s * Z[(size_t)kk * n + i] + c * f;
              Z[(size_t)kk * n + i] = c * Z[(size_t)kk * n + i] - s * f;
            }
          }
        }
        if (deflated) continue;
        d[l] -= pp;
        e[l] = g;
        e[m] = 0.0;
      }
    } while (m != l);
  }
}

// Symmetric eigen-decomposition: Householder reduction to tridiagonal form, then
// the implicit QL iteration with Wilkinson-type shifts of Bowdler, Martin, Reinsch and
// Wilkinson (the published tql2 algorithm, Numer. Math. 11, 1968); eigenvalues
// ascending, eigenvectors in the columns of Z (row-major n x n).
void symmetric_eigen(int n, const std::vector<double>& Ain, std::vector<double>& evals,
                     std::vector<double>& Z) {
  std::vector<double> A = Ain;
  Z.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Z[(size_t)i * n + i] = 1.0;
  std::vector<double> v(n), p(n), qv(n), zv(n);
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;  // length of the column below the diagonal
    double nrm = 0;
    for (int i = k + 1; i < n; ++i) nrm += A[(size_t)i * n + k] * A[(size_t)i * n + k];
    nrm = std::sqrt(nrm);
    if (nrm == 0.0) continue;
    const double x0 = A[(size_t)(k + 1) * n + k];
    const double alpha = (x0 > 0) ? -nrm : nrm;
    std::fill(v.begin(), v.end(), 0.0);
    for (int i = k + 1; i < n; ++i) v[i] = A[(size_t)i * n + k];
    v[k + 1] -= alpha;
    double vn = 0;
    for (int i = k + 1; i < n; ++i) vn += v[i] * v[i];
    vn = std::sqrt(vn);
    if (vn == 0.0) continue;
    for (int i = k + 1; i < n; ++i) v[i] /= vn;
    (void)m;
    // A <- H A H with H = I - 2 v v^T (acting on indices >= k)
    for (int i = k; i < n; ++i) {
      double s = 0;
      for (int j = k + 1; j < n; ++j) s += A[(size_t)i * n + j] * v[j];
      p[i] = s;
    }
    double K = 0;
    for (int i = k + 1; i < n; ++i) K += v[i] * p[i];
    for (int i = k; i < n; ++i) qv[i] = p[i] - K * v[i];
    for (int i = k; i < n; ++i)
      for (int j = k; j < n; ++j)
        A[(size_t)i * n + j] -= 2.0 * (v[i] * qv[j] + qv[i] * v[j]);
    // Z <- Z H
    for (int i = 0; i < n; ++i) {
      double s = 0;
      for (int j = k + 1; j < n; ++j) s += Z[(size_t)i * n + j] * v[j];
      zv[i] = s;
    }
    for (int i = 0; i < n; ++i)
      for (int j = k + 1; j < n; ++j) Z[(size_t)i * n + j] -= 2.0 * zv[i] * v[j];
  }
  std::vector<double> d(n), e(n, 0.0);
  for (int i = 0; i < n; ++i) d[i] = A[(size_t)i * n + i];
  for (int i = 0; i + 1 < n; ++i) e[i] = A[(size_t)(i + 1) * n + i];
  ql_implicit(n, d, e, Z.data());
  // sort ascending
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return d[a] < d[b]; });
  evals.resize(n);
  std::vector<double> Zs((size_t)n * n);
  for (int c2 = 0; c2 < n; ++c2) {
    evals[c2] = d[order[c2]];
    for (int i = 0; i < n; ++i) Zs[(size_t)i * n + c2] = Z[(size_t)i * n + order[c2]];
  }
  Z.swap(Zs);
}

// Orthonormal DST-II row j (1-based) at node i (1-based).
double dst2(int N, int j, int i) {
  double v = std::sqrt(2.0 / N) * std::sin(j * M_PI * (i - 0.5) / N);
  if (j == N) v /= std::sqrt(2.0);
  return v;
}

// Weights w, dw with f(x) = w . q and f'(x) = dw . q for a sine-DVR vector q:
// f = sum_j s_j a_j phi_j, a = S q, phi_j(x) = sqrt(2/L) sin(k_j (x - xa)).
void sine_interpolation_weights(double xa, double xb, int N, double x, std::vector<double>& w,
                                std::vector<double>& dw) {
  const double L = xb - xa;
  w.assign(N, 0.0);
  dw.assign(N, 0.0);
  for (int j = 1; j <= N; ++j) {
    const double k = j * M_PI / L;
    const double s = (j == N) ? 1.0 / std::sqrt(2.0) : 1.0;
    const double ph = std::sqrt(2.0 / L) * std::sin(k * (x - xa));
    const double dph = std::sqrt(2.0 / L) * k * std::cos(k * (x - xa));
    for (int i = 1; i <= N; ++i) {
      const double S = dst2(N, j, i);
      w[i - 1] += S * s * ph;
      dw[i - 1] += S * s * dph;
    }
  }
}

// ------------------------------------------------- product arrangement geometry
// Atom positions with the BC centre of mass at the origin, as alpha r + beta R:
// A = R, B = -(m_C / M_BC) r, C = (m_B / M_BC) r.
void product_jacobi_matrix(const double m[3], int arrangement, double M[2][2]) {
  const double MBC = m[1] + m[2];
  const double A[2] = {0.0, 1.0}, B[2] = {-m[2] / MBC, 0.0}, C[2] = {m[1] / MBC, 0.0};
  for (int c = 0; c < 2; ++c) {
    if (arrangement == 1) {            // AC + B
      M[0][c] = C[c] - A[c];
      M[1][c] = B[c] - (m[0] * A[c] + m[2] * C[c]) / (m[0] + m[2]);
    } else {                           // AB + C
      M[0][c] = B[c] - A[c];
      M[1][c] = C[c] - (m[0] * A[c] + m[1] * B[c]) / (m[0] + m[1]);
    }
  }
}

void product_masses(const double m[3], int arrangement, double* mu_p, double* m_p) {
  const double Mt = m[0] + m[1] + m[2];
  if (arrangement == 1) {
    *mu_p = m[1] * (m[0] + m[2]) / Mt;
    *m_p = m[0] * m[2] / (m[0] + m[2]);
  } else {
    *mu_p = m[2] * (m[0] + m[1]) / Mt;
    *m_p = m[0] * m[1] / (m[0] + m[1]);
  }
}

void product_point(const double masses[3], int arrangement, double Rp, double rp, double cosgp,
                   double* R, double* r, double* cosg, double* beta, int* sa, int* sc) {
  double M[2][2];
  product_jacobi_matrix(masses, arrangement, M);
  const double det = M[0][0] * M[1][1] - M[0][1] * M[1][0];
  const double Mi[2][2] = {{M[1][1] / det, -M[0][1] / det}, {-M[1][0] / det, M[0][0] / det}};
  // plane vectors (x, z) in the product body-fixed frame
  const double sg = std::sqrt(std::max(1.0 - cosgp * cosgp, 0.0));
  const double rpv[2] = {rp * sg, rp * cosgp}, Rpv[2] = {0.0, Rp};
  double rv[2], Rv[2];
  for (int c = 0; c < 2; ++c) {
    rv[c] = Mi[0][0] * rpv[c] + Mi[0][1] * Rpv[c];
    Rv[c] = Mi[1][0] * rpv[c] + Mi[1][1] * Rpv[c];
  }
  *R = std::hypot(Rv[0], Rv[1]);
  *r = std::hypot(rv[0], rv[1]);
  *cosg = (rv[0] * Rv[0] + rv[1] * Rv[1]) / (*r * *R);
  // reactant axes in product coordinates: z_r = R / |R|, x_r = unit part of r normal to R
  const double zr[2] = {Rv[0] / *R, Rv[1] / *R};
  const double rz = rv[0] * zr[0] + rv[1] * zr[1];
  double xr[2] = {rv[0] - rz * zr[0], rv[1] - rz * zr[1]};
  const double nx = std::hypot(xr[0], xr[1]);
  if (nx > 0) {
    xr[0] /= nx;
    xr[1] /= nx;
  }
  // y_r = z_r x x_r = sigma y' ; rho = R_z(a) R_y(beta) R_z(c) with a, c in {0, pi}:
  // rho_zz = z_r . z' = cos beta, rho_xz = x_r . z' = cos(a) sin(beta),
  // rho_zx = z_r . x' = -sin(beta) cos(c), rho_yy = sigma = cos(a) cos(c)
  const int sigma = (zr[1] * xr[0] - zr[0] * xr[1]) >= 0 ? 1 : -1;
  *beta = std::acos(std::max(-1.0, std::min(1.0, zr[1])));
  if (std::sin(*beta) > 1e-12) {
    *sa = xr[1] >= 0 ? 1 : -1;
    *sc = zr[0] <= 0 ? 1 : -1;
  } else {
    *sa = 1;
    *sc = sigma;
  }
}

// Wigner d^J_(m'm)(beta) in its Jacobi-polynomial form (mw3_wigner.h): the explicit
// alternating sum loses about nine digits at J = 40, this form keeps them.
double wigner_small_d(int J, int mp, int m, double beta) {
  return wigner_small_d_jacobi(J, mp, m, beta);
}

// Unadapted components: Phi'_m' = sum_m D_(m m')(rho) Phi_m with Phi_(-m) = (-1)^m Phi_m
// and the adapted block m = 0 scaled by sqrt(2).
void helicity_transform(int J, int nom, double beta, int sa, int sc, std::vector<double>& T) {
  auto D = [&](int m1, int m2) {   // D^J_(m1 m2)(rho), real
    double v = wigner_small_d(J, m1, m2, beta);
    if (sa < 0 && (m1 & 1)) v = -v;
    if (sc < 0 && (m2 & 1)) v = -v;
    return v;
  };
  T.assign((size_t)nom * nom, 0.0);
  for (int op = 0; op < nom; ++op)
    for (int om = 0; om < nom; ++om) {
      double v = (om == 0 ? std::sqrt(2.0) : 1.0) * D(om, op);
      if (om > 0) v += ((om & 1) ? -1.0 : 1.0) * D(-om, op);
      T[(size_t)op * nom + om] = v / (op == 0 ? std::sqrt(2.0) : 1.0);
    }
}

// --------------------------------------------------------------- LEPS surface
extern "C" int mw3_pes_leps(double r, double R, double cosg, double* potmat, void* user) {
  const mw3_leps_params* P = static_cast<const mw3_leps_params*>(user);
  if (!P || !potmat) return -1;
  const double mB = P->masses[1], mC = P->masses[2];
  const double MBC = mB + mC;
  const double sB = mC * r / MBC, sC = mB * r / MBC;
  double rab = std::sqrt(std::max(R * R + sB * sB + 2.0 * R * sB * cosg, 0.0));
  double rac = std::sqrt(std::max(R * R + sC * sC - 2.0 * R * sC * cosg, 0.0));
  double rbc = r;
  rab = std::max(rab, 0.25);
  rac = std::max(rac, 0.25);
  rbc = std::max(rbc, 0.25);
  auto qj = [&](double rr, double& Q, double& Jx) {
    const double e1 = std::exp(-P->beta * (rr - P->re));
    const double singlet = P->D * (e1 * e1 - 2.0 * e1);
    const double triplet = 0.5 * P->D * (e1 * e1 + 2.0 * e1);
    const double den = 2.0 * (1.0 + P->delta);
    Q = (singlet * (1.0 + P->delta) + triplet * (1.0 - P->delta)) / den;
    Jx = (singlet * (1.0 + P->delta) - triplet * (1.0 - P->delta)) / den;
  };
  double Qab, Jab, Qbc, Jbc, Qac, Jac;
  qj(rab, Qab, Jab);
  qj(rbc, Qbc, Jbc);
  qj(rac, Qac, Jac);
  const double ex = std::sqrt(0.5 * ((Jab - Jbc) * (Jab - Jbc) + (Jbc - Jac) * (Jbc - Jac) +
                                     (Jac - Jab) * (Jac - Jab)));
  const double v11 = Qab + Qbc + Qac - ex + P->D;
  if (!P->two_state) {
    potmat[0] = v11;
    return 0;
  }
  const double v22 = v11 + P->bump * std::exp(-(r - P->bump_r0) * (r - P->bump_r0) / P->bump_w2);
  const double v12 = P->coup * std::exp(-((R - P->coup_R0) * (R - P->coup_R0) +
                                          (r - P->coup_r0) * (r - P->coup_r0)) / P->coup_w2);
  potmat[0] = v11;
  potmat[1] = v12;
  potmat[2] = v12;
  potmat[3] = v22;
  return 0;
}

// J_k(x), k = 0..n-1: the recurrence J_(k-1) = (2k/x) J_k - J_(k+1) run downwards from an
// index well above both n and x (where J is negligible) with arbitrary small start values is
// stable in that direction (Miller's algorithm); the sequence is then scaled so that
// J_0 + 2 (J_2 + J_4 + ...) = 1, the generating-function identity at angle 0.
void bessel_j_sequence(double x, int n, std::vector<double>& J) {
  J.assign(std::max(n, 0), 0.0);
  if (n <= 0) return;
  if (x == 0.0) {
    J[0] = 1.0;
    return;
  }
  const double m = std::max((double)n, x);
  int top = (int)(m + 40.0 + 12.0 * std::cbrt(m));
  top += top & 1;
  std::vector<double> t((size_t)top + 1, 0.0);
  double jk1 = 0.0, jk = 1e-280;   // J_(top+1), J_top up to a common factor
  t[top] = jk;
  for (int k = top; k >= 1; --k) {
    const double jm = (2.0 * k / x) * jk - jk1;
    jk1 = jk;
    jk = jm;
    t[k - 1] = jm;
    if (std::fabs(jm) > 1e250) {   // rescale everything computed so far
      for (int i = k - 1; i <= top; ++i) t[i] *= 1e-250;
      jk *= 1e-250;
      jk1 *= 1e-250;
    }
  }
  double s = t[0];
  for (int i = 2; i <= top; i += 2) s += 2.0 * t[i];
  for (int k = 0; k < n; ++k) J[k] = t[k] / s;
}

// Eigenvalues (ascending) of the symmetric tridiagonal matrix with diagonal d[0..n-1] and
// off-diagonal e[0..n-2] (e[i] couples i and i+1): the implicit QL above without vectors.
void tridiagonal_eigenvalues(const std::vector<double>& d_in, const std::vector<double>& e_in,
                             std::vector<double>& evals) {
  const int n = (int)d_in.size();
  std::vector<double> d = d_in, e(n, 0.0);
  for (int i = 0; i + 1 < n; ++i) e[i] = e_in[i];
  ql_implicit(n, d, e, nullptr);
  std::sort(d.begin(), d.end());
  evals = d;
}

// Eigenvector of the same tridiagonal matrix for the eigenvalue lam by inverse iteration:
// three solves of (T - (lam + delta) I) x = x_prev by Gaussian elimination with partial
// pivoting (the band grows to two super-diagonals), delta a relative 1e-12 offset that keeps
// the shifted matrix nonsingular. x is normalised.
void tridiagonal_eigenvector(const std::vector<double>& d, const std::vector<double>& e,
                             double lam, std::vector<double>& x) {
  const int n = (int)d.size();
  const double scale = std::max(1.0, std::fabs(lam));
  const double mu = lam + 1e-12 * scale;
  x.assign(n, 1.0 / std::sqrt((double)n));
  for (int it = 0; it < 3; ++it) {
    // rows i: a[i] (sub), b[i] (diag), c[i] (super), f[i] (second super after pivoting)
    std::vector<double> a(n, 0.0), b(n), c(n, 0.0), f(n, 0.0), r = x;
    for (int i = 0; i < n; ++i) {
      b[i] = d[i] - mu;
      if (i > 0) a[i] = e[i - 1];
      if (i + 1 < n) c[i] = e[i];
    }
    for (int i = 0; i + 1 < n; ++i) {
      // eliminate a[i+1] using row i or the swapped row i+1
      if (std::fabs(a[i + 1]) > std::fabs(b[i])) {
        std::swap(b[i], a[i + 1]);
        std::swap(c[i], b[i + 1]);
        std::swap(f[i], c[i + 1]);
        std::swap(r[i], r[i + 1]);
      }
      const double piv = b[i] != 0.0 ? b[i] : 1e-300;
      const double mlt = a[i + 1] / piv;
      b[i + 1] -= mlt * c[i];
      c[i + 1] -= mlt * f[i];
      r[i + 1] -= mlt * r[i];
      a[i + 1] = 0.0;
    }
    for (int i = n - 1; i >= 0; --i) {
      double v = r[i];
      if (i + 1 < n) v -= c[i] * x[i + 1];
      if (i + 2 < n) v -= f[i] * x[i + 2];
      x[i] = v / (b[i] != 0.0 ? b[i] : 1e-300);
    }
    double nrm = 0;
    for (double v : x) nrm += v * v;
    nrm = std::sqrt(nrm);
    for (double& v : x) v /= nrm;
  }
}

}  // namespace mw3
