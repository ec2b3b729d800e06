// Host-side set-up mathematics of libmw3 (private).
#pragma once

#include <vector>

#include "../../include/mw3.h"

namespace mw3 {

void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);
void norm_assoc_legendre(int jmax, int om, const std::vector<double>& x, std::vector<double>& out);
void fbr_matrix(int om, int n, const std::vector<double>& x, const std::vector<double>& w,
                std::vector<double>& T);
void symmetric_eigen(int n, const std::vector<double>& A, std::vector<double>& evals,
                     std::vector<double>& Z);
double dst2(int N, int j, int i);
void sine_interpolation_weights(double xa, double xb, int N, double x, std::vector<double>& w,
                                std::vector<double>& dw);

// ------------------------------------------------- product arrangement geometry
// Product Jacobi vectors as (r', R') = M (r, R). arrangement 1: products AC + B
// (r' = C - A, R' from the AC centre of mass to B); 2: products AB + C.
void product_jacobi_matrix(const double masses[3], int arrangement, double M[2][2]);
// Reduced masses (mu' of R', m' of r') of the product arrangement.
void product_masses(const double masses[3], int arrangement, double* mu_p, double* m_p);
// Reactant (R, r, cos gamma) of the product point (R', r', cos gamma') and the signs and
// angle of the rotation between the body-fixed frames: D^J_(m'm)(rho) =
// sa^m' d^J_(m'm)(beta) sc^m, rho taking the reactant axes (z along R, r in x > 0) to the
// product axes (z along R', r' in x > 0).
void product_point(const double masses[3], int arrangement, double Rp, double rp, double cosgp,
                   double* R, double* r, double* cosg, double* beta, int* sa, int* sc);
// Wigner d^J_(m'm)(beta).
double wigner_small_d(int J, int mp, int m, double beta);

// Symmetric tridiagonal matrix (diagonal d, off-diagonal e, e[i] coupling i and i+1):
// ascending eigenvalues by implicit QL, and one normalised eigenvector by inverse iteration.
void tridiagonal_eigenvalues(const std::vector<double>& d, const std::vector<double>& e,
                             std::vector<double>& evals);
void tridiagonal_eigenvector(const std::vector<double>& d, const std::vector<double>& e,
                             double lam, std::vector<double>& x);

// Bessel functions of the first kind J_0(x) .. J_(n-1)(x) for x >= 0 (Miller's backward
// recurrence normalised by J_0 + 2 sum_m J_2m = 1).
void bessel_j_sequence(double x, int n, std::vector<double>& J);
// Helicity transform of the parity-adapted blocks Omega = 0..nom-1 (parity (-1)^J):
// T[op * nom + om] with Phi'_op = sum_om T[op][om] Phi_om.
void helicity_transform(int J, int nom, double beta, int sa, int sc, std::vector<double>& T);

}  // namespace mw3
