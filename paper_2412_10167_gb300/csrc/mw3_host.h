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

}  // namespace mw3
