// Host-side FP64 numerics of the RIDG library: 1D Legendre tables, Gauss rules, the
// region system of eq. pred_full_system for a linear flux and its centre-row solution
// operator, and the quadrature / triple-product tables the nonlinear kernels use.
#pragma once

#include <vector>

namespace ridg {

// P_n(x) and P_n'(x) by the three-term recurrence.
void legendre(int n, double x, double* p, double* dp);
// phi_b(x) = sqrt(2b+1) P_b(x), b < nb; values and derivatives.
void phi_values(int nb, double x, double* v, double* dv);
// Gauss-Legendre nodes / weights on [-1, 1] (Newton on P_n).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);

struct Tables1D {
  int nb = 0;
  std::vector<double> ep, em;  // phi_b(+1), phi_b(-1)
  std::vector<double> D;       // D[a*nb+b] = int phi_a' phi_b
};
Tables1D tables1d(int nb);

// Centre-row solution operator of the linear region system (Sec. 2.2):
//   W_centre = P X,  X = the region's Q stacked (3^d blocks of theta_S, x fastest),
// P has theta_T rows and K = 3^d theta_S columns (row-major).  nu[d] = a_d dt / h_d.
// Returns false if the region matrix is singular.
bool linear_operator(int dim, int M, const double* nu, std::vector<double>& P);

// Dense LU with partial pivoting, in place (row-major n x n); perm[i] = original row of
// row i of the factors.  Returns false on a zero pivot.
bool lu_factor(int n, double* A, std::vector<int>& perm);
// Solve A^T z = b with the factors of A.
void lu_solve_transpose(int n, const double* LU, const std::vector<int>& perm, double* b);
// Solve A z = b with the factors of A.
void lu_solve(int n, const double* LU, const std::vector<int>& perm, double* b);

}  // namespace ridg
