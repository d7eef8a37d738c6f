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

// The region cells a linear flux's prediction depends on (Sec. 2.2).  With upwind face
// values the region system of eq. pred_full_system is block triangular in the flow
// direction: a cell's equations reference only itself and its upstream face neighbours, so
// the centre's solution depends only on the cells upstream of it.  Per dimension d that is
// offsets {-1, 0} for a_d > 0, {0, +1} for a_d < 0 and {0} for a_d = 0: a box of
// cnt[0] x cnt[1] x cnt[2] cells starting at offset lo[], x fastest.
struct RegionBox {
  int lo[3] = {0, 0, 0};
  int cnt[3] = {1, 1, 1};
  int n = 1;
};
RegionBox upwind_box(int dim, const double* vel);

// Centre-row solution operator of the linear region system (Sec. 2.2):
//   W_centre = P X,  X = the Q of the box's cells stacked (box.n blocks of theta_S, x fastest),
// P has theta_T rows and K = box.n theta_S columns (row-major); the region cells outside
// the box have exactly zero columns and are left out.  nu[d] = a_d dt / h_d must have the
// sign of the velocity the box was made from (or be zero).  The system is solved by block
// substitution over the box (one dense LU per box cell's diagonal block).  Returns false if
// a diagonal block is singular.
bool linear_operator(int dim, int M, const double* nu, const RegionBox& box,
                     std::vector<double>& P);

// The fused step operator G = C P-bar of the mixed path (dim 2 or 3): C maps a cell's time
// mean W-bar (theta_S modes, x fastest) to the correction's linear functionals of it --
// rows 0 .. theta_S - 1 the volume term sum_d nu_d (D along d) W-bar (Sec. 2.3), then per
// direction d and line t of the nb^(dim-1) lines of modes along d (the other indices, the
// lower one fastest) the upwind trace nu_d tr(W-bar) on the cell's downstream d-face
// (phi_b(+1) for nu_d >= 0, phi_b(-1) for nu_d < 0): row theta_S + d nb^(dim-1) + t.  Pbar
// holds the theta_S time-mean rows of the prediction operator (theta_S x K); G gets
// (theta_S + dim nb^(dim-1)) x K.
void fused_step_operator(int dim, int nb, const double* nu, const std::vector<double>& Pbar,
                         int K, std::vector<double>& G);

// Dense LU with partial pivoting, in place (row-major n x n); perm[i] = original row of
// row i of the factors.  Returns false on a zero pivot.
bool lu_factor(int n, double* A, std::vector<int>& perm);
// Solve A^T z = b with the factors of A.
void lu_solve_transpose(int n, const double* LU, const std::vector<int>& perm, double* b);
// Solve A z = b with the factors of A.
void lu_solve(int n, const double* LU, const std::vector<int>& perm, double* b);

}  // namespace ridg
