// Host-built FP64 tables of the nonlinear (Newton) RIDG path in 2D: basis values at the
// Gauss points of the residual and of the quasi-quadrature-free projection, and the sparse
// lists of nonzero triple-product integrals (Sec. 3, eqs. Jacproj and Jacobian2).
#pragma once

#include <vector>

namespace ridg {

struct SparseTriple {
  // for every (k, l) pair (k * thT + l): entries [ptr[kl], ptr[kl + 1]) of (p, value)
  std::vector<int> ptr, p;
  std::vector<double> val;
};

struct NlHostTables {
  int nb = 0, thS = 0, thT = 0;
  int nq = 0, Qv = 0, Qf = 0;     // residual rule: nq points per dimension
  int np = 0, QP = 0, QPf = 0;    // projection rule: 2M + 1 points per dimension
  std::vector<double> Mt;         // nb x nb: psi_a(1) psi_g(1) - int psi_a' psi_g
  std::vector<double> em;         // psi_a(-1)
  std::vector<double> PsiV, dPsiV;   // thT x Qv, 2 x thT x Qv (d/dxi_x, d/dxi_y)
  std::vector<double> wV;            // Qv (tau slowest, then y, x)
  // the same rule in 1D (for sum-factorised evaluation): phi_b(x_q) as nb x nq and nq x nb,
  // phi_b'(x_q) as nb x nq, and the traces phi_b(+1), phi_b(-1)
  std::vector<double> V1, V1T, dV1, ep1, em1;
  std::vector<double> PsiF;          // [dim][side (+1, -1)][thT][Qf]
  std::vector<double> wF;            // [dim][Qf] (tau slowest, then the other dimension)
  std::vector<double> PhiV, dPhiV;   // thS x Qv, 2 x thS x Qv (spatial basis, for the correction)
  std::vector<double> PhiF;          // [dim][side][thS][Qf]
  std::vector<double> PsiAtP;        // thT x QP: solution basis at the projection points
  std::vector<double> PsiAtFP;       // [dim][side][thT][QPf]
  // 1D projection factor P1[p][q] = phi_p(x_q) w_q / 2 (np x np); the projections of
  // eq. Jacproj onto Psi_p (volume) and onto the face basis are its tensor products
  std::vector<double> P1;
  SparseTriple beta[2];              // [dim]: int d_dim Psi_k Psi_l Psi_p (volume)
  // the 1D factors of those triple products, [a][b][p] (a, b < nb, p < np): int phi_a phi_b
  // phi_p, and the same with phi_a' (for the sum-factorised assembly)
  std::vector<double> T0, T1;
  SparseTriple gamma[2][2][2];       // [dim][side_k][side_l]: face integrals
};

// Build the tables for degree M in 2D.
NlHostTables build_nl_tables(int M);

// The Jacobian's triple-product lists merged per (k, l) pair for assembly.  The diagonal
// block of a region cell takes, for every pair, the volume lists of both directions and the
// own-side face lists of its four faces; an entry is (offset, coefficient) with the offset
// (in units of m x m matrices) into the cell's projected arrays laid out as
//   [F'_x (QP) | F'_y (QP) | own face 0..3 (QPf each) | neighbour face 0..3 (QPf each)].
// The block towards the neighbour across face f takes the neighbour-side list of face f.
struct NlAsmLists {
  std::vector<int> dptr, doff;
  std::vector<double> dval;
  std::vector<int> optr[4], ooff[4];
  std::vector<double> oval[4];
};
NlAsmLists build_asm_lists(const NlHostTables& t);

}  // namespace ridg
