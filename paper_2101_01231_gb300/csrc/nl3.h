// The 3D nonlinear (Newton) RIDG path for Burgers' flux: host tables and launchers.
#pragma once

#include <cuda_runtime.h>

#include <vector>

namespace ridg {

struct Nl3HostTables {
  int nb = 0, thS = 0, thT = 0, nf = 0, nq = 0;
  std::vector<double> w1, V1, dV1;  // 1D Gauss rule of the residual: weights, phi_b(x_q), phi_b'
  std::vector<double> ep, em;       // phi_b(+1), phi_b(-1)
  std::vector<double> Mt;           // nb x nb time term psi_a(1) psi_g(1) - int psi_a' psi_g
  std::vector<double> beta;         // [d][k][l][p], p < thT: int d_d Psi_k Psi_l Psi_p
  std::vector<double> gamma;        // [d][sk][sl][k][l][pf]: face products with the traces
};
Nl3HostTables build_nl3_tables(int M);

// Device copies (one allocation) of the tables, read by the kernels.
struct Nl3Dev {
  const double *w1, *V1, *dV1, *ep, *em, *Mt, *beta, *gamma;
  int nq;
};
// bytes of the device copy, and the upload (mem == nullptr: size only)
int nl3_tables_upload(int nb, Nl3Dev& out, void* mem, size_t* bytes, cudaStream_t s);

struct Newton3Args {
  Nl3Dev tb;
  const double* Q;
  double* W;             // centre prediction, cells x theta_T
  int n[3];
  long long ncell;
  double lam[3];         // dt / h_d
  int max_iters;
  double tol;
  void* scratch;         // per CTA: the region Jacobian (n x n) and the pivot rows
  size_t scratch_per_cta;
  int* counter;          // region counter (zeroed by the launcher)
  int* stats;            // as the 2D kernel: [0] unconverged, [1] max iters, [2] flags, [7..22]
  unsigned long long* iters_total;
};
bool newton3_supported(int nb);
size_t newton3_scratch_per_cta(int nb, bool fp32);
// one persistent CTA per SM; fp32: the region Jacobian factorised in FP32 (the residual,
// the iterate and the stopping test stay FP64)
cudaError_t launch_newton3(int nb, bool fp32, const Newton3Args& a, int grid, cudaStream_t s);
cudaError_t launch_nl3_correct(int nb, const Nl3Dev& tb, double* Q, const double* W, const int* n,
                               long long ncell, const double* lam, cudaStream_t s);
// largest |q| over a 6 x 6 x 6 equispaced grid of every cell -> *out (as bits)
cudaError_t launch_max_speed3(int nb, const double* Q, long long ncell, unsigned long long* out,
                              cudaStream_t s);

}  // namespace ridg
