// Physical fluxes of the nonlinear path in 2D (FP64): F_d(w), its Jacobian dF_d/dw and the
// largest wave speed in direction d, for Burgers' equation (eq. burger2d: F_d = w^2 / 2)
// and the compressible Euler equations of an ideal gas (conserved rho, rho u, rho v, E).
#pragma once

#include "../../include/ridg.h"

namespace ridg {
namespace nlflux {

template <int FLUX>
__device__ __forceinline__ void F(const double* w, int dd, double* f, double g);
template <int FLUX>
__device__ __forceinline__ void dF(const double* w, int dd, double* J, double g);
template <int FLUX>
__device__ __forceinline__ double speed(const double* w, int dd, double g);

// ---- Burgers ----
template <>
__device__ __forceinline__ void F<RIDG_FLUX_BURGERS>(const double* w, int, double* f, double) {
  f[0] = 0.5 * w[0] * w[0];
}
template <>
__device__ __forceinline__ void dF<RIDG_FLUX_BURGERS>(const double* w, int, double* J, double) {
  J[0] = w[0];
}
template <>
__device__ __forceinline__ double speed<RIDG_FLUX_BURGERS>(const double* w, int, double) {
  return fabs(w[0]);
}

// ---- Euler ----
template <>
__device__ __forceinline__ void F<RIDG_FLUX_EULER>(const double* w, int dd, double* f, double g) {
  const double rho = w[0], u = w[1] / rho, v = w[2] / rho, E = w[3];
  const double p = (g - 1.0) * (E - 0.5 * rho * (u * u + v * v));
  if (dd == 0) {
    f[0] = rho * u;
    f[1] = rho * u * u + p;
    f[2] = rho * u * v;
    f[3] = u * (E + p);
  } else {
    f[0] = rho * v;
    f[1] = rho * u * v;
    f[2] = rho * v * v + p;
    f[3] = v * (E + p);
  }
}
template <>
__device__ __forceinline__ void dF<RIDG_FLUX_EULER>(const double* w, int dd, double* J, double g) {
  const double g1 = g - 1.0;
  const double rho = w[0], u = w[1] / rho, v = w[2] / rho, E = w[3];
  const double q2 = u * u + v * v;
  const double p = g1 * (E - 0.5 * rho * q2);
  const double H = (E + p) / rho;
  if (dd == 0) {
    J[0] = 0.0;                       J[1] = 1.0;             J[2] = 0.0;        J[3] = 0.0;
    J[4] = 0.5 * g1 * q2 - u * u;     J[5] = (3.0 - g) * u;   J[6] = -g1 * v;    J[7] = g1;
    J[8] = -u * v;                    J[9] = v;               J[10] = u;         J[11] = 0.0;
    J[12] = u * (0.5 * g1 * q2 - H);  J[13] = H - g1 * u * u; J[14] = -g1 * u * v; J[15] = g * u;
  } else {
    J[0] = 0.0;                       J[1] = 0.0;             J[2] = 1.0;        J[3] = 0.0;
    J[4] = -u * v;                    J[5] = v;               J[6] = u;          J[7] = 0.0;
    J[8] = 0.5 * g1 * q2 - v * v;     J[9] = -g1 * u;         J[10] = (3.0 - g) * v; J[11] = g1;
    J[12] = v * (0.5 * g1 * q2 - H);  J[13] = -g1 * u * v;    J[14] = H - g1 * v * v; J[15] = g * v;
  }
}
template <>
__device__ __forceinline__ double speed<RIDG_FLUX_EULER>(const double* w, int dd, double g) {
  const double rho = w[0], u = w[1] / rho, v = w[2] / rho, E = w[3];
  const double p = (g - 1.0) * (E - 0.5 * rho * (u * u + v * v));
  return fabs(dd == 0 ? u : v) + sqrt(g * p / rho);
}

}  // namespace nlflux
}  // namespace ridg
