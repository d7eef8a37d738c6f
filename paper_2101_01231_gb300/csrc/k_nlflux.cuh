// Physical fluxes of the nonlinear path in 2D: F_d(w), its Jacobian dF_d/dw (row-major m x m)
// and the largest wave speed in direction d, for Burgers' equation (eq. burger2d: F_d = w^2
// / 2) and the compressible Euler equations of an ideal gas (conserved rho, rho u, rho v, E).
// S is double for the residual, the correction and the FP64 Jacobian, float for the FP32
// Jacobian of the mixed form.
#pragma once

#include "../../include/ridg.h"

namespace ridg {
namespace nlflux {

template <int FLUX, typename S>
__device__ __forceinline__ void F(const S* w, int dd, S* f, S g) {
  if constexpr (FLUX == RIDG_FLUX_BURGERS) {
    f[0] = S(0.5) * w[0] * w[0];
  } else {
    const S rho = w[0], u = w[1] / rho, v = w[2] / rho, E = w[3];
    const S p = (g - S(1)) * (E - S(0.5) * rho * (u * u + v * v));
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
}

template <int FLUX, typename S>
__device__ __forceinline__ void dF(const S* w, int dd, S* J, S g) {
  if constexpr (FLUX == RIDG_FLUX_BURGERS) {
    J[0] = w[0];
  } else {
    const S g1 = g - S(1);
    const S rho = w[0], u = w[1] / rho, v = w[2] / rho, E = w[3];
    const S q2 = u * u + v * v;
    const S p = g1 * (E - S(0.5) * rho * q2);
    const S H = (E + p) / rho;
    const S k = S(0.5) * g1 * q2;
    if (dd == 0) {
      J[0] = S(0);          J[1] = S(1);             J[2] = S(0);            J[3] = S(0);
      J[4] = k - u * u;     J[5] = (S(3) - g) * u;   J[6] = -g1 * v;         J[7] = g1;
      J[8] = -u * v;        J[9] = v;                J[10] = u;              J[11] = S(0);
      J[12] = u * (k - H);  J[13] = H - g1 * u * u;  J[14] = -g1 * u * v;    J[15] = g * u;
    } else {
      J[0] = S(0);          J[1] = S(0);             J[2] = S(1);            J[3] = S(0);
      J[4] = -u * v;        J[5] = v;                J[6] = u;               J[7] = S(0);
      J[8] = k - v * v;     J[9] = -g1 * u;          J[10] = (S(3) - g) * v; J[11] = g1;
      J[12] = v * (k - H);  J[13] = -g1 * u * v;     J[14] = H - g1 * v * v; J[15] = g * v;
    }
  }
}

template <int FLUX, typename S>
__device__ __forceinline__ S speed(const S* w, int dd, S g) {
  if constexpr (FLUX == RIDG_FLUX_BURGERS) {
    return fabs(w[0]);
  } else {
    const S rho = w[0], u = w[1] / rho, v = w[2] / rho, E = w[3];
    const S p = (g - S(1)) * (E - S(0.5) * rho * (u * u + v * v));
    return fabs(dd == 0 ? u : v) + sqrt(g * p / rho);
  }
}

}  // namespace nlflux
}  // namespace ridg
