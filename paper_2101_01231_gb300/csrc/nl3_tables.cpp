// Host-built FP64 tables of the 3D nonlinear (Newton) RIDG path for Burgers' flux
// F_d(q) = q^2 / 2 (see nl3.h).
//
// Space-time basis Psi_k = psi_a(tau) phi_bx(xi_x) phi_by(xi_y) phi_bz(xi_z), k = a thS + s,
// s = bx + nb (by + nb bz).  For Burgers F'(w) = w lies in the solution's own space, so the
// projection of eq. Jacproj onto Psi_p is w's own coefficients and the triple products of
// eq. Jacobian2 are needed only for p of degree <= M per dimension: beta (volume) and gamma
// (faces) below are those products, built from the 1D integrals int phi_a phi_b phi_c and
// int phi_a' phi_b phi_c by exact Gauss quadrature.
#include "nl3.h"

#include <cmath>

#include "tables.h"

namespace ridg {
namespace {

// int_{-1}^{1} f_a phi_b phi_c, f = phi or phi' (deriv), a, b, c < nb
std::vector<double> triple(int nb, bool deriv) {
  std::vector<double> x, w;
  gauss_legendre(3 * nb / 2 + 2, x, w);
  const int n = (int)x.size();
  std::vector<double> V((size_t)nb * n), dV((size_t)nb * n), v(nb), dv(nb);
  for (int q = 0; q < n; ++q) {
    phi_values(nb, x[q], v.data(), dv.data());
    for (int b = 0; b < nb; ++b) {
      V[(size_t)b * n + q] = v[b];
      dV[(size_t)b * n + q] = dv[b];
    }
  }
  std::vector<double> T((size_t)nb * nb * nb, 0.0);
  for (int a = 0; a < nb; ++a)
    for (int b = 0; b < nb; ++b)
      for (int c = 0; c < nb; ++c) {
        double s = 0.0;
        for (int q = 0; q < n; ++q)
          s += w[q] * (deriv ? dV[(size_t)a * n + q] : V[(size_t)a * n + q]) *
               V[(size_t)b * n + q] * V[(size_t)c * n + q];
        T[((size_t)a * nb + b) * nb + c] = s;
      }
  return T;
}

}  // namespace

Nl3HostTables build_nl3_tables(int M) {
  Nl3HostTables t;
  const int nb = t.nb = M + 1;
  t.thS = nb * nb * nb;
  t.thT = nb * t.thS;
  t.nf = nb * nb * nb;  // face modes: (a, two transverse degrees)
  t.nq = (3 * M + 2) / 2;  // ceil((3M + 1) / 2): exact for the quadratic flux
  std::vector<double> x, w;
  gauss_legendre(t.nq, x, w);
  t.w1 = w;
  t.V1.assign((size_t)nb * t.nq, 0.0);
  t.dV1.assign((size_t)nb * t.nq, 0.0);
  std::vector<double> v(nb), dv(nb);
  for (int q = 0; q < t.nq; ++q) {
    phi_values(nb, x[q], v.data(), dv.data());
    for (int b = 0; b < nb; ++b) {
      t.V1[(size_t)b * t.nq + q] = v[b];
      t.dV1[(size_t)b * t.nq + q] = dv[b];
    }
  }
  Tables1D t1 = tables1d(nb);
  t.ep = t1.ep;
  t.em = t1.em;
  // time term psi_a(1) psi_g(1) - int psi_a' psi_g (per time index pair; identity in space)
  t.Mt.assign((size_t)nb * nb, 0.0);
  for (int a = 0; a < nb; ++a)
    for (int g = 0; g < nb; ++g) t.Mt[(size_t)a * nb + g] = t1.ep[a] * t1.ep[g] - t1.D[a * nb + g];
  const std::vector<double> T0 = triple(nb, false), T1 = triple(nb, true);
  auto t0 = [&](int a, int b, int c) { return T0[((size_t)a * nb + b) * nb + c]; };
  auto t1d = [&](int a, int b, int c) { return T1[((size_t)a * nb + b) * nb + c]; };
  auto digits = [&](int k, int* dg) {  // k -> (bx, by, bz, a)
    dg[0] = k % nb;
    dg[1] = (k / nb) % nb;
    dg[2] = (k / (nb * nb)) % nb;
    dg[3] = k / t.thS;
  };
  const int T = t.thT;
  t.beta.assign((size_t)3 * T * T * T, 0.0);
  for (int d = 0; d < 3; ++d)
    for (int k = 0; k < T; ++k)
      for (int l = 0; l < T; ++l)
        for (int p = 0; p < T; ++p) {
          int dk[4], dl[4], dp[4];
          digits(k, dk);
          digits(l, dl);
          digits(p, dp);
          double v2 = t0(dk[3], dl[3], dp[3]);
          for (int e = 0; e < 3; ++e)
            v2 *= e == d ? t1d(dk[e], dl[e], dp[e]) : t0(dk[e], dl[e], dp[e]);
          t.beta[(((size_t)d * T + k) * T + l) * T + p] = v2;
        }
  // faces: gamma[d][sk][sl][k][l][pf], pf = a + nb (c1 + nb c2) over the time degree and the
  // two transverse degrees (increasing dimension order); sides 0 = +1, 1 = -1
  const int F = t.nf;
  t.gamma.assign((size_t)3 * 4 * T * T * F, 0.0);
  for (int d = 0; d < 3; ++d) {
    const int e1 = d == 0 ? 1 : 0, e2 = d == 2 ? 1 : 2;
    for (int sk = 0; sk < 2; ++sk)
      for (int sl = 0; sl < 2; ++sl)
        for (int k = 0; k < T; ++k)
          for (int l = 0; l < T; ++l)
            for (int pf = 0; pf < F; ++pf) {
              int dk[4], dl[4];
              digits(k, dk);
              digits(l, dl);
              const int pa = pf % nb, p1 = (pf / nb) % nb, p2 = pf / (nb * nb);
              const double trk = sk == 0 ? t1.ep[dk[d]] : t1.em[dk[d]];
              const double trl = sl == 0 ? t1.ep[dl[d]] : t1.em[dl[d]];
              const double v2 = t0(dk[3], dl[3], pa) * t0(dk[e1], dl[e1], p1) *
                                t0(dk[e2], dl[e2], p2) * trk * trl;
              t.gamma[((((size_t)(d * 4 + sk * 2 + sl) * T + k) * T + l) * F) + pf] = v2;
            }
  }
  return t;
}

}  // namespace ridg
