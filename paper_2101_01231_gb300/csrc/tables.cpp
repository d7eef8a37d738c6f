// Host-side FP64 numerics (see tables.h).
#include "tables.h"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace ridg {

void legendre(int n, double x, double* p, double* dp) {
  // P_0 = 1, P_1 = x, (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1};
  // P_k' = k (x P_k - P_{k-1}) / (x^2 - 1) away from +-1, closed form k(k+1)/2 (+-1)^(k+1) at +-1.
  double p0 = 1.0, p1 = x;
  if (n == 0) { *p = 1.0; *dp = 0.0; return; }
  for (int k = 1; k < n; ++k) {
    double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  *p = p1;
  if (std::fabs(std::fabs(x) - 1.0) < 1e-15) {
    double s = (x > 0 || (n + 1) % 2 == 0) ? 1.0 : -1.0;
    *dp = s * 0.5 * n * (n + 1.0);
  } else {
    *dp = n * (x * p1 - p0) / (x * x - 1.0);
  }
}

void phi_values(int nb, double x, double* v, double* dv) {
  // derivatives by the recurrence P_{k+1}' = P_{k-1}' + (2k+1) P_k (valid everywhere)
  std::vector<double> P(nb + 1), dP(nb + 1);
  P[0] = 1.0;
  dP[0] = 0.0;
  if (nb > 1) { P[1] = x; dP[1] = 1.0; }
  for (int k = 1; k + 1 < nb; ++k) {
    P[k + 1] = ((2.0 * k + 1.0) * x * P[k] - k * P[k - 1]) / (k + 1.0);
    dP[k + 1] = dP[k - 1] + (2.0 * k + 1.0) * P[k];
  }
  for (int b = 0; b < nb; ++b) {
    double s = std::sqrt(2.0 * b + 1.0);
    if (v) v[b] = s * P[b];
    if (dv) dv[b] = s * dP[b];
  }
}

void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5));
    double p = 0, dp = 1;
    for (int it = 0; it < 100; ++it) {
      legendre(n, z, &p, &dp);
      double dz = p / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    legendre(n, z, &p, &dp);
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

Tables1D tables1d(int nb) {
  Tables1D t;
  t.nb = nb;
  t.ep.resize(nb);
  t.em.resize(nb);
  phi_values(nb, 1.0, t.ep.data(), nullptr);
  phi_values(nb, -1.0, t.em.data(), nullptr);
  // D[a][b] = int phi_a' phi_b by Gauss with nb points (integrand degree <= 2 nb - 3)
  std::vector<double> x, w;
  gauss_legendre(nb + 1, x, w);
  t.D.assign(nb * nb, 0.0);
  std::vector<double> v(nb), dv(nb);
  for (size_t q = 0; q < x.size(); ++q) {
    phi_values(nb, x[q], v.data(), dv.data());
    for (int a = 0; a < nb; ++a)
      for (int b = 0; b < nb; ++b) t.D[a * nb + b] += w[q] * dv[a] * v[b];
  }
  return t;
}

bool lu_factor(int n, double* A, std::vector<int>& perm) {
  perm.resize(n);
  for (int i = 0; i < n; ++i) perm[i] = i;
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = std::fabs(A[(size_t)k * n + k]);
    for (int i = k + 1; i < n; ++i) {
      double v = std::fabs(A[(size_t)i * n + k]);
      if (v > best) { best = v; p = i; }
    }
    if (best == 0.0) return false;
    if (p != k) {
      for (int j = 0; j < n; ++j) std::swap(A[(size_t)k * n + j], A[(size_t)p * n + j]);
      std::swap(perm[k], perm[p]);
    }
    const double inv = 1.0 / A[(size_t)k * n + k];
    const double* rowk = A + (size_t)k * n;
#pragma omp parallel for schedule(static) if (n - k > 256)
    for (int i = k + 1; i < n; ++i) {
      double* rowi = A + (size_t)i * n;
      double l = rowi[k] * inv;
      rowi[k] = l;
      if (l != 0.0)
        for (int j = k + 1; j < n; ++j) rowi[j] -= l * rowk[j];
    }
  }
  return true;
}

void lu_solve(int n, const double* LU, const std::vector<int>& perm, double* b) {
  std::vector<double> y(n);
  for (int i = 0; i < n; ++i) y[i] = b[perm[i]];
  for (int i = 0; i < n; ++i) {
    double s = y[i];
    for (int j = 0; j < i; ++j) s -= LU[(size_t)i * n + j] * y[j];
    y[i] = s;
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = y[i];
    for (int j = i + 1; j < n; ++j) s -= LU[(size_t)i * n + j] * y[j];
    y[i] = s / LU[(size_t)i * n + i];
  }
  std::memcpy(b, y.data(), sizeof(double) * n);
}

void lu_solve_transpose(int n, const double* LU, const std::vector<int>& perm, double* b) {
  // (P A) = L U  =>  A^T z = b  <=>  U^T L^T (P z) = b
  std::vector<double> v(b, b + n);
  for (int i = 0; i < n; ++i) {  // U^T v = b (U^T lower)
    double s = v[i];
    for (int j = 0; j < i; ++j) s -= LU[(size_t)j * n + i] * v[j];
    v[i] = s / LU[(size_t)i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {  // L^T u = v (unit upper)
    double s = v[i];
    for (int j = i + 1; j < n; ++j) s -= LU[(size_t)j * n + i] * v[j];
    v[i] = s;
  }
  for (int i = 0; i < n; ++i) b[perm[i]] = v[i];  // z = P^T u
}

namespace {
inline int ipow(int b, int e) {
  int r = 1;
  while (e--) r *= b;
  return r;
}
}  // namespace

RegionBox upwind_box(int dim, const double* vel) {
  RegionBox b;
  for (int d = 0; d < dim; ++d) {
    if (vel[d] > 0) {
      b.lo[d] = -1;
      b.cnt[d] = 2;
    } else if (vel[d] < 0) {
      b.lo[d] = 0;
      b.cnt[d] = 2;
    }
  }
  b.n = b.cnt[0] * b.cnt[1] * b.cnt[2];
  return b;
}

bool linear_operator(int dim, int M, const double* nu, const RegionBox& box,
                     std::vector<double>& P) {
  const int nb = M + 1, thS = ipow(nb, dim), thT = nb * thS, nc = box.n;
  const int K = nc * thS;
  Tables1D t = tables1d(nb);
  auto D = [&](int a, int b) { return t.D[a * nb + b]; };
  auto digit = [&](int s, int dd) { return (s / ipow(nb, dd)) % nb; };
  // box cell i <-> region offsets o[] (x fastest)
  auto offsets = [&](int i, int* o) {
    o[0] = box.lo[0] + i % box.cnt[0];
    o[1] = box.lo[1] + (i / box.cnt[0]) % box.cnt[1];
    o[2] = box.lo[2] + i / (box.cnt[0] * box.cnt[1]);
  };
  auto box_index = [&](const int* o) {
    return (o[0] - box.lo[0]) + box.cnt[0] * ((o[1] - box.lo[1]) + box.cnt[1] * (o[2] - box.lo[2]));
  };
  // Diagonal block of region cell o, stored transposed (At[l][k] = A[k][l]): time term,
  // internal flux, and the cell's own trace on each face -- the upwind trace on a face
  // shared with a region neighbour, the cell's own (interior) trace on the region boundary.
  std::vector<std::vector<double>> LU(nc);
  std::vector<std::vector<int>> perm(nc);
  for (int i = 0; i < nc; ++i) {
    int o[3];
    offsets(i, o);
    std::vector<double>& At = LU[i];
    At.assign((size_t)thT * thT, 0.0);
    auto add = [&](int k, int l, double v) { At[(size_t)l * thT + k] += v; };
    for (int k = 0; k < thT; ++k) {
      const int al = k / thS, s = k % thS;
      for (int g = 0; g < nb; ++g) add(k, g * thS + s, t.ep[al] * t.ep[g] - D(al, g));
      for (int dd = 0; dd < dim; ++dd) {
        const int st = ipow(nb, dd), bd = digit(s, dd), base = s - bd * st;
        const double nud = nu[dd], nup = nud > 0 ? nud : 0.0, num = nud < 0 ? nud : 0.0;
        const bool has_plus = o[dd] + 1 <= 1, has_minus = o[dd] - 1 >= -1;
        for (int b2 = 0; b2 < nb; ++b2) {
          const int l = al * thS + base + b2 * st;
          add(k, l, -nud * D(bd, b2));
          add(k, l, (has_plus ? nup : nud) * t.ep[bd] * t.ep[b2]);
          add(k, l, -(has_minus ? num : nud) * t.em[bd] * t.em[b2]);
        }
      }
    }
    if (!lu_factor(thT, At.data(), perm[i])) return false;
  }
  // Box cells in sweep order: the centre first, then by the number of nonzero offsets, so
  // that a cell's downstream neighbours (offset moved to 0 in one dimension) come earlier.
  std::vector<int> order(nc);
  for (int i = 0; i < nc; ++i) order[i] = i;
  auto nonzero = [&](int i) {
    int o[3];
    offsets(i, o);
    return (o[0] != 0) + (o[1] != 0) + (o[2] != 0);
  };
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return nonzero(a) < nonzero(b); });
  // Coupling of cell r to its downstream neighbour r' along dd: row (r', k') of A holds
  // C[bd][b2] at column (r, l) for k' = (al, base + bd st), l = (al, base + b2 st), with
  // C = -nu em (x) ep for nu > 0 (face -1 of r') and nu ep (x) em for nu < 0 (face +1).
  // P[c][(i, s)] = sum_a z_i[(a, s)] psi_a(-1), where A^T z = e_(centre, c).
  P.assign((size_t)thT * K, 0.0);
  int o0[3] = {0, 0, 0};
  const int centre = box_index(o0);
  // The theta_T right-hand sides e_(centre, c) in blocks of CB columns: every row operation
  // below runs over a block's columns at once, so each box cell's LU factors are read once
  // per block rather than once per column (each column's arithmetic is unchanged).
  constexpr int CB = 32;
  const int nblk = (thT + CB - 1) / CB;
#pragma omp parallel for schedule(dynamic)
  for (int blk = 0; blk < nblk; ++blk) {
    const int c0 = blk * CB, cw = std::min(CB, thT - c0);
    std::vector<double> z((size_t)nc * thT * CB, 0.0);  // z[i][l][cc], cc < cw
    std::vector<double> y((size_t)thT * CB);
    for (int i : order) {
      int o[3];
      offsets(i, o);
      double* zi = z.data() + (size_t)i * thT * CB;
      if (i == centre)
        for (int cc = 0; cc < cw; ++cc) zi[(size_t)(c0 + cc) * CB + cc] = 1.0;
      for (int dd = 0; dd < dim; ++dd) {
        if (o[dd] == 0) continue;
        int od[3] = {o[0], o[1], o[2]};
        od[dd] = 0;
        const double* zd = z.data() + (size_t)box_index(od) * thT * CB;
        const int st = ipow(nb, dd);
        const double nud = nu[dd];
        for (int l = 0; l < thT; ++l) {
          const int al = l / thS, s = l % thS, b2 = digit(s, dd), base = s - b2 * st;
          double acc[CB] = {};
          for (int bd = 0; bd < nb; ++bd) {
            const double C = nud > 0 ? -nud * t.em[bd] * t.ep[b2] : nud * t.ep[bd] * t.em[b2];
            const double* zr = zd + (size_t)(al * thS + base + bd * st) * CB;
            for (int cc = 0; cc < CB; ++cc) acc[cc] += C * zr[cc];
          }
          double* zl = zi + (size_t)l * CB;
          for (int cc = 0; cc < CB; ++cc) zl[cc] -= acc[cc];
        }
      }
      // zi = (A_ii^T)^-1 zi with the factors of A_ii^T (P A = L U, perm[r] = original row)
      const double* A = LU[i].data();
      const std::vector<int>& pr = perm[i];
      for (int r = 0; r < thT; ++r)
        std::memcpy(y.data() + (size_t)r * CB, zi + (size_t)pr[r] * CB, sizeof(double) * CB);
      for (int r = 0; r < thT; ++r) {
        double* yr = y.data() + (size_t)r * CB;
        const double* Ar = A + (size_t)r * thT;
        for (int jj = 0; jj < r; ++jj) {
          const double a = Ar[jj];
          if (a == 0.0) continue;
          const double* yj = y.data() + (size_t)jj * CB;
          for (int cc = 0; cc < CB; ++cc) yr[cc] -= a * yj[cc];
        }
      }
      for (int r = thT - 1; r >= 0; --r) {
        double* yr = y.data() + (size_t)r * CB;
        const double* Ar = A + (size_t)r * thT;
        for (int jj = r + 1; jj < thT; ++jj) {
          const double a = Ar[jj];
          if (a == 0.0) continue;
          const double* yj = y.data() + (size_t)jj * CB;
          for (int cc = 0; cc < CB; ++cc) yr[cc] -= a * yj[cc];
        }
        const double d = Ar[r];
        for (int cc = 0; cc < CB; ++cc) yr[cc] /= d;
      }
      std::memcpy(zi, y.data(), sizeof(double) * (size_t)thT * CB);
    }
    for (int cc = 0; cc < cw; ++cc)
      for (int i = 0; i < nc; ++i)
        for (int s = 0; s < thS; ++s) {
          double acc = 0.0;
          for (int a = 0; a < nb; ++a)
            acc += z[((size_t)i * thT + a * thS + s) * CB + cc] * t.em[a];
          P[(size_t)(c0 + cc) * K + i * thS + s] = acc;
        }
  }
  return true;
}

void fused_step_operator(int dim, int nb, const double* nu, const std::vector<double>& Pbar,
                         int K, std::vector<double>& G) {
  const Tables1D t1 = tables1d(nb);
  int thS = 1, NT = 1;
  for (int d = 0; d < dim; ++d) thS *= nb;
  NT = thS / nb;  // lines of modes along a direction
  const int nout = thS + dim * NT;
  std::vector<double> C((size_t)nout * thS, 0.0);
  for (int d = 0; d < dim; ++d) {
    int st = 1;
    for (int e = 0; e < d; ++e) st *= nb;
    for (int s = 0; s < thS; ++s) {
      const int ad = (s / st) % nb, base = s - ad * st;
      for (int b = 0; b < nb; ++b) C[(size_t)s * thS + base + b * st] += nu[d] * t1.D[ad * nb + b];
    }
    const std::vector<double>& tr = nu[d] >= 0 ? t1.ep : t1.em;
    for (int t = 0; t < NT; ++t) {
      // line t: the modes with the other indices fixed; its first mode (index 0 along d)
      const int base = (t % st) + (t / st) * st * nb;
      for (int b = 0; b < nb; ++b) C[(size_t)(thS + d * NT + t) * thS + base + b * st] = nu[d] * tr[b];
    }
  }
  G.assign((size_t)nout * K, 0.0);
  for (int r = 0; r < nout; ++r)
    for (int s = 0; s < thS; ++s) {
      const double c = C[(size_t)r * thS + s];
      if (c == 0.0) continue;
      for (int k = 0; k < K; ++k) G[(size_t)r * K + k] += c * Pbar[(size_t)s * K + k];
    }
}

}  // namespace ridg
