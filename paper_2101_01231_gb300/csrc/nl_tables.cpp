// Host-built FP64 tables of the nonlinear RIDG path (see nl_tables.h).
//
// Reference coordinates (tau, xi_x, xi_y) in [-1, 1]^3; the space-time basis is
// Psi_k = psi_a(tau) phi_bx(xi_x) phi_by(xi_y), k = a thS + bx + nb by, phi_b =
// sqrt(2b+1) P_b.  Point indices run tau slowest, then y, then x.  The projection basis
// (degree 2M per dimension) has the same construction with np = 2M + 1 functions.
#include "nl_tables.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <set>
#include <utility>

#include "ridg_internal.h"
#include "tables.h"

namespace ridg {
namespace {

struct Rule1D {
  std::vector<double> x, w;
};

Rule1D rule(int n) {
  Rule1D r;
  gauss_legendre(n, r.x, r.w);
  return r;
}

// V[b][q] and dV[b][q] for b < nb at the rule's points
void values(int nb, const Rule1D& r, std::vector<double>& V, std::vector<double>& dV) {
  const int n = (int)r.x.size();
  V.assign((size_t)nb * n, 0.0);
  dV.assign((size_t)nb * n, 0.0);
  std::vector<double> v(nb), dv(nb);
  for (int q = 0; q < n; ++q) {
    phi_values(nb, r.x[q], v.data(), dv.data());
    for (int b = 0; b < nb; ++b) {
      V[(size_t)b * n + q] = v[b];
      dV[(size_t)b * n + q] = dv[b];
    }
  }
}

// int_{-1}^{1} f_a g_b h_c with f, g, h in {phi, phi'}: exact Gauss quadrature
std::vector<double> triple1d(int na, int nbb, int nc, bool deriv_a) {
  const int n = (na + nbb + nc) / 2 + 2;
  Rule1D r = rule(n);
  std::vector<double> Va, dVa, Vb, dVb, Vc, dVc;
  values(na, r, Va, dVa);
  values(nbb, r, Vb, dVb);
  values(nc, r, Vc, dVc);
  std::vector<double> T((size_t)na * nbb * nc, 0.0);
  for (int a = 0; a < na; ++a)
    for (int b = 0; b < nbb; ++b)
      for (int c = 0; c < nc; ++c) {
        double s = 0.0;
        for (int q = 0; q < n; ++q)
          s += r.w[q] * (deriv_a ? dVa[(size_t)a * n + q] : Va[(size_t)a * n + q]) *
               Vb[(size_t)b * n + q] * Vc[(size_t)c * n + q];
        T[((size_t)a * nbb + b) * nc + c] = s;
      }
  return T;
}

}  // namespace

NlHostTables build_nl_tables(int M) {
  NlHostTables t;
  const int nb = t.nb = M + 1;
  t.thS = nb * nb;
  t.thT = nb * t.thS;
  const int nq = t.nq = (3 * M + 2) / 2;  // ceil((3M + 1) / 2)
  t.Qv = nq * nq * nq;
  t.Qf = nq * nq;
  const int np = t.np = 2 * M + 1;
  t.QP = np * np * np;
  t.QPf = np * np;
  const int thS = t.thS, thT = t.thT;

  Tables1D t1 = tables1d(nb);
  t.Mt.assign((size_t)nb * nb, 0.0);
  for (int a = 0; a < nb; ++a)
    for (int g = 0; g < nb; ++g) t.Mt[(size_t)a * nb + g] = t1.ep[a] * t1.ep[g] - t1.D[a * nb + g];
  t.em = t1.em;

  // --- residual rule ---
  Rule1D rq = rule(nq);
  std::vector<double> V, dV;
  values(nb, rq, V, dV);
  auto v1 = [&](int b, int q) { return V[(size_t)b * nq + q]; };
  auto d1 = [&](int b, int q) { return dV[(size_t)b * nq + q]; };
  t.V1 = V;
  t.dV1 = dV;
  t.V1T.assign((size_t)nq * nb, 0.0);
  for (int b = 0; b < nb; ++b)
    for (int q = 0; q < nq; ++q) t.V1T[(size_t)q * nb + b] = V[(size_t)b * nq + q];
  t.ep1 = t1.ep;
  t.em1 = t1.em;
  t.wV.assign(t.Qv, 0.0);
  t.PsiV.assign((size_t)thT * t.Qv, 0.0);
  t.dPsiV.assign((size_t)2 * thT * t.Qv, 0.0);
  t.PhiV.assign((size_t)thS * t.Qv, 0.0);
  t.dPhiV.assign((size_t)2 * thS * t.Qv, 0.0);
  for (int qt = 0; qt < nq; ++qt)
    for (int qy = 0; qy < nq; ++qy)
      for (int qx = 0; qx < nq; ++qx) {
        const int q = (qt * nq + qy) * nq + qx;
        t.wV[q] = rq.w[qt] * rq.w[qy] * rq.w[qx];
        for (int k = 0; k < thT; ++k) {
          const int a = k / thS, s = k % thS, bx = s % nb, by = s / nb;
          t.PsiV[(size_t)k * t.Qv + q] = v1(a, qt) * v1(by, qy) * v1(bx, qx);
          t.dPsiV[(size_t)k * t.Qv + q] = v1(a, qt) * v1(by, qy) * d1(bx, qx);
          t.dPsiV[(size_t)(thT + k) * t.Qv + q] = v1(a, qt) * d1(by, qy) * v1(bx, qx);
        }
        for (int s = 0; s < thS; ++s) {
          const int bx = s % nb, by = s / nb;
          t.PhiV[(size_t)s * t.Qv + q] = v1(by, qy) * v1(bx, qx);
          t.dPhiV[(size_t)s * t.Qv + q] = v1(by, qy) * d1(bx, qx);
          t.dPhiV[(size_t)(thS + s) * t.Qv + q] = d1(by, qy) * v1(bx, qx);
        }
      }
  // faces: dim dd at xi_dd = side; points (tau, other dimension)
  t.wF.assign((size_t)2 * t.Qf, 0.0);
  t.PsiF.assign((size_t)4 * thT * t.Qf, 0.0);
  t.PhiF.assign((size_t)4 * thS * t.Qf, 0.0);
  for (int dd = 0; dd < 2; ++dd)
    for (int si = 0; si < 2; ++si) {
      const double* tr = si == 0 ? t1.ep.data() : t1.em.data();
      for (int qt = 0; qt < nq; ++qt)
        for (int qo = 0; qo < nq; ++qo) {
          const int q = qt * nq + qo;
          if (si == 0) t.wF[(size_t)dd * t.Qf + q] = rq.w[qt] * rq.w[qo];
          for (int k = 0; k < thT; ++k) {
            const int a = k / thS, s = k % thS, bx = s % nb, by = s / nb;
            const double vx = dd == 0 ? tr[bx] : v1(bx, qo);
            const double vy = dd == 1 ? tr[by] : v1(by, qo);
            t.PsiF[((size_t)(dd * 2 + si) * thT + k) * t.Qf + q] = v1(a, qt) * vx * vy;
          }
          for (int s = 0; s < thS; ++s) {
            const int bx = s % nb, by = s / nb;
            const double vx = dd == 0 ? tr[bx] : v1(bx, qo);
            const double vy = dd == 1 ? tr[by] : v1(by, qo);
            t.PhiF[((size_t)(dd * 2 + si) * thS + s) * t.Qf + q] = vx * vy;
          }
        }
    }

  // --- projection rule (quasi-quadrature-free) ---
  Rule1D rp = rule(np);
  std::vector<double> Vp, dVp, Vs, dVs;
  values(np, rp, Vp, dVp);  // projection basis (degree 2M)
  values(nb, rp, Vs, dVs);  // solution basis at the projection points
  auto vp = [&](int b, int q) { return Vp[(size_t)b * np + q]; };
  auto vs = [&](int b, int q) { return Vs[(size_t)b * np + q]; };
  t.PsiAtP.assign((size_t)thT * t.QP, 0.0);
  for (int qt = 0; qt < np; ++qt)
    for (int qy = 0; qy < np; ++qy)
      for (int qx = 0; qx < np; ++qx) {
        const int q = (qt * np + qy) * np + qx;
        for (int k = 0; k < thT; ++k) {
          const int a = k / thS, s = k % thS, bx = s % nb, by = s / nb;
          t.PsiAtP[(size_t)k * t.QP + q] = vs(a, qt) * vs(by, qy) * vs(bx, qx);
        }
      }
  t.P1.assign((size_t)np * np, 0.0);
  for (int p = 0; p < np; ++p)
    for (int q = 0; q < np; ++q) t.P1[(size_t)p * np + q] = vp(p, q) * rp.w[q] / 2.0;
  t.PsiAtFP.assign((size_t)4 * thT * t.QPf, 0.0);
  for (int dd = 0; dd < 2; ++dd)
    for (int si = 0; si < 2; ++si) {
      const double* tr = si == 0 ? t1.ep.data() : t1.em.data();
      for (int qt = 0; qt < np; ++qt)
        for (int qo = 0; qo < np; ++qo) {
          const int q = qt * np + qo;
          for (int k = 0; k < thT; ++k) {
            const int a = k / thS, s = k % thS, bx = s % nb, by = s / nb;
            const double vx = dd == 0 ? tr[bx] : vs(bx, qo);
            const double vy = dd == 1 ? tr[by] : vs(by, qo);
            t.PsiAtFP[((size_t)(dd * 2 + si) * thT + k) * t.QPf + q] = vs(a, qt) * vx * vy;
          }
        }
    }

  // --- sparse triple-product lists ---
  const std::vector<double> T0 = triple1d(nb, nb, np, false);  // int phi_a phi_b phi_c
  const std::vector<double> T1 = triple1d(nb, nb, np, true);   // int phi_a' phi_b phi_c
  t.T0 = T0;
  t.T1 = T1;
  auto t0 = [&](int a, int b, int c) { return T0[((size_t)a * nb + b) * np + c]; };
  auto t1d = [&](int a, int b, int c) { return T1[((size_t)a * nb + b) * np + c]; };
  const double tol = 1e-13;
  for (int dd = 0; dd < 2; ++dd) {
    SparseTriple& B = t.beta[dd];
    B.ptr.assign(1, 0);
    for (int k = 0; k < thT; ++k)
      for (int l = 0; l < thT; ++l) {
        const int ak = k / thS, sk = k % thS, bxk = sk % nb, byk = sk / nb;
        const int al = l / thS, sl = l % thS, bxl = sl % nb, byl = sl / nb;
        for (int pt = 0; pt < np; ++pt) {
          const double ft = t0(ak, al, pt);
          if (std::fabs(ft) < tol) continue;
          for (int py = 0; py < np; ++py) {
            const double fy = dd == 1 ? t1d(byk, byl, py) : t0(byk, byl, py);
            if (std::fabs(fy) < tol) continue;
            for (int px = 0; px < np; ++px) {
              const double fx = dd == 0 ? t1d(bxk, bxl, px) : t0(bxk, bxl, px);
              if (std::fabs(fx) < tol) continue;
              B.p.push_back((pt * np + py) * np + px);
              B.val.push_back(ft * fy * fx);
            }
          }
        }
        B.ptr.push_back((int)B.p.size());
      }
    // faces: int over the face of Psi_k Psi_l Psi^f_p, Psi^f_p = psi_pt(tau) phi_po(other)
    for (int sk = 0; sk < 2; ++sk)
      for (int sl = 0; sl < 2; ++sl) {
        const double* trk = sk == 0 ? t1.ep.data() : t1.em.data();
        const double* trl = sl == 0 ? t1.ep.data() : t1.em.data();
        SparseTriple& G = t.gamma[dd][sk][sl];
        G.ptr.assign(1, 0);
        for (int k = 0; k < thT; ++k)
          for (int l = 0; l < thT; ++l) {
            const int ak = k / thS, s1 = k % thS, bxk = s1 % nb, byk = s1 / nb;
            const int al = l / thS, s2 = l % thS, bxl = s2 % nb, byl = s2 / nb;
            const double fn = dd == 0 ? trk[bxk] * trl[bxl] : trk[byk] * trl[byl];
            const int ok = dd == 0 ? byk : bxk, ol = dd == 0 ? byl : bxl;
            for (int pt = 0; pt < np; ++pt) {
              const double ft = t0(ak, al, pt);
              if (std::fabs(ft) < tol) continue;
              for (int po = 0; po < np; ++po) {
                const double fo = t0(ok, ol, po);
                if (std::fabs(fo) < tol) continue;
                G.p.push_back(pt * np + po);
                G.val.push_back(fn * ft * fo);
              }
            }
            G.ptr.push_back((int)G.p.size());
          }
      }
  }
  return t;
}

NlAsmLists build_asm_lists(const NlHostTables& t) {
  NlAsmLists L;
  const int npair = t.thT * t.thT;
  L.dptr.assign(1, 0);
  for (int kl = 0; kl < npair; ++kl) {
    for (int d = 0; d < 2; ++d) {
      const SparseTriple& B = t.beta[d];
      for (int e = B.ptr[kl]; e < B.ptr[kl + 1]; ++e) {
        L.doff.push_back(d * t.QP + B.p[e]);
        L.dval.push_back(B.val[e]);
      }
    }
    for (int f = 0; f < 4; ++f) {
      const int d = f >> 1, si = f & 1;
      const SparseTriple& G = t.gamma[d][si][si];
      for (int e = G.ptr[kl]; e < G.ptr[kl + 1]; ++e) {
        L.doff.push_back(2 * t.QP + f * t.QPf + G.p[e]);
        L.dval.push_back(G.val[e]);
      }
    }
    L.dptr.push_back((int)L.doff.size());
  }
  for (int f = 0; f < 4; ++f) {
    const int d = f >> 1, si = f & 1;
    const SparseTriple& G = t.gamma[d][si][si ^ 1];
    L.optr[f].assign(1, 0);
    for (int kl = 0; kl < npair; ++kl) {
      for (int e = G.ptr[kl]; e < G.ptr[kl + 1]; ++e) {
        L.ooff[f].push_back(2 * t.QP + (4 + f) * t.QPf + G.p[e]);
        L.oval[f].push_back(G.val[e]);
      }
      L.optr[f].push_back((int)L.ooff[f].size());
    }
  }
  return L;
}

// ---------------------------------------------------------------------------------------
// elimination plan
// ---------------------------------------------------------------------------------------
NlPlan build_elim_plan() {
  NlPlan p;
  std::memset(&p, 0, sizeof(p));
  const int order[9] = {0, 2, 6, 8, 1, 3, 5, 7, 4};  // corners, edges, centre
  int pos[9];
  for (int t = 0; t < 9; ++t) {
    p.order[t] = order[t];
    pos[order[t]] = t;
    p.pos[order[t]] = t;
  }
  std::set<std::pair<int, int>> nz;
  for (int r = 0; r < 9; ++r) {
    nz.insert({r, r});
    const int rx = r % 3, ry = r / 3;
    if (rx < 2) nz.insert({r, r + 1}), nz.insert({r + 1, r});
    if (ry < 2) nz.insert({r, r + 3}), nz.insert({r + 3, r});
  }
  for (int i = 0; i < 81; ++i) p.slot[i] = -1;
  int ns = 0;
  for (int r = 0; r < 9; ++r) p.slot[r * 9 + r] = ns++;
  for (auto& ij : nz)
    if (ij.first != ij.second) p.slot[ij.first * 9 + ij.second] = ns++;
  for (int t = 0; t < 9; ++t) {
    const int k = order[t];
    std::vector<int> nb;
    for (int j = 0; j < 9; ++j)
      if (pos[j] > t && (nz.count({k, j}) || nz.count({j, k}))) nb.push_back(j);
    std::sort(nb.begin(), nb.end(), [&](int a, int b) { return pos[a] < pos[b]; });
    p.nn[t] = (int)nb.size();
    for (int a = 0; a < (int)nb.size(); ++a) p.nbr[t][a] = nb[a];
    for (int a = 0; a < (int)nb.size(); ++a)
      for (int b = 0; b < (int)nb.size(); ++b) {
        const std::pair<int, int> ij{nb[a], nb[b]};
        if (!nz.count(ij)) {
          nz.insert(ij);
          p.slot[ij.first * 9 + ij.second] = ns++;
          p.first[t][a][b] = 1;
        }
      }
  }
  p.nslots = ns;
  return p;
}

}  // namespace ridg
