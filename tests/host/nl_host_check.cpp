// Host-side checks of the nonlinear (Newton) path's C++ tables, built by the tests with g++
// against the library's host sources (no GPU):
//   nl_host_check tables M out.txt   -- write the tables of degree M (name, count, values)
//   nl_host_check plan               -- block elimination with the plan's order and fill on a
//                                       random matrix with the region's block sparsity,
//                                       against a dense LU solve; exit 0 on agreement
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <vector>

#include "nl_tables.h"
#include "ridg_internal.h"
#include "tables.h"

using namespace ridg;

static void put(FILE* f, const char* name, const std::vector<double>& v) {
  fprintf(f, "%s %zu\n", name, v.size());
  for (double x : v) fprintf(f, "%.17g\n", x);
}
static void puti(FILE* f, const char* name, const std::vector<int>& v) {
  fprintf(f, "%s %zu\n", name, v.size());
  for (int x : v) fprintf(f, "%d\n", x);
}

static int dump_tables(int M, const char* path) {
  NlHostTables t = build_nl_tables(M);
  NlAsmLists L = build_asm_lists(t);
  FILE* f = fopen(path, "w");
  if (!f) return 2;
  put(f, "Mt", t.Mt);
  put(f, "em", t.em);
  put(f, "PsiV", t.PsiV);
  put(f, "dPsiV", t.dPsiV);
  put(f, "wV", t.wV);
  put(f, "PsiF", t.PsiF);
  put(f, "wF", t.wF);
  put(f, "PhiV", t.PhiV);
  put(f, "dPhiV", t.dPhiV);
  put(f, "PhiF", t.PhiF);
  put(f, "PsiAtP", t.PsiAtP);
  put(f, "PsiAtFP", t.PsiAtFP);
  put(f, "P1", t.P1);
  put(f, "V1", t.V1);
  put(f, "dV1", t.dV1);
  put(f, "ep1", t.ep1);
  put(f, "em1", t.em1);
  put(f, "T0", t.T0);
  put(f, "T1", t.T1);
  puti(f, "dptr", L.dptr);
  puti(f, "doff", L.doff);
  put(f, "dval", L.dval);
  for (int k = 0; k < 4; ++k) {
    char n[16];
    snprintf(n, sizeof(n), "optr%d", k);
    puti(f, n, L.optr[k]);
    snprintf(n, sizeof(n), "ooff%d", k);
    puti(f, n, L.ooff[k]);
    snprintf(n, sizeof(n), "oval%d", k);
    put(f, n, L.oval[k]);
  }
  fclose(f);
  return 0;
}

static int check_plan() {
  const NlPlan p = build_elim_plan();
  const int b = 5, n = 9 * b;
  std::mt19937 rng(1);
  std::uniform_real_distribution<double> U(-1, 1);
  std::vector<double> A((size_t)n * n, 0.0), rhs(n);
  std::vector<std::vector<double>> S(p.nslots, std::vector<double>(b * b, 0.0));
  for (int i = 0; i < 9; ++i)
    for (int j = 0; j < 9; ++j) {
      const bool adj = i == j || std::abs(i % 3 - j % 3) + std::abs(i / 3 - j / 3) == 1;
      if (adj && p.slot[i * 9 + j] < 0) return 3;  // every structural block has a slot
      if (!adj) continue;
      for (int r = 0; r < b; ++r)
        for (int c = 0; c < b; ++c) {
          const double v = U(rng) + (i == j && r == c ? 8.0 : 0.0);
          A[(size_t)(i * b + r) * n + j * b + c] = v;
          S[p.slot[i * 9 + j]][r * b + c] = v;
        }
    }
  for (int i = 0; i < n; ++i) rhs[i] = U(rng);
  std::vector<double> LU = A, x = rhs;
  std::vector<int> perm;
  if (!lu_factor(n, LU.data(), perm)) return 4;
  lu_solve(n, LU.data(), perm, x.data());
  auto inverse = [&](std::vector<double> Mx) {
    std::vector<int> pr;
    lu_factor(b, Mx.data(), pr);
    std::vector<double> out(b * b);
    for (int c = 0; c < b; ++c) {
      std::vector<double> col(b, 0.0);
      col[c] = 1.0;
      lu_solve(b, Mx.data(), pr, col.data());
      for (int r = 0; r < b; ++r) out[r * b + c] = col[r];
    }
    return out;
  };
  std::vector<double> y = rhs;
  for (int t = 0; t < 9; ++t) {
    const int k = p.order[t];
    const std::vector<double> Ik = inverse(S[p.slot[k * 9 + k]]);
    std::vector<double> yk(b, 0.0);
    for (int r = 0; r < b; ++r)
      for (int c = 0; c < b; ++c) yk[r] += Ik[r * b + c] * y[k * b + c];
    for (int r = 0; r < b; ++r) y[k * b + r] = yk[r];
    for (int a = 0; a < p.nn[t]; ++a) {
      std::vector<double>& B = S[p.slot[k * 9 + p.nbr[t][a]]];
      std::vector<double> o(b * b, 0.0);
      for (int r = 0; r < b; ++r)
        for (int c = 0; c < b; ++c)
          for (int q = 0; q < b; ++q) o[r * b + c] += Ik[r * b + q] * B[q * b + c];
      B = o;
    }
    for (int a = 0; a < p.nn[t]; ++a) {
      const int i = p.nbr[t][a];
      const std::vector<double>& Aik = S[p.slot[i * 9 + k]];
      for (int r = 0; r < b; ++r)
        for (int c = 0; c < b; ++c) y[i * b + r] -= Aik[r * b + c] * y[k * b + c];
      for (int c2 = 0; c2 < p.nn[t]; ++c2) {
        const int j = p.nbr[t][c2];
        if (p.slot[i * 9 + j] < 0) return 5;  // fill without a slot
        std::vector<double>& C = S[p.slot[i * 9 + j]];
        const std::vector<double>& Ukj = S[p.slot[k * 9 + j]];
        if (p.first[t][a][c2])
          for (double& v : C) v = 0.0;  // the kernel writes the first update of a fill block
        for (int r = 0; r < b; ++r)
          for (int c = 0; c < b; ++c) {
            double s = 0.0;
            for (int q = 0; q < b; ++q) s += Aik[r * b + q] * Ukj[q * b + c];
            C[r * b + c] -= s;
          }
      }
    }
  }
  for (int t = 8; t >= 0; --t) {
    const int k = p.order[t];
    for (int a = 0; a < p.nn[t]; ++a) {
      const int j = p.nbr[t][a];
      const std::vector<double>& Ukj = S[p.slot[k * 9 + j]];
      for (int r = 0; r < b; ++r)
        for (int c = 0; c < b; ++c) y[k * b + r] -= Ukj[r * b + c] * y[j * b + c];
    }
  }
  double md = 0.0, mx = 0.0;
  for (int i = 0; i < n; ++i) {
    md = std::fmax(md, std::fabs(y[i] - x[i]));
    mx = std::fmax(mx, std::fabs(x[i]));
  }
  printf("slots %d, max |x_plan - x_dense| = %.3e of %.3e\n", p.nslots, md, mx);
  return md <= 1e-12 * mx ? 0 : 1;
}

int main(int argc, char** argv) {
  if (argc >= 4 && !strcmp(argv[1], "tables")) return dump_tables(atoi(argv[2]), argv[3]);
  if (argc >= 2 && !strcmp(argv[1], "plan")) return check_plan();
  fprintf(stderr, "usage: nl_host_check tables M out.txt | plan\n");
  return 2;
}
