// Host-side check of the linear path's centre-row operator (built by the tests with g++
// against the library's tables.cpp, no GPU):
//   lin_host_check dim M nu0 nu1 nu2 out.txt [fused]
// writes the upwind box (lo[3], cnt[3]) and P (theta_T rows, box.n theta_S columns), one
// value per line, for the velocity signs of nu and nu itself; with "fused" (dim 2, 3) the
// mixed path's fused step operator G = C P-bar instead of P.
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "tables.h"

int main(int argc, char** argv) {
  if (argc != 7 && argc != 8) return 2;
  const bool fused = argc == 8 && std::string(argv[7]) == "fused";
  const int dim = atoi(argv[1]), M = atoi(argv[2]);
  const double nu[3] = {atof(argv[3]), atof(argv[4]), atof(argv[5])};
  const ridg::RegionBox box = ridg::upwind_box(dim, nu);
  std::vector<double> P;
  const auto t0 = std::chrono::steady_clock::now();
  if (!ridg::linear_operator(dim, M, nu, box, P)) return 3;
  const double secs =
      std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (fused) {
    int thS = 1;
    for (int d = 0; d < dim; ++d) thS *= M + 1;
    const int K = box.n * thS;
    std::vector<double> Pbar(P.begin(), P.begin() + (size_t)thS * K), G;
    ridg::fused_step_operator(dim, M + 1, nu, Pbar, K, G);
    P.swap(G);
  }
  FILE* f = fopen(argv[6], "w");
  if (!f) return 2;
  fprintf(f, "%d %d %d %d %d %d %d\n", box.lo[0], box.lo[1], box.lo[2], box.cnt[0], box.cnt[1],
          box.cnt[2], box.n);
  fprintf(f, "%zu\n", P.size());
  for (double v : P) fprintf(f, "%.17g\n", v);
  fclose(f);
  printf("seconds %.3f\n", secs);
  return 0;
}
