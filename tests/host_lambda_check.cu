// Reads symmetric matrices from stdin ("r" then r*r values, row-major, repeated until EOF) and
// prints the smallest eigenvalue the library's host routine (Householder tridiagonalisation and
// Sturm bisection) returns for each, one per line with 17 significant digits.
#include <cstdio>
#include <vector>

#include "../paper_1503_03004_gb300/csrc/sfr_internal.h"

int main() {
  int r;
  while (std::scanf("%d", &r) == 1) {
    std::vector<double> A((size_t)r * r);
    for (auto& x : A)
      if (std::scanf("%lf", &x) != 1) return 2;
    std::printf("%.17g\n", sfr::host_lambda_min(A, r));
  }
  return 0;
}
