// Host-only check of the quaternion sign tables: reads A, B (4 parts of m x m each) from
// stdin, writes stack(A B) = Lq(A) stack(B) and stack(A+ B) = Lq(A+) stack(B) to stdout.
#include <cstdio>
#include <vector>

#include "../../paper_1303_4446_gb300/csrc/common.cuh"

int main() {
  int m;
  if (scanf("%d", &m) != 1) return 1;
  std::vector<double> A(4 * m * m), B(4 * m * m);
  for (auto &x : A) if (scanf("%lf", &x) != 1) return 1;
  for (auto &x : B) if (scanf("%lf", &x) != 1) return 1;
  for (int adj = 0; adj < 2; ++adj) {
    for (int p = 0; p < 4; ++p)
      for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) {
          double s = 0;
          for (int q = 0; q < 4; ++q) {
            const int c = p ^ q;
            for (int k = 0; k < m; ++k) {
              const double a = adj ? x2c::quat_sign_adj(p, q) * A[(c * m + k) * m + i]
                                   : x2c::quat_sign(p, q) * A[(c * m + i) * m + k];
              s += a * B[(q * m + k) * m + j];
            }
          }
          printf("%.17g\n", s);
        }
  }
  return 0;
}
