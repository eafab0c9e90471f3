// Host build of the device integral formulas (integrals_math.cuh): reads n_nuc, then
// x y z Z per nucleus, then n, then x y z alpha per primitive from stdin, and prints
// S T V W0 of every pair (i, j), row-major, one pair per line.
#include <cstdio>
#include <vector>

#include "../../paper_1303_4446_gb300/csrc/integrals_math.cuh"

int main() {
  int nn = 0, n = 0;
  if (scanf("%d", &nn) != 1) return 1;
  std::vector<double> nxyz(3 * nn), nz(nn);
  for (int c = 0; c < nn; ++c)
    if (scanf("%lf %lf %lf %lf", &nxyz[3 * c], &nxyz[3 * c + 1], &nxyz[3 * c + 2], &nz[c]) != 4) return 1;
  if (scanf("%d", &n) != 1) return 1;
  std::vector<double> xyz(3 * n), al(n);
  for (int i = 0; i < n; ++i)
    if (scanf("%lf %lf %lf %lf", &xyz[3 * i], &xyz[3 * i + 1], &xyz[3 * i + 2], &al[i]) != 4) return 1;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s, t, v, w;
      x2c::s_pair_integrals(&xyz[3 * i], al[i], &xyz[3 * j], al[j], nn, nxyz.data(), nz.data(), s, t, v, w);
      printf("%.17g %.17g %.17g %.17g\n", s, t, v, w);
    }
  return 0;
}
