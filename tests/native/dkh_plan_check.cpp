// Prints, for n = 2..14, the number of matrix products of the DKHn Hamiltonian plan
// (dkh_plan.h) and its number of device operations.
#include <cstdio>

#include "../../paper_1303_4446_gb300/csrc/dkh_plan.h"

int main() {
  for (int n = 2; n <= 14; ++n) {
    x2c::dkh::Plan p(n);
    for (int k = 1; k <= n / 2; ++k) p.transform(k);
    p.hamiltonian_slots();
    printf("%d %d %zu %d\n", n, p.products(), p.ops().size(), x2c::dkh::hamiltonian_products(n));
  }
  return 0;
}
