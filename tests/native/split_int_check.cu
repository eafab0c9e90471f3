// Host driver for the split-precision integer helpers: reads commands from stdin and prints
// results, so tests/test_split_int_cpu.py can compare them with exact Python arithmetic.
#include <cstdio>
#include <cstring>

#include "../../paper_1303_4446_gb300/csrc/split_int.cuh"

int main() {
  char cmd[16];
  while (scanf("%15s", cmd) == 1) {
    if (!strcmp(cmd, "fp")) {  // fixed_point: hex bits of x, shift
      unsigned long long b;
      int sh;
      if (scanf("%llx %d", &b, &sh) != 2) return 1;
      double x;
      memcpy(&x, &b, 8);
      printf("%lld %d\n", x2c::fixed_point(x, sh), x2c::frexp_exp(x));
    } else if (!strcmp(cmd, "dg")) {  // digits S=5 and S=6 of F
      long long F;
      if (scanf("%lld", &F) != 1) return 1;
      int d5[5], d6[6];
      x2c::digits<5>(F, d5);
      x2c::digits<6>(F, d6);
      for (int i = 0; i < 5; ++i) printf("%d ", d5[i]);
      for (int i = 0; i < 6; ++i) printf("%d ", d6[i]);
      printf("\n");
    } else if (!strcmp(cmd, "sd")) {  // scaled_to_double: I, E
      long long I;
      int E;
      if (scanf("%lld %d", &I, &E) != 2) return 1;
      double v = x2c::scaled_to_double(I, E);
      unsigned long long b;
      memcpy(&b, &v, 8);
      printf("%llx\n", b);
    }
  }
  return 0;
}
