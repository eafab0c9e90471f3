/* Prints sizeof / offsetof of the public structs so the ctypes binding can be checked. */
#include <stddef.h>
#include <stdio.h>

#include "x2c.h"

int main(void) {
  printf("options %zu %zu %zu %zu %zu %zu\n", sizeof(x2c_options), offsetof(x2c_options, two_component),
         offsetof(x2c_options, precision), offsetof(x2c_options, so_same_atom_only),
         offsetof(x2c_options, n_slices), offsetof(x2c_options, reserved));
  printf("mats %zu %zu %zu\n", sizeof(x2c_mats), offsetof(x2c_mats, S), offsetof(x2c_mats, Wz));
  printf("hout %zu\n", sizeof(x2c_hout));
  printf("uout %zu %zu\n", sizeof(x2c_uout), offsetof(x2c_uout, US));
  printf("layout %zu %zu %zu %zu\n", sizeof(x2c_layout), offsetof(x2c_layout, atom_offset),
         offsetof(x2c_layout, n_kinds), offsetof(x2c_layout, kinds));
  printf("counters %zu %zu\n", sizeof(x2c_counters), offsetof(x2c_counters, credited_flops));
  return 0;
}
