/* Prints sizeof / offsetof of the public structs so the ctypes binding can be checked. */
#include <stddef.h>
#include <stdio.h>

#include "x2c.h"

int main(void) {
  printf("options %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(x2c_options), offsetof(x2c_options, two_component),
         offsetof(x2c_options, precision), offsetof(x2c_options, so_same_atom_only),
         offsetof(x2c_options, n_slices), offsetof(x2c_options, local_approx), offsetof(x2c_options, h_upper_only),
         offsetof(x2c_options, decoupling));
  printf("property %zu %zu %zu\n", sizeof(x2c_property), offsetof(x2c_property, LL), offsetof(x2c_property, SS));
  printf("mats %zu %zu %zu\n", sizeof(x2c_mats), offsetof(x2c_mats, S), offsetof(x2c_mats, Wz));
  printf("hout %zu\n", sizeof(x2c_hout));
  printf("uout %zu %zu\n", sizeof(x2c_uout), offsetof(x2c_uout, US));
  printf("layout %zu %zu %zu %zu\n", sizeof(x2c_layout), offsetof(x2c_layout, atom_offset),
         offsetof(x2c_layout, n_kinds), offsetof(x2c_layout, kinds));
  printf("counters %zu %zu\n", sizeof(x2c_counters), offsetof(x2c_counters, credited_flops));
  printf("server_options %zu %zu %zu\n", sizeof(x2c_server_options), offsetof(x2c_server_options, hbm_budget_bytes),
         offsetof(x2c_server_options, reserved));
  printf("request %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(x2c_request), offsetof(x2c_request, kind),
         offsetof(x2c_request, layout), offsetof(x2c_request, kind_key), offsetof(x2c_request, mol),
         offsetof(x2c_request, ld), offsetof(x2c_request, out), offsetof(x2c_request, t_arrival));
  printf("result %zu %zu %zu %zu\n", sizeof(x2c_result), offsetof(x2c_result, h), offsetof(x2c_result, t_end),
         offsetof(x2c_result, slot));
  printf("server_stats %zu %zu %zu %zu\n", sizeof(x2c_server_stats), offsetof(x2c_server_stats, latency_p50_ms),
         offsetof(x2c_server_stats, bytes_in_use), offsetof(x2c_server_stats, max_concurrent));
  printf("graph_stats %zu %zu %zu\n", sizeof(x2c_graph_stats), offsetof(x2c_graph_stats, cached),
         offsetof(x2c_graph_stats, last_replayed));
  return 0;
}
