// Split-precision (Ozaki) BF16 pair assembly -- not provided yet.
#include "common.cuh"

namespace x2c {
x2c_status assemble_pairs_split(x2c_ctx *ctx, cudaStream_t st, double c, int nc, int so_all_pairs,
                                const std::vector<PairDesc> &pairs, const MolDesc *d_mols,
                                UTable ut, int max_n, int n_slices, Arena &ar) {
  (void)ctx; (void)st; (void)c; (void)nc; (void)so_all_pairs; (void)pairs; (void)d_mols;
  (void)ut; (void)max_n; (void)n_slices; (void)ar;
  return X2C_ERR_ARG;
}
}  // namespace x2c
