// x2c_s_integrals: the input matrices S, T, V, W0 over primitive s Gaussians on the device
// (one thread per matrix element of the upper triangle, mirrored; the nuclei staged in
// shared memory).  The formulas are in integrals_math.cuh.
#include <algorithm>

#include "common.cuh"
#include "integrals_math.cuh"

namespace {

__global__ void s_integrals_kernel(int n_nuc, const double *__restrict__ nuc_xyz, const double *__restrict__ nuc_z,
                                   int n, const double *__restrict__ bf_xyz, const double *__restrict__ bf_alpha,
                                   double *S, double *T, double *V, double *W0) {
  extern __shared__ double nuc[];  // [3 n_nuc coordinates][n_nuc charges]
  for (int i = threadIdx.x; i < 4 * n_nuc; i += blockDim.x) nuc[i] = i < 3 * n_nuc ? nuc_xyz[i] : nuc_z[i - 3 * n_nuc];
  __syncthreads();
  const int64_t nn = static_cast<int64_t>(n) * n;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < nn;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(idx / n), j = static_cast<int>(idx - static_cast<int64_t>(i) * n);
    if (i > j) continue;
    double s, t, v, w;
    x2c::s_pair_integrals(bf_xyz + 3 * i, bf_alpha[i], bf_xyz + 3 * j, bf_alpha[j], n_nuc, nuc, nuc + 3 * n_nuc, s,
                          t, v, w);
    const int64_t o = idx, m = static_cast<int64_t>(j) * n + i;
    if (S) S[o] = S[m] = s;
    if (T) T[o] = T[m] = t;
    if (V) V[o] = V[m] = v;
    if (W0) W0[o] = W0[m] = w;
  }
}

}  // namespace

extern "C" x2c_status x2c_s_integrals(const x2c_s_basis *basis, double *S, double *T, double *V, double *W0,
                                      void *stream) {
  if (!basis || basis->n < 1 || basis->n_nuc < 0 || !basis->bf_xyz || !basis->bf_alpha ||
      (basis->n_nuc > 0 && (!basis->nuc_xyz || !basis->nuc_z)))
    return X2C_ERR_ARG;
  if (basis->n_nuc > 1536) return X2C_ERR_ARG;  // the nuclei must fit in 48 KB of shared memory
  if (!S && !T && !V && !W0) return X2C_OK;
  const int64_t nn = static_cast<int64_t>(basis->n) * basis->n;
  const int blocks = static_cast<int>(std::min<int64_t>((nn + 255) / 256, 152 * 16));
  const size_t smem = sizeof(double) * 4 * std::max(1, basis->n_nuc);
  s_integrals_kernel<<<blocks, 256, smem, static_cast<cudaStream_t>(stream)>>>(
      basis->n_nuc, basis->nuc_xyz, basis->nuc_z, basis->n, basis->bf_xyz, basis->bf_alpha, S, T, V, W0);
  return cudaGetLastError() == cudaSuccess ? X2C_OK : X2C_ERR_CUDA;
}
