// x2c_build_dlu_host: DLU build from host buffers (copy in, build, copy out).
#include <cstring>

#include "common.cuh"

using x2c::ensure_stage;

namespace {

// Copy the diagonal blocks of an N x N host matrix into the same places of a device matrix.
x2c_status copy_diag_blocks(x2c_ctx *ctx, double *dst, const double *src, int64_t N,
                            const x2c_layout *lay, cudaStream_t st) {
  for (int a = 0; a < lay->n_atoms; ++a) {
    const int64_t o = lay->atom_offset[a], n = lay->atom_offset[a + 1] - o;
    X2C_TRY_CUDA(ctx, cudaMemcpy2DAsync(dst + o * N + o, N * sizeof(double), src + o * N + o,
                                        N * sizeof(double), n * sizeof(double), n,
                                        cudaMemcpyHostToDevice, st));
  }
  return X2C_OK;
}

// Copy the upper block triangle (rows of atom a, columns from the atom's first function to
// N - 1) of an N x N host matrix into the same places of a device matrix.
x2c_status copy_upper_blocks(x2c_ctx *ctx, double *dst, const double *src, int64_t N, const x2c_layout *lay,
                             cudaStream_t st) {
  for (int a = 0; a < lay->n_atoms; ++a) {
    const int64_t o = lay->atom_offset[a], n = lay->atom_offset[a + 1] - o;
    X2C_TRY_CUDA(ctx, cudaMemcpy2DAsync(dst + o * N + o, N * sizeof(double), src + o * N + o, N * sizeof(double),
                                        (N - o) * sizeof(double), n, cudaMemcpyHostToDevice, st));
  }
  return X2C_OK;
}

}  // namespace

extern "C" x2c_status x2c_build_dlu_host(x2c_ctx *ctx, const x2c_options *opt, const x2c_layout *lay,
                                         const x2c_mats *mol, const x2c_hout *h, void *stream) {
  if (!ctx || !opt || !lay || !mol || !h || mol->n < 1 || lay->n_atoms < 1 || !lay->atom_offset)
    return X2C_ERR_ARG;
  X2C_TRY_CUDA(ctx, cudaSetDevice(ctx->device));
  const int nc = opt->two_component ? 4 : 1;
  const int64_t N = mol->n, N2 = N * N;
  const bool mb = opt->dlu_potential == X2C_DLU_MOLECULAR_BLOCK;
  const bool so_blocks = nc == 4 && opt->so_same_atom_only;
  if (!mol->S || !mol->T || !mol->V || !mol->W0) return X2C_ERR_ARG;
  if (nc == 4 && (!mol->Wx || !mol->Wy || !mol->Wz)) return X2C_ERR_ARG;
  for (int q = 0; q < nc; ++q)
    if (!h->h[q]) return X2C_ERR_ARG;
  int64_t kind_doubles = 0;
  if (!mb) {
    if (!lay->kinds || lay->n_kinds < 1) return X2C_ERR_ARG;
    for (int k = 0; k < lay->n_kinds; ++k) kind_doubles += (int64_t)(3 + nc + 1) * lay->kinds[k].n * lay->kinds[k].n;
  }
  // staging layout: S, T, V, W0, Wx, Wy, Wz (as needed), h parts, kinds
  const int64_t mats = 4 + (nc == 4 ? 3 : 0);
  const size_t bytes = sizeof(double) * ((mats + nc) * N2 + kind_doubles) + 1024;
  X2C_TRY(ensure_stage(ctx, bytes));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double *base = reinterpret_cast<double *>(ctx->stage);
  double *dS = base, *dT = dS + N2, *dV = dT + N2, *dW0 = dV + N2;
  double *dW[3] = {nullptr, nullptr, nullptr};
  double *next = dW0 + N2;
  if (nc == 4)
    for (int k = 0; k < 3; ++k) { dW[k] = next; next += N2; }
  double *dh[4] = {nullptr, nullptr, nullptr, nullptr};
  for (int q = 0; q < nc; ++q) { dh[q] = next; next += N2; }
  const size_t full = N2 * sizeof(double);
  // The copies are spread over the call's stream and three side streams of the context, so
  // that several copy engines move the matrices at once; the side streams start after the
  // work already on `st` and `st` waits for them before the build (and again for the copies
  // of h back).
  X2C_TRY(x2c::ensure_aux_streams(ctx, 3));
  cudaStream_t cs[4] = {st, ctx->aux[0], ctx->aux[1], ctx->aux[2]};
  auto fork = [&]() -> x2c_status {
    X2C_TRY_CUDA(ctx, cudaEventRecord(ctx->aux_fork, st));
    for (int i = 1; i < 4; ++i) X2C_TRY_CUDA(ctx, cudaStreamWaitEvent(cs[i], ctx->aux_fork, 0));
    return X2C_OK;
  };
  auto join = [&]() -> x2c_status {
    for (int i = 1; i < 4; ++i) {
      X2C_TRY_CUDA(ctx, cudaEventRecord(ctx->aux_join[i - 1], cs[i]));
      X2C_TRY_CUDA(ctx, cudaStreamWaitEvent(st, ctx->aux_join[i - 1], 0));
    }
    return X2C_OK;
  };
  X2C_TRY(fork());
  // the pair assembly reads the blocks A <= B; DLH reads T and V everywhere and W0 on the
  // same-atom blocks only
  if (opt->local_approx == X2C_LOCAL_DLH) {
    X2C_TRY_CUDA(ctx, cudaMemcpyAsync(dT, mol->T, full, cudaMemcpyHostToDevice, cs[0]));
    X2C_TRY_CUDA(ctx, cudaMemcpyAsync(dV, mol->V, full, cudaMemcpyHostToDevice, cs[1]));
    X2C_TRY(copy_diag_blocks(ctx, dW0, mol->W0, N, lay, cs[2]));
  } else {
    X2C_TRY(copy_upper_blocks(ctx, dT, mol->T, N, lay, cs[0]));
    X2C_TRY(copy_upper_blocks(ctx, dV, mol->V, N, lay, cs[1]));
    X2C_TRY(copy_upper_blocks(ctx, dW0, mol->W0, N, lay, cs[2]));
  }
  if (mb) X2C_TRY(copy_diag_blocks(ctx, dS, mol->S, N, lay, cs[3]));
  const double *hw[3] = {mol->Wx, mol->Wy, mol->Wz};
  for (int k = 0; k < 3 && nc == 4; ++k) {
    if (so_blocks) X2C_TRY(copy_diag_blocks(ctx, dW[k], hw[k], N, lay, cs[3]));
    else X2C_TRY(copy_upper_blocks(ctx, dW[k], hw[k], N, lay, cs[(k + 1) % 4]));
  }
  std::vector<x2c_mats> dk;
  if (!mb) {
    for (int k = 0; k < lay->n_kinds; ++k) {
      const x2c_mats &km = lay->kinds[k];
      const size_t nb = (size_t)km.n * km.n * sizeof(double);
      x2c_mats d{};
      d.n = km.n;
      const double *src[7] = {km.S, km.T, km.V, km.W0, km.Wx, km.Wy, km.Wz};
      double *dst[7] = {nullptr};
      for (int i = 0; i < 3 + (nc == 4 ? 4 : 1); ++i) {
        if (!src[i]) return X2C_ERR_ARG;
        dst[i] = next;
        next += (size_t)km.n * km.n;
        X2C_TRY_CUDA(ctx, cudaMemcpyAsync(dst[i], src[i], nb, cudaMemcpyHostToDevice, cs[3]));
      }
      d.S = dst[0]; d.T = dst[1]; d.V = dst[2]; d.W0 = dst[3];
      d.Wx = dst[4]; d.Wy = dst[5]; d.Wz = dst[6];
      dk.push_back(d);
    }
  }
  x2c_mats dm{};
  dm.n = (int32_t)N;
  dm.S = dS; dm.T = dT; dm.V = dV; dm.W0 = dW0;
  dm.Wx = dW[0]; dm.Wy = dW[1]; dm.Wz = dW[2];
  x2c_layout dl = *lay;
  if (!mb) dl.kinds = dk.data();
  x2c_hout dho{};
  for (int q = 0; q < nc; ++q) dho.h[q] = dh[q];
  X2C_TRY(join());
  X2C_TRY(x2c_build_dlu(ctx, opt, &dl, &dm, &dho, stream));
  X2C_TRY(fork());
  for (int q = 0; q < nc; ++q)
    X2C_TRY_CUDA(ctx, cudaMemcpyAsync(h->h[q], dh[q], full, cudaMemcpyDeviceToHost, cs[q]));
  X2C_TRY(join());
  X2C_TRY_CUDA(ctx, cudaStreamSynchronize(st));
  return X2C_OK;
}
