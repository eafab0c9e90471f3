// x2c_build_dlu_host: DLU build from host buffers (copy in, build, copy out).
//
// Free-atom DLU runs as a pipeline over chunks of row atoms: the pair blocks (A, B >= A) of
// Eq. 42 are independent, so chunk k is assembled while the upper-block rows of chunk k+1
// cross to the device and the h rows of chunk k-1 come back; the per-kind decoupling solve
// runs while the first chunk is still copying.  Other modes copy everything in, build, and
// copy everything out.
#include <cstdlib>
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

// The diagonal blocks of an N x N matrix in pinned host memory (src: its device mapping),
// gathered by one kernel (CTA a copies atom a's block) instead of one copy per block.
__global__ void gather_diag_kernel(const double *src, double *dst, int64_t N, const int32_t *off) {
  const int a = blockIdx.x;
  const int64_t o = off[a], n = off[a + 1] - o;
  for (int64_t idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int64_t i = idx / n, j = idx - i * n;
    dst[(o + i) * N + o + j] = src[(o + i) * N + o + j];
  }
}

// Device mapping of a host pointer the GPU can read directly (pinned or registered), else NULL.
const double *device_readable(const double *p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type == cudaMemoryTypeHost && a.devicePointer) return static_cast<const double *>(a.devicePointer);
  return nullptr;
}

// Copy the upper block triangle of rows of atoms [a0, a1) (rows of atom a, columns from the
// atom's first function to N - 1) between an N x N host and device matrix.
x2c_status copy_upper_rows(x2c_ctx *ctx, double *dst, const double *src, int64_t N, const x2c_layout *lay, int a0,
                           int a1, cudaMemcpyKind kind, cudaStream_t st) {
  for (int a = a0; a < a1; ++a) {
    const int64_t o = lay->atom_offset[a], n = lay->atom_offset[a + 1] - o;
    X2C_TRY_CUDA(ctx, cudaMemcpy2DAsync(dst + o * N + o, N * sizeof(double), src + o * N + o, N * sizeof(double),
                                        (N - o) * sizeof(double), n, kind, st));
  }
  return X2C_OK;
}

x2c_status copy_upper_blocks(x2c_ctx *ctx, double *dst, const double *src, int64_t N, const x2c_layout *lay,
                             cudaStream_t st) {
  return copy_upper_rows(ctx, dst, src, N, lay, 0, lay->n_atoms, cudaMemcpyHostToDevice, st);
}

// The row band of atoms [a0, a1) from the band's first column to N - 1, as ONE 2D copy: the
// upper block triangle of those rows plus the blocks below the diagonal inside the band
// (a few per cent more bytes, but one copy call instead of one per atom: the host's copy
// calls, not the link, bound a pipeline of thousands of per-atom copies).
x2c_status copy_band(x2c_ctx *ctx, double *dst, const double *src, int64_t N, const x2c_layout *lay, int a0, int a1,
                     cudaMemcpyKind kind, cudaStream_t st) {
  const int64_t r0 = lay->atom_offset[a0], r1 = lay->atom_offset[a1];
  X2C_TRY_CUDA(ctx, cudaMemcpy2DAsync(dst + r0 * N + r0, N * sizeof(double), src + r0 * N + r0, N * sizeof(double),
                                      (N - r0) * sizeof(double), r1 - r0, kind, st));
  return X2C_OK;
}

// Row-atom chunks of about equal copy volume: atom a carries n_a (N - offset_a) elements of
// the upper block triangle.
std::vector<int> row_chunks(const x2c_layout *lay, int64_t N, int chunks) {
  const int L = lay->n_atoms;
  std::vector<double> cum(L + 1, 0.0);
  for (int a = 0; a < L; ++a)
    cum[a + 1] = cum[a] + double(lay->atom_offset[a + 1] - lay->atom_offset[a]) * double(N - lay->atom_offset[a]);
  std::vector<int> cut{0};
  for (int k = 1; k < chunks; ++k) {
    const double target = cum[L] * k / chunks;
    int a = cut.back() + 1;
    while (a < L && cum[a] < target) ++a;
    if (a < L && a > cut.back()) cut.push_back(a);
  }
  cut.push_back(L);
  return cut;
}

struct Events {
  std::vector<cudaEvent_t> ev;
  ~Events() {
    for (auto e : ev) cudaEventDestroy(e);
  }
  x2c_status make(x2c_ctx *ctx, size_t n) {
    ev.assign(n, nullptr);
    for (auto &e : ev) X2C_TRY_CUDA(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return X2C_OK;
  }
};

// Row-atom chunks of the pipeline (X2C_HOST_CHUNKS overrides, 1..64).  Measured on the
// Ag309 two-component build (ms per call): 6 chunks 29.3, 8 27.4, 12 26.0.
int pipeline_chunks() {
  static const int n = [] {
    const char *e = std::getenv("X2C_HOST_CHUNKS");
    const int v = e ? std::atoi(e) : 0;
    return (v >= 1 && v <= 64) ? v : 12;
  }();
  return n;
}

}  // namespace

extern "C" x2c_status x2c_build_dlu_host(x2c_ctx *ctx, const x2c_options *opt, const x2c_layout *lay,
                                         const x2c_mats *mol, const x2c_hout *h, void *stream) {
  if (!ctx || !opt || !lay || !mol || !h || mol->n < 1 || lay->n_atoms < 1 || !lay->atom_offset)
    return X2C_ERR_ARG;
  if (opt->h_upper_only != 0 && opt->h_upper_only != 1) return X2C_ERR_ARG;
  X2C_TRY_CUDA(ctx, cudaSetDevice(ctx->device));
  x2c_options o = *opt;  // the build calls below take no host-copy options
  o.h_upper_only = 0;
  X2C_TRY(x2c::check_options(&o));
  const bool upper_only = opt->h_upper_only == 1;
  const int nc = opt->two_component ? 4 : 1;
  const int64_t N = mol->n, N2 = N * N;
  const int L = lay->n_atoms;
  const bool mb = opt->dlu_potential == X2C_DLU_MOLECULAR_BLOCK;
  const bool dlh = opt->local_approx == X2C_LOCAL_DLH;
  const bool so_blocks = nc == 4 && opt->so_same_atom_only;
  if (!mol->S || !mol->T || !mol->V || !mol->W0) return X2C_ERR_ARG;
  if (nc == 4 && (!mol->Wx || !mol->Wy || !mol->Wz)) return X2C_ERR_ARG;
  for (int q = 0; q < nc; ++q)
    if (!h->h[q]) return X2C_ERR_ARG;
  if (lay->atom_offset[0] != 0 || lay->atom_offset[L] != N) return X2C_ERR_ARG;
  for (int a = 0; a < L; ++a)
    if (lay->atom_offset[a + 1] <= lay->atom_offset[a]) return X2C_ERR_ARG;
  int64_t kind_doubles = 0, kind_u_doubles = 0;
  if (!mb) {
    if (!lay->kinds || lay->n_kinds < 1) return X2C_ERR_ARG;
    for (int k = 0; k < lay->n_kinds; ++k) {
      const int64_t n2 = (int64_t)lay->kinds[k].n * lay->kinds[k].n;
      if (lay->kinds[k].n < 1) return X2C_ERR_ARG;
      kind_doubles += (int64_t)(3 + nc + 1) * n2;
      kind_u_doubles += 2 * nc * n2;
    }
  }
  const bool pipelined = !mb && !dlh && L >= 2;
  // staging layout: S (molecular-block mode only), T, V, W0, Wx, Wy, Wz (as needed), h
  // parts, kinds, kind transforms (pipelined path)
  const int64_t mats = (mb ? 1 : 0) + 3 + (nc == 4 ? 3 : 0);
  const size_t bytes =
      sizeof(double) * ((mats + nc) * N2 + kind_doubles + (pipelined ? kind_u_doubles : 0) + (L + 1) / 2 + 64) + 1024;
  X2C_TRY(ensure_stage(ctx, bytes));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double *next = reinterpret_cast<double *>(ctx->stage);
  double *dS = nullptr;
  if (mb) { dS = next; next += N2; }
  double *dT = next, *dV = dT + N2, *dW0 = dV + N2;
  next = dW0 + N2;
  if (!mb) dS = dT;  // free-atom mode never reads the molecular S
  double *dW[3] = {nullptr, nullptr, nullptr};
  if (nc == 4)
    for (int k = 0; k < 3; ++k) { dW[k] = next; next += N2; }
  double *dh[4] = {nullptr, nullptr, nullptr, nullptr};
  for (int q = 0; q < nc; ++q) { dh[q] = next; next += N2; }
  const size_t full = N2 * sizeof(double);
  // The copies are spread over the call's stream and three side streams of the context, so
  // that several copy engines move the matrices at once; the side streams start after the
  // work already on `st`, and `st` waits for them before it reads what they copied.
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
  // kinds (small) first, on the last side stream
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
  const double *hw[3] = {mol->Wx, mol->Wy, mol->Wz};
  if (so_blocks) {
    // same-atom spin-orbit blocks: one gather kernel per matrix when the host buffers are
    // device-readable (pinned), so that hundreds of small copies do not sit on the copy engine
    // ahead of the row bands; else one copy per block
    const double *mw[3] = {device_readable(hw[0]), device_readable(hw[1]), device_readable(hw[2])};
    if (mw[0] && mw[1] && mw[2]) {
      int32_t *doff = reinterpret_cast<int32_t *>(next);
      next += (L + 1 + 1) / 2 + 32;
      X2C_TRY(x2c::upload(ctx, cs[3], doff, lay->atom_offset, sizeof(int32_t) * (L + 1)));
      for (int k = 0; k < 3; ++k) {
        x2c::tbegin(ctx, cs[3]);
        gather_diag_kernel<<<L, 256, 0, cs[3]>>>(mw[k], dW[k], N, doff);
        X2C_TRY(x2c::launched(ctx, "gather_diag_kernel", cs[3]));
      }
    } else {
      for (int k = 0; k < 3; ++k) X2C_TRY(copy_diag_blocks(ctx, dW[k], hw[k], N, lay, cs[3]));
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

  if (!pipelined) {
    if (dlh) {  // DLH reads T and V everywhere and W0 on the same-atom blocks only
      X2C_TRY_CUDA(ctx, cudaMemcpyAsync(dT, mol->T, full, cudaMemcpyHostToDevice, cs[0]));
      X2C_TRY_CUDA(ctx, cudaMemcpyAsync(dV, mol->V, full, cudaMemcpyHostToDevice, cs[1]));
      X2C_TRY(copy_diag_blocks(ctx, dW0, mol->W0, N, lay, cs[2]));
    } else {
      X2C_TRY(copy_upper_blocks(ctx, dT, mol->T, N, lay, cs[0]));
      X2C_TRY(copy_upper_blocks(ctx, dV, mol->V, N, lay, cs[1]));
      X2C_TRY(copy_upper_blocks(ctx, dW0, mol->W0, N, lay, cs[2]));
    }
    if (mb) X2C_TRY(copy_diag_blocks(ctx, dS, mol->S, N, lay, cs[3]));
    if (nc == 4 && !so_blocks)
      for (int k = 0; k < 3; ++k) X2C_TRY(copy_upper_blocks(ctx, dW[k], hw[k], N, lay, cs[(k + 1) % 4]));
    X2C_TRY(join());
    X2C_TRY(x2c_build_dlu(ctx, &o, &dl, &dm, &dho, stream));
    X2C_TRY(fork());
    for (int q = 0; q < nc; ++q) {
      if (upper_only)
        X2C_TRY(copy_upper_rows(ctx, h->h[q], dh[q], N, lay, 0, L, cudaMemcpyDeviceToHost, cs[q]));
      else
        X2C_TRY_CUDA(ctx, cudaMemcpyAsync(h->h[q], dh[q], full, cudaMemcpyDeviceToHost, cs[q]));
    }
    X2C_TRY(join());
    X2C_TRY_CUDA(ctx, cudaStreamSynchronize(st));
    return X2C_OK;
  }

  // ---- pipelined free-atom DLU
  // 1. per-kind transforms, as soon as the kinds are on the device (side stream 3 copied them)
  const int nk = lay->n_kinds;
  std::vector<x2c_uout> ku_out(nk);
  std::vector<const double *> ul(nk), us(nk);
  for (int k = 0; k < nk; ++k) {
    const int64_t n2 = (int64_t)lay->kinds[k].n * lay->kinds[k].n;
    x2c_uout u{};
    for (int q = 0; q < nc; ++q) { u.UL[q] = next + q * n2; u.US[q] = next + (nc + q) * n2; }
    ul[k] = next;
    us[k] = next + nc * n2;
    next += 2 * nc * n2;
    ku_out[k] = u;
  }
  const std::vector<int> cut = row_chunks(lay, N, pipeline_chunks());
  const int nch = (int)cut.size() - 1;
  Events ev;
  X2C_TRY(ev.make(ctx, 2 * (size_t)nch + 2));
  cudaEvent_t ev_kinds = ev.ev[2 * nch], ev_out = ev.ev[2 * nch + 1];
  X2C_TRY_CUDA(ctx, cudaEventRecord(ev_kinds, cs[3]));
  X2C_TRY_CUDA(ctx, cudaStreamWaitEvent(st, ev_kinds, 0));
  X2C_TRY(x2c_atomic_transforms(ctx, &o, nk, dk.data(), ku_out.data(), stream));
  const x2c::KindTransforms kt{ul.data(), us.data()};
  // 2. chunk k: rows in on side stream 1 (one stream, so that the copy engine delivers the
  //    chunks in order), assembly on `st`, h rows out on side stream 3
  for (int c = 0; c < nch; ++c) {
    const int a0 = cut[c], a1 = cut[c + 1];
    cudaStream_t in = cs[1];
    X2C_TRY(copy_band(ctx, dT, mol->T, N, lay, a0, a1, cudaMemcpyHostToDevice, in));
    X2C_TRY(copy_band(ctx, dV, mol->V, N, lay, a0, a1, cudaMemcpyHostToDevice, in));
    X2C_TRY(copy_band(ctx, dW0, mol->W0, N, lay, a0, a1, cudaMemcpyHostToDevice, in));
    if (nc == 4 && !so_blocks)
      for (int k = 0; k < 3; ++k) X2C_TRY(copy_band(ctx, dW[k], hw[k], N, lay, a0, a1, cudaMemcpyHostToDevice, in));
    X2C_TRY_CUDA(ctx, cudaEventRecord(ev.ev[2 * c], in));
    X2C_TRY_CUDA(ctx, cudaStreamWaitEvent(st, ev.ev[2 * c], 0));
    X2C_TRY(x2c::dlu_build(ctx, &o, 1, &dl, &dm, &dho, &kt, st, nullptr, a0, a1));
    X2C_TRY_CUDA(ctx, cudaEventRecord(ev.ev[2 * c + 1], st));
    // the rows of this chunk are complete now: their blocks left of the diagonal are the
    // mirrors written by this and the earlier chunks, the rest by this chunk
    cudaStream_t out = cs[3];
    X2C_TRY_CUDA(ctx, cudaStreamWaitEvent(out, ev.ev[2 * c + 1], 0));
    const int64_t r0 = lay->atom_offset[a0], r1 = lay->atom_offset[a1];
    for (int q = 0; q < nc; ++q) {
      if (upper_only)
        X2C_TRY(copy_band(ctx, h->h[q], dh[q], N, lay, a0, a1, cudaMemcpyDeviceToHost, out));
      else
        X2C_TRY_CUDA(ctx, cudaMemcpyAsync(h->h[q] + r0 * N, dh[q] + r0 * N, (r1 - r0) * N * sizeof(double),
                                          cudaMemcpyDeviceToHost, out));
    }
  }
  X2C_TRY_CUDA(ctx, cudaEventRecord(ev_out, cs[3]));
  X2C_TRY_CUDA(ctx, cudaStreamWaitEvent(st, ev_out, 0));
  X2C_TRY(join());
  X2C_TRY_CUDA(ctx, cudaStreamSynchronize(st));
  return X2C_OK;
}
