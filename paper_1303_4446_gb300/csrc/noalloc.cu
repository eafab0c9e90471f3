// x2c_atomic_transforms_noalloc: the batched decoupling solve of x2c_atomic_transforms for
// callers that cannot allocate device memory.  Its scratch lives in one fixed, file-scope
// device array instead of a context workspace, so the call performs no cudaMalloc/cudaFree
// and needs no context (whose creation allocates).
#include <cstring>
#include <mutex>

#include "common.cuh"

namespace {

// The scratch array.  Every GPU that loads this library holds it until the process exits.
// In host code `g_noalloc_scratch` is only a stand-in for the symbol, not a device address:
// the address used by the kernels comes from cudaGetSymbolAddress (see scratch_base).
static __device__ __align__(256) unsigned char g_noalloc_scratch[X2C_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
char *g_base[kMaxDevices] = {};
void *g_ctx[kMaxDevices] = {};  // the context the cached address belongs to

// Current driver context (CUcontext as an opaque pointer), through the driver entry point
// the runtime exposes, so the library needs no link against the driver library.
void *current_context() {
  using GetCurrent = int (*)(void **);
  static GetCurrent fn = [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPoint("cuCtxGetCurrent", &f, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      f = nullptr;
    }
    return reinterpret_cast<GetCurrent>(f);
  }();
  void *c = nullptr;
  if (!fn || fn(&c) != 0) return nullptr;
  return c;
}

// Set-up, once per device (and again after that device's context was torn down and
// re-created, e.g. by cudaDeviceReset), with that device current: the device address of the
// array.  The first lookup may load the module that holds the array.
x2c_status scratch_base(int device, char **out) {
  if (device < 0 || device >= kMaxDevices) return X2C_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_mutex);
  void *ctx = current_context();
  if (!g_base[device] || !ctx || ctx != g_ctx[device]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      g_base[device] = nullptr;
      return X2C_ERR_CUDA;
    }
    g_base[device] = static_cast<char *>(p);
    g_ctx[device] = current_context();
  }
  *out = g_base[device];
  return X2C_OK;
}

size_t round256(size_t b) { return ((b + 255) / 256) * 256; }

}  // namespace

extern "C" x2c_status x2c_atomic_transforms_noalloc(const x2c_options *opt, int32_t n_problems,
                                                    const x2c_mats *inputs, const x2c_uout *U,
                                                    void *stream) {
  if (!opt || n_problems < 1 || !inputs || !U) return X2C_ERR_ARG;
  if (opt->two_component != 0 && opt->two_component != 1) return X2C_ERR_ARG;
  if (opt->decoupling != X2C_DEC_X2C || opt->h_upper_only != 0) return X2C_ERR_ARG;  // X2C transforms only
  const int nc = opt->two_component ? 4 : 1;
  const int n = inputs[0].n;
  if (n < 1 || n > x2c::kMaxSolveN) return X2C_ERR_ARG;
  for (int i = 0; i < n_problems; ++i) {
    const x2c_mats &m = inputs[i];
    if (m.n != n || !m.S || !m.T || !m.V || !m.W0) return X2C_ERR_ARG;
    if (nc == 4 && (!m.Wx || !m.Wy || !m.Wz)) return X2C_ERR_ARG;
    for (int q = 0; q < nc; ++q)
      if (!U[i].UL[q] || !U[i].US[q]) return X2C_ERR_ARG;
  }
  // Layout of the array: status word | input descriptors | U^L, U^S | solve scratch.
  const size_t nb = (size_t)n_problems, n2 = (size_t)n * n;
  const size_t desc_off = 256;
  const size_t u_off = desc_off + round256(nb * sizeof(x2c::InputDesc));
  const size_t solve_off = u_off + round256(2 * nb * nc * n2 * sizeof(double));
  const size_t need = solve_off + x2c::solve_workspace_bytes((int)nb, n, nc);
  if (need > (size_t)X2C_NOALLOC_SCRATCH_BYTES) return X2C_ERR_NOMEM;

  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) {
    cudaGetLastError();
    return X2C_ERR_CUDA;
  }
  char *base = nullptr;
  x2c_status s = scratch_base(device, &base);
  if (s != X2C_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  x2c_ctx local;  // host-side bookkeeping only; its status word is inside the array
  local.device = device;
  local.d_status = reinterpret_cast<int *>(base);
  // The array keeps the previous call's contents: the status word must start at zero
  // (everything else is fully written before it is read).
  if (cudaMemsetAsync(local.d_status, 0, sizeof(int), st) != cudaSuccess) {
    cudaGetLastError();
    return X2C_ERR_CUDA;
  }
  std::vector<x2c::InputDesc> hd(nb);
  for (size_t i = 0; i < nb; ++i) {
    const x2c_mats &m = inputs[i];
    x2c::InputDesc d{};
    d.S = m.S;
    d.T = m.T;
    d.V = m.V;
    d.W[0] = m.W0;
    if (nc == 4) {
      d.W[1] = m.Wx;
      d.W[2] = m.Wy;
      d.W[3] = m.Wz;
    }
    d.ld = n;
    hd[i] = d;
  }
  auto *d_desc = reinterpret_cast<x2c::InputDesc *>(base + desc_off);
  if (cudaMemcpyAsync(d_desc, hd.data(), nb * sizeof(x2c::InputDesc), cudaMemcpyHostToDevice, st) != cudaSuccess) {
    cudaGetLastError();
    return X2C_ERR_CUDA;
  }
  double *UL = reinterpret_cast<double *>(base + u_off);
  double *US = UL + nb * nc * n2;
  x2c::Arena ar;
  ar.base = base + solve_off;
  ar.cap = (size_t)X2C_NOALLOC_SCRATCH_BYTES - solve_off;
  ar.off = 0;
  const double c = x2c::speed_of_light(opt);
  s = x2c::solve_transforms(&local, st, c, (int)nb, n, nc, d_desc, UL, US, ar);
  if (s != X2C_OK) return s;
  for (size_t i = 0; i < nb; ++i) {
    for (int q = 0; q < nc; ++q) {
      if (cudaMemcpyAsync(U[i].UL[q], UL + (i * nc + q) * n2, n2 * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
          cudaMemcpyAsync(U[i].US[q], US + (i * nc + q) * n2, n2 * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
        cudaGetLastError();
        return X2C_ERR_CUDA;
      }
    }
  }
  // Synchronous: wait for the stream and report the device-side status of this call.
  int code = 0;
  if (cudaStreamSynchronize(st) != cudaSuccess ||
      cudaMemcpy(&code, local.d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return X2C_ERR_CUDA;
  }
  return static_cast<x2c_status>(code);
}
