// Internal definitions shared by the CUDA translation units of the X2C library.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "../../include/x2c.h"

// Device-side error codes latched in the context's status word (same values as x2c_status).
#define X2C_DEV_NOT_POSDEF 4
#define X2C_DEV_NOCONV 5
#define X2C_DEV_DECOUPLING 6
#define X2C_DEV_NONFINITE 7

// Split-precision workspace cap of the server's slots, and the fallback of a context whose
// larger workspace could not be allocated (the pair assembly then runs in chunks of this size).
constexpr size_t kSplitWsCapSmall = (size_t)3 << 30;

struct x2c_ctx {
  int device = 0;
  int *d_status = nullptr;      // first device-side error code (0 = none)
  char *ws = nullptr;           // growable device workspace
  size_t ws_bytes = 0;
  char *stage = nullptr;        // growable device staging area of the host-buffer calls
  size_t stage_bytes = 0;
  std::string last_error;
  x2c_counters counters{};
  int64_t launches = 0;         // kernels launched by the current call
  // optional per-kernel timing (x2c_ctx_set_timing): events around every launch
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  struct Pending {
    std::string name;
    size_t begin;  // index of its begin event
    double flops;  // algorithmic flops of the launch (0 where the launcher does not count them)
  };
  struct KernelTotals {
    double ms = 0, flops = 0;
    int64_t launches = 0;
  };
  std::vector<Pending> pending;
  std::map<std::string, KernelTotals> kernel_ms;
  std::string names_buf;
  // when set, the workspace grows stream-ordered from this pool on the call's stream
  // (no device-wide synchronisation; used by the server, whose slots run concurrently)
  cudaMemPool_t pool = nullptr;
  // largest workspace a split-precision pair assembly asks for (it runs in chunks of what
  // fits); the server keeps its slots at kSplitWsCapSmall so that admission under its budget
  // is unchanged, and a context whose large workspace cannot be allocated falls back to it
  size_t split_ws_cap = (size_t)24 << 30;
  // streams on which independent size groups of a batched solve run concurrently
  std::vector<cudaStream_t> aux;
  std::vector<cudaEvent_t> aux_join;
  cudaEvent_t aux_fork = nullptr;
  // pinned staging ring for the small descriptor uploads (see x2c::upload)
  struct Staged {
    size_t start, end;
    cudaEvent_t done;
  };
  char *ring = nullptr;
  size_t ring_cap = 0, ring_head = 0;
  std::vector<Staged> ring_inflight;  // oldest first
  std::vector<cudaEvent_t> ring_events;
  // autotuner: tile choice per workload shape, chosen by timing the candidates once
  bool autotune = true;
  int split_variant = -1;  // >= 0: always this candidate (x2c_ctx_set_split_variant)
  int cta_cap = 0;         // > 0: the persistent split kernels use at most this many CTAs
  std::map<uint64_t, int> tuned;
  std::string tune_log;
  cudaEvent_t tune_ev[2] = {nullptr, nullptr};
  // CUDA-graph replay of repeated identical builds (x2c_ctx_set_graphs; abi.cu)
  struct GraphEntry;
  bool graphs = false;
  bool capturing = false;                 // a build is being captured into a graph
  uint64_t ws_generation = 0;             // bumped whenever the workspace moves
  std::vector<GraphEntry *> graph_cache;  // least recently used first
  std::map<uint64_t, int> graph_seen;     // plan hash -> eager calls with that plan
  std::vector<char *> cap_pinned;         // pinned sources of the current capture's uploads
  size_t cap_off = 0, cap_cap = 0;
  cudaStream_t cap_stream = nullptr;
  int64_t graph_captures = 0, graph_replays = 0;
  bool last_replayed = false;
};

namespace x2c {

constexpr double kDefaultC = 137.035999;

inline double speed_of_light(const x2c_options *o) { return (o && o->c > 0) ? o->c : kDefaultC; }

// Record a CUDA error in the context and return X2C_ERR_CUDA.
inline x2c_status cuda_fail(x2c_ctx *ctx, cudaError_t e, const char *what) {
  if (ctx) {
    ctx->last_error = std::string(what) + ": " + cudaGetErrorString(e);
  }
  return X2C_ERR_CUDA;
}

#define X2C_TRY_CUDA(ctx, call)                                  \
  do {                                                           \
    cudaError_t e__ = (call);                                    \
    if (e__ != cudaSuccess) return x2c::cuda_fail(ctx, e__, #call); \
  } while (0)

#define X2C_TRY(expr)                 \
  do {                                \
    x2c_status s__ = (expr);          \
    if (s__ != X2C_OK) return s__;    \
  } while (0)

// Timing: tbegin() records a begin event before a launch, launched() the end event after
// it (both on the launching stream); x2c_ctx_kernel_times() turns them into durations.
inline cudaEvent_t next_event(x2c_ctx *ctx) {
  if (ctx->ev_used == ctx->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    ctx->ev_pool.push_back(e);
  }
  return ctx->ev_pool[ctx->ev_used++];
}
// Inside a stream capture the record must become a node of the graph (an external record);
// a plain record would only order the captured work.
inline void record_timing_event(x2c_ctx *ctx, cudaEvent_t e, cudaStream_t st) {
  if (ctx->capturing) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
  else cudaEventRecord(e, st);
}
inline void tbegin(x2c_ctx *ctx, cudaStream_t st) {
  if (!ctx->timing) return;
  cudaEvent_t e = next_event(ctx);
  if (e) record_timing_event(ctx, e, st);
}

// Check the launch that was just enqueued and count it; `flops` = the launch's algorithmic
// flops, reported with its time when timing is enabled.
inline x2c_status launched(x2c_ctx *ctx, const char *name, cudaStream_t st = nullptr, double flops = 0) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, name);
  ctx->launches++;
  if (ctx->timing && ctx->ev_used > 0) {
    const size_t begin = ctx->ev_used - 1;
    cudaEvent_t ev = next_event(ctx);
    if (ev) {
      record_timing_event(ctx, ev, st);
      ctx->pending.push_back({name, begin, flops});
    }
  }
  return X2C_OK;
}

__device__ __forceinline__ void flag_error(int *st, int code) { atomicCAS(st, 0, code); }

// ---------------------------------------------------------------------------------------
// Quaternion (time-reversal) algebra of Eq. 5.  A two-component matrix
//   M = I2 (x) M0 + i sum_k sigma_k (x) Mk
// is stored as its four real parts M0..M3 (component-major).  With the Pauli product
// sigma_k sigma_j = delta_kj + i eps_kjl sigma_l, the product C = A B has
//   C0 = A0 B0 - sum_k Ak Bk
//   Cl = A0 Bl + Al B0 - sum_kj eps_kjl Ak Bj
// i.e. stack(C) = Lq(A) stack(B) with the 4 x 4 block matrix Lq(A) whose block (p, q) is
// sign(p, q) * A_{p xor q}; the negative blocks are (0,1) (0,2) (0,3) (1,3) (2,1) (3,2).
// The adjoint A+ has parts (A0^T, -A1^T, -A2^T, -A3^T).
__host__ __device__ __forceinline__ double quat_sign(int p, int q) {
  constexpr unsigned kNeg = (1u << 1) | (1u << 2) | (1u << 3) | (1u << 7) | (1u << 9) | (1u << 14);
  return ((kNeg >> (p * 4 + q)) & 1u) ? -1.0 : 1.0;
}
// Block (p, q) of Lq(A+): sign * A_{p xor q}^T with the adjoint's extra minus on parts 1-3.
__host__ __device__ __forceinline__ double quat_sign_adj(int p, int q) {
  return ((p ^ q) == 0) ? quat_sign(p, q) : -quat_sign(p, q);
}

// Workspace bump allocator for one library call (256-byte aligned slices).
struct Arena {
  char *base = nullptr;
  size_t cap = 0, off = 0;
  double *take(size_t n_doubles) {
    size_t bytes = ((n_doubles * sizeof(double) + 255) / 256) * 256;
    if (off + bytes > cap) return nullptr;
    double *p = reinterpret_cast<double *>(base + off);
    off += bytes;
    return p;
  }
  void *take_bytes(size_t bytes) {
    bytes = ((bytes + 255) / 256) * 256;
    if (off + bytes > cap) return nullptr;
    void *p = base + off;
    off += bytes;
    return p;
  }
};
inline size_t arena_doubles(size_t n) { return ((n * sizeof(double) + 255) / 256) * 256; }

// Grow the context workspace to at least `bytes` (synchronises the device when it grows,
// unless the context has a pool: then the growth is stream-ordered on `st`).  Growth
// bumps ctx->ws_generation and is refused while a build is being captured.
x2c_status ensure_workspace(x2c_ctx *ctx, size_t bytes, Arena *out, cudaStream_t st);
// Copy `bytes` of host memory to the device on `st` through the context's pinned staging
// ring, so that the call returns at once: cudaMemcpyAsync from pageable memory would first
// wait for all work already queued on the stream.  The host data may be reused on return.
x2c_status upload(x2c_ctx *ctx, cudaStream_t st, void *dst, const void *src, size_t bytes);
// Device-side copy and byte fill (kernels, so that they never wait behind bulk transfers on
// the copy engines); src may be pinned host memory's device mapping.
x2c_status device_copy(x2c_ctx *ctx, cudaStream_t st, void *dst, const void *src, size_t bytes);
x2c_status device_fill(x2c_ctx *ctx, cudaStream_t st, void *dst, int value, size_t bytes);

// Destroy the context's captured graphs (waits for the device first).
void drop_graphs(x2c_ctx *ctx);

// Auxiliary streams of the context (created on first use, at most kMaxAuxStreams).
constexpr int kMaxAuxStreams = 4;
x2c_status ensure_aux_streams(x2c_ctx *ctx, int count);
// Workspace size the context holds after a call that needs `bytes`.
size_t workspace_after_growth(const x2c_ctx *ctx, size_t bytes);
// Grow the staging area of the host-buffer calls (synchronises the device when it grows).
x2c_status ensure_stage(x2c_ctx *ctx, size_t bytes);

// Argument checks shared by the entry points.
bool mats_ok(const x2c_mats *m, int nc);
x2c_status check_options(const x2c_options *o);

// Entry points shared by the C ABI and the server.  With dry_bytes non-NULL nothing is
// enqueued: *dry_bytes receives the workspace the call needs.
struct KindTransforms {
  const double *const *UL;  // host arrays indexed by kind: device U^L, U^S of that kind,
  const double *const *US;  // nc n^2 doubles each, part-major (NULL entry = solve it)
};
x2c_status full_build(x2c_ctx *ctx, const x2c_options *opt, const x2c_mats *mol, const x2c_hout *h,
                      const x2c_uout *U, cudaStream_t st, size_t *dry_bytes);
// a_begin, a_end (one molecule only): assemble only the pair blocks (A, B >= A) whose row
// atom A lies in [a_begin, a_end); a_end < 0 means the last atom.  nbr (one molecule, host
// n_atoms^2 mask): only neighbouring pairs are assembled, every other block is T + V.
x2c_status dlu_build(x2c_ctx *ctx, const x2c_options *opt, int n_mol, const x2c_layout *layouts,
                     const x2c_mats *mols, const x2c_hout *h, const KindTransforms *ku, cudaStream_t st,
                     size_t *dry_bytes, int a_begin = 0, int a_end = -1, const uint8_t *nbr = nullptr);
x2c_status transforms_build(x2c_ctx *ctx, const x2c_options *opt, int n_problems, const x2c_mats *inputs,
                            const x2c_uout *U, cudaStream_t st, size_t *dry_bytes);

// Descriptor of one decoupling problem's inputs (device pointers, leading dimension ld).
struct InputDesc {
  const double *S, *T, *V;
  const double *W[4];  // W0, Wx, Wy, Wz (Wx..Wz NULL when spin-free)
  int64_t ld;
};

// Batched decoupling transforms (the matrix function of Eqs. 43 / 22): nb problems of
// size n with nc = 1 (scalar) or 4 (two-component) parts.  d_in: device array of nb
// descriptors.  UL, US: device, nb * nc * n * n doubles each (problem-major, then part).
// Scratch comes from `ar` (passed by value: the caller's arena is not advanced).
constexpr int kMaxSolveN = 168;  // largest n factorised in one CTA (bigger: blocked)
x2c_status solve_transforms(x2c_ctx *ctx, cudaStream_t st, double c, int nb, int n, int nc,
                            const InputDesc *d_in, double *UL, double *US, Arena ar);
// BSS (decoupling = 1) and DKHn (decoupling = n >= 2) transforms of nb problems of size n
// (solve_fw.cuh); problems of n <= 160 (fw_supported).
constexpr int kMaxDkhOrder = X2C_DEC_MAX_DKH_ORDER;
bool fw_supported(int n, int decoupling);
size_t solve_fw_workspace_bytes(int nb, int n, int nc, int decoupling);
x2c_status solve_transforms_fw(x2c_ctx *ctx, cudaStream_t st, double c, int nb, int n, int nc, int decoupling,
                               const InputDesc *d_in, double *UL, double *US, Arena ar);
// The DKHn Hamiltonian of one whole system (h: nc device parts of n x n).
size_t dkh_hamiltonian_workspace_bytes(int n, int nc, int order);
x2c_status dkh_hamiltonian(x2c_ctx *ctx, cudaStream_t st, double c, int n, int nc, int order, const InputDesc *d_in,
                           double *const *h, Arena ar);
size_t solve_workspace_bytes(int nb, int n, int nc);

// Pair-block assembly of h = U+ D U for block-diagonal U (Eq. 8 with Eq. 42).
struct PairDesc {
  int32_t offA, offB;   // first basis function of atoms A and B (within the molecule)
  int32_t nA, nB;       // atom sizes
  int32_t uA, uB;       // index of the atoms' transforms in the U table
  int32_t mol;          // molecule index (batched builds)
  int32_t diag;         // 1 when A == B
  int64_t r_off;        // offset (doubles) of this pair's intermediate in the R buffer
};
struct MolDesc {
  const double *V, *T, *W0;
  const double *W[3];   // Wx, Wy, Wz (NULL when spin-free)
  double *h[4];
  int64_t ld;
};
struct UTable {
  const double *const *UL;  // device array: per transform index, pointer to nc*n*n doubles
  const double *const *US;
};
x2c_status assemble_pairs_fp64(x2c_ctx *ctx, cudaStream_t st, double c, int nc, int so_all_pairs,
                               const std::vector<PairDesc> &pairs, const MolDesc *d_mols,
                               UTable ut, int max_n, Arena &ar);
// hUL/hUS: host copies of the U table (device pointers), used to build per-kind operands.
x2c_status assemble_pairs_split(x2c_ctx *ctx, cudaStream_t st, double c, int nc, int so_all_pairs,
                                const std::vector<PairDesc> &pairs, const MolDesc *d_mols, UTable ut,
                                const std::vector<const double *> &hUL, const std::vector<const double *> &hUS,
                                int n_slices, Arena &ar);
size_t assemble_workspace_bytes(const std::vector<PairDesc> &pairs, int nc, int max_n, int precision,
                                size_t split_cap);
// DLH: h = T + V (spin parts 0) on every block of molecule `mol` outside the same-atom
// blocks; d_off: device copy of the molecule's L + 1 atom offsets, N = d_off[L].
x2c_status fill_nonrel_offdiag(x2c_ctx *ctx, cudaStream_t st, const MolDesc *d_mols, int mol, const int32_t *d_off,
                               int L, int N, int nc);

}  // namespace x2c
