// extern "C" entry points of the X2C library (include/x2c.h).
#include <algorithm>
#include <cstring>
#include <map>
#include <tuple>

#include "common.cuh"
#include "dkh_plan.h"

// A build captured into a CUDA graph (x2c_ctx_set_graphs), keyed by its launch plan.
struct x2c_ctx::GraphEntry {
  std::string key;
  uint64_t hash = 0;
  uint64_t ws_generation = 0;  // the workspace the graph's kernels point into
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<char *> pinned;  // sources of the captured descriptor uploads
  struct Timed {
    std::string name;
    double flops;
    cudaGraphNode_t begin, end;  // event-record nodes around the launch
  };
  std::vector<Timed> timed;
  int64_t launches = 0, pair_blocks = 0, atomic_solves = 0;
  double credited = 0;
};

namespace x2c {

x2c_status ensure_workspace(x2c_ctx *ctx, size_t bytes, Arena *out, cudaStream_t st) {
  if (bytes > ctx->ws_bytes) {
    if (ctx->capturing) {  // the graph would hold pointers into a buffer freed here
      ctx->last_error = "workspace growth inside a graph capture";
      return X2C_ERR_ARG;
    }
    ctx->ws_generation++;
    const size_t want = bytes + bytes / 8;
    cudaError_t e;
    if (ctx->pool) {
      // stream-ordered: the old workspace is only ever used on this stream
      if (ctx->ws) cudaFreeAsync(ctx->ws, st);
      ctx->ws = nullptr;
      ctx->ws_bytes = 0;
      e = cudaMallocFromPoolAsync(reinterpret_cast<void **>(&ctx->ws), want, ctx->pool, st);
    } else {
      X2C_TRY_CUDA(ctx, cudaDeviceSynchronize());
      if (ctx->ws) cudaFree(ctx->ws);
      ctx->ws = nullptr;
      ctx->ws_bytes = 0;
      e = cudaMalloc(&ctx->ws, want);
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      ctx->ws = nullptr;
      ctx->last_error = std::string("workspace allocation: ") + cudaGetErrorString(e);
      return X2C_ERR_NOMEM;
    }
    ctx->ws_bytes = want;
  }
  out->base = ctx->ws;
  out->cap = ctx->ws_bytes;
  out->off = 0;
  return X2C_OK;
}

size_t workspace_after_growth(const x2c_ctx *ctx, size_t bytes) {
  return bytes > ctx->ws_bytes ? bytes + bytes / 8 : ctx->ws_bytes;
}

// Copies and fills of the build path run as kernels, not on the copy engines: a host-buffer
// build keeps the copy engines busy with its bulk transfers, and a small copy queued behind
// them would hold up the build's kernels until those transfers finish.  Sources in pinned
// host memory are read through their device mapping.
__global__ void copy_bytes_kernel(unsigned char *dst, const unsigned char *src, size_t bytes) {
  const size_t tid = blockIdx.x * (size_t)blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
  if ((((uintptr_t)dst | (uintptr_t)src) & 15) == 0) {
    const size_t words = bytes / 16;
    for (size_t i = tid; i < words; i += stride)
      reinterpret_cast<uint4 *>(dst)[i] = reinterpret_cast<const uint4 *>(src)[i];
    for (size_t i = words * 16 + tid; i < bytes; i += stride) dst[i] = src[i];
  } else {
    for (size_t i = tid; i < bytes; i += stride) dst[i] = src[i];
  }
}
__global__ void fill_bytes_kernel(unsigned char *dst, unsigned char v, size_t bytes) {
  const size_t tid = blockIdx.x * (size_t)blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = tid; i < bytes; i += stride) dst[i] = v;
}
int copy_grid(size_t bytes) { return (int)std::min<size_t>(std::max<size_t>(1, (bytes / 16 + 255) / 256), 152 * 4); }

x2c_status device_copy(x2c_ctx *ctx, cudaStream_t st, void *dst, const void *src, size_t bytes) {
  if (bytes == 0) return X2C_OK;
  tbegin(ctx, st);
  copy_bytes_kernel<<<copy_grid(bytes), 256, 0, st>>>(static_cast<unsigned char *>(dst),
                                                      static_cast<const unsigned char *>(src), bytes);
  return launched(ctx, "copy_kernel", st);
}

x2c_status device_fill(x2c_ctx *ctx, cudaStream_t st, void *dst, int value, size_t bytes) {
  if (bytes == 0) return X2C_OK;
  tbegin(ctx, st);
  fill_bytes_kernel<<<copy_grid(bytes), 256, 0, st>>>(static_cast<unsigned char *>(dst), (unsigned char)value, bytes);
  return launched(ctx, "copy_kernel", st);
}

// Device address of a pinned host allocation (the same pointer under unified addressing).
x2c_status mapped(x2c_ctx *ctx, const void *host, const void **dev) {
  void *d = nullptr;
  X2C_TRY_CUDA(ctx, cudaHostGetDevicePointer(&d, const_cast<void *>(host), 0));
  *dev = d;
  return X2C_OK;
}

x2c_status upload(x2c_ctx *ctx, cudaStream_t st, void *dst, const void *src, size_t bytes) {
  if (bytes == 0) return X2C_OK;
  const size_t need = (bytes + 255) & ~static_cast<size_t>(255);
  if (ctx->capturing) {
    // a captured copy reads its source at every replay: the source is a pinned block that
    // belongs to the graph and is never rewritten
    if (ctx->cap_pinned.empty() || ctx->cap_off + need > ctx->cap_cap) {
      const size_t cap = std::max<size_t>(need, 1u << 20);
      char *blk = nullptr;
      cudaError_t e = cudaHostAlloc(reinterpret_cast<void **>(&blk), cap, cudaHostAllocDefault);
      if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->last_error = std::string("pinned graph source allocation: ") + cudaGetErrorString(e);
        return X2C_ERR_NOMEM;
      }
      ctx->cap_pinned.push_back(blk);
      ctx->cap_off = 0;
      ctx->cap_cap = cap;
    }
    char *h = ctx->cap_pinned.back() + ctx->cap_off;
    ctx->cap_off += need;
    std::memcpy(h, src, bytes);
    const void *hd = nullptr;
    X2C_TRY(mapped(ctx, h, &hd));
    return device_copy(ctx, st, dst, hd, bytes);
  }
  auto retire = [&](const x2c_ctx::Staged &f) -> x2c_status {
    X2C_TRY_CUDA(ctx, cudaEventSynchronize(f.done));
    ctx->ring_events.push_back(f.done);
    return X2C_OK;
  };
  // drop uploads the device has finished
  while (!ctx->ring_inflight.empty() && cudaEventQuery(ctx->ring_inflight.front().done) == cudaSuccess) {
    ctx->ring_events.push_back(ctx->ring_inflight.front().done);
    ctx->ring_inflight.erase(ctx->ring_inflight.begin());
  }
  cudaGetLastError();  // cudaErrorNotReady from the query above
  if (need > ctx->ring_cap) {  // grow: wait for everything staged in the old buffer
    for (auto &f : ctx->ring_inflight) X2C_TRY(retire(f));
    ctx->ring_inflight.clear();
    if (ctx->ring) cudaFreeHost(ctx->ring);
    ctx->ring = nullptr;
    ctx->ring_cap = 0;
    const size_t cap = std::max<size_t>(need, 16u << 20);
    cudaError_t e = cudaHostAlloc(reinterpret_cast<void **>(&ctx->ring), cap, cudaHostAllocDefault);
    if (e != cudaSuccess) {
      cudaGetLastError();
      ctx->ring = nullptr;
      ctx->last_error = std::string("pinned staging allocation: ") + cudaGetErrorString(e);
      return X2C_ERR_NOMEM;
    }
    ctx->ring_cap = cap;
    ctx->ring_head = 0;
  }
  size_t start = ctx->ring_head;
  if (start + need > ctx->ring_cap) start = 0;  // wrap around
  const size_t end = start + need;
  // the region may still be the source of an older upload the device has not performed yet
  while (!ctx->ring_inflight.empty()) {
    const auto &f = ctx->ring_inflight.front();
    if (!(f.start < end && start < f.end)) break;
    X2C_TRY(retire(f));
    ctx->ring_inflight.erase(ctx->ring_inflight.begin());
  }
  std::memcpy(ctx->ring + start, src, bytes);
  const void *hd = nullptr;
  X2C_TRY(mapped(ctx, ctx->ring + start, &hd));
  X2C_TRY(device_copy(ctx, st, dst, hd, bytes));
  cudaEvent_t ev;
  if (!ctx->ring_events.empty()) {
    ev = ctx->ring_events.back();
    ctx->ring_events.pop_back();
  } else {
    X2C_TRY_CUDA(ctx, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  }
  X2C_TRY_CUDA(ctx, cudaEventRecord(ev, st));
  ctx->ring_inflight.push_back({start, end, ev});
  ctx->ring_head = end;
  return X2C_OK;
}

x2c_status ensure_aux_streams(x2c_ctx *ctx, int count) {
  if (!ctx->aux_fork) X2C_TRY_CUDA(ctx, cudaEventCreateWithFlags(&ctx->aux_fork, cudaEventDisableTiming));
  while ((int)ctx->aux.size() < count) {
    cudaStream_t s;
    cudaEvent_t e;
    X2C_TRY_CUDA(ctx, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    X2C_TRY_CUDA(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ctx->aux.push_back(s);
    ctx->aux_join.push_back(e);
  }
  return X2C_OK;
}

bool mats_ok(const x2c_mats *m, int nc) {
  if (!m || m->n < 1 || !m->S || !m->T || !m->V || !m->W0) return false;
  if (nc == 4 && (!m->Wx || !m->Wy || !m->Wz)) return false;
  return true;
}

x2c_status check_options(const x2c_options *o) {
  if (!o) return X2C_ERR_ARG;
  if (o->two_component != 0 && o->two_component != 1) return X2C_ERR_ARG;
  if (o->precision != X2C_PREC_FP64 && o->precision != X2C_PREC_SPLIT_BF16) return X2C_ERR_ARG;
  if (o->dlu_potential != X2C_DLU_FREE_ATOM && o->dlu_potential != X2C_DLU_MOLECULAR_BLOCK) return X2C_ERR_ARG;
  if (o->n_slices < 0 || o->n_slices > 8) return X2C_ERR_ARG;
  if (o->local_approx != X2C_LOCAL_DLU && o->local_approx != X2C_LOCAL_DLH) return X2C_ERR_ARG;
  if (o->h_upper_only != 0) return X2C_ERR_ARG;  // only x2c_build_dlu_host takes it (and clears it)
  if (o->decoupling < 0 || o->decoupling > X2C_DEC_MAX_DKH_ORDER) return X2C_ERR_ARG;
  return X2C_OK;
}

namespace {

double credited_pair_flops(int nA, int nB, int nc, bool diag, bool so) {
  const double a = nA, b = nB;
  if (nc == 1) return 2.0 * (4.0 * a * b * b + 2.0 * a * a * b);
  double f = 2.0 * (16.0 * a * b * b + 32.0 * a * a * b);
  if (diag || so) f += 24.0 * a * b * b;
  return f;
}

// Conventional counts of the paper's operation list (Tables II and III) for one
// decoupling problem of size n: eigen 9 m^3, inversion 2 m^3, product 2 m^3, complex x4.
// The DKHn Hamiltonian of one system: the kinetic basis (one diagonalisation of n, K^-1, the
// potential transforms) and the P(n) products of Table I, conventional counts (eigen with
// vectors 9 n^3, inverse 2 n^3, product 2 n^3; a quaternion product 16 real products) plus
// the back transformation (2 products per part).
double hamiltonian_flops(int n, int nc, int order) {
  const double n3 = (double)n * n * n;
  const double qp = (nc == 4 ? 16.0 : 1.0) * 2.0 * n3;
  return 9 * n3 + 2 * n3 + 2 * (1 + nc) * 2 * n3 + dkh::hamiltonian_products(order) * qp + nc * 2 * 2 * n3;
}

double credited_solve_flops(int n, int nc) {
  const double N3 = (double)n * n * n;
  if (nc == 1) return (2 * 9 + 9 * 8 + 2 * 2 + 15 * 2) * N3;
  return (9 + 4 * 9 * 8 + 4 * 9 * 64 + 2 + 4 * 2 * 8 + 10 * 2 + 11 * 4 * 2 * 8) * N3;
}

struct Problem {
  InputDesc in;
  int n;
  const double *preUL = nullptr;  // precomputed transforms (device, nc n^2 each): no solve
  const double *preUS = nullptr;
};

// One logical build: a set of decoupling problems (grouped by size), a U table indexed by
// problem, molecules and their pair list.
struct NonRelFill {  // DLH: a molecule whose atom-other-atom blocks are T + V
  int mol;
  std::vector<int32_t> off;
};

struct BuildPlan {
  std::vector<Problem> problems;
  std::vector<MolDesc> mols;
  std::vector<PairDesc> pairs;
  std::vector<NonRelFill> fills;
  int nc = 1;
  int max_n = 0;
  double credited = 0;
};

// Scratch of one size group's decoupling solve (X2C, or BSS / DKHn).
size_t solve_bytes(const x2c_options *opt, int nb, int n, int nc) {
  return opt->decoupling == X2C_DEC_X2C ? solve_workspace_bytes(nb, n, nc)
                                        : solve_fw_workspace_bytes(nb, n, nc, opt->decoupling);
}

x2c_status run_plan(x2c_ctx *ctx, const x2c_options *opt, BuildPlan &plan, cudaStream_t st,
                    std::vector<double *> *UL_out = nullptr, std::vector<double *> *US_out = nullptr,
                    size_t *dry_bytes = nullptr) {
  const double c = speed_of_light(opt);
  const int nc = plan.nc;
  // group the problems that need a solve by size
  std::map<int, std::vector<int>> groups;
  for (size_t i = 0; i < plan.problems.size(); ++i)
    if (!plan.problems[i].preUL) groups[plan.problems[i].n].push_back((int)i);
  size_t u_doubles = 0, solve_ws = 0, desc_bytes = 0;
  if (opt->decoupling != X2C_DEC_X2C)
    for (auto &g : groups)
      if (!fw_supported(g.first, opt->decoupling)) return X2C_ERR_ARG;
  for (auto &g : groups) {
    const size_t n2 = (size_t)g.first * g.first;
    u_doubles += 2 * g.second.size() * nc * n2;
    solve_ws += solve_bytes(opt, (int)g.second.size(), g.first, nc) + 256;  // groups run concurrently
    desc_bytes += ((g.second.size() * sizeof(InputDesc) + 255) / 256) * 256;
  }
  const size_t np = plan.problems.size();
  const size_t table_bytes = 2 * (((np * sizeof(double *) + 255) / 256) * 256);
  const size_t mol_bytes = ((plan.mols.size() * sizeof(MolDesc) + 255) / 256) * 256;
  size_t fill_bytes = 0;
  for (const auto &f : plan.fills) fill_bytes += ((f.off.size() * sizeof(int32_t) + 255) / 256) * 256;
  auto total_for = [&](size_t cap) {
    const size_t asm_ws = assemble_workspace_bytes(plan.pairs, nc, plan.max_n, opt->precision, cap);
    return arena_doubles(u_doubles) + desc_bytes + table_bytes + mol_bytes + fill_bytes +
           std::max(solve_ws, asm_ws) + 8192;
  };
  const size_t total = total_for(ctx->split_ws_cap);
  if (dry_bytes) {
    *dry_bytes = total;
    return X2C_OK;
  }
  Arena ar;
  x2c_status ws = ensure_workspace(ctx, total, &ar, st);
  if (ws == X2C_ERR_NOMEM && ctx->split_ws_cap > kSplitWsCapSmall) {
    // the one-chunk workspace does not fit: this context assembles in smaller chunks from now on
    ctx->split_ws_cap = kSplitWsCapSmall;
    ws = ensure_workspace(ctx, total_for(ctx->split_ws_cap), &ar, st);
  }
  X2C_TRY(ws);
  double *Ustore = ar.take(std::max<size_t>(1, u_doubles));
  double **dUL = reinterpret_cast<double **>(ar.take_bytes(np * sizeof(double *)));
  double **dUS = reinterpret_cast<double **>(ar.take_bytes(np * sizeof(double *)));
  MolDesc *dmols = reinterpret_cast<MolDesc *>(ar.take_bytes(std::max<size_t>(1, plan.mols.size()) * sizeof(MolDesc)));
  if (!Ustore || !dUL || !dUS || !dmols) return X2C_ERR_NOMEM;
  std::vector<int32_t *> doffs;
  for (const auto &f : plan.fills) {
    doffs.push_back(reinterpret_cast<int32_t *>(ar.take_bytes(f.off.size() * sizeof(int32_t))));
    if (!doffs.back()) return X2C_ERR_NOMEM;
  }
  std::vector<double *> hUL(np), hUS(np);
  for (size_t i = 0; i < np; ++i)
    if (plan.problems[i].preUL) {
      hUL[i] = const_cast<double *>(plan.problems[i].preUL);
      hUS[i] = const_cast<double *>(plan.problems[i].preUS);
    }
  // solve each size group
  size_t uoff = 0;
  std::vector<InputDesc *> ddescs;
  for (auto &g : groups) {
    const int n = g.first, nb = (int)g.second.size();
    const size_t n2 = (size_t)n * n;
    double *UL = Ustore + uoff;
    double *US = UL + (size_t)nb * nc * n2;
    uoff += 2 * (size_t)nb * nc * n2;
    std::vector<InputDesc> hd(nb);
    for (int i = 0; i < nb; ++i) {
      hd[i] = plan.problems[g.second[i]].in;
      hUL[g.second[i]] = UL + (size_t)i * nc * n2;
      hUS[g.second[i]] = US + (size_t)i * nc * n2;
    }
    InputDesc *dd = reinterpret_cast<InputDesc *>(ar.take_bytes(nb * sizeof(InputDesc)));
    if (!dd) return X2C_ERR_NOMEM;
    X2C_TRY(upload(ctx, st, dd, hd.data(), nb * sizeof(InputDesc)));
    ddescs.push_back(dd);
    plan.credited += nb * credited_solve_flops(n, nc);
  }
  // Size groups are independent: each runs on its own stream (the first on the caller's)
  // with its own part of the scratch region that follows; the caller's stream then waits
  // for all of them (the assembly reuses the region afterwards).
  {
    const int ng = (int)groups.size();
    std::vector<cudaStream_t> gs(ng, st);
    if (ng > 1) {
      X2C_TRY(ensure_aux_streams(ctx, std::min(ng - 1, kMaxAuxStreams)));
      X2C_TRY_CUDA(ctx, cudaEventRecord(ctx->aux_fork, st));
      for (int i = 1; i < ng; ++i) {
        gs[i] = ctx->aux[(i - 1) % kMaxAuxStreams];
        if (i <= kMaxAuxStreams) X2C_TRY_CUDA(ctx, cudaStreamWaitEvent(gs[i], ctx->aux_fork, 0));
      }
    }
    size_t gi = 0, uo = 0;
    Arena scratch = ar;
    for (auto &g : groups) {
      const int n = g.first, nb = (int)g.second.size();
      const size_t n2 = (size_t)n * n;
      double *UL = Ustore + uo;
      double *US = UL + (size_t)nb * nc * n2;
      uo += 2 * (size_t)nb * nc * n2;
      const size_t need = solve_bytes(opt, nb, n, nc);
      Arena mine;
      mine.base = static_cast<char *>(scratch.take_bytes(need));
      mine.cap = need;
      if (!mine.base) return X2C_ERR_NOMEM;
      if (opt->decoupling == X2C_DEC_X2C)
        X2C_TRY(solve_transforms(ctx, gs[gi], c, nb, n, nc, ddescs[gi], UL, US, mine));
      else
        X2C_TRY(solve_transforms_fw(ctx, gs[gi], c, nb, n, nc, opt->decoupling, ddescs[gi], UL, US, mine));
      ++gi;
    }
    for (int i = 1; i < ng && i <= kMaxAuxStreams; ++i) {
      X2C_TRY_CUDA(ctx, cudaEventRecord(ctx->aux_join[i - 1], ctx->aux[i - 1]));
      X2C_TRY_CUDA(ctx, cudaStreamWaitEvent(st, ctx->aux_join[i - 1], 0));
    }
  }
  size_t solved = 0;
  for (auto &g : groups) solved += g.second.size();
  ctx->counters.atomic_solves = (int64_t)solved;
  if (UL_out) *UL_out = hUL;
  if (US_out) *US_out = hUS;
  if (plan.pairs.empty()) return X2C_OK;
  X2C_TRY(upload(ctx, st, dUL, hUL.data(), np * sizeof(double *)));
  X2C_TRY(upload(ctx, st, dUS, hUS.data(), np * sizeof(double *)));
  X2C_TRY(upload(ctx, st, dmols, plan.mols.data(), plan.mols.size() * sizeof(MolDesc)));
  for (size_t i = 0; i < plan.fills.size(); ++i) {
    const auto &f = plan.fills[i];
    const int L = (int)f.off.size() - 1;
    X2C_TRY(upload(ctx, st, doffs[i], f.off.data(), f.off.size() * sizeof(int32_t)));
    X2C_TRY(fill_nonrel_offdiag(ctx, st, dmols, f.mol, doffs[i], L, f.off[L], nc));
  }
  UTable ut{dUL, dUS};
  const int so_all = (nc == 4 && !opt->so_same_atom_only) ? 1 : 0;
  for (const auto &P : plan.pairs) plan.credited += credited_pair_flops(P.nA, P.nB, nc, P.diag, so_all);
  ctx->counters.pair_blocks = (int64_t)plan.pairs.size();
  if (opt->precision == X2C_PREC_SPLIT_BF16) {
    const int slices = opt->n_slices ? opt->n_slices : 5;
    std::vector<const double *> cUL(hUL.begin(), hUL.end()), cUS(hUS.begin(), hUS.end());
    return assemble_pairs_split(ctx, st, c, nc, so_all, plan.pairs, dmols, ut, cUL, cUS, slices, ar);
  }
  return assemble_pairs_fp64(ctx, st, c, nc, so_all, plan.pairs, dmols, ut, plan.max_n, ar);
}

MolDesc mol_desc(const x2c_mats *m, const x2c_hout *h, int nc) {
  MolDesc d{};
  d.V = m->V;
  d.T = m->T;
  d.W0 = m->W0;
  if (nc == 4) {
    d.W[0] = m->Wx;
    d.W[1] = m->Wy;
    d.W[2] = m->Wz;
  }
  for (int q = 0; q < nc; ++q) d.h[q] = h->h[q];
  d.ld = m->n;
  return d;
}

InputDesc input_desc(const x2c_mats *m, int nc, int64_t off, int64_t ld) {
  InputDesc d{};
  const int64_t o = off * ld + off;
  d.S = m->S + o;
  d.T = m->T + o;
  d.V = m->V + o;
  d.W[0] = m->W0 + o;
  if (nc == 4) {
    d.W[1] = m->Wx + o;
    d.W[2] = m->Wy + o;
    d.W[3] = m->Wz + o;
  }
  d.ld = ld;
  return d;
}

// Add one molecule's problems (molecular-block mode) or kind references and its pairs.
using KindIndex = std::map<std::tuple<const double *, const double *, const double *, const double *,
                                      const double *>, int>;

x2c_status add_molecule(BuildPlan &plan, const x2c_options *opt, const x2c_layout *lay,
                        const x2c_mats *mol, const x2c_hout *h, int mol_index, KindIndex &kind_index,
                        const KindTransforms *ku = nullptr, int a_begin = 0, int a_end = -1,
                        const uint8_t *nbr = nullptr) {
  const int nc = plan.nc;
  if (!lay || lay->n_atoms < 1 || !lay->atom_offset || !mats_ok(mol, nc) || !h) return X2C_ERR_ARG;
  for (int q = 0; q < nc; ++q)
    if (!h->h[q]) return X2C_ERR_ARG;
  const int L = lay->n_atoms;
  if (lay->atom_offset[0] != 0 || lay->atom_offset[L] != mol->n) return X2C_ERR_ARG;
  for (int a = 0; a < L; ++a)
    if (lay->atom_offset[a + 1] <= lay->atom_offset[a]) return X2C_ERR_ARG;
  std::vector<int> uidx(L);
  if (opt->dlu_potential == X2C_DLU_MOLECULAR_BLOCK) {
    for (int a = 0; a < L; ++a) {
      const int n = lay->atom_offset[a + 1] - lay->atom_offset[a];
      uidx[a] = (int)plan.problems.size();
      plan.problems.push_back({input_desc(mol, nc, lay->atom_offset[a], mol->n), n});
    }
  } else {
    if (!lay->atom_kind || lay->n_kinds < 1 || !lay->kinds) return X2C_ERR_ARG;
    for (int a = 0; a < L; ++a) {
      const int k = lay->atom_kind[a];
      if (k < 0 || k >= lay->n_kinds) return X2C_ERR_ARG;
      const x2c_mats *km = &lay->kinds[k];
      const int n = lay->atom_offset[a + 1] - lay->atom_offset[a];
      const bool pre = ku && ku->UL && ku->UL[k] && ku->US && ku->US[k];
      if (pre) {
        if (km->n != n) return X2C_ERR_ARG;
        auto key = std::make_tuple(ku->UL[k], ku->US[k], (const double *)nullptr, (const double *)nullptr,
                                   (const double *)nullptr);
        auto it = kind_index.find(key);
        if (it == kind_index.end()) {
          Problem p{};
          p.n = n;
          p.preUL = ku->UL[k];
          p.preUS = ku->US[k];
          const int id = (int)plan.problems.size();
          plan.problems.push_back(p);
          it = kind_index.emplace(key, id).first;
        }
        uidx[a] = it->second;
        continue;
      }
      if (!mats_ok(km, nc) || km->n != n) return X2C_ERR_ARG;
      auto key = std::make_tuple(km->S, km->T, km->V, km->W0, nc == 4 ? km->Wx : nullptr);
      auto it = kind_index.find(key);
      if (it == kind_index.end()) {
        const int id = (int)plan.problems.size();
        plan.problems.push_back({input_desc(km, nc, 0, n), n});
        it = kind_index.emplace(key, id).first;
      }
      uidx[a] = it->second;
    }
  }
  plan.mols.push_back(mol_desc(mol, h, nc));
  // DLH: only the same-atom blocks are transformed; the rest is filled with T + V.  With a
  // neighbour mask (neighbouring-atomic-blocks approximation) the blocks of neighbouring atoms
  // are transformed as in DLU after that fill.
  const bool dlh = opt->local_approx == X2C_LOCAL_DLH;
  if (dlh || nbr) plan.fills.push_back({mol_index, std::vector<int32_t>(lay->atom_offset, lay->atom_offset + L + 1)});
  if (a_end < 0) a_end = L;
  if (a_begin < 0 || a_begin >= a_end || a_end > L) return X2C_ERR_ARG;
  for (int A = a_begin; A < a_end; ++A) {
    const int nA = lay->atom_offset[A + 1] - lay->atom_offset[A];
    plan.max_n = std::max(plan.max_n, nA);
    for (int B = A; B < (dlh ? A + 1 : L); ++B) {
      if (nbr && B != A && !nbr[(int64_t)A * L + B] && !nbr[(int64_t)B * L + A]) continue;
      PairDesc P{};
      P.offA = lay->atom_offset[A];
      P.offB = lay->atom_offset[B];
      P.nA = nA;
      P.nB = lay->atom_offset[B + 1] - lay->atom_offset[B];
      P.uA = uidx[A];
      P.uB = uidx[B];
      P.mol = mol_index;
      P.diag = (A == B);
      plan.pairs.push_back(P);
    }
  }
  return X2C_OK;
}

__global__ void quat_to_dense_kernel(const double *h0, const double *h1, const double *h2,
                                     const double *h3, int n, double *out) {
  const int64_t N = n;
  const int64_t total = N * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / N, j = idx % N;
    const double a = h0[idx], x = h1 ? h1[idx] : 0.0, y = h2 ? h2[idx] : 0.0, z = h3 ? h3[idx] : 0.0;
    const int64_t ld = 2 * N;  // complex elements per row
    double *o = out;
    // [[h0 + i h3, h2 + i h1], [-h2 + i h1, h0 - i h3]]
    o[2 * (i * ld + j)] = a;              o[2 * (i * ld + j) + 1] = z;
    o[2 * (i * ld + N + j)] = y;          o[2 * (i * ld + N + j) + 1] = x;
    o[2 * ((N + i) * ld + j)] = -y;       o[2 * ((N + i) * ld + j) + 1] = x;
    o[2 * ((N + i) * ld + N + j)] = a;    o[2 * ((N + i) * ld + N + j) + 1] = -z;
  }
}

x2c_status begin_call(x2c_ctx *ctx) {
  if (!ctx) return X2C_ERR_ARG;
  ctx->launches = 0;
  X2C_TRY_CUDA(ctx, cudaSetDevice(ctx->device));
  return X2C_OK;
}

void end_call(x2c_ctx *ctx, const BuildPlan &plan) {
  ctx->counters.kernel_launches = ctx->launches;
  ctx->counters.credited_flops = plan.credited;
}

// ---------------------------------------------------------------------------------------
// CUDA-graph replay.  A build's host work (plan, descriptor uploads, a few hundred launches)
// is the same for every call with the same plan; with graphs enabled the second such call
// captures the enqueued work on a private stream and every later one launches the
// instantiated graph on the caller's stream.

constexpr size_t kMaxGraphs = 32;
constexpr size_t kMaxSeenPlans = 4096;

struct KeyBuf {
  std::string b;
  template <class T>
  void put(const T &v) { b.append(reinterpret_cast<const char *>(&v), sizeof(T)); }
};

// Everything that decides what a build enqueues: the entry point, the options, every
// problem, molecule and pair descriptor (so every input and output pointer), extra output
// pointers, and the context's kernel choices.
std::string plan_key(const x2c_ctx *ctx, int entry, const x2c_options *opt, const BuildPlan &plan,
                     const x2c_uout *U, int nU) {
  static_assert(sizeof(PairDesc) == 40 && sizeof(MolDesc) == 88, "descriptors without padding");
  KeyBuf k;
  k.put(entry);
  k.put(opt->c);
  k.put(opt->two_component);
  k.put(opt->precision);
  k.put(opt->dlu_potential);
  k.put(opt->so_same_atom_only);
  k.put(opt->n_slices);
  k.put(opt->local_approx);
  k.put(opt->decoupling);
  k.put(plan.nc);
  k.put(plan.max_n);
  k.put(ctx->split_variant);
  k.put(ctx->cta_cap);
  k.put(ctx->timing);
  k.put(plan.problems.size());
  for (const auto &p : plan.problems) {
    k.put(p.in.S);
    k.put(p.in.T);
    k.put(p.in.V);
    for (const double *w : p.in.W) k.put(w);
    k.put(p.in.ld);
    k.put(p.n);
    k.put(p.preUL);
    k.put(p.preUS);
  }
  k.put(plan.mols.size());
  k.b.append(reinterpret_cast<const char *>(plan.mols.data()), plan.mols.size() * sizeof(MolDesc));
  k.put(plan.pairs.size());
  k.b.append(reinterpret_cast<const char *>(plan.pairs.data()), plan.pairs.size() * sizeof(PairDesc));
  for (const auto &f : plan.fills) {
    k.put(f.mol);
    k.put(f.off.size());
    k.b.append(reinterpret_cast<const char *>(f.off.data()), f.off.size() * sizeof(int32_t));
  }
  for (int i = 0; i < nU; ++i)
    for (int q = 0; q < 4; ++q) {
      k.put(U[i].UL[q]);
      k.put(U[i].US[q]);
    }
  return std::move(k.b);
}

// Hash of a plan key, eight bytes at a time (keys of large builds are megabytes; a match is
// always confirmed by comparing the whole key).
uint64_t fnv1a(const std::string &b) {
  uint64_t h = 1469598103934665603ull;
  size_t i = 0;
  for (; i + 8 <= b.size(); i += 8) {
    uint64_t w;
    std::memcpy(&w, b.data() + i, 8);
    h = (h ^ w) * 1099511628211ull;
    h ^= h >> 29;
  }
  for (; i < b.size(); ++i) h = (h ^ static_cast<unsigned char>(b[i])) * 1099511628211ull;
  return h;
}

void destroy_entry(x2c_ctx::GraphEntry *e) {
  if (e->exec) cudaGraphExecDestroy(e->exec);
  if (e->graph) cudaGraphDestroy(e->graph);
  for (char *p : e->pinned) cudaFreeHost(p);
  delete e;
}

// Launch a captured build on `st`: fresh timing events for its record nodes, the call's
// counters as the capture counted them.
x2c_status replay(x2c_ctx *ctx, x2c_ctx::GraphEntry *e, cudaStream_t st, BuildPlan &plan) {
  if (ctx->timing)
    for (const auto &t : e->timed) {
      cudaEvent_t b = next_event(ctx), en = next_event(ctx);
      if (!b || !en) return cuda_fail(ctx, cudaErrorMemoryAllocation, "timing event");
      X2C_TRY_CUDA(ctx, cudaGraphExecEventRecordNodeSetEvent(e->exec, t.begin, b));
      X2C_TRY_CUDA(ctx, cudaGraphExecEventRecordNodeSetEvent(e->exec, t.end, en));
      ctx->pending.push_back({t.name, ctx->ev_used - 2, t.flops});
    }
  X2C_TRY_CUDA(ctx, cudaGraphLaunch(e->exec, st));
  ctx->launches += e->launches;
  ctx->counters.pair_blocks = e->pair_blocks;
  ctx->counters.atomic_solves = e->atomic_solves;
  plan.credited += e->credited;
  ctx->graph_replays++;
  ctx->last_replayed = true;
  return X2C_OK;
}

// Run one build: eagerly (graphs off, or a plan seen for the first time), else as a launch of
// the graph captured for this plan.  enqueue(stream, dry_bytes) enqueues the build's work on
// `stream`, or with dry_bytes non-NULL only sizes its workspace.
template <class KeyFn, class F>
x2c_status graph_run(x2c_ctx *ctx, cudaStream_t st, KeyFn &&make_key, BuildPlan &plan, F &&enqueue) {
  ctx->last_replayed = false;
  if (!ctx->graphs || ctx->pool) return enqueue(st, nullptr);
  const std::string key = make_key();
  const uint64_t hash = fnv1a(key);
  auto &cache = ctx->graph_cache;
  // graphs that point into a workspace that has moved since
  {
    bool stale = false;
    for (auto *e : cache) stale |= e->ws_generation != ctx->ws_generation;
    if (stale) {
      X2C_TRY_CUDA(ctx, cudaDeviceSynchronize());
      std::vector<x2c_ctx::GraphEntry *> keep;
      for (auto *e : cache)
        if (e->ws_generation == ctx->ws_generation) keep.push_back(e);
        else destroy_entry(e);
      cache.swap(keep);
    }
  }
  for (size_t i = 0; i < cache.size(); ++i)
    if (cache[i]->hash == hash && cache[i]->key == key) {
      auto *e = cache[i];
      cache.erase(cache.begin() + i);
      cache.push_back(e);
      return replay(ctx, e, st, plan);
    }
  if (ctx->graph_seen.size() > kMaxSeenPlans) ctx->graph_seen.clear();
  if (++ctx->graph_seen[hash] < 2) return enqueue(st, nullptr);  // first call: eager (and tuned)

  // capture: size the workspace first (no growth may happen inside the capture)
  size_t need = 0;
  X2C_TRY(enqueue(st, &need));
  Arena unused;
  x2c_status ws = ensure_workspace(ctx, need, &unused, st);
  if (ws == X2C_ERR_NOMEM && ctx->split_ws_cap > kSplitWsCapSmall) {
    ctx->split_ws_cap = kSplitWsCapSmall;  // smaller chunks from now on (see dlu_build)
    X2C_TRY(enqueue(st, &need));
    ws = ensure_workspace(ctx, need, &unused, st);
  }
  X2C_TRY(ws);
  if (!ctx->cap_stream) X2C_TRY_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
  const size_t ev0 = ctx->ev_used, pend0 = ctx->pending.size();
  const int64_t launches0 = ctx->launches;
  const double credited0 = plan.credited;
  X2C_TRY_CUDA(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeRelaxed));
  ctx->capturing = true;
  ctx->cap_pinned.clear();
  ctx->cap_off = ctx->cap_cap = 0;
  const x2c_status s = enqueue(ctx->cap_stream, nullptr);
  ctx->capturing = false;
  cudaGraph_t graph = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(ctx->cap_stream, &graph);
  auto *e = new x2c_ctx::GraphEntry();
  e->pinned.swap(ctx->cap_pinned);
  e->graph = graph;
  e->key = key;
  e->hash = hash;
  e->ws_generation = ctx->ws_generation;
  e->launches = ctx->launches - launches0;
  e->pair_blocks = ctx->counters.pair_blocks;
  e->atomic_solves = ctx->counters.atomic_solves;
  e->credited = plan.credited - credited0;
  ctx->launches = launches0;
  plan.credited = credited0;
  // the timing events of the capture name its event-record nodes
  std::vector<x2c_ctx::Pending> timed(ctx->pending.begin() + pend0, ctx->pending.end());
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> tev;
  for (const auto &p : timed) tev.push_back({ctx->ev_pool[p.begin], ctx->ev_pool[p.begin + 1]});
  ctx->pending.resize(pend0);
  ctx->ev_used = ev0;
  if (s != X2C_OK || ce != cudaSuccess || !graph) {
    cudaGetLastError();
    destroy_entry(e);
    return s != X2C_OK ? s : cuda_fail(ctx, ce, "graph capture");
  }
  if (!timed.empty()) {
    size_t nn = 0;
    X2C_TRY_CUDA(ctx, cudaGraphGetNodes(graph, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    X2C_TRY_CUDA(ctx, cudaGraphGetNodes(graph, nodes.data(), &nn));
    std::map<cudaEvent_t, cudaGraphNode_t> rec;
    for (auto nd : nodes) {
      cudaGraphNodeType ty;
      X2C_TRY_CUDA(ctx, cudaGraphNodeGetType(nd, &ty));
      if (ty != cudaGraphNodeTypeEventRecord) continue;
      cudaEvent_t ev;
      X2C_TRY_CUDA(ctx, cudaGraphEventRecordNodeGetEvent(nd, &ev));
      rec[ev] = nd;
    }
    for (size_t i = 0; i < timed.size(); ++i) {
      auto b = rec.find(tev[i].first), en = rec.find(tev[i].second);
      if (b == rec.end() || en == rec.end()) {
        destroy_entry(e);
        ctx->last_error = "graph capture: timing event without a record node";
        return X2C_ERR_CUDA;
      }
      e->timed.push_back({timed[i].name, timed[i].flops, b->second, en->second});
    }
  }
  const cudaError_t ie = cudaGraphInstantiate(&e->exec, graph, 0);
  if (ie != cudaSuccess) {
    cudaGetLastError();
    e->exec = nullptr;
    destroy_entry(e);
    return cuda_fail(ctx, ie, "cudaGraphInstantiate");
  }
  if (cache.size() >= kMaxGraphs) {  // least recently used; a replay may still read its sources
    X2C_TRY_CUDA(ctx, cudaDeviceSynchronize());
    destroy_entry(cache.front());
    cache.erase(cache.begin());
  }
  cache.push_back(e);
  ctx->graph_captures++;
  return replay(ctx, e, st, plan);
}

}  // namespace

x2c_status ensure_stage(x2c_ctx *ctx, size_t bytes) {
  if (bytes <= ctx->stage_bytes) return X2C_OK;
  X2C_TRY_CUDA(ctx, cudaDeviceSynchronize());
  if (ctx->stage) cudaFree(ctx->stage);
  ctx->stage = nullptr;
  ctx->stage_bytes = 0;
  cudaError_t e = cudaMalloc(&ctx->stage, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ctx->last_error = std::string("staging allocation: ") + cudaGetErrorString(e);
    return X2C_ERR_NOMEM;
  }
  ctx->stage_bytes = bytes;
  return X2C_OK;
}

void drop_graphs(x2c_ctx *ctx) {
  if (!ctx->graph_cache.empty()) {
    cudaDeviceSynchronize();  // a replay in flight still reads the pinned sources
    for (auto *e : ctx->graph_cache) destroy_entry(e);
  }
  ctx->graph_cache.clear();
  ctx->graph_seen.clear();
}

x2c_status full_build(x2c_ctx *ctx, const x2c_options *opt, const x2c_mats *mol, const x2c_hout *h,
                      const x2c_uout *U, cudaStream_t st, size_t *dry_bytes) {
  X2C_TRY(begin_call(ctx));
  X2C_TRY(check_options(opt));
  const int nc = opt->two_component ? 4 : 1;
  if (!mats_ok(mol, nc) || !h) return X2C_ERR_ARG;
  x2c_options o = *opt;
  o.dlu_potential = X2C_DLU_MOLECULAR_BLOCK;
  o.precision = X2C_PREC_FP64;
  o.so_same_atom_only = 1;  // one atom: the only pair is the diagonal one
  o.local_approx = X2C_LOCAL_DLU;
  int32_t offs[2] = {0, mol->n};
  x2c_layout lay{1, offs, nullptr, 0, nullptr};
  BuildPlan plan;
  plan.nc = nc;
  KindIndex kinds;
  X2C_TRY(add_molecule(plan, &o, &lay, mol, h, 0, kinds));
  const bool dkh = o.decoupling >= 2;
  if (dkh) {
    // DKHn: h is the DKHn Hamiltonian itself (Sec. II.C), not Eq. 8 with the cut transforms;
    // the plan then only solves for the transforms, when they are asked for
    if (!fw_supported(mol->n, o.decoupling)) return X2C_ERR_ARG;
    plan.pairs.clear();
  }
  std::vector<double *> ULp, USp;
  auto enqueue = [&](cudaStream_t s, size_t *dry) -> x2c_status {
    if (dkh) {
      const size_t need = dkh_hamiltonian_workspace_bytes(mol->n, nc, o.decoupling) + 1024;
      size_t u_need = 0;
      if (U) X2C_TRY(run_plan(ctx, &o, plan, s, nullptr, nullptr, &u_need));
      if (dry) {
        *dry = std::max(need, u_need);
        return X2C_OK;
      }
      Arena ar;
      X2C_TRY(ensure_workspace(ctx, std::max(need, u_need), &ar, s));
      auto *dd = reinterpret_cast<InputDesc *>(ar.take_bytes(sizeof(InputDesc)));
      if (!dd) return X2C_ERR_NOMEM;
      const InputDesc hd = input_desc(mol, nc, 0, mol->n);
      X2C_TRY(upload(ctx, s, dd, &hd, sizeof(InputDesc)));
      X2C_TRY(dkh_hamiltonian(ctx, s, speed_of_light(&o), mol->n, nc, o.decoupling, dd, h->h, ar));
      plan.credited += hamiltonian_flops(mol->n, nc, o.decoupling);
      if (!U) return X2C_OK;
      X2C_TRY(run_plan(ctx, &o, plan, s, &ULp, &USp, nullptr));
    } else {
      X2C_TRY(run_plan(ctx, &o, plan, s, &ULp, &USp, dry));
    }
    if (dry || !U) return X2C_OK;
    const size_t n2 = (size_t)mol->n * mol->n;
    for (int q = 0; q < nc; ++q) {
      if (U->UL[q]) X2C_TRY(device_copy(ctx, s, U->UL[q], ULp[0] + q * n2, n2 * sizeof(double)));
      if (U->US[q]) X2C_TRY(device_copy(ctx, s, U->US[q], USp[0] + q * n2, n2 * sizeof(double)));
    }
    return X2C_OK;
  };
  if (dry_bytes) return enqueue(st, dry_bytes);
  X2C_TRY(graph_run(ctx, st, [&] { return plan_key(ctx, 0, &o, plan, U, U ? 1 : 0); }, plan, enqueue));
  end_call(ctx, plan);
  return X2C_OK;
}

x2c_status dlu_build(x2c_ctx *ctx, const x2c_options *opt, int n_mol, const x2c_layout *layouts,
                     const x2c_mats *mols, const x2c_hout *h, const KindTransforms *ku, cudaStream_t st,
                     size_t *dry_bytes, int a_begin, int a_end, const uint8_t *nbr) {
  X2C_TRY(begin_call(ctx));
  X2C_TRY(check_options(opt));
  if (n_mol < 1 || !layouts || !mols || !h) return X2C_ERR_ARG;
  if ((a_begin != 0 || a_end >= 0 || nbr) && n_mol != 1) return X2C_ERR_ARG;
  if (nbr && opt->local_approx != X2C_LOCAL_DLU) return X2C_ERR_ARG;
  BuildPlan plan;
  plan.nc = opt->two_component ? 4 : 1;
  KindIndex kinds;
  for (int i = 0; i < n_mol; ++i)
    X2C_TRY(add_molecule(plan, opt, &layouts[i], &mols[i], &h[i], i, kinds, ku ? &ku[i] : nullptr, a_begin, a_end,
                         nbr));
  auto enqueue = [&](cudaStream_t s, size_t *dry) { return run_plan(ctx, opt, plan, s, nullptr, nullptr, dry); };
  if (dry_bytes) return enqueue(st, dry_bytes);
  X2C_TRY(graph_run(ctx, st, [&] { return plan_key(ctx, 1, opt, plan, nullptr, 0); }, plan, enqueue));
  end_call(ctx, plan);
  return X2C_OK;
}

x2c_status transforms_build(x2c_ctx *ctx, const x2c_options *opt, int n_problems, const x2c_mats *inputs,
                            const x2c_uout *U, cudaStream_t st, size_t *dry_bytes) {
  X2C_TRY(begin_call(ctx));
  X2C_TRY(check_options(opt));
  if (n_problems < 1 || !inputs || !U) return X2C_ERR_ARG;
  BuildPlan plan;
  plan.nc = opt->two_component ? 4 : 1;
  for (int i = 0; i < n_problems; ++i) {
    if (!mats_ok(&inputs[i], plan.nc)) return X2C_ERR_ARG;
    for (int q = 0; q < plan.nc; ++q)
      if (!U[i].UL[q] || !U[i].US[q]) return X2C_ERR_ARG;
    plan.problems.push_back({input_desc(&inputs[i], plan.nc, 0, inputs[i].n), inputs[i].n});
  }
  std::vector<double *> ULp, USp;
  auto enqueue = [&](cudaStream_t s, size_t *dry) -> x2c_status {
    X2C_TRY(run_plan(ctx, opt, plan, s, &ULp, &USp, dry));
    if (dry) return X2C_OK;
    for (int i = 0; i < n_problems; ++i) {
      const size_t n2 = (size_t)inputs[i].n * inputs[i].n;
      for (int q = 0; q < plan.nc; ++q) {
        X2C_TRY(device_copy(ctx, s, U[i].UL[q], ULp[i] + q * n2, n2 * sizeof(double)));
        X2C_TRY(device_copy(ctx, s, U[i].US[q], USp[i] + q * n2, n2 * sizeof(double)));
      }
    }
    return X2C_OK;
  };
  if (dry_bytes) return enqueue(st, dry_bytes);
  X2C_TRY(graph_run(ctx, st, [&] { return plan_key(ctx, 2, opt, plan, U, n_problems); }, plan, enqueue));
  end_call(ctx, plan);
  return X2C_OK;
}

// DLU assembly from given per-kind transforms, gathered part-major into the staging area.
// With P (picture change) instead of mol, the assembly runs on the property: V = P^LL,
// T = 0, W = P^SS and 4c^2 = 1 turn the middle matrix [[V, T], [T, W/4c^2 - T]] of Eq. 8
// into [[P^LL, 0], [0, P^SS]]; the zero matrix (and absent spin parts) sit in the staging area.
x2c_status with_transforms(x2c_ctx *ctx, const x2c_options *opt, const x2c_layout *layout, const x2c_uout *kind_U,
                           const x2c_mats *mol, const x2c_property *P, const x2c_hout *h, cudaStream_t st) {
  X2C_TRY(begin_call(ctx));
  X2C_TRY(check_options(opt));
  if (!layout || !kind_U || (!mol && !P) || layout->n_kinds < 1 || !layout->kinds ||
      opt->dlu_potential != X2C_DLU_FREE_ATOM)
    return X2C_ERR_ARG;
  const int nc = opt->two_component ? 4 : 1;
  const int nk = layout->n_kinds;
  // the assembly reads each kind's parts contiguously (part-major): gather them into the
  // staging area unless they already are
  std::vector<size_t> off(nk + 1, 0);
  for (int k = 0; k < nk; ++k) {
    const int n = layout->kinds[k].n;
    if (n < 1) return X2C_ERR_ARG;
    for (int q = 0; q < nc; ++q)
      if (!kind_U[k].UL[q] || !kind_U[k].US[q]) return X2C_ERR_ARG;
    off[k + 1] = off[k] + 2 * (size_t)nc * n * n;
  }
  const size_t zero_doubles = P ? ((size_t)P->n * P->n + 31) / 32 * 32 : 0;
  X2C_TRY(ensure_stage(ctx, (off[nk] + zero_doubles) * sizeof(double)));
  double *stage = reinterpret_cast<double *>(ctx->stage);
  std::vector<const double *> ul(nk), us(nk);
  for (int k = 0; k < nk; ++k) {
    const size_t n2 = (size_t)layout->kinds[k].n * layout->kinds[k].n;
    double *dst = stage + off[k];
    for (int q = 0; q < nc; ++q) {
      X2C_TRY(device_copy(ctx, st, dst + q * n2, kind_U[k].UL[q], n2 * sizeof(double)));
      X2C_TRY(device_copy(ctx, st, dst + (nc + q) * n2, kind_U[k].US[q], n2 * sizeof(double)));
    }
    ul[k] = dst;
    us[k] = dst + nc * n2;
  }
  KindTransforms ku{ul.data(), us.data()};
  if (!P) return dlu_build(ctx, opt, 1, layout, mol, h, &ku, st, nullptr);
  double *zero = stage + off[nk];
  X2C_TRY(device_fill(ctx, st, zero, 0, zero_doubles * sizeof(double)));
  x2c_mats pm{};
  pm.n = P->n;
  pm.S = P->LL;  // not read: the transforms are given
  pm.T = zero;
  pm.V = P->LL;
  pm.W0 = P->SS[0];
  pm.Wx = P->SS[1] ? P->SS[1] : zero;
  pm.Wy = P->SS[2] ? P->SS[2] : zero;
  pm.Wz = P->SS[3] ? P->SS[3] : zero;
  x2c_options o = *opt;
  o.c = 0.5;
  o.local_approx = X2C_LOCAL_DLU;
  return dlu_build(ctx, &o, 1, layout, &pm, h, &ku, st, nullptr);
}

}  // namespace x2c

using namespace x2c;

extern "C" {

const char *x2c_status_string(x2c_status s) {
  switch (s) {
    case X2C_OK: return "ok";
    case X2C_ERR_ARG: return "invalid argument";
    case X2C_ERR_NOMEM: return "out of memory";
    case X2C_ERR_CUDA: return "CUDA error";
    case X2C_ERR_NOT_POSDEF: return "S or T is not positive definite";
    case X2C_ERR_NOCONV: return "iteration did not converge";
    case X2C_ERR_DECOUPLING: return "positive/negative energy spectrum does not split at -c^2";
    case X2C_ERR_NONFINITE: return "non-finite value";
    case X2C_ERR_ADMISSION: return "request exceeds the memory budget";
    case X2C_ERR_TIMEOUT: return "timed out";
    case X2C_ERR_CANCELLED: return "cancelled";
    case X2C_ERR_NOT_FOUND: return "unknown ticket";
  }
  return "unknown status";
}

x2c_status x2c_ctx_create(int device, x2c_ctx **out) {
  if (!out) return X2C_ERR_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return X2C_ERR_ARG;
  }
  x2c_ctx *ctx = new x2c_ctx();
  ctx->device = device;
  if (cudaSetDevice(device) != cudaSuccess || cudaMalloc(&ctx->d_status, sizeof(int)) != cudaSuccess ||
      cudaMemset(ctx->d_status, 0, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return X2C_ERR_CUDA;
  }
  *out = ctx;
  return X2C_OK;
}

x2c_status x2c_ctx_destroy(x2c_ctx *ctx) {
  if (!ctx) return X2C_OK;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  drop_graphs(ctx);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->stage) cudaFree(ctx->stage);
  for (auto e : ctx->ev_pool) cudaEventDestroy(e);
  for (auto e : ctx->tune_ev)
    if (e) cudaEventDestroy(e);
  for (auto &f : ctx->ring_inflight) cudaEventDestroy(f.done);
  for (auto e : ctx->ring_events) cudaEventDestroy(e);
  if (ctx->ring) cudaFreeHost(ctx->ring);
  for (auto s : ctx->aux) cudaStreamDestroy(s);
  for (auto e : ctx->aux_join) cudaEventDestroy(e);
  if (ctx->aux_fork) cudaEventDestroy(ctx->aux_fork);
  if (ctx->d_status) cudaFree(ctx->d_status);
  delete ctx;
  return X2C_OK;
}

const char *x2c_last_error_message(x2c_ctx *ctx) { return ctx ? ctx->last_error.c_str() : ""; }

x2c_status x2c_ctx_status(x2c_ctx *ctx, void *stream) {
  if (!ctx) return X2C_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  X2C_TRY_CUDA(ctx, cudaSetDevice(ctx->device));
  X2C_TRY_CUDA(ctx, cudaStreamSynchronize(st));
  int code = 0;
  X2C_TRY_CUDA(ctx, cudaMemcpy(&code, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (code) X2C_TRY_CUDA(ctx, cudaMemset(ctx->d_status, 0, sizeof(int)));
  return static_cast<x2c_status>(code);
}

x2c_status x2c_ctx_counters(x2c_ctx *ctx, x2c_counters *out) {
  if (!ctx || !out) return X2C_ERR_ARG;
  *out = ctx->counters;
  return X2C_OK;
}

x2c_status x2c_ctx_set_timing(x2c_ctx *ctx, int32_t enable) {
  if (!ctx) return X2C_ERR_ARG;
  X2C_TRY_CUDA(ctx, cudaSetDevice(ctx->device));
  if (!ctx->pending.empty()) X2C_TRY_CUDA(ctx, cudaDeviceSynchronize());
  ctx->timing = enable != 0;
  ctx->pending.clear();
  ctx->ev_used = 0;
  ctx->kernel_ms.clear();
  return X2C_OK;
}

x2c_status x2c_query_workspace(x2c_ctx *ctx, const x2c_options *opt, int32_t n_mol, const x2c_layout *layouts,
                               const x2c_mats *mols, size_t *bytes) {
  if (!bytes) return X2C_ERR_ARG;
  *bytes = 0;
  if (!ctx || !opt || n_mol < 0) return X2C_ERR_ARG;
  size_t need = 0;
  if (n_mol == 0) {  // full X2C of mols[0]
    if (!mols) return X2C_ERR_ARG;
    const int nc = opt->two_component ? 4 : 1;
    x2c_hout h{};
    static double dummy;
    for (int q = 0; q < nc; ++q) h.h[q] = &dummy;
    X2C_TRY(full_build(ctx, opt, mols, &h, nullptr, nullptr, &need));
  } else {
    if (!layouts || !mols) return X2C_ERR_ARG;
    std::vector<x2c_hout> h(n_mol);
    static double dummy;
    for (auto &o : h)
      for (int q = 0; q < 4; ++q) o.h[q] = &dummy;
    X2C_TRY(dlu_build(ctx, opt, n_mol, layouts, mols, h.data(), nullptr, nullptr, &need));
  }
  *bytes = need;
  return X2C_OK;
}

x2c_status x2c_ctx_set_autotune(x2c_ctx *ctx, int32_t enable) {
  if (!ctx || (enable != 0 && enable != 1)) return X2C_ERR_ARG;
  ctx->autotune = enable != 0;
  return X2C_OK;
}

const char *x2c_ctx_tuning_log(x2c_ctx *ctx) { return ctx ? ctx->tune_log.c_str() : ""; }

x2c_status x2c_ctx_set_split_variant(x2c_ctx *ctx, int32_t variant) {
  if (!ctx || variant < -1 || variant > 2) return X2C_ERR_ARG;
  ctx->split_variant = variant;
  return X2C_OK;
}

x2c_status x2c_ctx_set_graphs(x2c_ctx *ctx, int32_t enable) {
  if (!ctx || (enable != 0 && enable != 1)) return X2C_ERR_ARG;
  X2C_TRY_CUDA(ctx, cudaSetDevice(ctx->device));
  if (!enable) drop_graphs(ctx);
  ctx->graphs = enable != 0;
  return X2C_OK;
}

x2c_status x2c_ctx_graph_stats(x2c_ctx *ctx, x2c_graph_stats *out) {
  if (!ctx || !out) return X2C_ERR_ARG;
  out->captures = ctx->graph_captures;
  out->replays = ctx->graph_replays;
  out->cached = (int32_t)ctx->graph_cache.size();
  out->last_replayed = ctx->last_replayed ? 1 : 0;
  return X2C_OK;
}

x2c_status x2c_ctx_kernel_times(x2c_ctx *ctx, int32_t max_entries, char *names, double *ms,
                                int64_t *launches, double *flops, int32_t *n_entries) {
  if (!ctx || max_entries < 0 || !n_entries) return X2C_ERR_ARG;
  X2C_TRY_CUDA(ctx, cudaSetDevice(ctx->device));
  for (auto &p : ctx->pending) {
    cudaEvent_t b = ctx->ev_pool[p.begin], e = ctx->ev_pool[p.begin + 1];
    X2C_TRY_CUDA(ctx, cudaEventSynchronize(e));
    float t = 0.f;
    X2C_TRY_CUDA(ctx, cudaEventElapsedTime(&t, b, e));
    auto &acc = ctx->kernel_ms[p.name];
    acc.ms += t;
    acc.flops += p.flops;
    acc.launches += 1;
  }
  ctx->pending.clear();
  ctx->ev_used = 0;
  int32_t i = 0;
  for (auto &kv : ctx->kernel_ms) {
    if (i >= max_entries) break;
    if (names) {
      std::strncpy(names + 32 * i, kv.first.c_str(), 31);
      names[32 * i + 31] = 0;
    }
    if (ms) ms[i] = kv.second.ms;
    if (launches) launches[i] = kv.second.launches;
    if (flops) flops[i] = kv.second.flops;
    ++i;
  }
  *n_entries = i;
  return X2C_OK;
}

x2c_status x2c_build_full(x2c_ctx *ctx, const x2c_options *opt, const x2c_mats *mol,
                          const x2c_hout *h, const x2c_uout *U, void *stream) {
  return full_build(ctx, opt, mol, h, U, static_cast<cudaStream_t>(stream), nullptr);
}

x2c_status x2c_build_dlu(x2c_ctx *ctx, const x2c_options *opt, const x2c_layout *layout,
                         const x2c_mats *mol, const x2c_hout *h, void *stream) {
  return dlu_build(ctx, opt, 1, layout, mol, h, nullptr, static_cast<cudaStream_t>(stream), nullptr);
}

x2c_status x2c_build_dlu_rows(x2c_ctx *ctx, const x2c_options *opt, const x2c_layout *layout, const x2c_mats *mol,
                              const x2c_hout *h, int32_t a_begin, int32_t a_end, void *stream) {
  if (!layout || a_begin < 0 || a_end <= a_begin || a_end > layout->n_atoms) return X2C_ERR_ARG;
  return dlu_build(ctx, opt, 1, layout, mol, h, nullptr, static_cast<cudaStream_t>(stream), nullptr, a_begin, a_end);
}

x2c_status x2c_build_dlu_nab(x2c_ctx *ctx, const x2c_options *opt, const x2c_layout *layout, const x2c_mats *mol,
                             const uint8_t *neighbours, const x2c_hout *h, void *stream) {
  if (!neighbours) return X2C_ERR_ARG;
  return dlu_build(ctx, opt, 1, layout, mol, h, nullptr, static_cast<cudaStream_t>(stream), nullptr, 0, -1,
                   neighbours);
}

x2c_status x2c_dlu_partition(const x2c_layout *layout, int32_t rank, int32_t world, int32_t *a_begin,
                             int32_t *a_end) {
  if (!layout || !layout->atom_offset || layout->n_atoms < 1 || world < 1 || rank < 0 || rank >= world || !a_begin ||
      !a_end)
    return X2C_ERR_ARG;
  const int L = layout->n_atoms;
  std::vector<double> n(L);
  for (int a = 0; a < L; ++a) {
    n[a] = layout->atom_offset[a + 1] - layout->atom_offset[a];
    if (n[a] < 1) return X2C_ERR_ARG;
  }
  // work of row atom A: its pair blocks (A, B >= A), each about n_A n_B (n_A + n_B) products
  std::vector<double> cum(L + 1, 0.0), tail_n(L + 1, 0.0), tail_n2(L + 1, 0.0);
  for (int b = L - 1; b >= 0; --b) {
    tail_n[b] = tail_n[b + 1] + n[b];
    tail_n2[b] = tail_n2[b + 1] + n[b] * n[b];
  }
  for (int a = 0; a < L; ++a) cum[a + 1] = cum[a] + n[a] * (n[a] * tail_n[a] + tail_n2[a]);
  // rank r takes the rows whose cumulative work starts in [r W / world, (r + 1) W / world)
  auto cut = [&](int r) {
    if (r <= 0) return 0;
    if (r >= world) return L;
    const double target = cum[L] * r / world;
    int a = 0;
    while (a < L && cum[a] < target) ++a;
    return a;
  };
  *a_begin = cut(rank);
  *a_end = cut(rank + 1);
  return X2C_OK;
}

x2c_status x2c_build_dlu_batched(x2c_ctx *ctx, const x2c_options *opt, int32_t n_mol,
                                 const x2c_layout *layouts, const x2c_mats *mols,
                                 const x2c_hout *h, void *stream) {
  return dlu_build(ctx, opt, n_mol, layouts, mols, h, nullptr, static_cast<cudaStream_t>(stream), nullptr);
}

x2c_status x2c_build_dlu_with_transforms(x2c_ctx *ctx, const x2c_options *opt, const x2c_layout *layout,
                                         const x2c_uout *kind_U, const x2c_mats *mol, const x2c_hout *h,
                                         void *stream) {
  return with_transforms(ctx, opt, layout, kind_U, mol, nullptr, h, static_cast<cudaStream_t>(stream));
}

x2c_status x2c_picture_change(x2c_ctx *ctx, const x2c_options *opt, const x2c_layout *layout,
                              const x2c_uout *kind_U, const x2c_property *P, const x2c_hout *out,
                              void *stream) {
  if (!P || P->n < 1 || !P->LL || !P->SS[0]) return X2C_ERR_ARG;
  return with_transforms(ctx, opt, layout, kind_U, nullptr, P, out, static_cast<cudaStream_t>(stream));
}

x2c_status x2c_atomic_transforms(x2c_ctx *ctx, const x2c_options *opt, int32_t n_problems,
                                 const x2c_mats *inputs, const x2c_uout *U, void *stream) {
  return transforms_build(ctx, opt, n_problems, inputs, U, static_cast<cudaStream_t>(stream), nullptr);
}

x2c_status x2c_quaternion_to_dense(const double *const h[4], int32_t n, double *out, void *stream) {
  if (!h || !h[0] || n < 1 || !out) return X2C_ERR_ARG;
  const int64_t total = (int64_t)n * n;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
  quat_to_dense_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(h[0], h[1], h[2], h[3], n, out);
  return cudaGetLastError() == cudaSuccess ? X2C_OK : X2C_ERR_CUDA;
}

}  // extern "C"
