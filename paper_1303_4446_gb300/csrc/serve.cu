// x2c_server_*: a device-resident request loop with continuous batching, a device cache of
// atomic transforms and admission under a device-memory budget (include/x2c.h).
//
// One scheduler thread owns the slots (stream + context each), the memory pool and the
// cache; client threads only queue requests and read results, under one mutex.  A slot's
// work is: input copies -> missing kinds' transforms (cached) -> one batched DLU build (or a
// full X2C build) -> optional copies of h to the host -> the device status word -> an event
// the scheduler polls.  The scheduling decisions themselves live in serve_policy.h.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>

#include "common.cuh"
#include "serve_policy.h"

namespace {

using x2c::serve::Candidate;
using Clock = std::chrono::steady_clock;

constexpr uint64_t kDefaultBudget = 150ull * 1000 * 1000 * 1000;
// Split-precision workspace cap of a slot: requests larger than it run their pair assembly in
// chunks, and the admission budget counts no more than this per slot.
constexpr size_t kSlotSplitCap = ::kSplitWsCapSmall;
constexpr size_t kLargePairs = 2000;  // builds above this many pair blocks count as large
constexpr int kFreeSMs = 32;          // SMs a large build leaves to the other slots

struct CacheEntry {
  std::tuple<uint64_t, int, int, uint64_t> key;  // kind key, n, nc | decoupling << 8, bits of c
  double *U = nullptr;                           // U^L (nc n^2) then U^S (nc n^2)
  size_t bytes = 0;
  cudaEvent_t ready = nullptr;                   // recorded after the solve, on its slot
  int solver_slot = -1;
  int state = 0;                                 // 0 being solved, 1 ready, 2 failed
  int fail_status = 0;
  int refs = 0;                                  // requests in flight that use it
  uint64_t last_use = 0;
  bool in_map = true;
};
using EntryPtr = std::shared_ptr<CacheEntry>;

struct Request {
  uint64_t ticket = 0;
  x2c_request rq{};
  std::vector<int32_t> offsets, atom_kind;
  std::vector<x2c_mats> kinds;
  std::vector<uint64_t> keys;
  std::vector<char> used;     // kinds some atom refers to
  int nc = 1;
  int64_t n = 0, ld = 0;
  bool copy_in = false;       // inputs are copied into a server slab
  size_t in_bytes = 0;        // that slab
  size_t out_bytes = 0;       // outputs the server allocates (kept until release unless host)
  bool out_kept = false;      // server-allocated device outputs handed to the caller
  uint64_t group = 0;
  bool batchable = false;
  int state = X2C_STATE_QUEUED;
  x2c_status status = X2C_OK;
  char *in_slab = nullptr;
  double *out_dev = nullptr;
  x2c_mats dmol{};
  std::vector<x2c_mats> dkinds;
  x2c_hout dout{};
  std::vector<EntryPtr> deps;
  double t_arrival = 0, t_submit = 0, t_admit = -1, t_start = -1, t_end = -1;
  int batch = 0, hits = 0, misses = 0, slot = -1;

  size_t own_bytes() const { return in_bytes + out_bytes; }
};
using ReqPtr = std::shared_ptr<Request>;

struct Slot {
  cudaStream_t st = nullptr;      // normal priority: large builds
  cudaStream_t st_hi = nullptr;   // highest priority: small builds
  cudaStream_t cur = nullptr;     // the stream of the batch in flight
  x2c_ctx *ctx = nullptr;
  cudaEvent_t ev_start = nullptr, ev_done = nullptr;
  int *h_status = nullptr;  // pinned: the context's device status word after the build
  bool busy = false;
  x2c_status host_fail = X2C_OK;
  std::vector<ReqPtr> batch;
  std::vector<EntryPtr> solving;
  size_t reserved = 0;      // bytes taken at launch for the batch's inputs and outputs
};

size_t mat_bytes(int64_t n) { return static_cast<size_t>(n) * n * sizeof(double); }
size_t round256(size_t b) { return (b + 255) / 256 * 256; }
uint64_t dbits(double x) {
  uint64_t u;
  std::memcpy(&u, &x, sizeof u);
  return u;
}

}  // namespace

struct x2c_server {
  int device = 0;
  int max_batch = 16;
  uint64_t budget = kDefaultBudget;
  cudaMemPool_t pool = nullptr;
  cudaStream_t misc = nullptr;
  cudaEvent_t ev_ref = nullptr;
  Clock::time_point t0;
  double t_ref = 0;  // server-clock time of ev_ref
  x2c_ctx *planner = nullptr;  // dry runs only (under the mutex)
  int sms_ = 152;
  std::vector<Slot> slots;

  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  std::thread thread;

  uint64_t next_ticket = 1;
  std::deque<ReqPtr> queue;
  std::map<uint64_t, ReqPtr> requests;
  std::map<std::tuple<uint64_t, int, int, uint64_t>, EntryPtr> cache;
  uint64_t use_clock = 0;

  // memory accounting (bytes the server holds from its pool)
  uint64_t in_use = 0, peak = 0;
  // statistics
  x2c_server_stats st{};
  std::vector<double> lat_ms;
  int running = 0;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
  double dev_time(cudaEvent_t e) const {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ev_ref, e) != cudaSuccess) {
      cudaGetLastError();
      return -1.0;
    }
    return t_ref + ms * 1e-3;
  }
  void take(uint64_t b) {
    in_use += b;
    if (in_use > peak) peak = in_use;
  }
  void give(uint64_t b) { in_use -= std::min(in_use, b); }

  void loop();
  bool plan_batch(Slot &sl, std::vector<ReqPtr> &batch);
  size_t extra_bytes(Slot &sl, const std::vector<ReqPtr> &batch, size_t *ws_need);
  bool evict_for(size_t need);
  void launch(int slot_index, std::vector<ReqPtr> &batch);
  void finish(int slot_index, cudaError_t e);
  void fill_result(const Request &r, x2c_result *res) const;
};

namespace {

// Memory-independent checks of a request and its byte counts.
x2c_status prepare(x2c_server *s, const x2c_request *in, Request &r) {
  r.rq = *in;
  x2c_status cs = x2c::check_options(&in->opt);
  if (cs != X2C_OK) return cs;
  if (in->kind != X2C_REQ_DLU && in->kind != X2C_REQ_FULL) return X2C_ERR_ARG;
  if (in->memory != X2C_MEM_DEVICE && in->memory != X2C_MEM_HOST) return X2C_ERR_ARG;
  if (in->reserved0 != 0) return X2C_ERR_ARG;
  r.nc = in->opt.two_component ? 4 : 1;
  if (!x2c::mats_ok(&in->mol, r.nc)) return X2C_ERR_ARG;
  r.n = in->mol.n;
  r.ld = in->ld ? in->ld : r.n;
  if (r.ld < r.n) return X2C_ERR_ARG;
  const bool free_atom = in->kind == X2C_REQ_DLU && in->opt.dlu_potential == X2C_DLU_FREE_ATOM;
  if (in->kind != X2C_REQ_FULL) {
    const x2c_layout &L = in->layout;
    if (L.n_atoms < 1 || !L.atom_offset) return X2C_ERR_ARG;
    r.offsets.assign(L.atom_offset, L.atom_offset + L.n_atoms + 1);
    if (r.offsets[0] != 0 || r.offsets[L.n_atoms] != r.n) return X2C_ERR_ARG;
    for (int a = 0; a < L.n_atoms; ++a) {
      const int na = r.offsets[a + 1] - r.offsets[a];
      if (na < 1) return X2C_ERR_ARG;
    }
    if (free_atom) {
      if (!L.atom_kind || L.n_kinds < 1 || !L.kinds) return X2C_ERR_ARG;
      r.atom_kind.assign(L.atom_kind, L.atom_kind + L.n_atoms);
      r.kinds.assign(L.kinds, L.kinds + L.n_kinds);
      r.keys.assign(L.n_kinds, 0);
      if (in->kind_key) r.keys.assign(in->kind_key, in->kind_key + L.n_kinds);
      r.used.assign(L.n_kinds, 0);
      for (int a = 0; a < L.n_atoms; ++a) {
        const int k = r.atom_kind[a];
        if (k < 0 || k >= L.n_kinds) return X2C_ERR_ARG;
        r.used[k] = 1;
        if (!x2c::mats_ok(&r.kinds[k], r.nc) || r.kinds[k].n != r.offsets[a + 1] - r.offsets[a]) return X2C_ERR_ARG;
      }
    }
    r.rq.layout.atom_offset = r.offsets.data();
    r.rq.layout.atom_kind = r.atom_kind.empty() ? nullptr : r.atom_kind.data();
    r.rq.layout.kinds = r.kinds.empty() ? nullptr : r.kinds.data();
    r.rq.kind_key = nullptr;
  }
  // inputs the build reads: T, V, W0 always; S unless free-atom DLU; Wx..Wz when 2c
  const int n_in = (free_atom ? 3 : 4) + (r.nc == 4 ? 3 : 0);
  r.copy_in = in->memory == X2C_MEM_HOST || r.ld != r.n;
  r.in_bytes = 0;
  if (r.copy_in) r.in_bytes += n_in * round256(mat_bytes(r.n));
  if (in->memory == X2C_MEM_HOST && free_atom)
    for (size_t k = 0; k < r.kinds.size(); ++k)
      if (r.used[k]) r.in_bytes += (4 + (r.nc == 4 ? 3 : 0)) * round256(mat_bytes(r.kinds[k].n));
  const bool server_out = in->out.h[0] == nullptr || in->memory == X2C_MEM_HOST;
  if (in->out.h[0]) {
    for (int q = 0; q < r.nc; ++q)
      if (!in->out.h[q]) return X2C_ERR_ARG;
  }
  r.out_bytes = server_out ? r.nc * round256(mat_bytes(r.n)) : 0;
  r.out_kept = in->out.h[0] == nullptr;
  r.batchable = free_atom;
  r.group = r.batchable ? (static_cast<uint64_t>(in->opt.two_component) | (uint64_t)in->opt.precision << 1 |
                           (uint64_t)in->opt.n_slices << 4 | (uint64_t)in->opt.so_same_atom_only << 8 |
                           (uint64_t)in->opt.local_approx << 9) ^
                              (dbits(x2c::speed_of_light(&in->opt)) * 0x9E3779B97F4A7C15ull)
                        : 0;
  (void)s;
  return X2C_OK;
}

}  // namespace

// Extra bytes a batch needs beyond its requests' own: new cache entries and workspace growth.
size_t x2c_server::extra_bytes(Slot &sl, const std::vector<ReqPtr> &batch, size_t *ws_need) {
  const ReqPtr &h = batch[0];
  const x2c_options &opt = h->rq.opt;
  const int nc = h->nc;
  size_t need = 0, entries = 0;
  std::vector<x2c_mats> solve;
  std::map<std::tuple<uint64_t, int, int, uint64_t>, const double *> fresh;
  static const double placeholder[256] = {};
  std::vector<std::vector<const double *>> ul(batch.size()), us(batch.size());
  std::vector<x2c::KindTransforms> ku(batch.size());
  std::vector<x2c_layout> lays;
  std::vector<x2c_mats> mols;
  std::vector<x2c_hout> outs(batch.size());
  if (h->rq.kind == X2C_REQ_FULL) {
    x2c_hout o{};
    for (int q = 0; q < nc; ++q) o.h[q] = const_cast<double *>(placeholder);
    x2c::full_build(planner, &opt, &h->rq.mol, &o, nullptr, nullptr, &need);
    *ws_need = need;
    return x2c::workspace_after_growth(sl.ctx, need) - sl.ctx->ws_bytes;
  }
  for (size_t i = 0; i < batch.size(); ++i) {
    const Request &r = *batch[i];
    lays.push_back(r.rq.layout);
    mols.push_back(r.rq.mol);
    for (int q = 0; q < nc; ++q) outs[i].h[q] = const_cast<double *>(placeholder);
    if (opt.dlu_potential == X2C_DLU_FREE_ATOM) {
      ul[i].assign(r.kinds.size(), nullptr);
      us[i].assign(r.kinds.size(), nullptr);
      for (size_t k = 0; k < r.kinds.size(); ++k) {
        if (!r.keys[k] || !r.used[k]) continue;
        auto key = std::make_tuple(r.keys[k], r.kinds[k].n, nc | (opt.decoupling << 8), dbits(x2c::speed_of_light(&opt)));
        auto it = cache.find(key);
        const double *p;
        if (it != cache.end()) {
          p = it->second->U;
        } else {
          auto f = fresh.find(key);
          if (f == fresh.end()) {
            // a distinct (never dereferenced) address per new kind for the planner's de-duplication
            p = reinterpret_cast<const double *>(reinterpret_cast<uintptr_t>(placeholder) + 4096 * (fresh.size() + 1));
            fresh.emplace(key, p);
            solve.push_back(r.kinds[k]);
            entries += 2 * round256(nc * mat_bytes(r.kinds[k].n));
          } else {
            p = f->second;
          }
        }
        ul[i][k] = p;
        us[i][k] = p + 1;
      }
      ku[i] = x2c::KindTransforms{ul[i].data(), us[i].data()};
    }
  }
  size_t b_build = 0, b_solve = 0;
  x2c::dlu_build(planner, &opt, (int)batch.size(), lays.data(), mols.data(), outs.data(),
                 opt.dlu_potential == X2C_DLU_FREE_ATOM ? ku.data() : nullptr, nullptr, &b_build);
  if (!solve.empty()) {
    std::vector<x2c_uout> uo(solve.size());
    for (auto &u : uo)
      for (int q = 0; q < nc; ++q) u.UL[q] = u.US[q] = const_cast<double *>(placeholder);
    x2c::transforms_build(planner, &opt, (int)solve.size(), solve.data(), uo.data(), nullptr, &b_solve);
  }
  need = std::max(b_build, b_solve);
  *ws_need = need;
  return entries + (x2c::workspace_after_growth(sl.ctx, need) - sl.ctx->ws_bytes);
}

bool x2c_server::evict_for(size_t need) {
  std::vector<x2c::serve::CacheView> view;
  std::vector<EntryPtr> ents;
  for (auto &kv : cache) {
    ents.push_back(kv.second);
    view.push_back({kv.second->last_use, kv.second->bytes, kv.second->state == 1 && kv.second->refs == 0});
  }
  auto pick = x2c::serve::choose_evictions(view, need);
  if (pick.empty()) return false;
  for (size_t i : pick) {
    EntryPtr e = ents[i];
    cache.erase(e->key);
    e->in_map = false;
    cudaFreeAsync(e->U, misc);
    cudaEventDestroy(e->ready);
    e->U = nullptr;
    give(e->bytes);
    st.cache_evictions++;
  }
  return true;
}

// Choose the batch for a free slot (policy + memory); false when the head must wait.
bool x2c_server::plan_batch(Slot &sl, std::vector<ReqPtr> &batch) {
  for (int attempt = 0; attempt < 2; ++attempt) {
    std::vector<Candidate> cand;
    for (auto &r : queue) cand.push_back({r->own_bytes(), r->group, r->batchable});
    const uint64_t free_b = budget > in_use ? budget - in_use : 0;
    auto pick = x2c::serve::choose_batch(cand, free_b, max_batch);
    if (!pick.empty()) {
      batch.clear();
      for (size_t i : pick) batch.push_back(queue[i]);
      while (!batch.empty()) {
        size_t own = 0, ws_need = 0;
        for (auto &r : batch) own += r->own_bytes();
        const size_t extra = extra_bytes(sl, batch, &ws_need);
        if (own + extra <= free_b) return true;
        if (batch.size() == 1) {
          if (attempt == 0 && evict_for(own + extra - free_b)) break;  // retry with the freed memory
          return false;
        }
        batch.pop_back();
      }
      if (batch.empty()) return false;
      continue;
    }
    if (queue.empty()) return false;
    const size_t need = queue[0]->own_bytes();
    if (attempt == 0 && need > free_b && evict_for(need - free_b)) continue;
    return false;
  }
  return false;
}

void x2c_server::launch(int si, std::vector<ReqPtr> &batch) {
  Slot &sl = slots[si];
  sl.batch = batch;
  sl.solving.clear();
  sl.host_fail = X2C_OK;
  sl.busy = true;
  sl.reserved = 0;
  // Small builds run on the slot's high-priority stream, so that their CTAs are scheduled
  // ahead of the remaining CTAs of large builds on other slots; large builds leave some SMs
  // free of their persistent tensor-core kernels.
  size_t batch_pairs = 0;
  for (auto &rp : batch) {
    const size_t L = rp->offsets.empty() ? 1 : rp->offsets.size() - 1;
    batch_pairs += L * (L + 1) / 2;
  }
  const bool large = batch_pairs > kLargePairs;
  cudaStream_t s = large ? sl.st : sl.st_hi;
  sl.cur = s;
  sl.ctx->cta_cap = large ? std::max(1, sms_ - kFreeSMs) : 0;
  const ReqPtr &h = batch[0];
  const x2c_options opt = h->rq.opt;
  const int nc = h->nc;
  const double t_adm = now();
  const size_t ws_before = sl.ctx->ws_bytes;
  auto fail = [&](x2c_status code) {
    if (sl.host_fail == X2C_OK) sl.host_fail = code;
  };
  cudaEventRecord(sl.ev_start, s);
  st.builds_launched++;
  running += (int)batch.size();
  st.max_concurrent = std::max<int32_t>(st.max_concurrent, running);
  for (auto &rp : batch) {
    Request &r = *rp;
    r.state = X2C_STATE_RUNNING;
    r.t_admit = t_adm;
    r.slot = si;
    r.batch = (int)batch.size();
    const size_t own = r.own_bytes();
    take(own);
    sl.reserved += own;
    const size_t nb = mat_bytes(r.n);
    // outputs
    if (r.out_bytes) {
      if (cudaMallocFromPoolAsync(reinterpret_cast<void **>(&r.out_dev), r.out_bytes, pool, s) != cudaSuccess) {
        cudaGetLastError();
        r.out_dev = nullptr;
        fail(X2C_ERR_NOMEM);
      }
    }
    for (int q = 0; q < nc; ++q)
      r.dout.h[q] = (r.rq.memory == X2C_MEM_DEVICE && r.rq.out.h[0])
                        ? r.rq.out.h[q]
                        : (r.out_dev ? reinterpret_cast<double *>(reinterpret_cast<char *>(r.out_dev) + q * round256(nb))
                                     : nullptr);
    // inputs
    r.dmol = r.rq.mol;
    r.dkinds = r.kinds;
    if (r.in_bytes) {
      if (cudaMallocFromPoolAsync(reinterpret_cast<void **>(&r.in_slab), r.in_bytes, pool, s) != cudaSuccess) {
        cudaGetLastError();
        r.in_slab = nullptr;
        fail(X2C_ERR_NOMEM);
        continue;
      }
      char *p = r.in_slab;
      const cudaMemcpyKind kind = r.rq.memory == X2C_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
      // Blocks a build reads: everything (full X2C), the upper block triangle A <= B (pair
      // blocks of DLU), or the same-atom blocks only (DLU: S in molecular-block mode, and
      // Wx, Wy, Wz when they vanish across atoms).  The copy keeps the n x n layout.
      enum Blocks { kAll, kUpper, kDiag };
      auto put = [&](const double *src, int64_t n, int64_t ld, Blocks which) -> const double * {
        double *dst = reinterpret_cast<double *>(p);
        p += round256(mat_bytes(n));
        auto copy = [&](int64_t r0, int64_t c0, int64_t rows, int64_t cols) {
          if (cudaMemcpy2DAsync(dst + r0 * n + c0, n * sizeof(double), src + r0 * ld + c0, ld * sizeof(double),
                                cols * sizeof(double), rows, kind, s) != cudaSuccess) {
            cudaGetLastError();
            fail(X2C_ERR_CUDA);
          }
        };
        if (which == kAll || r.offsets.empty()) {
          copy(0, 0, n, n);
        } else {
          for (size_t a = 0; a + 1 < r.offsets.size(); ++a) {
            const int64_t o = r.offsets[a], na = r.offsets[a + 1] - o;
            copy(o, o, na, which == kUpper ? n - o : na);
          }
        }
        return dst;
      };
      const bool free_atom = r.rq.kind == X2C_REQ_DLU && opt.dlu_potential == X2C_DLU_FREE_ATOM;
      const Blocks pair = r.rq.kind == X2C_REQ_FULL ? kAll : kUpper;
      const Blocks same = r.rq.kind == X2C_REQ_FULL ? kAll : kDiag;
      const Blocks so = (r.rq.kind == X2C_REQ_FULL || !opt.so_same_atom_only) ? pair : kDiag;
      // DLH fills the atom-other-atom blocks with T + V: all of T and V, W0 on the same-atom
      // blocks only
      const bool dlh = r.rq.kind == X2C_REQ_DLU && opt.local_approx == X2C_LOCAL_DLH;
      if (r.copy_in) {
        r.dmol.T = put(r.rq.mol.T, r.n, r.ld, dlh ? kAll : pair);
        r.dmol.V = put(r.rq.mol.V, r.n, r.ld, dlh ? kAll : pair);
        r.dmol.W0 = put(r.rq.mol.W0, r.n, r.ld, dlh ? kDiag : pair);
        // free-atom DLU never reads the molecular S: any valid device address will do
        r.dmol.S = free_atom ? r.dmol.T : put(r.rq.mol.S, r.n, r.ld, same);
        if (nc == 4) {
          r.dmol.Wx = put(r.rq.mol.Wx, r.n, r.ld, so);
          r.dmol.Wy = put(r.rq.mol.Wy, r.n, r.ld, so);
          r.dmol.Wz = put(r.rq.mol.Wz, r.n, r.ld, so);
        }
      }
      if (r.rq.memory == X2C_MEM_HOST && free_atom) {
        for (size_t ki = 0; ki < r.dkinds.size(); ++ki) {
          if (!r.used[ki]) continue;
          x2c_mats &k = r.dkinds[ki];
          k.S = put(k.S, k.n, k.n, kAll);
          k.T = put(k.T, k.n, k.n, kAll);
          k.V = put(k.V, k.n, k.n, kAll);
          k.W0 = put(k.W0, k.n, k.n, kAll);
          if (nc == 4) {
            k.Wx = put(k.Wx, k.n, k.n, kAll);
            k.Wy = put(k.Wy, k.n, k.n, kAll);
            k.Wz = put(k.Wz, k.n, k.n, kAll);
          }
        }
      }
    }
  }
  // cached transforms: hits, and kinds to solve now (once per key)
  std::vector<std::vector<const double *>> ul(batch.size()), us(batch.size());
  std::vector<x2c::KindTransforms> ku(batch.size());
  std::vector<x2c_mats> solve_in;
  std::vector<x2c_uout> solve_out;
  const bool free_atom = h->rq.kind == X2C_REQ_DLU && opt.dlu_potential == X2C_DLU_FREE_ATOM;
  if (free_atom && sl.host_fail == X2C_OK) {
    for (size_t i = 0; i < batch.size(); ++i) {
      Request &r = *batch[i];
      ul[i].assign(r.kinds.size(), nullptr);
      us[i].assign(r.kinds.size(), nullptr);
      for (size_t k = 0; k < r.kinds.size(); ++k) {
        if (!r.used[k]) continue;
        if (!r.keys[k]) {
          r.misses++;
          continue;
        }
        const int n = r.kinds[k].n;
        auto key = std::make_tuple(r.keys[k], n, nc | (opt.decoupling << 8), dbits(x2c::speed_of_light(&opt)));
        auto it = cache.find(key);
        EntryPtr e;
        if (it != cache.end()) {
          e = it->second;
          r.hits++;
          st.cache_hits++;
          if (e->state == 0 && e->solver_slot != si) cudaStreamWaitEvent(s, e->ready, 0);
        } else {
          e = std::make_shared<CacheEntry>();
          e->key = key;
          e->bytes = 2 * round256(nc * mat_bytes(n));
          e->solver_slot = si;
          if (cudaEventCreateWithFlags(&e->ready, cudaEventDisableTiming) != cudaSuccess ||
              cudaMallocFromPoolAsync(reinterpret_cast<void **>(&e->U), e->bytes, pool, s) != cudaSuccess) {
            cudaGetLastError();
            fail(X2C_ERR_NOMEM);
            break;
          }
          take(e->bytes);
          cache.emplace(key, e);
          sl.solving.push_back(e);
          x2c_uout u{};
          const size_t n2 = static_cast<size_t>(n) * n;
          double *us0 = reinterpret_cast<double *>(reinterpret_cast<char *>(e->U) + e->bytes / 2);
          for (int q = 0; q < nc; ++q) {
            u.UL[q] = e->U + q * n2;
            u.US[q] = us0 + q * n2;
          }
          solve_in.push_back(r.dkinds[k]);
          solve_out.push_back(u);
          r.misses++;
          st.cache_misses++;
        }
        e->refs++;
        e->last_use = ++use_clock;
        r.deps.push_back(e);
        ul[i][k] = e->U;
        us[i][k] = reinterpret_cast<const double *>(reinterpret_cast<const char *>(e->U) + e->bytes / 2);
      }
      ku[i] = x2c::KindTransforms{ul[i].data(), us[i].data()};
    }
    if (sl.host_fail == X2C_OK && !solve_in.empty()) {
      x2c_status s2 = x2c::transforms_build(sl.ctx, &opt, (int)solve_in.size(), solve_in.data(), solve_out.data(), s,
                                            nullptr);
      st.kernel_launches += sl.ctx->launches;
      if (s2 != X2C_OK) fail(s2);
    }
    for (auto &e : sl.solving) cudaEventRecord(e->ready, s);
  }
  // the build
  if (sl.host_fail == X2C_OK) {
    x2c_status sb;
    if (h->rq.kind == X2C_REQ_FULL) {
      sb = x2c::full_build(sl.ctx, &opt, &h->dmol, &h->dout, nullptr, s, nullptr);
    } else {
      std::vector<x2c_layout> lays;
      std::vector<x2c_mats> mols;
      std::vector<x2c_hout> outs;
      for (auto &rp : batch) {
        x2c_layout L = rp->rq.layout;
        L.kinds = rp->dkinds.empty() ? nullptr : rp->dkinds.data();
        lays.push_back(L);
        mols.push_back(rp->dmol);
        outs.push_back(rp->dout);
      }
      sb = x2c::dlu_build(sl.ctx, &opt, (int)batch.size(), lays.data(), mols.data(), outs.data(),
                          free_atom ? ku.data() : nullptr, s, nullptr);
    }
    st.kernel_launches += sl.ctx->launches;
    if (sb != X2C_OK) fail(sb);
  }
  // results to host buffers
  if (sl.host_fail == X2C_OK) {
    for (auto &rp : batch) {
      Request &r = *rp;
      if (r.rq.memory != X2C_MEM_HOST || !r.rq.out.h[0]) continue;
      for (int q = 0; q < nc; ++q)
        if (cudaMemcpyAsync(r.rq.out.h[q], r.dout.h[q], mat_bytes(r.n), cudaMemcpyDeviceToHost, s) != cudaSuccess) {
          cudaGetLastError();
          fail(X2C_ERR_CUDA);
        }
    }
  }
  // the device status word of this build, then the completion event
  *sl.h_status = 0;
  cudaMemcpyAsync(sl.h_status, sl.ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaMemsetAsync(sl.ctx->d_status, 0, sizeof(int), s);
  cudaEventRecord(sl.ev_done, s);
  if (cudaGetLastError() != cudaSuccess) fail(X2C_ERR_CUDA);
  // workspace growth is held by the slot from now on
  if (sl.ctx->ws_bytes > ws_before) take(sl.ctx->ws_bytes - ws_before);
}

void x2c_server::finish(int si, cudaError_t e) {
  Slot &sl = slots[si];
  x2c_status status = X2C_OK;
  if (e != cudaSuccess) {
    cudaGetLastError();
    status = X2C_ERR_CUDA;
  } else if (sl.host_fail != X2C_OK) {
    status = sl.host_fail;
  } else {
    status = static_cast<x2c_status>(*sl.h_status);
  }
  for (auto &ent : sl.solving) {
    if (status == X2C_OK) {
      ent->state = 1;
    } else {
      ent->state = 2;
      ent->fail_status = status;
      if (ent->in_map) {
        cache.erase(ent->key);
        ent->in_map = false;
      }
    }
  }
  const double t_s = dev_time(sl.ev_start), t_e = dev_time(sl.ev_done);
  for (auto &rp : sl.batch) {
    Request &r = *rp;
    r.status = status;
    for (auto &d : r.deps)
      if (d->state == 2 && r.status == X2C_OK) r.status = static_cast<x2c_status>(d->fail_status);
    r.t_start = t_s;
    r.t_end = t_e;
    if (r.in_slab) {
      cudaFreeAsync(r.in_slab, sl.cur);
      r.in_slab = nullptr;
    }
    give(r.in_bytes);
    if (!r.out_kept || r.status != X2C_OK) {
      if (r.out_dev) cudaFreeAsync(r.out_dev, sl.cur);
      r.out_dev = nullptr;
      give(r.out_bytes);
      r.out_kept = false;
    }
    for (auto &d : r.deps) {
      d->refs--;
      if (!d->in_map && d->refs == 0 && d->U) {
        cudaFreeAsync(d->U, sl.cur);
        cudaEventDestroy(d->ready);
        d->U = nullptr;
        give(d->bytes);
      }
    }
    r.deps.clear();
    r.state = X2C_STATE_DONE;
    running--;
    if (r.status == X2C_OK) {
      st.completed++;
      lat_ms.push_back((r.t_end - r.t_arrival) * 1e3);
      if (st.completed == 1 || r.t_arrival < st.first_arrival) st.first_arrival = r.t_arrival;
      st.last_completion = std::max(st.last_completion, r.t_end);
    } else {
      st.failed++;
    }
  }
  sl.batch.clear();
  sl.solving.clear();
  sl.busy = false;
  cv_done.notify_all();
}

void x2c_server::loop() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  while (true) {
    bool busy = false;
    for (size_t i = 0; i < slots.size(); ++i) {
      if (!slots[i].busy) continue;
      cudaError_t e = cudaEventQuery(slots[i].ev_done);
      if (e == cudaErrorNotReady) {
        busy = true;
        continue;
      }
      // a batch that used transforms another slot was still solving completes only after
      // that slot has reported whether the solve succeeded
      bool waiting = false;
      for (auto &r : slots[i].batch)
        for (auto &d : r->deps)
          if (d->state == 0 && d->solver_slot != (int)i) waiting = true;
      if (waiting) {
        busy = true;
        continue;
      }
      finish((int)i, e);
    }
    if (stop && !busy) break;
    while (!stop && !queue.empty()) {
      int si = -1;
      for (size_t i = 0; i < slots.size(); ++i)
        if (!slots[i].busy) {
          si = (int)i;
          break;
        }
      if (si < 0) break;
      std::vector<ReqPtr> batch;
      if (!plan_batch(slots[si], batch)) break;
      for (auto &r : batch)
        for (auto it = queue.begin(); it != queue.end(); ++it)
          if (*it == r) {
            queue.erase(it);
            break;
          }
      launch(si, batch);
      busy = true;
    }
    if (busy)
      cv_work.wait_for(lk, std::chrono::microseconds(50));
    else
      cv_work.wait_for(lk, std::chrono::milliseconds(5));
  }
}

void x2c_server::fill_result(const Request &r, x2c_result *res) const {
  std::memset(res, 0, sizeof *res);
  res->state = r.state;
  res->status = r.state == X2C_STATE_DONE ? r.status : X2C_OK;
  if (r.state == X2C_STATE_DONE && r.status == X2C_OK && !(r.rq.memory == X2C_MEM_HOST && r.rq.out.h[0]))
    for (int q = 0; q < r.nc; ++q) res->h[q] = r.dout.h[q];
  res->t_arrival = r.t_arrival;
  res->t_submit = r.t_submit;
  res->t_admit = r.t_admit;
  res->t_start = r.t_start;
  res->t_end = r.t_end;
  res->batch_size = r.batch;
  res->cache_hits = r.hits;
  res->cache_misses = r.misses;
  res->slot = r.slot;
}

extern "C" {

x2c_status x2c_server_create(const x2c_server_options *opt, x2c_server **out) {
  if (!opt || !out) return X2C_ERR_ARG;
  *out = nullptr;
  if (opt->reserved0) return X2C_ERR_ARG;
  for (int r : opt->reserved)
    if (r) return X2C_ERR_ARG;
  const int slots = opt->max_inflight ? opt->max_inflight : 4;
  const int batch = opt->max_batch ? opt->max_batch : 16;
  if (slots < 1 || slots > 16 || batch < 1 || batch > 256) return X2C_ERR_ARG;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || opt->device < 0 || opt->device >= count) {
    cudaGetLastError();
    return X2C_ERR_ARG;
  }
  auto *s = new x2c_server();
  s->device = opt->device;
  s->max_batch = batch;
  s->budget = opt->hbm_budget_bytes ? opt->hbm_budget_bytes : kDefaultBudget;
  s->t0 = Clock::now();
  bool ok = cudaSetDevice(s->device) == cudaSuccess;
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = s->device;
  ok = ok && cudaMemPoolCreate(&s->pool, &props) == cudaSuccess;
  uint64_t keep = UINT64_MAX;
  ok = ok && cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep) == cudaSuccess;
  // no hidden cross-slot ordering: memory freed on one slot's stream is not handed to another
  // slot's stream by making that stream wait (the pool grows instead, within the budget)
  int no = 0;
  ok = ok && cudaMemPoolSetAttribute(s->pool, cudaMemPoolReuseAllowInternalDependencies, &no) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&s->misc, cudaStreamNonBlocking) == cudaSuccess;
  int prio_lo = 0, prio_hi = 0;
  ok = ok && cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) == cudaSuccess;
  ok = ok && cudaDeviceGetAttribute(&s->sms_, cudaDevAttrMultiProcessorCount, s->device) == cudaSuccess;
  ok = ok && cudaEventCreate(&s->ev_ref) == cudaSuccess;
  ok = ok && x2c_ctx_create(s->device, &s->planner) == X2C_OK;
  if (s->planner) s->planner->split_ws_cap = kSlotSplitCap;
  for (int i = 0; ok && i < slots; ++i) {
    Slot sl;
    ok = cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) == cudaSuccess &&
         cudaStreamCreateWithPriority(&sl.st_hi, cudaStreamNonBlocking, prio_hi) == cudaSuccess &&
         x2c_ctx_create(s->device, &sl.ctx) == X2C_OK && cudaEventCreate(&sl.ev_start) == cudaSuccess &&
         cudaEventCreate(&sl.ev_done) == cudaSuccess &&
         cudaHostAlloc(reinterpret_cast<void **>(&sl.h_status), sizeof(int), cudaHostAllocDefault) == cudaSuccess;
    if (sl.ctx) {
      sl.ctx->pool = s->pool;
      sl.ctx->split_ws_cap = kSlotSplitCap;
      // no timing runs inside the request loop: they would synchronise a slot stream while
      // the scheduler holds its lock; the slots take the untuned default variant
      sl.ctx->autotune = false;
    }
    s->slots.push_back(sl);
  }
  if (ok) {
    ok = cudaEventRecord(s->ev_ref, s->misc) == cudaSuccess && cudaEventSynchronize(s->ev_ref) == cudaSuccess;
    s->t_ref = s->now();
  }
  if (!ok) {
    cudaGetLastError();
    x2c_server_destroy(s);
    return X2C_ERR_CUDA;
  }
  s->st.budget_bytes = s->budget;
  s->thread = std::thread([s] { s->loop(); });
  *out = s;
  return X2C_OK;
}

x2c_status x2c_server_destroy(x2c_server *s) {
  if (!s) return X2C_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (auto &r : s->queue) {
      r->state = X2C_STATE_DONE;
      r->status = X2C_ERR_CANCELLED;
    }
    s->queue.clear();
  }
  s->cv_work.notify_all();
  if (s->thread.joinable()) s->thread.join();
  s->cv_done.notify_all();
  cudaSetDevice(s->device);
  for (auto &kv : s->requests)
    if (kv.second->out_dev) cudaFreeAsync(kv.second->out_dev, s->misc);
  for (auto &kv : s->cache)
    if (kv.second->U) {
      cudaFreeAsync(kv.second->U, s->misc);
      cudaEventDestroy(kv.second->ready);
    }
  for (auto &sl : s->slots) {
    if (sl.st) cudaStreamSynchronize(sl.st);
    if (sl.st_hi) cudaStreamSynchronize(sl.st_hi);
    if (sl.ctx && sl.ctx->ws) {
      cudaFreeAsync(sl.ctx->ws, sl.st ? sl.st : s->misc);
      sl.ctx->ws = nullptr;
      sl.ctx->ws_bytes = 0;
    }
  }
  cudaDeviceSynchronize();
  for (auto &sl : s->slots) {
    if (sl.ctx) x2c_ctx_destroy(sl.ctx);
    if (sl.ev_start) cudaEventDestroy(sl.ev_start);
    if (sl.ev_done) cudaEventDestroy(sl.ev_done);
    if (sl.h_status) cudaFreeHost(sl.h_status);
    if (sl.st) cudaStreamDestroy(sl.st);
    if (sl.st_hi) cudaStreamDestroy(sl.st_hi);
  }
  if (s->planner) x2c_ctx_destroy(s->planner);
  if (s->ev_ref) cudaEventDestroy(s->ev_ref);
  if (s->misc) cudaStreamDestroy(s->misc);
  if (s->pool) cudaMemPoolDestroy(s->pool);
  cudaGetLastError();
  delete s;
  return X2C_OK;
}

x2c_status x2c_server_now(x2c_server *s, double *t) {
  if (!s || !t) return X2C_ERR_ARG;
  *t = s->now();
  return X2C_OK;
}

x2c_status x2c_server_submit(x2c_server *s, const x2c_request *req, uint64_t *ticket) {
  if (!s || !req || !ticket) return X2C_ERR_ARG;
  auto r = std::make_shared<Request>();
  x2c_status ps = prepare(s, req, *r);
  if (ps != X2C_OK) return ps;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->stop) return X2C_ERR_CANCELLED;
  // a request that could never fit: its own bytes, its kinds' transforms and the workspace
  // of building it alone (with every slot's workspace grown to that size)
  {
    Slot probe;
    x2c_ctx empty;
    probe.ctx = &empty;
    std::vector<ReqPtr> one{r};
    size_t ws_need = 0;
    const size_t extra = s->extra_bytes(probe, one, &ws_need);
    if (r->own_bytes() + extra > s->budget) return X2C_ERR_ADMISSION;
  }
  r->ticket = s->next_ticket++;
  r->t_submit = s->now();
  r->t_arrival = req->t_arrival >= 0 ? req->t_arrival : r->t_submit;
  s->queue.push_back(r);
  s->requests.emplace(r->ticket, r);
  s->st.submitted++;
  *ticket = r->ticket;
  lk.unlock();
  s->cv_work.notify_all();
  return X2C_OK;
}

x2c_status x2c_server_poll(x2c_server *s, uint64_t ticket, x2c_result *res) {
  if (!s || !res) return X2C_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->requests.find(ticket);
  if (it == s->requests.end()) return X2C_ERR_NOT_FOUND;
  s->fill_result(*it->second, res);
  return X2C_OK;
}

x2c_status x2c_server_wait(x2c_server *s, uint64_t ticket, uint32_t timeout_ms, x2c_result *res) {
  if (!s) return X2C_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->requests.find(ticket);
  if (it == s->requests.end()) return X2C_ERR_NOT_FOUND;
  ReqPtr r = it->second;
  const bool done = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                        [&] { return r->state == X2C_STATE_DONE; });
  if (res) s->fill_result(*r, res);
  return done ? X2C_OK : X2C_ERR_TIMEOUT;
}

x2c_status x2c_server_cancel(x2c_server *s, uint64_t ticket) {
  if (!s) return X2C_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->requests.find(ticket);
  if (it == s->requests.end()) return X2C_ERR_NOT_FOUND;
  ReqPtr r = it->second;
  if (r->state != X2C_STATE_QUEUED) return X2C_ERR_ARG;
  for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
    if (*q == r) {
      s->queue.erase(q);
      break;
    }
  r->state = X2C_STATE_DONE;
  r->status = X2C_ERR_CANCELLED;
  s->st.cancelled++;
  s->cv_done.notify_all();
  s->cv_work.notify_all();
  return X2C_OK;
}

x2c_status x2c_server_release(x2c_server *s, uint64_t ticket) {
  if (!s) return X2C_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->requests.find(ticket);
  if (it == s->requests.end()) return X2C_ERR_NOT_FOUND;
  ReqPtr r = it->second;
  if (r->state != X2C_STATE_DONE) return X2C_ERR_ARG;
  if (r->out_dev) {
    cudaSetDevice(s->device);
    cudaFreeAsync(r->out_dev, s->misc);
    r->out_dev = nullptr;
    s->give(r->out_bytes);
  }
  s->requests.erase(it);
  s->cv_work.notify_all();
  return X2C_OK;
}

x2c_status x2c_server_get_stats(x2c_server *s, x2c_server_stats *out) {
  if (!s || !out) return X2C_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  x2c_server_stats r = s->st;
  r.queued = (int64_t)s->queue.size();
  r.running = s->running;
  r.cache_entries = (int64_t)s->cache.size();
  r.bytes_in_use = s->in_use;
  r.peak_bytes = s->peak;
  r.budget_bytes = s->budget;
  r.latency_p50_ms = x2c::serve::percentile(s->lat_ms, 50.0);
  r.latency_p99_ms = x2c::serve::percentile(s->lat_ms, 99.0);
  double sum = 0, mx = 0;
  for (double v : s->lat_ms) {
    sum += v;
    mx = std::max(mx, v);
  }
  r.latency_mean_ms = s->lat_ms.empty() ? 0.0 : sum / s->lat_ms.size();
  r.latency_max_ms = mx;
  const double span = r.last_completion - r.first_arrival;
  r.builds_per_s = (r.completed > 0 && span > 0) ? r.completed / span : 0.0;
  *out = r;
  return X2C_OK;
}

x2c_status x2c_server_reset_stats(x2c_server *s) {
  if (!s) return X2C_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  const int64_t keep_entries = s->st.cache_entries;
  s->st = x2c_server_stats{};
  s->st.cache_entries = keep_entries;
  s->st.budget_bytes = s->budget;
  s->lat_ms.clear();
  s->peak = s->in_use;
  return X2C_OK;
}

}  // extern "C"
