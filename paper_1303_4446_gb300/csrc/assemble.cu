// Pair-block assembly of the decoupled Hamiltonian (Eq. 8) for block-diagonal U^L, U^S
// (DLU, Eq. 42), FP64 path.
//
// For a pair of atoms (A, B), A <= B, with Mid_AB = [[V_AB, T_AB], [T_AB, W'_AB]],
// W' = W/4c^2 - T, and the stacked transforms F_B = [U^L_B; U^S_B] (parts side by side):
//   stage 1:  R_AB = Mid_AB F_B                  (2 nA x nc nB)
//             (+ the spin-orbit part i sum_k sigma_k Wk_AB / 4c^2 times U^S_B, as a
//              quaternion product, on pairs whose Wk block is non-zero)
//   stage 2:  h_AB = [U^L_A+ U^S_A+] R_AB        (quaternion adjoint product, nc nA x nB)
// h_BA = h_AB+ is written by mirroring (part 0 transposed, parts 1-3 negated transposes).
// Credited work per pair: scalar 2 (4 nA nB^2 + 2 nA^2 nB); two-component
// 2 (16 nA nB^2 + 32 nA^2 nB) plus 24 nA nB^2 for the spin-orbit middle term.
#include <algorithm>

#include "common.cuh"
#include "gemm_f64.cuh"

namespace x2c {
namespace {

struct Stage1Dims {
  const PairDesc *p;
  int nc;
  __device__ int M(int b) const { return 2 * p[b].nA; }
  __device__ int N(int b) const { return nc * p[b].nB; }
  __device__ int K(int b) const { return 2 * p[b].nB; }
  __device__ int K0(int) const { return 0; }
};

// A operand of stage 1: Mid_AB gathered from the molecular V, T, W0.
struct MidOp {
  const PairDesc *p;
  const MolDesc *mols;
  double inv4c2;
  static constexpr bool k_contig = true;
  __device__ __forceinline__ double operator()(int b, int r, int k) const {
    const PairDesc &P = p[b];
    const MolDesc &m = mols[P.mol];
    const int Y = r >= P.nA, X = k >= P.nB;
    const int i = r - Y * P.nA, kk = k - X * P.nB;
    const int64_t o = (int64_t)(P.offA + i) * m.ld + (P.offB + kk);
    if (!Y && !X) return m.V[o];
    if (Y != X) return m.T[o];
    return m.W0[o] * inv4c2 - m.T[o];
  }
};

// B operand of stage 1: F_B[(X,kk), (q,j)] = U^X_{B,q}[kk][j].
struct FOp {
  const PairDesc *p;
  UTable ut;
  int nc;
  static constexpr bool n_contig = true;
  __device__ __forceinline__ double operator()(int b, int k, int col) const {
    const PairDesc &P = p[b];
    const int n = P.nB;
    const int X = k >= n;
    const int kk = k - X * n;
    const int q = col / n, j = col - q * n;
    const double *U = X ? ut.US[P.uB] : ut.UL[P.uB];
    return U[((int64_t)q * n + kk) * n + j];
  }
};

struct StoreR {
  const PairDesc *p;
  double *R;
  int nc;
  __device__ __forceinline__ void operator()(int b, int r, int c, double acc) const {
    const PairDesc &P = p[b];
    R[P.r_off + (int64_t)r * (nc * P.nB) + c] = acc;
  }
};

struct SoDims {
  const PairDesc *p;
  __device__ int M(int b) const { return 4 * p[b].nA; }
  __device__ int N(int b) const { return p[b].nB; }
  __device__ int K(int b) const { return 4 * p[b].nB; }
  __device__ int K0(int) const { return 0; }
};

// A operand: Lq(Wso) with Wso = (0, Wx, Wy, Wz)_AB / 4c^2.
struct SoLeftOp {
  const PairDesc *p;
  const MolDesc *mols;
  double inv4c2;
  static constexpr bool k_contig = true;
  __device__ __forceinline__ double operator()(int b, int r, int k) const {
    const PairDesc &P = p[b];
    const int pr = r / P.nA, i = r - pr * P.nA;
    const int pq = k / P.nB, kk = k - pq * P.nB;
    const int comp = pr ^ pq;
    if (comp == 0) return 0.0;
    const MolDesc &m = mols[P.mol];
    return quat_sign(pr, pq) * inv4c2 * m.W[comp - 1][(int64_t)(P.offA + i) * m.ld + (P.offB + kk)];
  }
};

// B operand: stacked parts of U^S_B, (4 nB) x nB.
struct UStackOp {
  const PairDesc *p;
  UTable ut;
  static constexpr bool n_contig = true;
  __device__ __forceinline__ double operator()(int b, int k, int j) const {
    const PairDesc &P = p[b];
    return ut.US[P.uB][(int64_t)k * P.nB + j];
  }
};

// Accumulate the quaternion product's part q, row i into R rows of the S block.
struct AccumulateRS {
  const PairDesc *p;
  double *R;
  __device__ __forceinline__ void operator()(int b, int r, int j, double acc) const {
    const PairDesc &P = p[b];
    const int q = r / P.nA, i = r - q * P.nA;
    R[P.r_off + (int64_t)(P.nA + i) * (4 * P.nB) + q * P.nB + j] += acc;
  }
};

struct Stage2Dims {
  const PairDesc *p;
  int nc;
  __device__ int M(int b) const { return nc * p[b].nA; }
  __device__ int N(int b) const { return p[b].nB; }
  __device__ int K(int b) const { return 2 * nc * p[b].nA; }
  __device__ int K0(int) const { return 0; }
};

// A operand of stage 2: G_A = [Lq(U^L_A+) Lq(U^S_A+)], element ((l,i), (X,q,kk)).
struct GOp {
  const PairDesc *p;
  UTable ut;
  int nc;
  static constexpr bool k_contig = false;
  __device__ __forceinline__ double operator()(int b, int r, int k) const {
    const PairDesc &P = p[b];
    const int n = P.nA;
    const int l = r / n, i = r - l * n;
    const int X = k / (nc * n);
    const int rem = k - X * nc * n;
    const int q = rem / n, kk = rem - q * n;
    const int comp = l ^ q;
    const double *U = X ? ut.US[P.uA] : ut.UL[P.uA];
    return quat_sign_adj(l, q) * U[((int64_t)comp * n + kk) * n + i];
  }
};

// B operand of stage 2: R''[(X,q,kk), j] = R[(X,kk), (q,j)].
struct RppOp {
  const PairDesc *p;
  const double *R;
  int nc;
  static constexpr bool n_contig = true;
  __device__ __forceinline__ double operator()(int b, int k, int j) const {
    const PairDesc &P = p[b];
    const int n = P.nA;
    const int X = k / (nc * n);
    const int rem = k - X * nc * n;
    const int q = rem / n, kk = rem - q * n;
    return R[P.r_off + (int64_t)(X * n + kk) * (nc * P.nB) + q * P.nB + j];
  }
};

struct StoreH {
  const PairDesc *p;
  const MolDesc *mols;
  __device__ __forceinline__ void operator()(int b, int r, int j, double acc) const {
    const PairDesc &P = p[b];
    const MolDesc &m = mols[P.mol];
    const int l = r / P.nA, i = r - l * P.nA;
    double *h = m.h[l];
    h[(int64_t)(P.offA + i) * m.ld + (P.offB + j)] = acc;
    if (!P.diag) h[(int64_t)(P.offB + j) * m.ld + (P.offA + i)] = (l == 0) ? acc : -acc;
  }
};

using TileStage1 = TileCfg<96, 64, 16, 6, 4>;
using TileStage2q = TileCfg<96, 48, 16, 6, 3>;
using TileStage2s = TileCfg<48, 48, 16, 3, 3>;

int64_t r_doubles(const PairDesc &P, int nc) { return (int64_t)2 * P.nA * nc * P.nB; }

constexpr int64_t kRChunkDoubles = (int64_t)1 << 27;  // 1 GiB of stage-1 intermediates

}  // namespace

size_t assemble_workspace_bytes(const std::vector<PairDesc> &pairs, int nc, int max_n, int precision,
                                size_t split_cap) {
  if (precision == X2C_PREC_SPLIT_BF16) {
    // split path: per pair about 2nA*KP*S*2 + nc nB*2nA*8 + nc nB*KP*S*2 bytes (S <= 6,
    // KP <= 128) plus per-kind operands; chunked inside.  The request is capped at split_cap
    // (24 GiB by default: a build of Ag309's 47895 two-component pairs, about 17 GB, runs in
    // one chunk, with fewer launches and kernel tails; larger ones in chunks of that size).
    const size_t kp = 128, S = 6;
    size_t need = 64u << 20;
    for (const auto &P : pairs)
      need += (size_t)2 * P.nA * kp * S * 2 + (size_t)nc * P.nB * 2 * P.nA * 8 + (size_t)nc * P.nB * kp * S * 2 + 4096;
    return std::min<size_t>(need, split_cap);
  }
  int64_t total = 0, chunk_max = 0, cur = 0;
  for (const auto &P : pairs) {
    const int64_t r = r_doubles(P, nc);
    total += r;
    if (cur + r > kRChunkDoubles && cur > 0) {
      chunk_max = std::max(chunk_max, cur);
      cur = 0;
    }
    cur += r;
  }
  chunk_max = std::max(chunk_max, cur);
  (void)total;
  (void)max_n;
  return arena_doubles(chunk_max) + arena_doubles(pairs.size() * sizeof(PairDesc) / sizeof(double) + 1) + 4096;
}

x2c_status assemble_pairs_fp64(x2c_ctx *ctx, cudaStream_t st, double c, int nc, int so_all_pairs,
                               const std::vector<PairDesc> &pairs_in, const MolDesc *d_mols,
                               UTable ut, int max_n, Arena &ar) {
  if (pairs_in.empty()) return X2C_OK;
  const double inv4c2 = 1.0 / (4.0 * c * c);
  // Split into chunks whose intermediates fit the R buffer; offsets relative to the chunk.
  std::vector<PairDesc> pairs = pairs_in;
  std::vector<std::pair<size_t, size_t>> chunks;
  {
    int64_t cur = 0;
    size_t start = 0;
    for (size_t i = 0; i < pairs.size(); ++i) {
      const int64_t r = r_doubles(pairs[i], nc);
      if (cur + r > kRChunkDoubles && cur > 0) {
        chunks.push_back({start, i});
        start = i;
        cur = 0;
      }
      pairs[i].r_off = cur;
      cur += r;
    }
    chunks.push_back({start, pairs.size()});
  }
  int64_t rmax = 0;
  for (auto &ch : chunks) {
    int64_t s = 0;
    for (size_t i = ch.first; i < ch.second; ++i) s += r_doubles(pairs[i], nc);
    rmax = std::max(rmax, s);
  }
  PairDesc *d_pairs = reinterpret_cast<PairDesc *>(ar.take_bytes(pairs.size() * sizeof(PairDesc)));
  double *R = ar.take(rmax);
  if (!d_pairs || !R) return X2C_ERR_NOMEM;
  X2C_TRY(upload(ctx, st, d_pairs, pairs.data(), pairs.size() * sizeof(PairDesc)));
  // Pairs needing the spin-orbit middle term: all pairs, or only A == B.
  std::vector<PairDesc> so_pairs;
  for (auto &ch : chunks) {
    const int np = (int)(ch.second - ch.first);
    const PairDesc *dp = d_pairs + ch.first;
    X2C_TRY((gemm_f64<TileStage1>(ctx, st, np, 2 * max_n, nc * max_n, MidOp{dp, d_mols, inv4c2},
                                  FOp{dp, ut, nc}, StoreR{dp, R, nc}, Stage1Dims{dp, nc}, "dlu_stage1")));
    if (nc == 4) {
      if (so_all_pairs) {
        X2C_TRY((gemm_f64<TileStage2q>(ctx, st, np, 4 * max_n, max_n, SoLeftOp{dp, d_mols, inv4c2},
                                       UStackOp{dp, ut}, AccumulateRS{dp, R}, SoDims{dp}, "dlu_spin_orbit")));
      } else {
        // same-atom blocks only: run the product over the diagonal pairs of the chunk, which
        // are gathered into a separate descriptor list at the end of the pair buffer
        std::vector<PairDesc> diag;
        for (size_t i = ch.first; i < ch.second; ++i)
          if (pairs[i].diag) diag.push_back(pairs[i]);
        if (!diag.empty()) {
          PairDesc *dd = reinterpret_cast<PairDesc *>(ar.take_bytes(diag.size() * sizeof(PairDesc)));
          if (!dd) return X2C_ERR_NOMEM;
          X2C_TRY(upload(ctx, st, dd, diag.data(), diag.size() * sizeof(PairDesc)));
          X2C_TRY((gemm_f64<TileStage2q>(ctx, st, (int)diag.size(), 4 * max_n, max_n,
                                         SoLeftOp{dd, d_mols, inv4c2}, UStackOp{dd, ut},
                                         AccumulateRS{dd, R}, SoDims{dd}, "dlu_spin_orbit")));
        }
      }
    }
    if (nc == 4) {
      X2C_TRY((gemm_f64<TileStage2q>(ctx, st, np, nc * max_n, max_n, GOp{dp, ut, nc}, RppOp{dp, R, nc},
                                     StoreH{dp, d_mols}, Stage2Dims{dp, nc}, "dlu_stage2")));
    } else {
      X2C_TRY((gemm_f64<TileStage2s>(ctx, st, np, nc * max_n, max_n, GOp{dp, ut, nc}, RppOp{dp, R, nc},
                                     StoreH{dp, d_mols}, Stage2Dims{dp, nc}, "dlu_stage2")));
    }
  }
  return X2C_OK;
}

// DLH (Sec. III.A): every atom-other-atom block of h is the non-relativistic T + V; the
// spin parts of those blocks are zero.  One CTA per row i (grid-strided): the atom of i by
// bisection of the offsets, then the row streamed outside [off[a], off[a+1]).
__global__ void nonrel_offdiag_kernel(const MolDesc *mols, int mol, const int32_t *off, int L, int nc) {
  const MolDesc &m = mols[mol];
  const int N = off[L];
  for (int i = blockIdx.x; i < N; i += gridDim.x) {
    int lo = 0, hi = L;  // off[lo] <= i < off[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (off[mid] <= i) lo = mid;
      else hi = mid;
    }
    const int a0 = off[lo], a1 = off[lo + 1];
    const int64_t row = static_cast<int64_t>(i) * m.ld;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
      if (j >= a0 && j < a1) continue;
      m.h[0][row + j] = m.T[row + j] + m.V[row + j];
      for (int q = 1; q < nc; ++q) m.h[q][row + j] = 0.0;
    }
  }
}

x2c_status fill_nonrel_offdiag(x2c_ctx *ctx, cudaStream_t st, const MolDesc *d_mols, int mol, const int32_t *d_off,
                               int L, int N, int nc) {
  if (L < 2) return X2C_OK;
  const int blocks = std::min(N, 152 * 8);
  tbegin(ctx, st);
  nonrel_offdiag_kernel<<<blocks, 256, 0, st>>>(d_mols, mol, d_off, L, nc);
  return launched(ctx, "dlh_offdiag", st, 0);
}

}  // namespace x2c
