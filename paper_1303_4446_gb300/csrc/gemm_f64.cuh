// Batched FP64 GEMM on the FMA pipe, C(b) = f(A(b) B(b)), with operand access through
// functors so that transposes, quaternion left-multiplication matrices and gathers from
// molecular pair blocks are read in place instead of being materialised.
//
// On GB300 the FP64 FMA rate (1.19 TFLOP/s measured) is above the FP64 tensor-core
// (mma.sync f64) rate (1.05 TFLOP/s measured), so the tile is register-blocked for DFMA:
// each thread owns TM x TN accumulators with rows ty + i*NTY and columns tx + j*NTX
// (interleaved, so shared-memory reads are broadcasts or conflict-free and the epilogue
// stores are coalesced).
#pragma once

#include <algorithm>

#include "common.cuh"

namespace x2c {

template <int BM_, int BN_, int KC_, int TM_, int TN_>
struct TileCfg {
  static constexpr int BM = BM_, BN = BN_, KC = KC_, TM = TM_, TN = TN_;
  static constexpr int NTY = BM / TM, NTX = BN / TN, NT = NTX * NTY;
  static_assert(BM % TM == 0 && BN % TN == 0, "tile");
};

// Shapes: M(b), N(b), K(b) per batch entry; the K loop runs over [K0(b), K(b)).
// An optional gate: with gate set, a launch for iteration `step` does nothing (M = 0, every
// CTA returns at once) when *gate <= step — iterations the device has found unnecessary.
__device__ __forceinline__ bool gated(const int *gate, int step) { return gate && *gate <= step; }

struct UniformDims {
  int m, n, k;
  const int *gate = nullptr;
  int step = 0;
  __device__ int M(int) const { return gated(gate, step) ? 0 : m; }
  __device__ int N(int) const { return n; }
  __device__ int K(int) const { return k; }
  __device__ int K0(int) const { return 0; }
};

// Shape of a product whose result is Hermitian in the quaternion sense (stacked parts of
// `part` rows; part 0 symmetric, parts 1-3 antisymmetric): tiles strictly below the diagonal
// of their part are skipped and the epilogue writes the mirror.
struct HermDims {
  int m, n, k, part;
  const int *gate = nullptr;
  int step = 0;
  __device__ int M(int) const { return gated(gate, step) ? 0 : m; }
  __device__ int N(int) const { return n; }
  __device__ int K(int) const { return k; }
  __device__ int K0(int) const { return 0; }
};
template <class Dims>
__device__ __forceinline__ bool tile_skip(const Dims &, int, int, int, int) { return false; }
__device__ __forceinline__ bool tile_skip(const HermDims &d, int m0, int n0, int BM, int BN) {
  const int p = m0 / d.part;
  if (m0 + BM - 1 >= (p + 1) * d.part) return false;  // the tile spans two parts
  return m0 - p * d.part > n0 + BN - 1;
}

// A plain strided matrix operand: element (r, k) (or (k, n) for B) of batch b.
//   trans = false: p[b*bs + r*ld + k];  trans = true: p[b*bs + k*ld + r]
template <bool TRANS>
struct Mat {
  const double *p;
  int64_t ld, bs;
  double scale;
  static constexpr bool k_contig = !TRANS;  // as A operand: is k the contiguous index?
  static constexpr bool n_contig = !TRANS;  // as B operand (k, n): is n contiguous?
  __device__ __forceinline__ double operator()(int b, int r, int k) const {
    return scale * (TRANS ? p[b * bs + (int64_t)k * ld + r] : p[b * bs + (int64_t)r * ld + k]);
  }
};

// Quaternion left-multiplication matrix Lq(A) (or Lq(A+) when ADJ) of a batch of
// quaternion matrices with parts of size m x m stored part-major (part q of batch b at
// p + b*bs + q*ps).  nc = 1 degenerates to A (or A^T).
template <bool ADJ>
struct QuatLeft {
  const double *p;
  int64_t ld, bs, ps;
  int m, nc;
  double scale;
  static constexpr bool k_contig = !ADJ;
  __device__ __forceinline__ double operator()(int b, int r, int k) const {
    int pr = 0, i = r, pq = 0, kk = k;
    if (nc == 4) {
      pr = r / m; i = r - pr * m;
      pq = k / m; kk = k - pq * m;
    }
    const int comp = pr ^ pq;
    const double *base = p + b * bs + comp * ps;
    if (!ADJ) return scale * quat_sign(pr, pq) * base[(int64_t)i * ld + kk];
    return scale * quat_sign_adj(pr, pq) * base[(int64_t)kk * ld + i];
  }
};

// Epilogue writing alpha*acc + beta*Cin into a strided output (Cin may alias nothing).
struct StoreAxpby {
  double *out;
  const double *cin;
  int64_t ld, bs;
  double alpha, beta;
  __device__ __forceinline__ void operator()(int b, int r, int c, double acc) const {
    const int64_t o = b * bs + (int64_t)r * ld + c;
    double v = alpha * acc;
    if (cin) v += beta * cin[o];
    out[o] = v;
  }
};

// Epilogue: out = alpha*acc + diag_shift*delta(r mod m, c) (identity part of a stacked
// quaternion lives only in rows of part 0, i.e. r < m).
struct StoreShiftIdentity {
  double *out;
  int64_t ld, bs;
  int m;
  double alpha, shift;
  __device__ __forceinline__ void operator()(int b, int r, int c, double acc) const {
    double v = alpha * acc;
    if (r == c && r < m) v += shift;
    out[b * bs + (int64_t)r * ld + c] = v;
  }
};

// Hermitian-product epilogues: write element (i, c) of part p for i <= c and its mirror
// (c, i) = +-value (part 0 symmetric, parts 1-3 antisymmetric); i > c is left to the mirror.
struct StoreAxpbyHerm {
  double *out;
  const double *cin;
  int64_t ld, bs;
  double alpha, beta;
  int m;
  __device__ __forceinline__ void operator()(int b, int r, int c, double acc) const {
    const int p = r / m, i = r - p * m;
    if (i > c) return;
    const int64_t o = b * bs + (int64_t)r * ld + c;
    double v = alpha * acc;
    if (cin) v += beta * cin[o];
    out[o] = v;
    if (i < c) out[b * bs + (int64_t)(p * m + c) * ld + i] = p == 0 ? v : -v;
  }
};
struct StoreShiftIdentityHerm {
  double *out;
  int64_t ld, bs;
  int m;
  double alpha, shift;
  __device__ __forceinline__ void operator()(int b, int r, int c, double acc) const {
    const int p = r / m, i = r - p * m;
    if (i > c) return;
    double v = alpha * acc;
    if (r == c && r < m) v += shift;
    out[b * bs + (int64_t)r * ld + c] = v;
    if (i < c) out[b * bs + (int64_t)(p * m + c) * ld + i] = p == 0 ? v : -v;
  }
};

// Newton-Schulz sign step with a per-problem coefficient a = a_k[b * stride] (device):
// out = (3a/2) Z - (a^3/2) acc, acc = Z Y.  The Herm variant writes i <= c and mirrors.
struct StoreSignStep {
  double *out;
  const double *z;
  int64_t ld, bs;
  const double *a;
  int stride;
  __device__ __forceinline__ void operator()(int b, int r, int c, double acc) const {
    const double av = a[b * stride];
    const int64_t o = b * bs + (int64_t)r * ld + c;
    double v = (-0.5 * av * av * av) * acc;
    v += (1.5 * av) * z[o];
    out[o] = v;
  }
};
struct StoreSignStepHerm {
  double *out;
  const double *z;
  int64_t ld, bs;
  const double *a;
  int stride, m;
  __device__ __forceinline__ void operator()(int b, int r, int c, double acc) const {
    const int p = r / m, i = r - p * m;
    if (i > c) return;
    const double av = a[b * stride];
    const int64_t o = b * bs + (int64_t)r * ld + c;
    double v = (-0.5 * av * av * av) * acc;
    v += (1.5 * av) * z[o];
    out[o] = v;
    if (i < c) out[b * bs + (int64_t)(p * m + c) * ld + i] = p == 0 ? v : -v;
  }
};

template <class Cfg, class AOp, class BOp, class COp, class Dims>
__global__ void __launch_bounds__(Cfg::NT) gemm_f64_kernel(AOp A, BOp B, COp C, Dims D, int tiles_n) {
  constexpr int BM = Cfg::BM, BN = Cfg::BN, KC = Cfg::KC, TM = Cfg::TM, TN = Cfg::TN;
  constexpr int NTX = Cfg::NTX, NTY = Cfg::NTY, NT = Cfg::NT;
  const int b = blockIdx.x;
  const int M = D.M(b), N = D.N(b), K = D.K(b);
  const int tile = blockIdx.y + blockIdx.z * gridDim.y;  // grid.z only when tiles > 65535
  const int tm = tile / tiles_n, tn = tile - (tile / tiles_n) * tiles_n;
  const int m0 = tm * BM, n0 = tn * BN;
  if (m0 >= M || n0 >= N || tile_skip(D, m0, n0, BM, BN)) return;

  __shared__ double As[KC][BM + 1];
  __shared__ double Bs[KC][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % NTX, ty = tid / NTX;
  double acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;

  for (int k0 = D.K0(b); k0 < K; k0 += KC) {
    for (int idx = tid; idx < BM * KC; idx += NT) {
      int r, kk;
      if (AOp::k_contig) { r = idx / KC; kk = idx - r * KC; }
      else { kk = idx / BM; r = idx - kk * BM; }
      const int gm = m0 + r, gk = k0 + kk;
      As[kk][r] = (gm < M && gk < K) ? A(b, gm, gk) : 0.0;
    }
    for (int idx = tid; idx < BN * KC; idx += NT) {
      int c, kk;
      if (BOp::n_contig) { kk = idx / BN; c = idx - kk * BN; }
      else { c = idx / KC; kk = idx - c * KC; }
      const int gn = n0 + c, gk = k0 + kk;
      Bs[kk][c] = (gn < N && gk < K) ? B(b, gk, gn) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      double a[TM], bv[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + i * NTY];
#pragma unroll
      for (int j = 0; j < TN; ++j) bv[j] = Bs[kk][tx + j * NTX];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gm = m0 + ty + i * NTY;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gn = n0 + tx + j * NTX;
      if (gn < N) C(b, gm, gn, acc[i][j]);
    }
  }
}

// Algorithmic flops of one launch, where the shape is uniform (0 otherwise).
template <class Dims>
inline double dims_flops(const Dims &, int) { return 0.0; }
// A gated launch reports no flops: the device decides whether it runs.
inline double dims_flops(const UniformDims &d, int batch) { return d.gate ? 0.0 : 2.0 * d.m * d.n * d.k * batch; }
// Hermitian products: the upper triangle of every part (about half of the full product).
inline double dims_flops(const HermDims &d, int batch) {
  return d.gate ? 0.0 : (double)d.m / d.part * d.part * (d.part + 1.0) * d.k * batch;
}
struct SplitDims;
inline double dims_flops(const SplitDims &d, int);

// Launch helper: grid.x = batch entries, grid.y (and z) = tiles of the largest M x N.
template <class Cfg, class AOp, class BOp, class COp, class Dims>
inline x2c_status gemm_f64(x2c_ctx *ctx, cudaStream_t st, int batch, int max_m, int max_n,
                           const AOp &A, const BOp &B, const COp &C, const Dims &D,
                           const char *name = "gemm_f64") {
  if (batch <= 0 || max_m <= 0 || max_n <= 0) return X2C_OK;
  const int tiles_m = (max_m + Cfg::BM - 1) / Cfg::BM;
  const int tiles_n = (max_n + Cfg::BN - 1) / Cfg::BN;
  const int tiles = tiles_m * tiles_n;
  dim3 grid(batch, std::min(tiles, 65535), (tiles + 65534) / 65535);
  tbegin(ctx, st);
  gemm_f64_kernel<Cfg><<<grid, Cfg::NT, 0, st>>>(A, B, C, D, tiles_n);
  return launched(ctx, name, st, dims_flops(D, batch));
}

// ---- split-K: batch entry b' = split * batch + b computes the K range of its split into a
// partial buffer; a second kernel sums the splits in a fixed order (deterministic) and
// applies the epilogue.
template <class Op>
struct SplitOp {
  Op op;
  int batch;
  static constexpr bool k_contig = Op::k_contig;
  __device__ __forceinline__ double operator()(int b, int r, int k) const { return op(b % batch, r, k); }
};
template <class Op>
struct SplitOpB {
  Op op;
  int batch;
  static constexpr bool n_contig = Op::n_contig;
  __device__ __forceinline__ double operator()(int b, int k, int n) const { return op(b % batch, k, n); }
};
struct SplitDims {
  int m, n, k, kc, batch;
  const int *gate = nullptr;
  int step = 0;
  __device__ int M(int) const { return gated(gate, step) ? 0 : m; }
  __device__ int N(int) const { return n; }
  __device__ int K0(int b) const { return (b / batch) * kc; }
  __device__ int K(int b) const { return min(k, (b / batch + 1) * kc); }
};
inline double dims_flops(const SplitDims &d, int) { return d.gate ? 0.0 : 2.0 * d.m * d.n * d.k * d.batch; }
struct PartialStore {
  double *part;
  int64_t mn;
  int n;
  __device__ __forceinline__ void operator()(int b, int r, int c, double acc) const {
    part[b * mn + static_cast<int64_t>(r) * n + c] = acc;
  }
};
template <class COp>
__global__ void splitk_reduce_kernel(const double *part, int splits, int batch, int m, int n, COp C,
                                     const int *gate, int step) {
  if (gated(gate, step)) return;
  const int64_t mn = static_cast<int64_t>(m) * n;
  const int64_t total = mn * batch;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int b = static_cast<int>(idx / mn);
    const int64_t rc = idx - b * mn;
    double s = 0.0;
    for (int sp = 0; sp < splits; ++sp) s += part[(static_cast<int64_t>(sp) * batch + b) * mn + rc];
    C(b, static_cast<int>(rc / n), static_cast<int>(rc % n), s);
  }
}

// Uniform-shape batched GEMM with split-K so that small products still fill the GPU.
// `part` must hold splits * batch * m * n doubles (splits chosen by the caller).
template <class Cfg, class AOp, class BOp, class COp>
inline x2c_status gemm_f64_splitk(x2c_ctx *ctx, cudaStream_t st, int batch, int m, int n, int k, int splits,
                                  double *part, const AOp &A, const BOp &B, const COp &C, const char *name,
                                  const int *gate = nullptr, int step = 0) {
  if (splits <= 1) return gemm_f64<Cfg>(ctx, st, batch, m, n, A, B, C, UniformDims{m, n, k, gate, step}, name);
  const int kc = ((k + splits - 1) / splits + Cfg::KC - 1) / Cfg::KC * Cfg::KC;
  splits = (k + kc - 1) / kc;
  X2C_TRY((gemm_f64<Cfg>(ctx, st, batch * splits, m, n, SplitOp<AOp>{A, batch}, SplitOpB<BOp>{B, batch},
                         PartialStore{part, static_cast<int64_t>(m) * n, n},
                         SplitDims{m, n, k, kc, batch, gate, step}, name)));
  const int64_t total = static_cast<int64_t>(m) * n * batch;
  const int blocks = static_cast<int>(std::min<int64_t>((total + 255) / 256, 152 * 8));
  tbegin(ctx, st);
  splitk_reduce_kernel<<<blocks, 256, 0, st>>>(part, splits, batch, m, n, C, gate, step);
  return launched(ctx, "splitk_reduce", st);
}

// Split count that gives about two waves of CTAs on 152 SMs, with at least `min_chunks`
// K steps per split.
template <class Cfg>
inline int choose_splits(int batch, int m, int n, int k, int min_chunks = 2) {
  const int tiles = ((m + Cfg::BM - 1) / Cfg::BM) * ((n + Cfg::BN - 1) / Cfg::BN) * batch;
  int s = (2 * 152 + tiles - 1) / tiles;
  s = std::max(1, std::min(s, k / (min_chunks * Cfg::KC)));
  return s;
}

// Default tile for the dense (square-ish) products of the decoupling solve.
using TileSolve = TileCfg<64, 64, 16, 4, 4>;
using TileSmall = TileCfg<32, 32, 16, 2, 2>;
// Tiny products (the decoupling solve of one small atom kind): one output per thread, so
// that a 60 x 60 product still spreads over dozens of CTAs.
using TileTiny = TileCfg<16, 16, 16, 1, 1>;
// Large dense products (full X2C of a whole molecule): 96 x 64 tiles, 24 accumulators.
using TileLarge = TileCfg<96, 64, 16, 6, 4>;

}  // namespace x2c
