// Batched X2C decoupling transforms U^L, U^S (Sec. II.A) by a GEMM-only route.
//
// The paper diagonalises T K = S K t (Eq. 11), builds the orthonormal 4c matrix H^p
// (Eq. 14), diagonalises it (Eq. 18), forms X' = C_S' C_L'^-1 (Eq. 19), R' =
// (1 + X'+ X')^-1/2 (Eq. 20) and U^L = K R' K^-1, U^S = 2c K p^-1 X' R' K^-1 (Eq. 22).
// Here the same transforms come from matrix functions evaluated with GEMMs:
//  1. Orthonormalisation by Cholesky factors instead of the eigenvectors of (T, S):
//       S = L L^T, T = M M^T,  K_L = L^-T,  K_S = sqrt(2) c M^-T
//     so H^p = [[L^-1 V L^-T, sqrt2 c L^-1 M], [.., (1/2) M^-1 W M^-T - 2c^2]].
//     (Any K_L with K_L+ S K_L = 1 and K_S+ (T/2c^2) K_S = 1 gives the same U: the
//     appendix argument, Eqs. A9-A17, only uses these two properties.)
//  2. The projector P onto the positive-energy solutions (eps + c^2 > 0) from the sign
//     function of Z = H^p + c^2, P = (1 + sign Z)/2, by a scaled Newton-Schulz iteration
//       Z <- (3 a/2) Z - (a^3/2) Z^3,   a = sqrt(3 / (1 + l + l^2))
//     with l the running lower bound of |eigenvalue| / ||Z|| (schedule fixed on the host).
//  3. With C+ the positive-energy eigenvectors, P_LL = C_L C_L+ and P_SL = C_S C_L+, so
//       X' = P_SL P_LL^-1   and   R' = (1 + X'+ X')^-1/2 = P_LL^1/2
//     (because 1 + X'+ X' = C_L^-+ C_L^-1 = P_LL^-1).  P_LL^(1/2) and P_LL^(-1/2) come
//     from the coupled Newton-Schulz iteration (eigenvalues of P_LL lie in (0, 1]).
//  4. U^L = K_L R' K_L^-1 = L^-T P_LL^1/2 L^T,
//     U^S = K_S X' R' K_L^-1 = sqrt2 c M^-T P_SL P_LL^-1/2 L^T.
// Two-component matrices are handled in the quaternion form (four real parts), so every
// product is a real GEMM with the quaternion left-multiplication matrix read in place.
#include <algorithm>
#include <climits>
#include <cmath>

#include "common.cuh"
#include "dkh_plan.h"
#include "gemm_f64.cuh"

namespace x2c {
namespace {

constexpr double kSignLowerBound = 1e-6;   // smallest min |eig| / ||Z|| the schedule allows for
// The per-problem schedule starts from l0 = kSignGap c^2 / G (G: the Gershgorin bound that
// scales Z), clamped to [kSignLowerBound, 0.5]: the eigenvalues of Z = H^p + c^2 are E + c^2,
// the negative-energy branch lies below -c^2 and the electronic one above -c^2 (1 - sqrt(1 -
// (Z/c)^2)) for a point nucleus, so |E + c^2| >= 0.5 c^2 up to Z = 118; the margin of 2 more
// covers basis and potential variations.  A violation costs iterations (up to the schedule of
// kSignLowerBound) or, beyond that, the convergence check's X2C_ERR_NOCONV: never a wrong h.
constexpr int kSqrtIters = 8;              // coupled Newton-Schulz steps for P_LL^(+-1/2)
constexpr double kSignTol = 1e-7;          // ||Z^2 - 1|| at the last sign step
constexpr double kSignGap = 0.25;
constexpr double kSqrtTol = 1e-7;          // ||T - 1|| at the last square-root step

constexpr int kSignMaxSteps = 64;  // bound on any schedule length (sign_schedule stops at 61)

std::vector<double> sign_schedule(double l0) {
  std::vector<double> a;
  double l = l0;
  auto f = [](double x) { return 1.5 * x - 0.5 * x * x * x; };
  while (1.0 - l > 1e-15 && a.size() < 60) {
    double al = std::sqrt(3.0 / (1.0 + l + l * l));
    a.push_back(al);
    l = std::fmin(f(al * l), f(al));
  }
  a.push_back(1.0);  // one plain step to settle the rounding level
  return a;
}

// Cholesky factor and its inverse of S (which = 0) or T (which = 1) of every problem.
// One CTA per matrix, factorisation in shared memory (n <= 168), inverse by column-wise
// forward substitution.  fac/inv: (2 * nb) blocks of n * n, lower triangular.
__global__ void chol_inv_kernel(const InputDesc *in, int n, double *fac, double *inv, int *status) {
  extern __shared__ double A[];
  const int prob = blockIdx.x >> 1, which = blockIdx.x & 1;
  const InputDesc d = in[prob];
  const double *src = which ? d.T : d.S;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx - i * n;
    A[idx] = src[(int64_t)i * d.ld + j];
  }
  __syncthreads();
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      double p = A[j * n + j];
      if (!(p > 0.0)) {   // also catches NaN
        bad = 1;
        p = 1.0;
      }
      A[j * n + j] = sqrt(p);
    }
    __syncthreads();
    const double piv = A[j * n + j];
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[i * n + j] /= piv;
    __syncthreads();
    const int w = n - j - 1;
    for (int idx = threadIdx.x; idx < w * w; idx += blockDim.x) {
      const int i = j + 1 + idx / w, k = j + 1 + idx % w;
      if (k <= i) A[i * n + k] -= A[i * n + j] * A[k * n + j];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && bad) flag_error(status, X2C_DEV_NOT_POSDEF);
  double *F = fac + (int64_t)blockIdx.x * n * n;
  double *X = inv + (int64_t)blockIdx.x * n * n;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, k = idx - i * n;
    F[idx] = (k <= i) ? A[idx] : 0.0;
    X[idx] = 0.0;
  }
  __syncthreads();
  // X = L^-1, column j by one thread: X_jj = 1/L_jj, X_ij = -(sum_k=j..i-1 L_ik X_kj) / L_ii
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    X[(int64_t)j * n + j] = 1.0 / A[j * n + j];
    for (int i = j + 1; i < n; ++i) {
      double s = 0.0;
      for (int k = j; k < i; ++k) s = fma(A[i * n + k], X[(int64_t)k * n + j], s);
      X[(int64_t)i * n + j] = -s / A[i * n + i];
    }
  }
}

// Leaf of the blocked factorisation of large matrices: Cholesky factor F (lower, zeros
// above the diagonal) and its inverse X of the n x n block at A (leading dimension lda),
// n <= kLeaf, one CTA, factorisation in shared memory as in chol_inv_kernel.
constexpr int kLeaf = 128;
__global__ void chol_leaf_kernel(const double *Ain, int64_t lda, int n, double *F, double *X, int64_t ld,
                                 int *status) {
  extern __shared__ double A[];
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx - i * n;
    A[idx] = Ain[(int64_t)i * lda + j];
  }
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      double p = A[j * n + j];
      if (!(p > 0.0)) {
        bad = 1;
        p = 1.0;
      }
      A[j * n + j] = sqrt(p);
    }
    __syncthreads();
    const double piv = A[j * n + j];
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[i * n + j] /= piv;
    __syncthreads();
    const int w = n - j - 1;
    for (int idx = threadIdx.x; idx < w * w; idx += blockDim.x) {
      const int i = j + 1 + idx / w, k = j + 1 + idx % w;
      if (k <= i) A[i * n + k] -= A[i * n + j] * A[k * n + j];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && bad) flag_error(status, X2C_DEV_NOT_POSDEF);
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, k = idx - i * n;
    F[(int64_t)i * ld + k] = (k <= i) ? A[idx] : 0.0;
    X[(int64_t)i * ld + k] = 0.0;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    X[(int64_t)j * ld + j] = 1.0 / A[j * n + j];
    for (int i = j + 1; i < n; ++i) {
      double s = 0.0;
      for (int k = j; k < i; ++k) s = fma(A[i * n + k], X[(int64_t)k * ld + j], s);
      X[(int64_t)i * ld + j] = -s / A[i * n + i];
    }
  }
}

// Copy S (which = 0) or T (which = 1) of problem `prob` into a dense n x n matrix.
__global__ void copy_input_kernel(const InputDesc *in, int prob, int which, int n, double *dst) {
  const InputDesc d = in[prob];
  const double *src = which ? d.T : d.S;
  const int64_t total = (int64_t)n * n;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / n, j = idx - i * n;
    dst[idx] = src[i * d.ld + j];
  }
}

// B operand reading an input matrix of problem bb / div (part bb % div for W).
struct InputOp {
  const InputDesc *d;
  int which;  // 0 S, 1 T, 2 V, 3 W[part]
  int div;
  static constexpr bool n_contig = true;
  __device__ __forceinline__ double operator()(int bb, int k, int nn) const {
    const InputDesc &D = d[bb / div];
    const double *p = which == 0 ? D.S : which == 1 ? D.T : which == 2 ? D.V : D.W[bb % div];
    return p[(int64_t)k * D.ld + nn];
  }
};

// Strided operand whose batch index is divided by `div` (shared by the parts of a problem).
template <bool TRANS>
struct MatDiv {
  const double *p;
  int64_t ld, bs;
  int div;
  double scale;
  static constexpr bool k_contig = !TRANS;
  static constexpr bool n_contig = !TRANS;
  __device__ __forceinline__ double operator()(int b, int r, int k) const {
    const double *q = p + (int64_t)(b / div) * bs;
    return scale * (TRANS ? q[(int64_t)k * ld + r] : q[(int64_t)r * ld + k]);
  }
};

// Z = H^p + c^2 (Eq. 14 in the Cholesky-orthonormal basis), parts of size 2n x 2n.
// grid.x = problem x part, grid.y strides over the elements.
__global__ void assemble_hp_kernel(int n, int nc, double c, const double *Vt, const double *LSm,
                                   const double *Wt, double *Z) {
  const int prob = blockIdx.x / nc, q = blockIdx.x % nc;
  const int64_t d = 2 * n;
  const double c2 = c * c;
  const double *vt = Vt + (int64_t)prob * n * n;
  const double *ls = LSm + (int64_t)prob * n * n;
  const double *wt = Wt + ((int64_t)prob * nc + q) * n * n;
  double *z = Z + ((int64_t)prob * nc + q) * d * d;
  for (int64_t idx = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; idx < d * d;
       idx += (int64_t)gridDim.y * blockDim.x) {
    const int64_t r = idx / d, col = idx - r * d;
    double v = 0.0;
    if (r < n && col < n) {
      if (q == 0) v = vt[r * n + col] + (r == col ? c2 : 0.0);
    } else if (r < n) {
      if (q == 0) v = ls[r * n + (col - n)];
    } else if (col < n) {
      if (q == 0) v = ls[col * n + (r - n)];
    } else {
      v = wt[(r - n) * n + (col - n)] - ((q == 0 && r == col) ? c2 : 0.0);
    }
    z[idx] = v;
  }
}

__device__ double block_max(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (l < (int)(blockDim.x >> 5)) ? red[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (l == 0) red[0] = v;
  }
  __syncthreads();
  v = red[0];
  __syncthreads();
  return v;
}

__device__ double block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (l < (int)(blockDim.x >> 5)) ? red[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (l == 0) red[0] = v;
  }
  __syncthreads();
  v = red[0];
  __syncthreads();
  return v;
}

// Maximum of non-negative doubles across CTAs: their bit patterns order like the values
// (a NaN compares above every finite value and is caught by the consumer).
__device__ void atomic_max_nonneg(unsigned long long *slot, double v) {
  atomicMax(slot, static_cast<unsigned long long>(__double_as_longlong(v)));
}

// Gershgorin bound of every problem's Z: the largest row sum of quaternion moduli (a bound
// of the spectral radius of the equivalent complex matrix).  One warp per row, grid.x =
// problem, grid.y strides over rows; the maximum goes to mx[problem] (zeroed before).
__global__ void gershgorin_kernel(int d, int nc, const double *Z, unsigned long long *mx) {
  __shared__ double red[32];
  const double *z = Z + (int64_t)blockIdx.x * nc * d * d;
  const int warps = blockDim.x >> 5, w = threadIdx.x >> 5, l = threadIdx.x & 31;
  double best = 0.0;
  for (int r = blockIdx.y * warps + w; r < d; r += gridDim.y * warps) {
    double s = 0.0;
    for (int col = l; col < d; col += 32) {
      double q2 = 0.0;
      for (int q = 0; q < nc; ++q) {
        const double v = z[(int64_t)q * d * d + (int64_t)r * d + col];
        q2 += v * v;
      }
      s += sqrt(q2);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    best = fmax(best, s);
  }
  best = block_max(best, red);
  if (threadIdx.x == 0) atomic_max_nonneg(&mx[blockIdx.x], best);
}

// Z /= its Gershgorin bound (a bad bound is flagged and the scale left at 1).
__global__ void scale_kernel(int64_t per, double *Z, const unsigned long long *mx, int *status) {
  double m = __longlong_as_double(static_cast<long long>(mx[blockIdx.x]));
  if (!(m > 0.0) || !isfinite(m)) {
    if (blockIdx.y == 0 && threadIdx.x == 0) flag_error(status, X2C_DEV_NONFINITE);
    m = 1.0;
  }
  const double inv = 1.0 / m;
  double *z = Z + (int64_t)blockIdx.x * per;
  for (int64_t idx = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; idx < per;
       idx += (int64_t)gridDim.y * blockDim.x)
    z[idx] *= inv;
}

// Per-problem scaled Newton-Schulz schedule (the host's sign_schedule, from the problem's own
// lower bound l0 = kSignGap c^2 / G): a[b * kmax + k] for k < kmax, then 1.0 (plain steps,
// which leave a converged sign unchanged).  *n_eff = the longest schedule, rounded up to the
// parity of kmax so that the last executed step leaves the iterate in the buffer the host
// expects after kmax steps; steps k >= *n_eff are skipped (the gate of their products).
__global__ void sign_schedule_kernel(int nb, double c2, const unsigned long long *mx, double *a, int kmax,
                                     int *n_eff) {
  __shared__ int nmax;
  if (threadIdx.x == 0) nmax = 0;
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    double g = __longlong_as_double(static_cast<long long>(mx[b]));
    if (!(g > 0.0) || !isfinite(g)) g = 1.0;
    double l = fmin(fmax(kSignGap * c2 / g, kSignLowerBound), 0.5);
    int k = 0;
    while (1.0 - l > 1e-15 && k < kmax - 1) {
      const double al = sqrt(3.0 / (1.0 + l + l * l));
      a[b * kmax + k++] = al;
      const double x = al * l;
      l = fmin(1.5 * x - 0.5 * x * x * x, 1.5 * al - 0.5 * al * al * al);
    }
    const int n = k + 1;  // and one plain step to settle the rounding level
    for (; k < kmax; ++k) a[b * kmax + k] = 1.0;
    atomicMax(&nmax, n);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int n = nmax;
    if ((kmax - n) & 1) ++n;
    *n_eff = min(n, kmax);
  }
}

// Convergence checks: ||Y - 1||_max of the last squared iterate (into dev[problem]) and,
// for the sign function, trace Z_0 (into tr[problem]); both zeroed before.
__global__ void deviation_kernel(int d, int nc, const double *Y, unsigned long long *dev) {
  __shared__ double red[32];
  const double *y = Y + (int64_t)blockIdx.x * nc * d * d;
  const int64_t total = (int64_t)nc * d * d;
  double mx = 0.0;
  for (int64_t idx = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.y * blockDim.x) {
    const int64_t rr = idx / d, col = idx % d;
    double v = y[idx] - ((rr == col) ? 1.0 : 0.0);  // part 0 rows are rr < d
    if (!isfinite(v)) v = 1e300;
    mx = fmax(mx, fabs(v));
  }
  mx = block_max(mx, red);
  if (threadIdx.x == 0) atomic_max_nonneg(&dev[blockIdx.x], mx);
}

__global__ void trace_kernel(int d, int nc, const double *Z, double *tr) {
  __shared__ double red[32];
  const double *z = Z + (int64_t)blockIdx.x * nc * d * d;
  double t = 0.0;
  for (int r = threadIdx.x; r < d; r += blockDim.x) t += z[(int64_t)r * d + r];
  t = block_sum(t, red);
  if (threadIdx.x == 0) tr[blockIdx.x] = t;
}

__global__ void check_final_kernel(int nb, const unsigned long long *dev, const double *tr, double tol,
                                   int *status) {
  for (int p = threadIdx.x; p < nb; p += blockDim.x) {
    const double m = __longlong_as_double(static_cast<long long>(dev[p]));
    if (!(m <= tol)) flag_error(status, m >= 1e299 ? X2C_DEV_NONFINITE : X2C_DEV_NOCONV);
    if (tr && !(fabs(tr[p]) < 0.5)) flag_error(status, X2C_DEV_DECOUPLING);
  }
}

// P = (1 + Z)/2 blocks: P_LL (Hermitian part of the LL block) and P_SL.
__global__ void projector_kernel(int n, int nc, const double *Z, double *PLL, double *PSL) {
  const int prob = blockIdx.x / nc, q = blockIdx.x % nc;
  const int64_t d = 2 * n;
  const double *z = Z + ((int64_t)prob * nc + q) * d * d;
  double *pll = PLL + ((int64_t)prob * nc + q) * n * n;
  double *psl = PSL + ((int64_t)prob * nc + q) * n * n;
  const double sgn = (q == 0) ? 1.0 : -1.0;  // part 0 symmetric, parts 1-3 antisymmetric
  const int64_t total = (int64_t)n * n;
  for (int64_t idx = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.y * blockDim.x) {
    const int64_t i = idx / n, j = idx - i * n;
    const double h = 0.5 * (z[i * d + j] + sgn * z[j * d + i]);
    pll[idx] = 0.5 * h + ((q == 0 && i == j) ? 0.5 : 0.0);
    psl[idx] = 0.5 * z[(n + i) * d + j];
  }
}

// Quaternion identity (part 0 = 1, others 0) for every problem.
__global__ void identity_kernel(int n, int nc, double *X) {
  const int prob = blockIdx.x;
  double *x = X + (int64_t)prob * nc * n * n;
  const int64_t total = (int64_t)nc * n * n;
  for (int64_t idx = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.y * blockDim.x) {
    const int64_t r = idx / n, col = idx % n;
    x[idx] = (r == col) ? 1.0 : 0.0;
  }
}

// Grid of an element-wise kernel: x = `rows` independent blocks of `elems` elements each,
// y = enough CTAs of 256 threads to cover them, about two waves in total.
dim3 aux_grid(int rows, int64_t elems) {
  int64_t y = (elems + 256 * 8 - 1) / (256 * 8);
  y = std::min<int64_t>(y, std::max<int64_t>(1, 152 * 16 / std::max(1, rows)));
  return dim3(rows, (unsigned)std::max<int64_t>(1, std::min<int64_t>(y, 65535)));
}

// Tile and split-K choice of the solve's products: products of a few million FMAs (one small
// atom kind) are latency-bound and get the smallest tile split along K down to single K
// steps; larger ones the 32 x 32 tile with split-K or the 64 x 64 / 96 x 64 tiles.
enum class SolveTile { Tiny, Small, Mid, Large };
struct SolvePlan {
  SolveTile tile;
  int splits;
};
constexpr double kTinyWork = 4.0 * 1024 * 1024;  // FMAs of one launch
SolvePlan plan_product(int nb, int M, int m, int K, bool can_split) {
  if ((double)nb * M * m * K <= kTinyWork)
    return {SolveTile::Tiny, can_split ? choose_splits<TileTiny>(nb, M, m, K, 1) : 1};
  if (m >= 512) return {SolveTile::Large, 1};
  const int s = can_split ? choose_splits<TileSmall>(nb, M, m, K) : 1;
  return {s > 1 ? SolveTile::Small : SolveTile::Mid, s};
}

// Quaternion product C = A B for nb problems (parts m x m): C_stack = Lq(A) B_stack.
// Small problems are split along K into a partial buffer (`part`, see quat_part_doubles).
template <class COp>
x2c_status quat_gemm(x2c_ctx *ctx, cudaStream_t st, int nb, int m, int nc, const double *A,
                     const double *B, double scale, const COp &C, double *part, const int *gate = nullptr,
                     int step = 0, const char *name = "solve_quat_gemm") {
  QuatLeft<false> a{A, m, (int64_t)nc * m * m, (int64_t)m * m, m, nc, scale};
  Mat<false> b{B, m, (int64_t)nc * m * m, 1.0};
  const int M = nc * m, K = nc * m;
  const SolvePlan p = plan_product(nb, M, m, K, part != nullptr);
  switch (p.tile) {
    case SolveTile::Tiny:
      if (p.splits > 1)
        return gemm_f64_splitk<TileTiny>(ctx, st, nb, M, m, K, p.splits, part, a, b, C, name, gate, step);
      return gemm_f64<TileTiny>(ctx, st, nb, M, m, a, b, C, UniformDims{M, m, K, gate, step}, name);
    case SolveTile::Small:
      return gemm_f64_splitk<TileSmall>(ctx, st, nb, M, m, K, p.splits, part, a, b, C, name, gate, step);
    case SolveTile::Large:
      return gemm_f64<TileLarge>(ctx, st, nb, M, m, a, b, C, UniformDims{M, m, K, gate, step}, name);
    default:
      return gemm_f64<TileSolve>(ctx, st, nb, M, m, a, b, C, UniformDims{M, m, K, gate, step}, name);
  }
}

// Quaternion product whose result is Hermitian (products of commuting Hermitian matrices:
// every Newton-Schulz product here): only the upper triangle of each part is computed, the
// epilogue mirrors.  Worth it for large parts (no split-K there).
constexpr int kHermMin = 256;
template <class COp>
x2c_status quat_gemm_herm(x2c_ctx *ctx, cudaStream_t st, int nb, int m, int nc, const double *A,
                          const double *B, const COp &C, const int *gate = nullptr, int step = 0,
                          const char *name = "solve_quat_gemm") {
  QuatLeft<false> a{A, m, (int64_t)nc * m * m, (int64_t)m * m, m, nc, 1.0};
  Mat<false> b{B, m, (int64_t)nc * m * m, 1.0};
  const int M = nc * m, K = nc * m;
  return gemm_f64<TileLarge>(ctx, st, nb, M, m, a, b, C, HermDims{M, m, K, m, gate, step}, name);
}

// Square-ish products of the solve (no split-K): tile by size.
template <class AOp, class BOp, class COp>
x2c_status gemm_sq(x2c_ctx *ctx, cudaStream_t st, int batch, int n, const AOp &A, const BOp &B, const COp &C) {
  const SolvePlan p = plan_product(batch, n, n, n, false);
  if (p.tile == SolveTile::Tiny) return gemm_f64<TileTiny>(ctx, st, batch, n, n, A, B, C, UniformDims{n, n, n});
  if (p.tile == SolveTile::Large) return gemm_f64<TileLarge>(ctx, st, batch, n, n, A, B, C, UniformDims{n, n, n});
  return gemm_f64<TileSolve>(ctx, st, batch, n, n, A, B, C, UniformDims{n, n, n});
}

// Size of the split-K partial buffer for quat_gemm on nb problems of part size m.
size_t quat_part_doubles(int nb, int m, int nc) {
  const int M = nc * m, K = nc * m;
  const SolvePlan p = plan_product(nb, M, m, K, true);
  return p.splits > 1 ? (size_t)(p.splits + 1) * nb * M * m : 0;
}

inline StoreAxpby store_plain(double *out, int m, int nc) {
  return StoreAxpby{out, nullptr, m, (int64_t)nc * m * m, 1.0, 0.0};
}

// Blocked Cholesky factor F and inverse X = F^-1 of the n x n matrix A (leading dimension
// lda; its lower part is overwritten by the trailing updates), by halves:
//   F11 X11 from A11;  F21 = A21 X11^T;  A22 -= F21 F21^T;  F22 X22 from A22;
//   X21 = -X22 (F21 X11).
// F and X (leading dimension ld) must be zero above the diagonal blocks beforehand; tmp
// holds n^2/4 + 32 n doubles (the largest F21 X11 product).
x2c_status chol_inv_blocked(x2c_ctx *ctx, cudaStream_t st, double *A, int64_t lda, int n, double *F,
                            double *X, int64_t ld, double *tmp, int *status) {
  if (n <= kLeaf) {
    const size_t smem = (size_t)n * n * sizeof(double);
    X2C_TRY_CUDA(ctx, cudaFuncSetAttribute(chol_leaf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(kLeaf * kLeaf * sizeof(double))));
    tbegin(ctx, st);
    chol_leaf_kernel<<<1, 256, smem, st>>>(A, lda, n, F, X, ld, status);
    return launched(ctx, "chol_leaf_kernel", st);
  }
  const int n1 = ((n / 2 + 31) / 32) * 32, n2 = n - n1;
  X2C_TRY(chol_inv_blocked(ctx, st, A, lda, n1, F, X, ld, tmp, status));
  double *F21 = F + (int64_t)n1 * ld, *X21 = X + (int64_t)n1 * ld;
  X2C_TRY((gemm_f64<TileLarge>(ctx, st, 1, n2, n1, Mat<false>{A + (int64_t)n1 * lda, lda, 0, 1.0},
                               Mat<true>{X, ld, 0, 1.0}, StoreAxpby{F21, nullptr, ld, 0, 1.0, 0.0},
                               UniformDims{n2, n1, n1}, "chol_gemm")));
  double *A22 = A + (int64_t)n1 * lda + n1;
  X2C_TRY((gemm_f64<TileLarge>(ctx, st, 1, n2, n2, Mat<false>{F21, ld, 0, 1.0}, Mat<true>{F21, ld, 0, 1.0},
                               StoreAxpby{A22, A22, lda, 0, -1.0, 1.0}, UniformDims{n2, n2, n1}, "chol_gemm")));
  X2C_TRY(chol_inv_blocked(ctx, st, A22, lda, n2, F21 + n1, X21 + n1, ld, tmp, status));
  X2C_TRY((gemm_f64<TileLarge>(ctx, st, 1, n2, n1, Mat<false>{F21, ld, 0, 1.0}, Mat<false>{X, ld, 0, 1.0},
                               StoreAxpby{tmp, nullptr, n1, 0, 1.0, 0.0}, UniformDims{n2, n1, n1}, "chol_gemm")));
  return gemm_f64<TileLarge>(ctx, st, 1, n2, n1, Mat<false>{X21 + n1, ld, 0, 1.0}, Mat<false>{tmp, n1, 0, 1.0},
                             StoreAxpby{X21, nullptr, ld, 0, -1.0, 0.0}, UniformDims{n2, n1, n2}, "chol_gemm");
}

// ||Y - 1||_max <= tol for every problem and, with Z, |trace Z_0| < 1/2 (equal numbers of
// positive- and negative-energy states); failures are latched in the status word.
x2c_status check(x2c_ctx *ctx, cudaStream_t st, int nb, int d, int nc, const double *Y, const double *Z,
                 double tol, unsigned long long *slot, double *trace, int *status) {
  X2C_TRY(device_fill(ctx, st, slot, 0, sizeof(unsigned long long) * nb));
  tbegin(ctx, st);
  deviation_kernel<<<aux_grid(nb, (int64_t)nc * d * d), 256, 0, st>>>(d, nc, Y, slot);
  X2C_TRY(launched(ctx, "check_kernel", st));
  if (Z) {
    tbegin(ctx, st);
    trace_kernel<<<nb, 256, 0, st>>>(d, nc, Z, trace);
    X2C_TRY(launched(ctx, "check_kernel", st));
  }
  tbegin(ctx, st);
  check_final_kernel<<<1, 256, 0, st>>>(nb, slot, Z ? trace : nullptr, tol, status);
  return launched(ctx, "check_kernel", st);
}

// Z <- sign(Z0), Z0 = H^p + c^2 assembled from the orthonormal blocks (Vt, the L-S
// coupling LSm, Wt; Eq. 14), scaled into [-1, 1] by its Gershgorin bound, by the per-problem
// scaled Newton-Schulz schedule; then the convergence (||Z^2 - 1||) and half/half split
// (|trace Z| < 1/2) checks.  Z, Zn, Y: nb nc (2n)^2 doubles each; Z and Zn are swapped so
// that Z holds the result.
x2c_status sign_of_hp(x2c_ctx *ctx, cudaStream_t st, int nb, int n, int nc, double c, const double *Vt,
                      const double *LSm, const double *Wt, double *&Z, double *&Zn, double *Y,
                      unsigned long long *slot, double *trace, double *sched, int *gate, double *part, int *status) {
  const int d = 2 * n;
  const int64_t d2 = (int64_t)d * d;
  tbegin(ctx, st);
  assemble_hp_kernel<<<aux_grid(nb * nc, d2), 256, 0, st>>>(n, nc, c, Vt, LSm, Wt, Z);
  X2C_TRY(launched(ctx, "assemble_hp_kernel", st));
  X2C_TRY(device_fill(ctx, st, slot, 0, sizeof(unsigned long long) * nb));
  tbegin(ctx, st);
  gershgorin_kernel<<<aux_grid(nb, (int64_t)d * 32 * nc), 256, 0, st>>>(d, nc, Z, slot);
  X2C_TRY(launched(ctx, "gershgorin_kernel", st));
  tbegin(ctx, st);
  scale_kernel<<<aux_grid(nb, nc * d2), 256, 0, st>>>(nc * d2, Z, slot, status);
  X2C_TRY(launched(ctx, "scale_kernel", st));
  // Sign function by the scaled Newton-Schulz schedule, per problem (sign_schedule_kernel);
  // the host enqueues the longest possible schedule and the device skips the steps past the
  // longest one it needs.
  const int kmax = static_cast<int>(sign_schedule(kSignLowerBound).size());
  if (kmax > kSignMaxSteps) return X2C_ERR_ARG;
  tbegin(ctx, st);
  sign_schedule_kernel<<<1, 256, 0, st>>>(nb, c * c, slot, sched, kmax, gate);
  X2C_TRY(launched(ctx, "sign_schedule_kernel", st));
  const bool herm_d = d >= kHermMin;
  for (int k = 0; k < kmax; ++k) {
    // Y = Z Z;  Zn = (3a/2) Z - (a^3/2) Z Y   (Z, Y commute and are Hermitian)
    // (named apart from the other products: how many of them run is decided on the device, so
    // they report no flops)
    const char *sign_name = "solve_sign_gemm";
    if (herm_d) {
      X2C_TRY(quat_gemm_herm(ctx, st, nb, d, nc, Z, Z, StoreAxpbyHerm{Y, nullptr, d, (int64_t)nc * d2, 1.0, 0.0, d},
                             gate, k, sign_name));
      X2C_TRY(quat_gemm_herm(ctx, st, nb, d, nc, Z, Y,
                             StoreSignStepHerm{Zn, Z, d, (int64_t)nc * d2, sched + k, kmax, d}, gate, k, sign_name));
    } else {
      X2C_TRY(quat_gemm(ctx, st, nb, d, nc, Z, Z, 1.0, store_plain(Y, d, nc), part, gate, k, sign_name));
      StoreSignStep upd{Zn, Z, d, (int64_t)nc * d2, sched + k, kmax};
      X2C_TRY(quat_gemm(ctx, st, nb, d, nc, Z, Y, 1.0, upd, part, gate, k, sign_name));
    }
    std::swap(Z, Zn);
  }
  X2C_TRY(check(ctx, st, nb, d, nc, Y, Z, kSignTol, slot, trace, status));
  return X2C_OK;
}

// Yk <- G^1/2 and Zk <- G^-1/2 of Hermitian G with eigenvalues in (0, 1] (coupled
// Newton-Schulz, kSqrtIters steps, then ||T - 1|| <= kSqrtTol checked on the device).  Every
// buffer holds nb nc n^2 doubles; Yk/Yk2 and Zk/Zk2 are swapped so Yk, Zk hold the result.
x2c_status coupled_sqrt(x2c_ctx *ctx, cudaStream_t st, int nb, int n, int nc, const double *G, double *&Yk,
                        double *&Zk, double *Tm, double *&Yk2, double *&Zk2, double *part, unsigned long long *slot,
                        int *status) {
  const int64_t n2 = (int64_t)n * n;
  const bool herm_n = n >= kHermMin;
  X2C_TRY(device_copy(ctx, st, Yk, G, sizeof(double) * nb * nc * n2));
  tbegin(ctx, st);
  identity_kernel<<<aux_grid(nb, nc * n2), 256, 0, st>>>(n, nc, Zk);
  X2C_TRY(launched(ctx, "identity_kernel", st));
  for (int it = 0; it < kSqrtIters; ++it) {
    // Tm = 3/2 - Zk Yk / 2;  Yk <- Yk Tm;  Zk <- Tm Zk   (all functions of P_LL: Hermitian)
    if (herm_n) {
      X2C_TRY(quat_gemm_herm(ctx, st, nb, n, nc, Zk, Yk, StoreShiftIdentityHerm{Tm, n, (int64_t)nc * n2, n, -0.5, 1.5}));
      X2C_TRY(quat_gemm_herm(ctx, st, nb, n, nc, Yk, Tm, StoreAxpbyHerm{Yk2, nullptr, n, (int64_t)nc * n2, 1.0, 0.0, n}));
      X2C_TRY(quat_gemm_herm(ctx, st, nb, n, nc, Tm, Zk, StoreAxpbyHerm{Zk2, nullptr, n, (int64_t)nc * n2, 1.0, 0.0, n}));
    } else {
      StoreShiftIdentity tm{Tm, n, (int64_t)nc * n2, n, -0.5, 1.5};
      X2C_TRY(quat_gemm(ctx, st, nb, n, nc, Zk, Yk, 1.0, tm, part));
      X2C_TRY(quat_gemm(ctx, st, nb, n, nc, Yk, Tm, 1.0, store_plain(Yk2, n, nc), part));
      X2C_TRY(quat_gemm(ctx, st, nb, n, nc, Tm, Zk, 1.0, store_plain(Zk2, n, nc), part));
    }
    std::swap(Yk, Yk2);
    std::swap(Zk, Zk2);
  }
  X2C_TRY(check(ctx, st, nb, n, nc, Tm, nullptr, kSqrtTol, slot, nullptr, status));
  return X2C_OK;
}

}  // namespace

size_t solve_workspace_bytes(int nb, int n, int nc) {
  const size_t n2 = (size_t)n * n;
  const size_t per = (6 + 23 * (size_t)nc) * n2;
  const size_t part = std::max(quat_part_doubles(nb, 2 * n, nc), quat_part_doubles(nb, n, nc));
  const size_t big = n > kMaxSolveN ? arena_doubles(n2) + arena_doubles(n2 / 4 + 32 * (size_t)n) : 0;
  return arena_doubles(per * nb) + arena_doubles(part) + big + 2 * arena_doubles(nb) +
         arena_doubles((size_t)nb * kSignMaxSteps) + arena_doubles(1) + 20 * 256;
}

x2c_status solve_transforms(x2c_ctx *ctx, cudaStream_t st, double c, int nb, int n, int nc,
                            const InputDesc *d_in, double *UL, double *US, Arena ar) {
  if (nb <= 0) return X2C_OK;
  if (n < 1 || 2 * (int64_t)n * 2 * n > INT32_MAX) return X2C_ERR_ARG;
  const int64_t n2 = (int64_t)n * n;
  const int d = 2 * n;
  const int64_t d2 = (int64_t)d * d;
  double *fac = ar.take(2 * nb * n2), *inv = ar.take(2 * nb * n2);
  double *Vt = ar.take(nb * n2), *LSm = ar.take(nb * n2);
  double *tmp = ar.take(nb * nc * n2), *Wt = ar.take(nb * nc * n2);
  double *Z = ar.take(nb * nc * d2), *Zn = ar.take(nb * nc * d2), *Y = ar.take(nb * nc * d2);
  double *PLL = ar.take(nb * nc * n2), *PSL = ar.take(nb * nc * n2);
  double *Yk = ar.take(nb * nc * n2), *Zk = ar.take(nb * nc * n2), *Tm = ar.take(nb * nc * n2);
  double *Yk2 = ar.take(nb * nc * n2), *Zk2 = ar.take(nb * nc * n2);
  double *XR = ar.take(nb * nc * n2), *tmp2 = ar.take(nb * nc * n2);
  auto *slot = reinterpret_cast<unsigned long long *>(ar.take(nb));
  double *trace = ar.take(nb);
  double *sched = ar.take((size_t)nb * kSignMaxSteps);
  int *gate = reinterpret_cast<int *>(ar.take(1));
  if (!tmp2 || !slot || !trace || !sched || !gate) return X2C_ERR_NOMEM;
  const size_t part_n = std::max(quat_part_doubles(nb, d, nc), quat_part_doubles(nb, n, nc));
  double *part = part_n ? ar.take(part_n) : nullptr;
  if (part_n && !part) return X2C_ERR_NOMEM;
  int *status = ctx->d_status;

  // 1. Cholesky factors and inverses of S and T.
  if (n <= kMaxSolveN) {
    const size_t smem = (size_t)n2 * sizeof(double);
    X2C_TRY_CUDA(ctx, cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    tbegin(ctx, st);
    chol_inv_kernel<<<2 * nb, 256, smem, st>>>(d_in, n, fac, inv, status);
    X2C_TRY(launched(ctx, "chol_inv_kernel", st));
  } else {
    // large matrices: blocked factorisation of a dense copy, one matrix at a time
    double *Acopy = ar.take(n2), *ctmp = ar.take(n2 / 4 + 32 * n);
    if (!ctmp) return X2C_ERR_NOMEM;
    X2C_TRY(device_fill(ctx, st, fac, 0, sizeof(double) * 2 * nb * n2));
    X2C_TRY(device_fill(ctx, st, inv, 0, sizeof(double) * 2 * nb * n2));
    for (int b = 0; b < nb; ++b)
      for (int which = 0; which < 2; ++which) {
        tbegin(ctx, st);
        copy_input_kernel<<<152 * 4, 256, 0, st>>>(d_in, b, which, n, Acopy);
        X2C_TRY(launched(ctx, "copy_input_kernel", st));
        X2C_TRY(chol_inv_blocked(ctx, st, Acopy, n, n, fac + (2 * b + which) * n2, inv + (2 * b + which) * n2, n,
                                 ctmp, status));
      }
  }
  // L_S at fac + 2b n2, L_T at fac + (2b+1) n2; inverses likewise in inv.
  const double rt2c = std::sqrt(2.0) * c;
  {
    // tmp = L^-1 V ;  Vt = tmp L^-T
    X2C_TRY((gemm_sq(ctx, st, nb, n, Mat<false>{inv, n, 2 * n2, 1.0},
                                 InputOp{d_in, 2, 1}, StoreAxpby{tmp, nullptr, n, n2, 1.0, 0.0})));
    X2C_TRY((gemm_sq(ctx, st, nb, n, Mat<false>{tmp, n, n2, 1.0},
                                 Mat<true>{inv, n, 2 * n2, 1.0}, StoreAxpby{Vt, nullptr, n, n2, 1.0, 0.0})));
    // LSm = sqrt2 c L^-1 M
    X2C_TRY((gemm_sq(ctx, st, nb, n, Mat<false>{inv, n, 2 * n2, 1.0},
                                 Mat<false>{fac + n2, n, 2 * n2, 1.0}, StoreAxpby{LSm, nullptr, n, n2, rt2c, 0.0})));
    // tmp_q = M^-1 W_q ;  Wt_q = (1/2) tmp_q M^-T      (batch over problem x part)
    X2C_TRY((gemm_sq(ctx, st, nb * nc, n, MatDiv<false>{inv + n2, n, 2 * n2, nc, 1.0},
                                 InputOp{d_in, 3, nc}, StoreAxpby{tmp, nullptr, n, n2, 1.0, 0.0})));
    X2C_TRY((gemm_sq(ctx, st, nb * nc, n, Mat<false>{tmp, n, n2, 1.0},
                                 MatDiv<true>{inv + n2, n, 2 * n2, nc, 1.0}, StoreAxpby{Wt, nullptr, n, n2, 0.5, 0.0})));
  }
  // 2-3. Z <- sign(H^p + c^2) (scaled Newton-Schulz), with its convergence and split checks.
  X2C_TRY(sign_of_hp(ctx, st, nb, n, nc, c, Vt, LSm, Wt, Z, Zn, Y, slot, trace, sched, gate, part, status));
  tbegin(ctx, st);
  projector_kernel<<<aux_grid(nb * nc, n2), 256, 0, st>>>(n, nc, Z, PLL, PSL);
  X2C_TRY(launched(ctx, "projector_kernel", st));
  // 4. Coupled Newton-Schulz: Yk -> P_LL^1/2, Zk -> P_LL^-1/2.
  X2C_TRY(coupled_sqrt(ctx, st, nb, n, nc, PLL, Yk, Zk, Tm, Yk2, Zk2, part, slot, status));
  // 5. X'R' = P_SL P_LL^-1/2
  X2C_TRY(quat_gemm(ctx, st, nb, n, nc, PSL, Zk, 1.0, store_plain(XR, n, nc), part));
  // 6. U^L_q = L^-T (R'_q L^T),  U^S_q = sqrt2 c M^-T (X'R'_q L^T)   (batch over problem x part)
  {
    X2C_TRY((gemm_sq(ctx, st, nb * nc, n, Mat<false>{Yk, n, n2, 1.0},
                                 MatDiv<true>{fac, n, 2 * n2, nc, 1.0}, StoreAxpby{tmp, nullptr, n, n2, 1.0, 0.0})));
    X2C_TRY((gemm_sq(ctx, st, nb * nc, n, MatDiv<true>{inv, n, 2 * n2, nc, 1.0},
                                 Mat<false>{tmp, n, n2, 1.0}, StoreAxpby{UL, nullptr, n, n2, 1.0, 0.0})));
    X2C_TRY((gemm_sq(ctx, st, nb * nc, n, Mat<false>{XR, n, n2, 1.0},
                                 MatDiv<true>{fac, n, 2 * n2, nc, 1.0}, StoreAxpby{tmp2, nullptr, n, n2, 1.0, 0.0})));
    X2C_TRY((gemm_sq(ctx, st, nb * nc, n, MatDiv<true>{inv + n2, n, 2 * n2, nc, 1.0},
                                 Mat<false>{tmp2, n, n2, 1.0}, StoreAxpby{US, nullptr, n, n2, rt2c, 0.0})));
  }
  return X2C_OK;
}

#include "solve_fw.cuh"

}  // namespace x2c
