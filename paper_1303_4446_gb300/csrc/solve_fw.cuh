// Decoupling transforms built on the free-particle transformation: BSS (Sec. II.B) and DKHn
// with the exponential parametrisation (Sec. II.C), batched over problems of one size; and
// the DKHn Hamiltonian of a whole system.  Included by solve.cu (it uses that file's GEMM,
// sign-function and square-root helpers).
//
// Both methods work in the orthonormal kinetic basis of Sec. II.A, T K = S K t, K+ S K = 1
// (Eq. 11): here S = L L^T (Cholesky), the symmetric t^ = L^-1 T L^-T is diagonalised by a
// one-CTA Jacobi iteration, t^ = Q t Q^T, and K = L^-T Q, K^-1 = Q^T L^T.  With p = sqrt(2t):
//   V~ = K^T V K,  W~ = p^-1 K^T W K p^-1,  H^p = [[V~, c p], [c p, W~ - 2c^2]]  (Eqs. 14-17),
// and the free-particle factors E0 = c sqrt(c^2 + p^2), A = sqrt((E0 + c^2)/2E0),
// B = sqrt((E0 - c^2)/2E0) (B^2 and E0 - c^2 evaluated as c^2 p^2 / ... without cancellation).
// U0 is the orthogonal matrix with the free electronic solutions [A; B] in its first block
// column (second [-B; A]).
//
// BSS: with P the projector onto the positive-energy solutions of H^p (the sign function of
// H^p + c^2, as for X2C) and H^0 = U0^T H^p U0, the BSS columns U0 [1; X''] R'' of Sec. II.B
// equal P [A; B] G^-1/2 with G = [A; B]^T P [A; B] (X'' = P''_SL P''_LL^-1 and R'' = P''_LL^1/2
// for the projector P'' = U0^T P U0 of H^0, and P''_LL = G): one more element-wise step and
// one more square root than X2C.
//
// DKHn: the operation list of dkh_plan.h on the blocks of H^0 (E1 = A V~ A + B W~ B,
// E1' = B V~ B + A W~ A, O1 = B W~ A - A V~ B, element-wise); the Hamiltonian is
// E0 - c^2 + sum of the even upper blocks up to order n; the transforms are the H^0-frame
// columns exp(-W_1) ... exp(-W_n) [1; 0] (each exponential cut after the powers of order <= n),
// renormalised by R'' = (Y+ Y)^-1/2 and taken through U0.
// Every transform ends as U^L = K Y_L K^-1, U^S = 2c K p^-1 Y_S K^-1.
// (solve.cu includes dkh_plan.h, the host-side DKH plan, before its namespace opens.)

namespace {

constexpr int kMaxJacobiN = 160;   // t^ lives in shared memory (n^2 doubles <= 200 KB)
constexpr int kJacobiSweeps = 40;

// Free-particle quantities of a kinetic eigenvalue t (p^2 = 2t).
__device__ __forceinline__ void fw_factors(double t, double c, double &E0, double &A, double &B, double &Ek) {
  const double c2 = c * c, p2 = 2.0 * t;
  E0 = c * sqrt(c2 + p2);
  Ek = c2 * p2 / (E0 + c2);  // E0 - c^2
  A = sqrt((E0 + c2) / (2.0 * E0));
  B = sqrt(Ek / (2.0 * E0));
}

// Eigen-decomposition of symmetric matrices (one CTA per matrix, cyclic Jacobi with the
// round-robin ordering: m/2 disjoint rotations per step, m - 1 steps per sweep, m = n rounded
// up to even; in step s, position k pairs with position m - 1 - k, position 0 holds index 0
// and position i >= 1 holds 1 + (i - 1 + s) mod (m - 1)).  A rotation is skipped when
// |a_pq| <= 1e-15 sqrt(a_pp a_qq) (relative criterion: small eigenvalues keep their relative
// accuracy); a sweep without rotations ends the iteration (no convergence within
// kJacobiSweeps is flagged).  The matrix lives in shared memory, and so do the eigenvectors
// when both fit (n <= kJacobiSmemV), else they are updated in global memory.  Output:
// eigenvalues evals[b n + i] and eigenvectors as the ROWS of QT (QT[b][i][:] belongs to
// evals[b n + i]).
constexpr int kJacobiSmemV = 110;  // 2 n^2 doubles <= 194 KB
__global__ void __launch_bounds__(256) jacobi_kernel(const double *Ain, int n, int64_t stride, double *evals,
                                                     double *QT, int *status) {
  extern __shared__ double A[];
  __shared__ int pp[kMaxJacobiN / 2], qq[kMaxJacobiN / 2];
  __shared__ double cs[kMaxJacobiN / 2], sn[kMaxJacobiN / 2];
  __shared__ int rotated;
  const int b = blockIdx.x;
  const double *a0 = Ain + b * stride;
  const int nn = n * n;
  const bool vsh = n <= kJacobiSmemV;
  double *qt = vsh ? A + nn : QT + b * stride;
  for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) {
    A[idx] = a0[idx];
    qt[idx] = (idx / n == idx % n) ? 1.0 : 0.0;
  }
  const int m = n + (n & 1), half = m / 2;
  __syncthreads();
  bool converged = n < 2;
  for (int sweep = 0; sweep < kJacobiSweeps && !converged; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int step = 0; step < m - 1; ++step) {
      for (int k = threadIdx.x; k < half; k += blockDim.x) {
        const int i1 = k, i2 = m - 1 - k;
        int p = i1 == 0 ? 0 : 1 + (i1 - 1 + step) % (m - 1);
        int q = 1 + (i2 - 1 + step) % (m - 1);
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        double c = 1.0, s = 0.0;
        if (q < n) {
          const double apq = A[p * n + q], app = A[p * n + p], aqq = A[q * n + q];
          if (fabs(apq) > 1e-15 * sqrt(fabs(app * aqq))) {
            const double tau = (aqq - app) / (2.0 * apq);
            const double t = fabs(tau) > 1e150 ? 0.5 / tau : copysign(1.0, tau) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
            rotated = 1;
          }
        }
        pp[k] = p;
        qq[k] = q;
        cs[k] = c;
        sn[k] = s;
      }
      __syncthreads();
      // A <- G A G^T for all the step's rotations at once, G_k = [[c, -s], [s, c]] on the
      // rows and columns (p_k, q_k): the 2 x 2 block of pairs (k, k') becomes
      // G_k B G_k'^T.  Only blocks k <= k' are computed (A is symmetric) and mirrored; each
      // thread reads and writes only its block and the mirror, so the update is in place.
      // The eigenvector rows p, q of QT take G_k in the same pass (disjoint data).
      for (int idx = threadIdx.x; idx < half * half; idx += blockDim.x) {
        const int k = idx / half, k2 = idx - k * half;
        if (k > k2) continue;
        const double c1 = cs[k], s1 = sn[k], c2 = cs[k2], s2 = sn[k2];
        if (s1 == 0.0 && s2 == 0.0) continue;
        const int r[2] = {pp[k], qq[k]}, q2[2] = {pp[k2], qq[k2]};
        double blk[2][2];
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int v = 0; v < 2; ++v) blk[u][v] = (r[u] < n && q2[v] < n) ? A[r[u] * n + q2[v]] : 0.0;
        double t[2][2];
#pragma unroll
        for (int v = 0; v < 2; ++v) {
          t[0][v] = c1 * blk[0][v] - s1 * blk[1][v];
          t[1][v] = s1 * blk[0][v] + c1 * blk[1][v];
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const double x0 = c2 * t[u][0] - s2 * t[u][1], x1 = s2 * t[u][0] + c2 * t[u][1];
          blk[u][0] = x0;
          blk[u][1] = x1;
        }
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int v = 0; v < 2; ++v)
            if (r[u] < n && q2[v] < n) {
              A[r[u] * n + q2[v]] = blk[u][v];
              A[q2[v] * n + r[u]] = blk[u][v];
            }
      }
      for (int idx = threadIdx.x; idx < half * n; idx += blockDim.x) {
        const int k = idx / n, j = idx - k * n;
        const double s = sn[k];
        if (s == 0.0) continue;
        const int p = pp[k], q = qq[k];
        const double c = cs[k];
        const double vp = qt[p * n + j], vq = qt[q * n + j];
        qt[p * n + j] = c * vp - s * vq;
        qt[q * n + j] = s * vp + c * vq;
      }
      __syncthreads();
    }
    converged = rotated == 0;
    __syncthreads();
  }
  if (!converged && threadIdx.x == 0) flag_error(status, X2C_DEV_NOCONV);
  for (int i = threadIdx.x; i < n; i += blockDim.x) evals[(int64_t)b * n + i] = A[i * n + i];
  if (vsh)
    for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) QT[b * stride + idx] = qt[idx];
}

// The right operand of a quaternion product as a stack of parts (or of the parts of its
// adjoint: (B+)_0 = B_0^T, (B+)_k = -B_k^T).
template <bool ADJ>
struct QuatStack {
  const double *p;
  int64_t bs, ps;
  int m, nc;
  static constexpr bool n_contig = !ADJ;
  static constexpr bool k_contig = ADJ;
  __device__ __forceinline__ double operator()(int b, int k, int col) const {
    int q = 0, kk = k;
    if (nc == 4) {
      q = k / m;
      kk = k - q * m;
    }
    const double *base = p + b * bs + q * ps;
    if (!ADJ) return base[(int64_t)kk * m + col];
    return (q == 0 ? 1.0 : -1.0) * base[(int64_t)col * m + kk];
  }
};

// C = alpha op(A) op(B) + beta C for nb problems of n x n quaternion matrices (part-major,
// nc n^2 doubles per problem), op = identity or adjoint.
template <bool AA, bool AB>
x2c_status quat_product(x2c_ctx *ctx, cudaStream_t st, int nb, int m, int nc, const double *A, const double *B,
                        double *C, double alpha, double beta, const char *name) {
  QuatLeft<AA> a{A, m, (int64_t)nc * m * m, (int64_t)m * m, m, nc, 1.0};
  QuatStack<AB> b{B, (int64_t)nc * m * m, (int64_t)m * m, m, nc};
  StoreAxpby cst{C, beta != 0.0 ? C : nullptr, m, (int64_t)nc * m * m, alpha, beta};
  const int M = nc * m, K = nc * m;
  const SolvePlan p = plan_product(nb, M, m, K, false);
  if (p.tile == SolveTile::Tiny) return gemm_f64<TileTiny>(ctx, st, nb, M, m, a, b, cst, UniformDims{M, m, K}, name);
  if (p.tile == SolveTile::Large) return gemm_f64<TileLarge>(ctx, st, nb, M, m, a, b, cst, UniformDims{M, m, K}, name);
  return gemm_f64<TileSolve>(ctx, st, nb, M, m, a, b, cst, UniformDims{M, m, K}, name);
}

x2c_status quat_product_op(x2c_ctx *ctx, cudaStream_t st, int nb, int m, int nc, bool aa, bool ab, const double *A,
                           const double *B, double *C, double alpha, double beta, const char *name) {
  if (aa && ab) return quat_product<true, true>(ctx, st, nb, m, nc, A, B, C, alpha, beta, name);
  if (aa) return quat_product<true, false>(ctx, st, nb, m, nc, A, B, C, alpha, beta, name);
  if (ab) return quat_product<false, true>(ctx, st, nb, m, nc, A, B, C, alpha, beta, name);
  return quat_product<false, false>(ctx, st, nb, m, nc, A, B, C, alpha, beta, name);
}

// Element-wise kernels: grid.x = problem x part (nc parts), grid.y strides over n^2 elements.
#define FW_ELEMENTS(n)                                                                    \
  for (int64_t idx = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)(n) * (n); \
       idx += (int64_t)gridDim.y * blockDim.x)

// LSm = diag(c p) (the L-S coupling of H^p in the kinetic basis), one block per problem.
__global__ void coupling_diag_kernel(int n, double c, const double *evals, double *LSm) {
  const int b = blockIdx.x;
  double *o = LSm + (int64_t)b * n * n;
  FW_ELEMENTS(n) {
    const int i = (int)(idx / n), j = (int)(idx - (int64_t)i * n);
    o[idx] = (i == j) ? c * sqrt(2.0 * evals[(int64_t)b * n + i]) : 0.0;
  }
}

// X_ij /= p_i p_j (W~ = p^-1 K^T W K p^-1).
__global__ void scale_pp_kernel(int n, int nc, const double *evals, double *X) {
  const int b = blockIdx.x / nc;
  double *x = X + (int64_t)blockIdx.x * n * n;
  const double *t = evals + (int64_t)b * n;
  FW_ELEMENTS(n) {
    const int i = (int)(idx / n), j = (int)(idx - (int64_t)i * n);
    x[idx] /= sqrt(4.0 * t[i] * t[j]);
  }
}

// BSS: Y = P [A; B] from Z = sign(H^p + c^2) (P = (1 + Z)/2; parts of size 2n):
// Y_L = P_LL A + P_LS B, Y_S = P_SL A + P_SS B (column scalings).
__global__ void bss_ref_kernel(int n, int nc, double c, const double *evals, const double *Z, double *YL,
                               double *YS) {
  const int b = blockIdx.x / nc, q = blockIdx.x % nc;
  const int64_t d = 2 * n;
  const double *z = Z + (int64_t)blockIdx.x * d * d;
  double *yl = YL + (int64_t)blockIdx.x * n * n, *ys = YS + (int64_t)blockIdx.x * n * n;
  const double *t = evals + (int64_t)b * n;
  FW_ELEMENTS(n) {
    const int i = (int)(idx / n), j = (int)(idx - (int64_t)i * n);
    double E0, A, B, Ek;
    fw_factors(t[j], c, E0, A, B, Ek);
    const double id = (q == 0) ? 1.0 : 0.0;
    const double pll = 0.5 * (z[i * d + j] + (i == j ? id : 0.0)), pls = 0.5 * z[i * d + n + j];
    const double psl = 0.5 * z[(n + i) * d + j], pss = 0.5 * (z[(n + i) * d + n + j] + (i == j ? id : 0.0));
    yl[idx] = pll * A + pls * B;
    ys[idx] = psl * A + pss * B;
  }
}

// BSS: G = A Y_L + B Y_S (row scalings), Hermitian part taken (part 0 symmetric, parts
// 1-3 antisymmetric).
__global__ void bss_gram_kernel(int n, int nc, double c, const double *evals, const double *YL, const double *YS,
                                double *G) {
  const int b = blockIdx.x / nc, q = blockIdx.x % nc;
  const double *yl = YL + (int64_t)blockIdx.x * n * n, *ys = YS + (int64_t)blockIdx.x * n * n;
  double *g = G + (int64_t)blockIdx.x * n * n;
  const double *t = evals + (int64_t)b * n;
  const double sgn = q == 0 ? 1.0 : -1.0;
  FW_ELEMENTS(n) {
    const int i = (int)(idx / n), j = (int)(idx - (int64_t)i * n);
    double E0, Ai, Bi, Aj, Bj, Ek;
    fw_factors(t[i], c, E0, Ai, Bi, Ek);
    fw_factors(t[j], c, E0, Aj, Bj, Ek);
    const double gij = Ai * yl[(int64_t)i * n + j] + Bi * ys[(int64_t)i * n + j];
    const double gji = Aj * yl[(int64_t)j * n + i] + Bj * ys[(int64_t)j * n + i];
    g[idx] = 0.5 * (gij + sgn * gji);
  }
}

// DKH: E1, E1', O1 of H^0 from V~ (spin-free) and W~ (nc parts).
__global__ void fw_blocks_kernel(int n, int nc, double c, const double *evals, const double *Vt, const double *Wt,
                                 double *E1, double *E1p, double *O1) {
  const int b = blockIdx.x / nc, q = blockIdx.x % nc;
  const double *v = Vt + (int64_t)b * n * n, *w = Wt + (int64_t)blockIdx.x * n * n;
  const int64_t o = (int64_t)blockIdx.x * n * n;
  const double *t = evals + (int64_t)b * n;
  FW_ELEMENTS(n) {
    const int i = (int)(idx / n), j = (int)(idx - (int64_t)i * n);
    double E0, Ai, Bi, Aj, Bj, Ek;
    fw_factors(t[i], c, E0, Ai, Bi, Ek);
    fw_factors(t[j], c, E0, Aj, Bj, Ek);
    const double vij = q == 0 ? v[idx] : 0.0, wij = w[idx];
    E1[o + idx] = Ai * Aj * vij + Bi * Bj * wij;
    E1p[o + idx] = Bi * Bj * vij + Ai * Aj * wij;
    O1[o + idx] = Bi * Aj * wij - Ai * Bj * vij;
  }
}

// DKH generator: W_ij = O_ij / (E0_i + E0_j).
__global__ void kin_div_kernel(int n, int nc, double c, const double *evals, const double *src, double *dst) {
  const int b = blockIdx.x / nc;
  const double *s = src + (int64_t)blockIdx.x * n * n;
  double *d = dst + (int64_t)blockIdx.x * n * n;
  const double *t = evals + (int64_t)b * n;
  FW_ELEMENTS(n) {
    const int i = (int)(idx / n), j = (int)(idx - (int64_t)i * n);
    double Ei, Ej, A, B, Ek;
    fw_factors(t[i], c, Ei, A, B, Ek);
    fw_factors(t[j], c, Ej, A, B, Ek);
    d[idx] = s[idx] / (Ei + Ej);
  }
}

// dst = alpha (src + src+): part 0 alpha (X + X^T), parts 1-3 alpha (X - X^T).
__global__ void herm_kernel(int n, int nc, double alpha, const double *src, double *dst) {
  const int q = blockIdx.x % nc;
  const double *s = src + (int64_t)blockIdx.x * n * n;
  double *d = dst + (int64_t)blockIdx.x * n * n;
  const double sgn = q == 0 ? 1.0 : -1.0;
  FW_ELEMENTS(n) {
    const int i = (int)(idx / n), j = (int)(idx - (int64_t)i * n);
    d[idx] = alpha * (s[idx] + sgn * s[(int64_t)j * n + i]);
  }
}

constexpr int kLinTerms = 8;
struct LinTerms {
  const double *src[kLinTerms];
  double coef[kLinTerms];
  int count;
  int accumulate;  // add to dst instead of writing it
};
// dst = (dst if accumulate) + sum coef_t src_t over whole problem x part blocks.
__global__ void lin_kernel(int64_t per, LinTerms L, double *dst) {
  const int64_t off = (int64_t)blockIdx.x * per;
  for (int64_t idx = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; idx < per;
       idx += (int64_t)gridDim.y * blockDim.x) {
    double v = L.accumulate ? dst[off + idx] : 0.0;
    for (int t = 0; t < L.count; ++t) v += L.coef[t] * L.src[t][off + idx];
    dst[off + idx] = v;
  }
}

// DKH Hamiltonian: part 0 diagonal += E0_i - c^2.
__global__ void add_free_diag_kernel(int n, int nc, double c, const double *evals, double *H) {
  const int b = blockIdx.x;
  double *h = H + (int64_t)b * nc * n * n;
  for (int i = blockIdx.y * blockDim.x + threadIdx.x; i < n; i += gridDim.y * blockDim.x) {
    double E0, A, B, Ek;
    fw_factors(evals[(int64_t)b * n + i], c, E0, A, B, Ek);
    h[(int64_t)i * n + i] += Ek;
  }
}

// U0 [top; bot]: L = A top - B bot, S = B top + A bot (row scalings).
__global__ void u0_apply_kernel(int n, int nc, double c, const double *evals, const double *top, const double *bot,
                                double *L, double *S) {
  const int b = blockIdx.x / nc;
  const int64_t o = (int64_t)blockIdx.x * n * n;
  const double *t = evals + (int64_t)b * n;
  FW_ELEMENTS(n) {
    const int i = (int)(idx / n);
    double E0, A, B, Ek;
    fw_factors(t[i], c, E0, A, B, Ek);
    L[o + idx] = A * top[o + idx] - B * bot[o + idx];
    S[o + idx] = B * top[o + idx] + A * bot[o + idx];
  }
}

// X_ij *= 2c / p_i (the 2c K p^-1 of U^S).
__global__ void row_scale_2cp_kernel(int n, int nc, double c, const double *evals, double *X) {
  const int b = blockIdx.x / nc;
  double *x = X + (int64_t)blockIdx.x * n * n;
  const double *t = evals + (int64_t)b * n;
  FW_ELEMENTS(n) {
    const int i = (int)(idx / n);
    x[idx] *= 2.0 * c / sqrt(2.0 * t[i]);
  }
}
#undef FW_ELEMENTS

template <class K, class... Args>
x2c_status fw_launch(x2c_ctx *ctx, cudaStream_t st, const char *name, K kernel, dim3 grid, Args... args) {
  tbegin(ctx, st);
  kernel<<<grid, 256, 0, st>>>(args...);
  return launched(ctx, name, st);
}

// The orthonormal kinetic basis of every problem: evals (t), K, K^-1, V~ and W~ (nc parts).
struct KineticBasis {
  double *fac, *inv, *evals, *QT, *K, *Kinv, *Vt, *Wt, *tmp;
};

size_t kinetic_bytes(int nb, int n, int nc) {  // arena_doubles(x) is the bytes of x doubles
  const size_t n2 = (size_t)n * n;
  return arena_doubles(4 * nb * n2) + arena_doubles((size_t)nb * n) + 4 * arena_doubles(nb * n2) +
         2 * arena_doubles(nb * nc * n2);
}

x2c_status kinetic_basis(x2c_ctx *ctx, cudaStream_t st, int nb, int n, int nc, const InputDesc *d_in, Arena &ar,
                         KineticBasis &kb) {
  const int64_t n2 = (int64_t)n * n;
  kb.fac = ar.take(2 * nb * n2);
  kb.inv = ar.take(2 * nb * n2);
  kb.evals = ar.take((size_t)nb * n);
  kb.QT = ar.take(nb * n2);
  kb.K = ar.take(nb * n2);
  kb.Kinv = ar.take(nb * n2);
  kb.Vt = ar.take(nb * n2);
  kb.Wt = ar.take(nb * nc * n2);
  kb.tmp = ar.take(nb * nc * n2);
  if (!kb.tmp) return X2C_ERR_NOMEM;
  int *status = ctx->d_status;
  const size_t smem = (size_t)n2 * sizeof(double);
  X2C_TRY_CUDA(ctx, cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  tbegin(ctx, st);
  chol_inv_kernel<<<2 * nb, 256, smem, st>>>(d_in, n, kb.fac, kb.inv, status);
  X2C_TRY(launched(ctx, "chol_inv_kernel", st));
  // t^ = L^-1 T L^-T (into Vt, used as scratch here)
  X2C_TRY((gemm_sq(ctx, st, nb, n, Mat<false>{kb.inv, n, 2 * n2, 1.0}, InputOp{d_in, 1, 1},
                   StoreAxpby{kb.tmp, nullptr, n, n2, 1.0, 0.0})));
  X2C_TRY((gemm_sq(ctx, st, nb, n, Mat<false>{kb.tmp, n, n2, 1.0}, Mat<true>{kb.inv, n, 2 * n2, 1.0},
                   StoreAxpby{kb.Vt, nullptr, n, n2, 1.0, 0.0})));
  const size_t jsmem = (n <= kJacobiSmemV ? 2 : 1) * smem;
  X2C_TRY_CUDA(ctx, cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)jsmem));
  tbegin(ctx, st);
  jacobi_kernel<<<nb, 256, jsmem, st>>>(kb.Vt, n, n2, kb.evals, kb.QT, status);
  X2C_TRY(launched(ctx, "jacobi_kernel", st));
  // K = L^-T Q,  K^-1 = Q^T L^T
  X2C_TRY((gemm_sq(ctx, st, nb, n, Mat<true>{kb.inv, n, 2 * n2, 1.0}, Mat<true>{kb.QT, n, n2, 1.0},
                   StoreAxpby{kb.K, nullptr, n, n2, 1.0, 0.0})));
  X2C_TRY((gemm_sq(ctx, st, nb, n, Mat<false>{kb.QT, n, n2, 1.0}, Mat<true>{kb.fac, n, 2 * n2, 1.0},
                   StoreAxpby{kb.Kinv, nullptr, n, n2, 1.0, 0.0})));
  // V~ = K^T V K;  W~_q = p^-1 K^T W_q K p^-1
  X2C_TRY((gemm_sq(ctx, st, nb, n, Mat<true>{kb.K, n, n2, 1.0}, InputOp{d_in, 2, 1},
                   StoreAxpby{kb.tmp, nullptr, n, n2, 1.0, 0.0})));
  X2C_TRY((gemm_sq(ctx, st, nb, n, Mat<false>{kb.tmp, n, n2, 1.0}, Mat<false>{kb.K, n, n2, 1.0},
                   StoreAxpby{kb.Vt, nullptr, n, n2, 1.0, 0.0})));
  X2C_TRY((gemm_sq(ctx, st, nb * nc, n, MatDiv<true>{kb.K, n, n2, nc, 1.0}, InputOp{d_in, 3, nc},
                   StoreAxpby{kb.tmp, nullptr, n, n2, 1.0, 0.0})));
  X2C_TRY((gemm_sq(ctx, st, nb * nc, n, Mat<false>{kb.tmp, n, n2, 1.0}, MatDiv<false>{kb.K, n, n2, nc, 1.0},
                   StoreAxpby{kb.Wt, nullptr, n, n2, 1.0, 0.0})));
  return fw_launch(ctx, st, "fw_elementwise", scale_pp_kernel, aux_grid(nb * nc, n2), n, nc,
                   (const double *)kb.evals, kb.Wt);
}

// U^L = K Y_L K^-1, U^S = 2c K p^-1 Y_S K^-1 (Y_S scaled in place).
x2c_status kinetic_back(x2c_ctx *ctx, cudaStream_t st, int nb, int n, int nc, double c, const KineticBasis &kb,
                        const double *YL, double *YS, double *UL, double *US) {
  const int64_t n2 = (int64_t)n * n;
  X2C_TRY(fw_launch(ctx, st, "fw_elementwise", row_scale_2cp_kernel, aux_grid(nb * nc, n2), n, nc, c,
                    (const double *)kb.evals, YS));
  const double *src[2] = {YL, YS};
  double *dst[2] = {UL, US};
  for (int w = 0; w < 2; ++w) {
    X2C_TRY((gemm_sq(ctx, st, nb * nc, n, MatDiv<false>{kb.K, n, n2, nc, 1.0}, Mat<false>{src[w], n, n2, 1.0},
                     StoreAxpby{kb.tmp, nullptr, n, n2, 1.0, 0.0})));
    X2C_TRY((gemm_sq(ctx, st, nb * nc, n, Mat<false>{kb.tmp, n, n2, 1.0}, MatDiv<false>{kb.Kinv, n, n2, nc, 1.0},
                     StoreAxpby{dst[w], nullptr, n, n2, 1.0, 0.0})));
  }
  return X2C_OK;
}

// Run a DKH plan's operations on slot buffers (slot s of every problem at slot0 + s nb nc n^2).
x2c_status run_dkh_ops(x2c_ctx *ctx, cudaStream_t st, int nb, int n, int nc, double c, const double *evals,
                       const std::vector<dkh::Op> &ops, double *slot0, size_t from) {
  const int64_t per = (int64_t)nc * n * n, sl = (int64_t)nb * per;
  auto S = [&](int s) { return slot0 + s * sl; };
  for (size_t i = from; i < ops.size(); ++i) {
    const dkh::Op &op = ops[i];
    switch (op.type) {
      case dkh::kGemm:
        X2C_TRY(quat_product_op(ctx, st, nb, n, nc, op.adj_a, op.adj_b, S(op.a), S(op.b), S(op.dst), op.alpha, op.beta,
                                "dkh_gemm"));
        break;
      case dkh::kHerm:
        X2C_TRY(fw_launch(ctx, st, "fw_elementwise", herm_kernel, aux_grid(nb * nc, (int64_t)n * n), n, nc, op.alpha,
                          (const double *)S(op.a), S(op.dst)));
        break;
      case dkh::kKin:
        X2C_TRY(fw_launch(ctx, st, "fw_elementwise", kin_div_kernel, aux_grid(nb * nc, (int64_t)n * n), n, nc, c,
                          evals, (const double *)S(op.a), S(op.dst)));
        break;
      default: {
        for (size_t t0 = 0; t0 < op.lin.size(); t0 += kLinTerms) {
          LinTerms L{};
          L.count = (int)std::min<size_t>(kLinTerms, op.lin.size() - t0);
          L.accumulate = t0 > 0;
          for (int t = 0; t < L.count; ++t) {
            L.src[t] = S(op.lin[t0 + t].second);
            L.coef[t] = op.lin[t0 + t].first;
          }
          X2C_TRY(fw_launch(ctx, st, "fw_elementwise", lin_kernel, aux_grid(nb, per), per, L, S(op.dst)));
        }
      }
    }
  }
  return X2C_OK;
}

}  // namespace

bool fw_supported(int n, int decoupling) {
  return decoupling >= 1 && decoupling <= kMaxDkhOrder && n >= 1 && n <= kMaxJacobiN;
}

// Slots of the DKH plan for transforms (order k generators up to `order`).
static dkh::Plan dkh_transform_plan(int order) {
  dkh::Plan p(order);
  for (int k = 1; k <= order; ++k)
    if (!p.transform(k)) break;
  p.generator_slots();
  return p;
}

size_t solve_fw_workspace_bytes(int nb, int n, int nc, int decoupling) {
  const size_t n2 = (size_t)n * n, q = nb * nc * n2;
  size_t d = kinetic_bytes(nb, n, nc) + 12 * arena_doubles(q);
  if (decoupling == 1) {
    const size_t d4 = 4 * n2;
    d += arena_doubles(nb * n2) + 3 * arena_doubles(nb * nc * d4) + 2 * arena_doubles(nb) +
         arena_doubles((size_t)nb * kSignMaxSteps) + arena_doubles(1) +
         arena_doubles(std::max(quat_part_doubles(nb, 2 * n, nc), quat_part_doubles(nb, n, nc)));
  } else {
    const dkh::Plan p = dkh_transform_plan(decoupling);
    d += (size_t)p.slots() * arena_doubles(q) + 8 * arena_doubles(q) + 2 * arena_doubles(nb) +
         arena_doubles(quat_part_doubles(nb, n, nc));
  }
  return d + 64 * 256;
}

x2c_status solve_transforms_fw(x2c_ctx *ctx, cudaStream_t st, double c, int nb, int n, int nc, int decoupling,
                               const InputDesc *d_in, double *UL, double *US, Arena ar) {
  if (nb <= 0) return X2C_OK;
  if (!fw_supported(n, decoupling)) return X2C_ERR_ARG;
  const int64_t n2 = (int64_t)n * n, q = (int64_t)nb * nc * n2;
  int *status = ctx->d_status;
  KineticBasis kb{};
  X2C_TRY(kinetic_basis(ctx, st, nb, n, nc, d_in, ar, kb));
  double *YL = ar.take(q), *YS = ar.take(q), *G = ar.take(q), *Yk = ar.take(q), *Zk = ar.take(q), *Tm = ar.take(q);
  double *Yk2 = ar.take(q), *Zk2 = ar.take(q), *UpL = ar.take(q), *UpS = ar.take(q);
  auto *slot = reinterpret_cast<unsigned long long *>(ar.take(nb));
  double *trace = ar.take(nb);
  if (!trace) return X2C_ERR_NOMEM;
  const dim3 eg = aux_grid(nb * nc, n2);
  if (decoupling == 1) {  // BSS
    const int64_t d2 = 4 * n2;
    double *LSm = ar.take(nb * n2), *Z = ar.take(nb * nc * d2), *Zn = ar.take(nb * nc * d2), *Y = ar.take(nb * nc * d2);
    double *sched = ar.take((size_t)nb * kSignMaxSteps);
    int *gate = reinterpret_cast<int *>(ar.take(1));
    const size_t part_n = std::max(quat_part_doubles(nb, 2 * n, nc), quat_part_doubles(nb, n, nc));
    double *part = part_n ? ar.take(part_n) : nullptr;
    if (!gate || (part_n && !part)) return X2C_ERR_NOMEM;
    X2C_TRY(fw_launch(ctx, st, "fw_elementwise", coupling_diag_kernel, aux_grid(nb, n2), n, c,
                      (const double *)kb.evals, LSm));
    X2C_TRY(sign_of_hp(ctx, st, nb, n, nc, c, kb.Vt, LSm, kb.Wt, Z, Zn, Y, slot, trace, sched, gate, part, status));
    X2C_TRY(fw_launch(ctx, st, "fw_elementwise", bss_ref_kernel, eg, n, nc, c, (const double *)kb.evals,
                      (const double *)Z, YL, YS));
    X2C_TRY(fw_launch(ctx, st, "fw_elementwise", bss_gram_kernel, eg, n, nc, c, (const double *)kb.evals,
                      (const double *)YL, (const double *)YS, G));
    X2C_TRY(coupled_sqrt(ctx, st, nb, n, nc, G, Yk, Zk, Tm, Yk2, Zk2, part, slot, status));
    X2C_TRY(quat_product_op(ctx, st, nb, n, nc, false, false, YL, Zk, UpL, 1.0, 0.0, "solve_quat_gemm"));
    X2C_TRY(quat_product_op(ctx, st, nb, n, nc, false, false, YS, Zk, UpS, 1.0, 0.0, "solve_quat_gemm"));
    return kinetic_back(ctx, st, nb, n, nc, c, kb, UpL, UpS, UL, US);
  }
  // DKHn: generators W_1 .. W_n, then exp(-W_1) ... exp(-W_n) [1; 0]
  const int order = decoupling;
  dkh::Plan plan = dkh_transform_plan(order);
  const auto gens = plan.generator_slots();
  double *slots = ar.take((size_t)plan.slots() * q);
  double *top = ar.take(q), *bot = ar.take(q), *ta = ar.take(q), *tb = ar.take(q), *na = ar.take(q),
         *nbt = ar.take(q), *acc_a = ar.take(q), *acc_b = ar.take(q);
  const size_t part_n = quat_part_doubles(nb, n, nc);
  double *part = part_n ? ar.take(part_n) : nullptr;
  if (!acc_b || (part_n && !part)) return X2C_ERR_NOMEM;
  X2C_TRY(fw_launch(ctx, st, "fw_elementwise", fw_blocks_kernel, eg, n, nc, c, (const double *)kb.evals,
                    (const double *)kb.Vt, (const double *)kb.Wt, slots + dkh::Plan::kSlotE1 * q,
                    slots + dkh::Plan::kSlotE1p * q, slots + dkh::Plan::kSlotO1 * q));
  X2C_TRY(run_dkh_ops(ctx, st, nb, n, nc, c, kb.evals, plan.ops(), slots, 0));
  X2C_TRY(fw_launch(ctx, st, "identity_kernel", identity_kernel, aux_grid(nb, nc * n2), n, nc, top));
  X2C_TRY(device_fill(ctx, st, bot, 0, sizeof(double) * q));
  const int64_t per = (int64_t)nc * n2;
  for (auto it = gens.rbegin(); it != gens.rend(); ++it) {
    const int k = it->first;
    const double *W = slots + (int64_t)it->second * q;
    // acc = Y; term = Y; for i = 1 .. order/k: term <- -(W term)/i, acc += term, where
    // W [a; b] = [W b; -W+ a]
    X2C_TRY(device_copy(ctx, st, acc_a, top, sizeof(double) * q));
    X2C_TRY(device_copy(ctx, st, acc_b, bot, sizeof(double) * q));
    const double *pa = top, *pb = bot;
    for (int i = 1; i <= order / k; ++i) {
      X2C_TRY(quat_product_op(ctx, st, nb, n, nc, false, false, W, pb, na, -1.0 / i, 0.0, "dkh_gemm"));
      X2C_TRY(quat_product_op(ctx, st, nb, n, nc, true, false, W, pa, nbt, 1.0 / i, 0.0, "dkh_gemm"));
      LinTerms L{};
      L.count = 1;
      L.accumulate = 1;
      L.coef[0] = 1.0;
      L.src[0] = na;
      X2C_TRY(fw_launch(ctx, st, "fw_elementwise", lin_kernel, aux_grid(nb, per), per, L, acc_a));
      L.src[0] = nbt;
      X2C_TRY(fw_launch(ctx, st, "fw_elementwise", lin_kernel, aux_grid(nb, per), per, L, acc_b));
      std::swap(na, ta);
      std::swap(nbt, tb);
      pa = ta;
      pb = tb;
    }
    std::swap(top, acc_a);
    std::swap(bot, acc_b);
  }
  // R'' = (Y+ Y)^-1/2;  U = U0 Y R''
  X2C_TRY(quat_product_op(ctx, st, nb, n, nc, true, false, top, top, G, 1.0, 0.0, "solve_quat_gemm"));
  X2C_TRY(quat_product_op(ctx, st, nb, n, nc, true, false, bot, bot, G, 1.0, 1.0, "solve_quat_gemm"));
  X2C_TRY(fw_launch(ctx, st, "fw_elementwise", herm_kernel, eg, n, nc, 0.5, (const double *)G, Tm));
  X2C_TRY(coupled_sqrt(ctx, st, nb, n, nc, Tm, Yk, Zk, G, Yk2, Zk2, part, slot, status));
  X2C_TRY(fw_launch(ctx, st, "fw_elementwise", u0_apply_kernel, eg, n, nc, c, (const double *)kb.evals,
                    (const double *)top, (const double *)bot, YL, YS));
  X2C_TRY(quat_product_op(ctx, st, nb, n, nc, false, false, YL, Zk, UpL, 1.0, 0.0, "solve_quat_gemm"));
  X2C_TRY(quat_product_op(ctx, st, nb, n, nc, false, false, YS, Zk, UpS, 1.0, 0.0, "solve_quat_gemm"));
  return kinetic_back(ctx, st, nb, n, nc, c, kb, UpL, UpS, UL, US);
}

size_t dkh_hamiltonian_workspace_bytes(int n, int nc, int order) {
  dkh::Plan p(order);
  for (int k = 1; k <= order / 2; ++k) p.transform(k);
  p.hamiltonian_slots();
  const size_t q = (size_t)nc * n * n;
  return kinetic_bytes(1, n, nc) + (size_t)(p.slots() + 2) * arena_doubles(q) + 64 * 256;
}

x2c_status dkh_hamiltonian(x2c_ctx *ctx, cudaStream_t st, double c, int n, int nc, int order, const InputDesc *d_in,
                           double *const *h, Arena ar) {
  if (!fw_supported(n, order) || order < 2) return X2C_ERR_ARG;
  const int64_t n2 = (int64_t)n * n, q = (int64_t)nc * n2;
  KineticBasis kb{};
  X2C_TRY(kinetic_basis(ctx, st, 1, n, nc, d_in, ar, kb));
  dkh::Plan plan(order);
  for (int k = 1; k <= order / 2; ++k) plan.transform(k);
  const std::vector<int> terms = plan.hamiltonian_slots();
  double *slots = ar.take((size_t)plan.slots() * q), *H = ar.take(q), *out = ar.take(q);
  if (!out) return X2C_ERR_NOMEM;
  const dim3 eg = aux_grid(nc, n2);
  X2C_TRY(fw_launch(ctx, st, "fw_elementwise", fw_blocks_kernel, eg, n, nc, c, (const double *)kb.evals,
                    (const double *)kb.Vt, (const double *)kb.Wt, slots + dkh::Plan::kSlotE1 * q,
                    slots + dkh::Plan::kSlotE1p * q, slots + dkh::Plan::kSlotO1 * q));
  X2C_TRY(run_dkh_ops(ctx, st, 1, n, nc, c, kb.evals, plan.ops(), slots, 0));
  // H = E0 - c^2 + sum_l E_l (upper blocks)
  X2C_TRY(device_fill(ctx, st, H, 0, sizeof(double) * q));
  for (size_t t0 = 0; t0 < terms.size(); t0 += kLinTerms) {
    LinTerms L{};
    L.count = (int)std::min<size_t>(kLinTerms, terms.size() - t0);
    L.accumulate = 1;
    for (int t = 0; t < L.count; ++t) {
      L.src[t] = slots + (int64_t)terms[t0 + t] * q;
      L.coef[t] = 1.0;
    }
    X2C_TRY(fw_launch(ctx, st, "fw_elementwise", lin_kernel, aux_grid(1, q), q, L, H));
  }
  X2C_TRY(fw_launch(ctx, st, "fw_elementwise", add_free_diag_kernel, dim3(1, 1), n, nc, c, (const double *)kb.evals, H));
  // h = (K^-1)^T H K^-1 per part
  X2C_TRY((gemm_sq(ctx, st, nc, n, MatDiv<true>{kb.Kinv, n, n2, nc, 1.0}, Mat<false>{H, n, n2, 1.0},
                   StoreAxpby{kb.tmp, nullptr, n, n2, 1.0, 0.0})));
  X2C_TRY((gemm_sq(ctx, st, nc, n, Mat<false>{kb.tmp, n, n2, 1.0}, MatDiv<false>{kb.Kinv, n, n2, nc, 1.0},
                   StoreAxpby{out, nullptr, n, n2, 1.0, 0.0})));
  for (int p = 0; p < nc; ++p)
    X2C_TRY(device_copy(ctx, st, h[p], out + p * n2, sizeof(double) * n2));
  return X2C_OK;
}
