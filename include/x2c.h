/*
 * x2c.h -- C ABI of the GB300 exact-decoupling (X2C) one-electron Hamiltonian library.
 *
 * Method: Peng, Middendorf, Weigend, Reiher, J. Chem. Phys. 138, 184105 (2013).
 * Given the primitive-basis matrices S, T, V and W (Sec. II, Eqs. 4-6) the library
 * returns the decoupled two-component (or scalar) Hamiltonian h of Eq. 8, either for the
 * whole system (X2C, Sec. II.A) or in the local DLU scheme (Sec. III.A, Eqs. 42-43), where
 * atomic U^L_AA, U^S_AA are computed once per atom kind and every pair block
 * h_AB = U^L_A+ V_AB U^L_B + U^L_A+ T_AB U^S_B + U^S_A+ T_AB U^L_B + U^S_A+ W'_AB U^S_B
 * (W' = W/4c^2 - T) is assembled from them.
 *
 * Conventions shared by every call
 *  - Matrices are FP64, row-major, n x n, with leading dimension n, in DEVICE memory unless
 *    a function says otherwise.  They are owned by the caller; the library never frees them.
 *  - Two-component matrices use the time-reversal (quaternion) form of Eq. 5:
 *        M = I2 (x) M0 + i (sigma_x (x) Mx + sigma_y (x) My + sigma_z (x) Mz),
 *    spin-blocked (alpha block first); M0, Mx, My, Mz are real n x n.  For W these are
 *    W0, Wx, Wy, Wz of Eq. 6 (W0 symmetric, Wx/Wy/Wz antisymmetric).  The output h is
 *    returned the same way: h0 (symmetric) and h1, h2, h3 (antisymmetric); the dense
 *    2n x 2n complex matrix is [[h0 + i h3, h2 + i h1], [-h2 + i h1, h0 - i h3]].
 *  - Calls are asynchronous on the caller's CUDA stream (passed as void*, NULL = the legacy
 *    default stream).  A non-OK return means nothing was enqueued or the enqueue failed.
 *    Numerical failures detected on the device (Cholesky pivot <= 0, non-convergence,
 *    failed positive/negative-energy split, non-finite values) are latched in the context
 *    and returned by x2c_ctx_status(), which synchronises the stream.
 *  - A context is bound to one device and is not thread-safe; use one per host thread.
 *    It owns a device workspace that grows on demand (the first call of a larger size
 *    allocates) and is freed by x2c_ctx_destroy().  A split-precision DLU assembly asks for
 *    up to 24 GiB (Ag309 two-component: about 17 GB, one chunk); if that cannot be
 *    allocated, the context falls back to chunks of 3 GiB for the rest of its life.
 *  - No function aborts, traps or exits; errors are returned as x2c_status.
 */
#ifndef X2C_H
#define X2C_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  X2C_OK = 0,
  X2C_ERR_ARG = 1,         /* invalid argument: NULL pointer, size out of range, bad option */
  X2C_ERR_NOMEM = 2,       /* device or pinned-host allocation failed */
  X2C_ERR_CUDA = 3,        /* a CUDA runtime call failed (see x2c_last_error_message) */
  X2C_ERR_NOT_POSDEF = 4,  /* S or T not positive definite (Cholesky pivot <= 0) */
  X2C_ERR_NOCONV = 5,      /* sign-function or matrix-square-root iteration did not converge */
  X2C_ERR_DECOUPLING = 6,  /* spectrum does not split at -c^2 into equal halves (Sec. II) */
  X2C_ERR_NONFINITE = 7,   /* NaN or Inf met in a result */
  X2C_ERR_ADMISSION = 8,   /* serving: request can never fit the memory budget */
  X2C_ERR_TIMEOUT = 9,     /* serving: wait timed out (the request keeps running) */
  X2C_ERR_CANCELLED = 10,  /* serving: request was cancelled */
  X2C_ERR_NOT_FOUND = 11   /* serving: unknown ticket */
} x2c_status;

typedef enum {
  X2C_PREC_FP64 = 0,       /* every product in FP64 */
  X2C_PREC_SPLIT_BF16 = 1  /* DLU pair assembly as split-precision (Ozaki) BF16 products
                              with FP32 accumulation on the tensor cores; every eigen-type
                              step (sign function, square roots, Cholesky) stays FP64.  The
                              assembly shares operands per class of pairs with the same
                              (U_A, U_B): at most 64 classes per build (free-atom mode: kinds
                              squared; molecular-block mode, one U per atom: up to ten atoms
                              in DLU, 64 in DLH), else X2C_ERR_ARG */
} x2c_precision;

typedef enum {
  X2C_DLU_FREE_ATOM = 0,      /* U_AA from each kind's free-atom inputs (x2c_layout.kinds) */
  X2C_DLU_MOLECULAR_BLOCK = 1 /* U_AA from the diagonal blocks S_AA, T_AA, V_AA, W_AA of the
                                 molecular matrices (Eq. 43 read literally); one solve per atom */
} x2c_dlu_potential;

/* The exact-decoupling or approximate transformation behind U^L, U^S (Sec. II):
 *  X2C_DEC_X2C  (0)  X2C, Sec. II.A: the X-operator transform of the positive-energy solutions.
 *  X2C_DEC_BSS  (1)  BSS, Sec. II.B: the same solutions reached through the free-particle
 *                    transformation first; exact decoupling in another unitary frame (same
 *                    eigenvalues as X2C, a different h).
 *  n = 2..14         DKHn, Sec. II.C: exponential parametrisation cut at order n in the
 *                    potential, with the operation count of Table I.  Full builds return the
 *                    DKHn Hamiltonian E0 - c^2 + sum_{l<=n} E_l; the transforms (atomic ones for
 *                    DLU, U of x2c_build_full) are the columns exp(-W_1) ... exp(-W_n) [1; 0]
 *                    cut at order n and renormalised (Eq. 9 holds).
 * BSS and DKHn diagonalise T in the metric S (Eq. 11) on the device, one CTA per matrix: they
 * take problems of n <= 160 functions (atoms for DLU; whole systems up to that size for full
 * builds); larger ones return X2C_ERR_ARG.  x2c_atomic_transforms_noalloc takes X2C only. */
typedef enum { X2C_DEC_X2C = 0, X2C_DEC_BSS = 1, X2C_DEC_DKH2 = 2 } x2c_decoupling;
#define X2C_DEC_MAX_DKH_ORDER 14

typedef enum {
  X2C_LOCAL_DLU = 0,  /* every pair block h_AB from the atomic transforms (Eq. 42 in Eq. 8) */
  X2C_LOCAL_DLH = 1   /* diagonal local Hamiltonian (Sec. III.A): only the same-atom blocks
                         h_AA are transformed (as in DLU); every atom-other-atom block is the
                         non-relativistic T_AB + V_AB (spin parts zero) */
} x2c_local_approx;

typedef struct {
  double c;                  /* speed of light (a.u.); <= 0 selects 137.035999 */
  int32_t two_component;     /* 0 = scalar (spin-free), 1 = two-component with Wx, Wy, Wz */
  int32_t precision;         /* x2c_precision */
  int32_t dlu_potential;     /* x2c_dlu_potential */
  int32_t so_same_atom_only; /* 1: Wx, Wy, Wz vanish outside same-atom blocks, so DLU reads
                                only those blocks and skips the rest (two-component only) */
  int32_t n_slices;          /* split precision: BF16 slices per operand, 0 = default (5) */
  int32_t local_approx;      /* x2c_local_approx of the DLU calls (ignored by full X2C) */
  int32_t h_upper_only;      /* x2c_build_dlu_host only: 1 = copy each h part back on its upper
                                block triangle (blocks A <= B) instead of whole: h0 is symmetric
                                and h1..h3 are antisymmetric, so the lower blocks follow from
                                the upper ones; this halves the device-to-host copy.  Blocks
                                below the diagonal are not written, except that some near the
                                diagonal (within the row bands the call copies at once) may
                                receive their values.  Other calls: must be 0 */
  int32_t decoupling;        /* x2c_decoupling: the decoupling transformation (default 0 = X2C) */
} x2c_options;

typedef struct {
  int32_t n;                       /* number of scalar basis functions */
  const double *S, *T, *V, *W0;    /* n x n symmetric */
  const double *Wx, *Wy, *Wz;      /* n x n antisymmetric; NULL when spin-free */
} x2c_mats;

typedef struct {
  double *h[4];    /* h0 (n x n), then h1, h2, h3 for two-component (NULL if spin-free) */
} x2c_hout;

typedef struct {
  double *UL[4];   /* U^L components (quaternion form, as h); UL[0] only if spin-free */
  double *US[4];   /* U^S components */
} x2c_uout;

typedef struct {
  int32_t n_atoms;
  const int32_t *atom_offset;  /* HOST array, n_atoms + 1 entries: first function of each
                                  atom, atom_offset[n_atoms] = n; atom-major basis order */
  const int32_t *atom_kind;    /* HOST array, n_atoms entries: index into kinds */
  int32_t n_kinds;
  const x2c_mats *kinds;       /* HOST array of n_kinds free-atom input sets (device
                                  matrices, sizes must match the atoms of that kind);
                                  ignored in X2C_DLU_MOLECULAR_BLOCK mode */
} x2c_layout;

typedef struct x2c_ctx x2c_ctx;

/* Create a context on CUDA device `device`.  Returns X2C_ERR_ARG for a bad device. */
x2c_status x2c_ctx_create(int device, x2c_ctx **out);

/* Destroy a context: waits for its work and frees its workspace.  NULL is allowed. */
x2c_status x2c_ctx_destroy(x2c_ctx *ctx);

/* Synchronise `stream`, return (and clear) the first device-side error latched since the
 * last call, else X2C_OK. */
x2c_status x2c_ctx_status(x2c_ctx *ctx, void *stream);

/* Static description of a status code. */
const char *x2c_status_string(x2c_status s);

/* Text of the last CUDA error seen by this context (empty if none). */
const char *x2c_last_error_message(x2c_ctx *ctx);

/* Full X2C (Sec. II.A): h of the whole system, and optionally U^L, U^S (Eq. 22) for
 * picture-change transformations (U may be NULL).  mol: device matrices.  Limits: n >= 1;
 * the library keeps O(n^2) workspace (about 60 n^2 doubles spin-free, 200 n^2 two-component). */
x2c_status x2c_build_full(x2c_ctx *ctx, const x2c_options *opt, const x2c_mats *mol,
                          const x2c_hout *h, const x2c_uout *U, void *stream);

/* DLU (Sec. III.A, Eqs. 42-43 with Eq. 8): h of the molecule from atomic transforms.
 * mol: the molecular matrices; only the blocks the method needs are read (V, T, W0 on
 * every pair block A <= B, the same-atom blocks of S, T, V, W for molecular-block mode, and
 * Wx, Wy, Wz on same-atom blocks only when so_same_atom_only = 1).  Atoms may have any
 * size >= 1; kinds must have the size of their atoms. */
x2c_status x2c_build_dlu(x2c_ctx *ctx, const x2c_options *opt, const x2c_layout *layout,
                         const x2c_mats *mol, const x2c_hout *h, void *stream);

/* Neighbouring-atomic-blocks approximation (named at the end of Sec. III.A as the way to
 * linear scaling; the paper does not spell it out): the pair blocks of neighbouring atoms are
 * assembled as in x2c_build_dlu (Eq. 42 in Eq. 8), every other atom-other-atom block is the
 * non-relativistic T_AB + V_AB with zero spin parts, as in DLH.  neighbours: HOST array of
 * n_atoms x n_atoms bytes, row-major; atoms A != B are neighbours when
 * neighbours[A n_atoms + B] or neighbours[B n_atoms + A] is non-zero (the caller's criterion:
 * a distance cutoff, an overlap threshold, ...); same-atom blocks are always transformed.  All
 * non-zero gives DLU, all zero DLH.  opt->local_approx must be X2C_LOCAL_DLU.  Reads T and V
 * on every block (W0 and the spin parts as DLU does on the neighbouring blocks). */
x2c_status x2c_build_dlu_nab(x2c_ctx *ctx, const x2c_options *opt, const x2c_layout *layout,
                             const x2c_mats *mol, const uint8_t *neighbours, const x2c_hout *h,
                             void *stream);

/* Pair-list partition of a DLU build over several GPUs (Sec. III.A: the pair blocks h_AB of
 * Eqs. 42-43 are independent, and the per-kind transforms are small enough to solve on every
 * GPU).  Rank `rank` of `world` is given the row atoms [*a_begin, *a_end): consecutive ranges
 * over 0..n_atoms, disjoint, covering every atom, with about equal shares of the work of the
 * upper block triangle (row atom A carries its blocks (A, B >= A), each weighted by
 * n_A n_B (n_A + n_B)).  A range may be empty (*a_begin == *a_end) when world > n_atoms.
 * Host-only: reads layout->atom_offset; no device work, no context. */
x2c_status x2c_dlu_partition(const x2c_layout *layout, int32_t rank, int32_t world, int32_t *a_begin,
                             int32_t *a_end);

/* One rank's share of a partitioned DLU build: as x2c_build_dlu, but only the pair blocks
 * (A, B >= A) with row atom A in [a_begin, a_end) are assembled (h_AB, and its mirror h_BA
 * for B > A); every other block of h is left as it was.  The per-kind transforms are solved
 * in full.  a_begin < a_end <= n_atoms, else X2C_ERR_ARG. */
x2c_status x2c_build_dlu_rows(x2c_ctx *ctx, const x2c_options *opt, const x2c_layout *layout,
                              const x2c_mats *mol, const x2c_hout *h, int32_t a_begin, int32_t a_end,
                              void *stream);

/* Batched DLU: n_mol independent molecules in one pass (one per-kind solve for the whole
 * batch and one grouped pair-assembly launch over all molecules' pair blocks).
 * layouts, mols, h: HOST arrays of n_mol entries. */
x2c_status x2c_build_dlu_batched(x2c_ctx *ctx, const x2c_options *opt, int32_t n_mol,
                                 const x2c_layout *layouts, const x2c_mats *mols,
                                 const x2c_hout *h, void *stream);

/* DLU (free-atom mode) from given atomic transforms: kind_U (HOST array, layout->n_kinds
 * entries, device matrices of the kinds' sizes, e.g. from x2c_atomic_transforms) replaces the
 * per-kind solve, and h is assembled from them exactly as in x2c_build_dlu (Eq. 42 with the
 * U_AA of Eq. 43 given).  Only layout->kinds[k].n is read from the kinds' input sets.
 * The transforms are copied into the context's staging area first (the staging area grows,
 * synchronising the device, when a larger call comes). */
x2c_status x2c_build_dlu_with_transforms(x2c_ctx *ctx, const x2c_options *opt, const x2c_layout *layout,
                                         const x2c_uout *kind_U, const x2c_mats *mol, const x2c_hout *h,
                                         void *stream);

/* Picture-change transformation of a one-electron property operator (Sec. II: the
 * decoupling transforms are kept for this): for an operator with no large-small coupling
 * (P^LS = 0, e.g. a multiplicative potential such as an electric field gradient or a contact
 * density) whose large- and small-component matrices in the primitive basis are P^LL and
 * P^SS, the two-component operator is
 *     P2c = U^L+ P^LL U^L + U^S+ P^SS U^S      (Eq. 8 with the property in place of D).
 * U^L, U^S: block-diagonal over the layout's atoms from kind_U (as in
 * x2c_build_dlu_with_transforms; DLU, Eq. 42), or the full-X2C transforms of
 * x2c_build_full(want_U) with a one-atom layout spanning the basis.  P^SS is quaternion-real
 * like W (Eq. 5): SS[0] symmetric, SS[1..3] antisymmetric spin parts (two-component; NULL
 * for a spin-free operator); P^LL is spin-free.  out: the quaternion parts of P2c (as h).
 * opt->c is ignored (the transforms carry it); precision, two_component and
 * so_same_atom_only apply as in the DLU calls (with so_same_atom_only = 1 the SS spin parts
 * are read on same-atom blocks only).  Device matrices, n x n, leading dimension n. */
typedef struct {
  int32_t n;
  const double *LL;     /* n x n symmetric */
  const double *SS[4];  /* SS[0] n x n symmetric; SS[1..3] antisymmetric or NULL */
} x2c_property;
x2c_status x2c_picture_change(x2c_ctx *ctx, const x2c_options *opt, const x2c_layout *layout,
                              const x2c_uout *kind_U, const x2c_property *P, const x2c_hout *out,
                              void *stream);

/* The input matrices over primitive s Gaussians g(r) = (2a/pi)^{3/4} exp(-a |r - A|^2) with
 * point nuclei, computed on the device (Sec. II: the modified Dirac equation needs S, T, V
 * and W; for s functions W is its scalar part W0 = sum_k p_k V p_k, the spin-orbit parts
 * vanish): S overlap, T kinetic energy, V nuclear attraction, W0 = <grad g_a|V|grad g_b>, in
 * closed form with the Boys functions F0, F1, F2.  All arrays are device memory: nuc_xyz
 * (3 n_nuc, bohr), nuc_z (n_nuc charges), bf_xyz (3 n centres), bf_alpha (n exponents);
 * outputs n x n row-major, exactly symmetric; any output may be NULL.  n_nuc <= 1536.
 * Asynchronous on `stream`; X2C_ERR_ARG for bad arguments. */
typedef struct {
  int32_t n_nuc;
  int32_t n;
  const double *nuc_xyz;
  const double *nuc_z;
  const double *bf_xyz;
  const double *bf_alpha;
} x2c_s_basis;
x2c_status x2c_s_integrals(const x2c_s_basis *basis, double *S, double *T, double *V, double *W0, void *stream);

/* Atomic (or any) decoupling transforms U^L, U^S of n_problems independent input sets in
 * one batched solve (the matrix function of Eq. 43).  inputs, U: HOST arrays. */
x2c_status x2c_atomic_transforms(x2c_ctx *ctx, const x2c_options *opt, int32_t n_problems,
                                 const x2c_mats *inputs, const x2c_uout *U, void *stream);

/* Size of the fixed device scratch array used by x2c_atomic_transforms_noalloc (32 MiB). */
#define X2C_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)

/* x2c_atomic_transforms without any device allocation, for callers that cannot call
 * cudaMalloc: code whose device memory is owned by another allocator (a serving process or
 * framework that reserved its memory budget up front), or that must not let an allocation
 * synchronise the device.  The paper has no counterpart; this is an interface variant of
 * the batched decoupling solve (same kernels, same results as x2c_atomic_transforms).
 *
 * No context is needed.  Scratch lives in one file-scope device array of
 * X2C_NOALLOC_SCRATCH_BYTES that every GPU loading this library holds until the process
 * exits.  The caller passes inputs and outputs (device pointers, as x2c_atomic_transforms);
 * all n_problems input sets must have the same n.  The call calls no cudaMalloc, cudaFree or
 * allocating library routine.  It returns X2C_ERR_NOMEM, before enqueueing anything, when the
 * problems need more scratch than the array holds: about 8 (2 nc + 6 + 23 nc) n^2 bytes per
 * problem plus about 6 KB (nc = 1 spin-free, 4 two-component): e.g. about 16 two-component
 * problems of n = 48, or 58 spin-free ones.
 *
 * The first call on a device looks up the array's device address (once per device, with
 * that device current, and again if that device's context was re-created); make that first
 * call before any stream capture.  That lookup may load the library's device module, which
 * holds the array: if device memory is already exhausted the first call fails with
 * X2C_ERR_CUDA (not X2C_ERR_NOMEM, which only reports a request larger than the array).
 * The call is synchronous: it waits for `stream` and returns the device-side status of this
 * call (X2C_ERR_NOT_POSDEF, X2C_ERR_NOCONV, ...).  Every call shares the one array, which keeps the
 * last call's contents; calls that overlap on the GPU (other host threads, other streams)
 * race on it and must be serialised by the caller. */
x2c_status x2c_atomic_transforms_noalloc(const x2c_options *opt, int32_t n_problems,
                                         const x2c_mats *inputs, const x2c_uout *U,
                                         void *stream);

/* DLU from HOST buffers (pageable or pinned): copies the inputs the method reads to the
 * device, builds, and copies h back into the caller's host buffers, all on `stream`;
 * returns after the stream has finished.  Arguments as x2c_build_dlu, but every matrix
 * pointer (mol, kinds, h) is a host pointer.  Only what the build reads crosses to the
 * device: the upper block triangle (blocks A <= B) of T, V and W0 (DLH: T and V whole, the
 * same-atom blocks of W0), the same-atom blocks of S (molecular-block mode) and of Wx, Wy,
 * Wz (so_same_atom_only = 1; else their upper block triangle); h comes back whole, or on its
 * upper block triangle (h_upper_only).  Free-atom DLU runs as a pipeline over row-atom chunks
 * (chunk k+1 copies in and chunk k-1 copies out while chunk k is assembled); a chunk's rows
 * cross as one band from its first column on, so a few blocks just below the diagonal are
 * copied too (the build does not read them). */
x2c_status x2c_build_dlu_host(x2c_ctx *ctx, const x2c_options *opt, const x2c_layout *layout,
                              const x2c_mats *mol, const x2c_hout *h, void *stream);

/* Dense spin-blocked 2n x 2n complex matrix (interleaved re, im; row-major) from the
 * quaternion parts h0..h3 (device).  out: device, 8 n^2 doubles. */
x2c_status x2c_quaternion_to_dense(const double *const h[4], int32_t n, double *out,
                                   void *stream);

/* Device workspace a build would need, without running it (for callers that budget device
 * memory; a context grows its workspace to this size on that build).  n_mol >= 1: DLU builds
 * of x2c_build_dlu_batched's arguments (layouts, mols: HOST arrays of n_mol entries; the
 * matrix pointers are not dereferenced); n_mol = 0: full X2C of mols[0].  The h outputs and
 * any transforms the caller passes are not included. */
x2c_status x2c_query_workspace(x2c_ctx *ctx, const x2c_options *opt, int32_t n_mol, const x2c_layout *layouts,
                               const x2c_mats *mols, size_t *bytes);

/* Counters of the last build on this context (for instrumentation and benchmarks). */
typedef struct {
  int64_t pair_blocks;       /* pair blocks assembled (A <= B) */
  int64_t atomic_solves;     /* decoupling problems solved (kinds or atoms) */
  int64_t kernel_launches;   /* kernels launched by the last call */
  double credited_flops;     /* algorithmic FP64-equivalent flops of the last call */
} x2c_counters;
x2c_status x2c_ctx_counters(x2c_ctx *ctx, x2c_counters *out);

/* Per-kernel timing for instrumentation.  With enable = 1 every kernel this context
 * launches is bracketed by CUDA events recorded on the launching stream (this adds a little
 * host overhead); enabling also clears the accumulated times.  x2c_ctx_kernel_times()
 * waits for the recorded events and returns, per kernel name (NUL-terminated, 32 bytes per
 * entry in `names`), the accumulated milliseconds, the number of launches and the
 * accumulated algorithmic flops (2 m n k per real GEMM product for the FP64 GEMM kernels; 0
 * for kernels whose launcher does not count them); any of names, ms, launches and flops may
 * be NULL.  At most max_entries entries are written and *n_entries receives the number
 * written. */
x2c_status x2c_ctx_set_timing(x2c_ctx *ctx, int32_t enable);

/* Autotuner (on by default): the first split-precision build of a workload shape (slices,
 * spin, atom sizes, order of magnitude of the pair count) on a context runs every candidate
 * N tile of the tensor-core kernels twice (a warm pass, then one timed with CUDA events on
 * the call's stream; that call synchronises the stream) and keeps the fastest for later
 * builds of the same shape.  All
 * candidates give bit-identical h.  x2c_ctx_tuning_log() returns one line per decision
 * (candidates with their times, and the choice); valid until the next call on the context. */
x2c_status x2c_ctx_set_autotune(x2c_ctx *ctx, int32_t enable);
const char *x2c_ctx_tuning_log(x2c_ctx *ctx);
/* Force one candidate of the split-precision kernels instead of the autotuner's choice:
 * -1 = automatic (default), 0 = 96-column (two-component) / 64-column (spin-free) N tiles,
 * 1 = 64 / 32-column N tiles, 2 = transposed-role stage 1 with 96-column stage 2 (two-
 * component, 5 slices, atoms of 17..48 functions; other classes fall back to 0).  With the
 * autotuner off and no forced variant the default is 2 where it applies, else 0.  All
 * variants give bit-identical h. */
x2c_status x2c_ctx_set_split_variant(x2c_ctx *ctx, int32_t variant);

/* CUDA-graph replay of repeated builds (off by default).  With enable = 1, a build call
 * (x2c_build_full, x2c_build_dlu, x2c_build_dlu_batched, x2c_build_dlu_with_transforms,
 * x2c_atomic_transforms, x2c_build_dlu_host) whose launch plan equals that of an earlier
 * call on this context -- the same options, sizes and layouts, the same input and output
 * pointers, the same kernel choices -- is not enqueued kernel by kernel: the second such
 * call captures its work into a CUDA graph (stream capture on a private stream of the
 * context, with the autotuner's choice from the first call) and launches it on the
 * caller's stream, and every later one launches that graph again.  The matrices are read
 * when the graph runs, so their contents may change between calls; a changed pointer makes
 * a new plan.  Per-kernel timing (x2c_ctx_set_timing) sees inside replays.  Graphs are kept
 * for the 32 most recently used plans and dropped when the workspace grows; enable = 0
 * drops them (and waits for the device).  Counters and x2c_ctx_counters() report a replayed
 * call like an eager one. */
x2c_status x2c_ctx_set_graphs(x2c_ctx *ctx, int32_t enable);
typedef struct {
  int64_t captures;       /* graphs captured on this context */
  int64_t replays;        /* build calls served by launching a captured graph */
  int32_t cached;         /* graphs held now */
  int32_t last_replayed;  /* 1 if the last build call launched a captured graph */
} x2c_graph_stats;
x2c_status x2c_ctx_graph_stats(x2c_ctx *ctx, x2c_graph_stats *out);
x2c_status x2c_ctx_kernel_times(x2c_ctx *ctx, int32_t max_entries, char *names, double *ms,
                                int64_t *launches, double *flops, int32_t *n_entries);

/* ---------------------------------------------------------------------------------------
 * Serving: a device-resident request loop with continuous batching.
 *
 * A server owns max_inflight slots (a CUDA stream and a context each), a device-memory pool
 * and a cache of atomic transforms U^L_A, U^S_A keyed by the caller's kind keys (element,
 * basis, spin-orbit blocks).  One scheduler thread takes requests in arrival order: when a
 * slot is free and the head request fits the memory budget it starts, together with later
 * queued requests of the same options (free-atom DLU) up to max_batch, as one batched build
 * (x2c_build_dlu_batched with the cached transforms); kinds missing from the cache are
 * solved once, in that build's slot, and cached for every later request.  Builds on
 * different slots overlap on the device.  The paper has no serving layer: this is the
 * interface around Eqs. 42-43 (DLU) and Sec. II.A (full X2C) for a stream of molecules.
 *
 * Memory: the budget covers everything the server allocates (copies of inputs, outputs it
 * allocates, cached transforms, the slots' workspaces); a request that could never fit is
 * refused at submission with X2C_ERR_ADMISSION, one that does not fit now waits (and the
 * requests behind it wait too: first come, first served).  Unused cache entries are evicted,
 * least recently used first, when the head request needs their memory.  Results the server
 * allocated stay counted until x2c_server_release().
 *
 * Clock: times are seconds since the server was created (x2c_server_now()); t_start and
 * t_end are device timestamps (CUDA events) on that clock.  Latency = t_end - t_arrival.
 * Thread safety: every x2c_server_* call may come from any host thread.
 * ------------------------------------------------------------------------------------- */
typedef struct x2c_server x2c_server;

typedef enum { X2C_REQ_DLU = 0, X2C_REQ_FULL = 1 } x2c_request_kind;
typedef enum { X2C_MEM_DEVICE = 0, X2C_MEM_HOST = 1 } x2c_memory;
typedef enum { X2C_STATE_QUEUED = 0, X2C_STATE_RUNNING = 1, X2C_STATE_DONE = 2 } x2c_request_state;

typedef struct {
  int32_t device;           /* CUDA device */
  int32_t max_inflight;     /* slots = builds running at once, 1..16 (0 = 4) */
  int32_t max_batch;        /* requests one build may hold, 1..256 (0 = 16) */
  int32_t reserved0;        /* must be zero */
  uint64_t hbm_budget_bytes;/* device memory the server may hold (0 = 150 GB) */
  int32_t reserved[4];      /* must be zero */
} x2c_server_options;

typedef struct {
  x2c_options opt;          /* as for the build calls */
  int32_t kind;             /* x2c_request_kind */
  int32_t memory;           /* x2c_memory: where mol, layout.kinds and out point */
  x2c_layout layout;        /* DLU: atoms and kinds (copied at submission); ignored for FULL */
  const uint64_t *kind_key; /* HOST, layout.n_kinds entries, or NULL: cache key of each kind's
                               transforms (0 = do not cache that kind).  Requests that give
                               the same key must give the same free-atom inputs for it. */
  x2c_mats mol;             /* molecular matrices (FULL: the whole system) */
  int32_t ld;               /* leading dimension (elements) of mol's matrices, 0 = mol.n */
  int32_t reserved0;        /* must be zero */
  x2c_hout out;             /* DEVICE: the caller's device outputs, or h[0] = NULL for
                               outputs the server allocates (valid until release).
                               HOST: the caller's host outputs, filled before the request
                               completes, or h[0] = NULL for server-allocated device outputs */
  double t_arrival;         /* scheduled arrival on the server clock, < 0 = at submission */
} x2c_request;

typedef struct {
  int32_t state;            /* x2c_request_state */
  int32_t status;           /* x2c_status of the build, once DONE */
  const double *h[4];       /* device result (NULL when delivered to host outputs) */
  double t_arrival, t_submit, t_admit, t_start, t_end;
  int32_t batch_size;       /* requests built in the same launch */
  int32_t cache_hits;       /* kinds whose transforms came from the cache */
  int32_t cache_misses;     /* kinds solved for this request */
  int32_t slot;
} x2c_result;

typedef struct {
  int64_t submitted, completed, failed, cancelled, queued, running;
  int64_t builds_launched;  /* batched builds started */
  int64_t cache_hits, cache_misses, cache_entries, cache_evictions;
  double latency_p50_ms, latency_p99_ms, latency_mean_ms, latency_max_ms; /* completed OK */
  double builds_per_s;      /* completed OK / (last completion - first arrival) */
  double first_arrival, last_completion;
  uint64_t bytes_in_use, peak_bytes, budget_bytes;
  int64_t kernel_launches;  /* kernels the builds launched */
  int32_t max_concurrent;   /* most requests running at once */
  int32_t reserved;
} x2c_server_stats;

/* Create a server (allocates its slots and starts its scheduler thread). */
x2c_status x2c_server_create(const x2c_server_options *opt, x2c_server **out);
/* Stop: cancel queued requests, wait for running builds, free everything.  NULL is allowed. */
x2c_status x2c_server_destroy(x2c_server *s);
/* Seconds since the server was created. */
x2c_status x2c_server_now(x2c_server *s, double *t);
/* Queue a request; *ticket identifies it.  The request's matrices must stay valid and
 * unchanged until it is DONE (host and device inputs are read when it starts).
 * X2C_ERR_ARG for an invalid request, X2C_ERR_ADMISSION if it can never fit the budget. */
x2c_status x2c_server_submit(x2c_server *s, const x2c_request *req, uint64_t *ticket);
/* Current state of a request (never blocks).  X2C_ERR_NOT_FOUND for an unknown ticket. */
x2c_status x2c_server_poll(x2c_server *s, uint64_t ticket, x2c_result *res);
/* Wait until the request is DONE or timeout_ms passes (X2C_ERR_TIMEOUT; it keeps running). */
x2c_status x2c_server_wait(x2c_server *s, uint64_t ticket, uint32_t timeout_ms, x2c_result *res);
/* Cancel a queued request (it completes with X2C_ERR_CANCELLED).  X2C_ERR_ARG if it has
 * already started or finished. */
x2c_status x2c_server_cancel(x2c_server *s, uint64_t ticket);
/* Forget a DONE request and free the outputs the server allocated for it.  The caller must
 * have finished reading them (stream work that reads them must have completed). */
x2c_status x2c_server_release(x2c_server *s, uint64_t ticket);
x2c_status x2c_server_get_stats(x2c_server *s, x2c_server_stats *out);
/* Clear the latency samples and counters (not the cache, budget or requests). */
x2c_status x2c_server_reset_stats(x2c_server *s);

#ifdef __cplusplus
}
#endif
#endif /* X2C_H */
