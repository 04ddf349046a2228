/*
 * ifmm.h -- C ABI of the GB300 inverse fast multipole method (IFMM).
 *
 * The library factorizes the dense BEM-type matrix
 *     A_ij = scale / |x_i - x_j|  (i != j),   A_ii = diag,
 * through its FMM representation (Eq. (1): the extended sparse system built from
 * the P2P, P2M, L2P, M2M, M2L, L2L operators of a uniform octree, Sec. 2.1-2.2,
 * with Chebyshev-interpolation operators), eliminates it level by level from the
 * leaves (Algorithm 1) with the nodes of a level processed color by color
 * (Sec. 3, Algorithm 3 coloring at separation sigma), recompresses every far-field
 * fill-in at relative accuracy eps (Sec. 5.1), and applies the result as a direct
 * solve (Algorithm 2) or as the preconditioner of GMRES(m) (Algorithms 4 and 5).
 *
 * Conventions for every entry point:
 *   - Status codes only; no exception or abort crosses the ABI.  On error the
 *     output handle is set to NULL and ifmm_last_error() describes the cause.
 *   - The caller owns every array it passes.  Handles are owned by the library
 *     and released with the matching *_free call (NULL is accepted).
 *   - Vectors are in the caller's point order; the tree's permutation is internal.
 *   - Pointers documented "host or device" may be either; the library inspects
 *     them with cudaPointerGetAttributes and copies host data in and out itself.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  All device
 *     work is enqueued on it.  Calls return after the stream has finished their
 *     work when a result the call returns depends on device values (ranks,
 *     singular pivots, GMRES convergence, host outputs); otherwise they may
 *     return early.
 *   - A handle must not be used from two threads at the same time.
 *   - There is no CPU fallback: without a CUDA device every compute call
 *     returns IFMM_ECUDA.
 */
#ifndef IFMM_H
#define IFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  IFMM_OK = 0,
  IFMM_EINVAL = 1,     /* bad argument (NULL, size out of range, inconsistent options) */
  IFMM_ENOMEM = 2,     /* host or device allocation failed */
  IFMM_ECUDA = 3,      /* CUDA runtime error, or no CUDA device */
  IFMM_ESINGULAR = 4,  /* a pivot block was numerically singular */
  IFMM_ENOCONV = 5,    /* GMRES stopped at maxit above tol (outputs still written) */
  IFMM_ETIMEOUT = 6,   /* a bounded device wait gave up */
  IFMM_ERANK = 7       /* a recompression needed more rank than max_rank allows */
} ifmm_status;

typedef struct ifmm_tree ifmm_tree; /* opaque, library-owned */
typedef struct ifmm_fact ifmm_fact; /* opaque, library-owned: the factor's block pool */

/* Matrix entries: A_ij = scale/|x_i - x_j| for i != j, A_ii = diag.
 * The collocation BEM system of the paper's electrostatic example (Sec. 2) with
 * area weight 4pi/N has scale = 1/N and diag = 0.5 + 1/sqrt(N).
 * arith selects how bem_matvec / bem_gmres apply the matrix:
 *   IFMM_ARITH_FP64 - direct summation in plain FP64;
 *   IFMM_ARITH_DF   - direct summation in pairs of floats with error-free
 *                     transformations: FP64-level accuracy at FP32 throughput
 *                     (about 1e-13 relative per interaction; for two points
 *                     closer than ~1e-3 of the domain the 48-bit pair
 *                     coordinates bound it at ~2^-46 R / r of the term);
 *   IFMM_ARITH_FMM  - the FMM representation A~ (Sec. 2.2, Eq. (1); the
 *                     paper's FMBEM matvec, Algorithm 4): P2M, M2M, M2L over
 *                     the interaction lists, L2L, L2P and the near field, with
 *                     the Chebyshev operators of order `order` (0: 4) that
 *                     ifmm_factor uses, in FP64.  It equals A only to the
 *                     interpolation error, and GMRES then solves A~ x = b.
 *                     The operator tables are built on first use and cached
 *                     on the tree. */
enum { IFMM_ARITH_FP64 = 0, IFMM_ARITH_DF = 1, IFMM_ARITH_FMM = 2 };
typedef struct {
  double scale;
  double diag;
  int arith;
  int order;         /* Chebyshev order of the FMM matvec (IFMM_ARITH_FMM), 0 = 4 */
  double wavenumber; /* Helmholtz: k != 0 (see below); 0 = Laplace               */
  double diag_im;    /* Helmholtz: imaginary part of A_ii                         */
} ifmm_kernel;
/* Helmholtz (the paper's acoustic BEM kernel, Sec. 4.1): with wavenumber k != 0
 * the entries are A_ij = scale e^{ik|x_i - x_j|}/|x_i - x_j| and A_ii = diag +
 * i diag_im, complex.  Every complex vector (right-hand sides, solutions; host or
 * device) is then N pairs (real, imaginary) of doubles -- the memory layout of
 * an array of N complex doubles -- and the factorization works on the real 2 x 2
 * form [[Re z, -Im z], [Im z, Re z]] of every complex entry: two real unknowns
 * per point, Chebyshev bases of 2 p^3 real columns, and every kernel of the
 * real path unchanged (twice the real operations of native complex
 * arithmetic).  A truncation that keeps k complex directions keeps 2k real ones
 * (the singular values of the real form come in equal pairs), and the ranks
 * reported and replayed are those real counts.  The matvec is the FP64 direct
 * sum (arith IFMM_ARITH_FP64; the float-pair and FMM matvecs, BD and the
 * allocation-free matvec are Laplace only and refuse k != 0 with IFMM_EINVAL). */

/* Arithmetic of the factorization outside the pivots (which are always FP64, as
 * are the solve, GMRES and its residual):
 *   FP64 - everything in FP64;
 *   FP32 - Schur-complement GEMMs, transforms and recompression (pivoted QR,
 *          Jacobi) computed in FP32 on FP64 storage;
 *   BF16 - as FP32, with the Schur-complement GEMM operands rounded to bfloat16
 *          (FP32 accumulation).  The fill-ins then carry bfloat16 rounding
 *          (~4e-3 relative), so truncation at eps much below that keeps noise. */
enum { IFMM_PREC_FP64 = 0, IFMM_PREC_FP32 = 1, IFMM_PREC_BF16 = 2 };
enum { IFMM_RANK_SVD = 0, IFMM_RANK_REPLAY = 1, IFMM_RANK_LEARNED = 2 };

typedef struct {
  int cheb_order;        /* Chebyshev points per axis p (2..6); r = p^3 per cell       */
  double eps;            /* relative truncation: keep s_j > eps*s_1; 0 = numerical rank */
  int precision;         /* IFMM_PREC_*: arithmetic of the Schur updates/recompression  */
  int rank_mode;         /* IFMM_RANK_*                                                 */
  const int32_t* replay; /* rank_mode REPLAY: host array of (level,node,event,rank)     */
  int64_t replay_len;    /*   quadruples, replay_len quadruples                         */
  int max_rank;          /* largest rank any node may need (0 = library default, 256);  */
                         /*   a recompression that needs more fails with IFMM_ERANK     */
  const float* mlp;      /* rank_mode LEARNED: host weights, IFMM_MLP_NWEIGHTS floats   */
  uint64_t seed;         /* seed of the randomized range finder (LEARNED mode)          */
} ifmm_opts;

/* Sec. 2.1: uniform octree of the given depth (>= 2, <= 10) over n >= 1 points.
 * xyz: n x 3 row-major doubles, host or device memory (device points are copied
 * to the host, where the tree and its lists are built).  The root is the tight
 * bounding cube of the points.  The tree keeps a device copy of the points in
 * tree order once a device call first needs them. */
ifmm_status ifmm_build_tree(const double* xyz, int64_t n, int depth, ifmm_tree** out);

/* Sec. 3.4, Algorithm 3: greedy coloring at separation sigma (>= 3) of every level
 * 2..depth.  Replaces any previous coloring of the tree.  ncolors_per_level, if not
 * NULL, receives depth+1 counts (levels 0 and 1 report 0). */
ifmm_status ifmm_color(ifmm_tree* t, int sigma, int32_t* ncolors_per_level);

/* The per-level strategy switch of Sec. 4.2 (Table 2, nIFMMs{sigma}t{tau}b{l}):
 * levels tau..depth are colored by Algorithm 3 at separation sigma and
 * eliminated a color at a time (node-parallel), levels 2..tau-1 get one node
 * per color, in node order, so their nodes are eliminated one after the other
 * with each node's large matrix operations spread over the GPU
 * (matrix-parallel).  tau in [2, depth]; tau = 2 is ifmm_color.  ncolors as
 * for ifmm_color. */
ifmm_status ifmm_color_levels(ifmm_tree* t, int sigma, int tau, int32_t* ncolors_per_level);

/* Integer views of the tree, for inspection and tests.  `what` is one of
 *   "cells"  (3 per node: ix iy iz)        "parent"  (per node, level >= 1)
 *   "nbr_ptr" "nbr"   neighbour CSR (Sec. 2.1, excluding the node itself)
 *   "il_ptr"  "il"    interaction-list CSR (Sec. 2.1)
 *   "color"           color per node      "group_ptr" "group"  colors as CSR lists
 *   "perm"            tree order -> caller index (level ignored)
 *   "leaf_ptr"        point CSR of the leaves (level ignored)
 *   "matvec_block"    2 values: the source tile (threads per CTA) and the targets
 *                     per thread of the float-pair matvec, chosen by its autotuner
 *                     on the first such product with this tree (0, 0 before); the
 *                     choice is remembered per device and N for the life of the
 *                     process, and trees of a size tuned before reuse it
 * Writes min(count, cap) int32 values to buf (may be NULL) and the full count to
 * *count. */
ifmm_status ifmm_tree_query(const ifmm_tree* t, int level, const char* what, int32_t* buf, int64_t cap,
                            int64_t* count);

/* Algorithm 1 with the coloring of ifmm_color (Sec. 3.2/3.3): initialise the
 * operators (Sec. 2.2), eliminate levels depth..2 color by color with eps-accurate
 * recompression of far-field fill-ins, and invert the remaining level-2 system
 * (explicit Gauss-Jordan inverse, partial pivoting).  Requires ifmm_color first.
 * The factor keeps its own reference to device data of the tree: the tree must
 * outlive it.  The call synchronizes the stream once per color (the ranks are
 * read back) and may use up to 8 host threads for its own descriptor building
 * (one inside ifmm_factor_batched workers); the result does not depend on the
 * number of threads.  Errors: IFMM_ESINGULAR when a pivot block (or the level-2
 * system) has an exactly zero pivot in Gauss-Jordan with partial pivoting;
 * IFMM_ERANK when a recompression keeps more than max_rank directions. */
ifmm_status ifmm_factor(const ifmm_tree* t, const ifmm_kernel* k, const ifmm_opts* o, void* stream,
                        ifmm_fact** out);

/* Sec. 4.3, BD / BDbot l_BD: the block-diagonal preconditioner the paper
 * compares the IFMM with.  For every non-empty cell of `level` (0..depth; the
 * leaf level is the paper's BD, a coarser level its BDbot l_BD) the self block
 * of A over the cell's points is inverted on the device (FP64 Gauss-Jordan
 * with partial pivoting); its application (Algorithm 5) solves each block
 * independently.  The result is a factor handle: ifmm_solve applies it and
 * bem_gmres takes it as `precond`, like an IFMM factor; ifmm_fact_stats reports
 * bd_level, bd_blocks, bd_max_block and time_factor.  Level 0 is a single dense
 * block: the exact inverse.  Errors: IFMM_ESINGULAR for a singular block. */
ifmm_status ifmm_bd_factor(const ifmm_tree* t, const ifmm_kernel* k, int level, void* stream, ifmm_fact** out);

/* Algorithm 2 (+ the dense level-2 solve): v = A~^{-1} r approximately, where A~ is
 * the FMM representation of A.  r and v: n x nrhs column-major doubles, host or
 * device (both on the same side).  r and v may alias. */
ifmm_status ifmm_solve(const ifmm_fact* f, const double* r, double* v, int nrhs, void* stream);

/* Algorithms 4 and 5: GMRES(restart) on A x = b from x = 0 with right
 * preconditioning by ifmm_solve (precond may be NULL: no preconditioner), the
 * matrix applied by direct summation on the device.  Stops when the true relative
 * residual ||b - A x|| / ||b|| <= tol or after maxit matrix-vector products.
 * b, x: n doubles, host or device (same side).  iters and relres may be NULL. */
ifmm_status bem_gmres(const ifmm_tree* t, const ifmm_kernel* k, const ifmm_fact* precond, const double* b,
                      double* x, int restart, double tol, int maxit, int* iters, double* relres, void* stream);

/* Independent problems together (a batch of many BEM problems; the paper factors
 * one problem at a time).  Problem i uses trees[i], kernels[i], opts[i]; out[i]
 * receives its factor.  nworkers host threads (<= 0: 8), each with its own CUDA
 * stream, take problems in index order, so kernels of different problems
 * overlap on the GPU.  Each factor equals what ifmm_factor gives for the same
 * problem.  On error every out[i] is NULL and the message names the problem.
 * Trees are uploaded to the device first, in the calling thread. */
ifmm_status ifmm_factor_batched(const ifmm_tree* const* trees, const ifmm_kernel* kernels, const ifmm_opts* opts,
                                int nprob, int nworkers, ifmm_fact** out);

/* bem_gmres for nprob independent problems on worker threads and streams as
 * above.  b[i], x[i]: N_i doubles (host or device); precond may be NULL (no
 * preconditioner for any problem) or hold NULL entries; iters/relres may be NULL.
 * Returns the first failing problem's status (IFMM_ENOCONV if one did not
 * converge); every x[i] is written. */
ifmm_status bem_gmres_batched(const ifmm_tree* const* trees, const ifmm_kernel* kernels, const ifmm_fact* const* precond,
                              const double* const* b, double* const* x, int nprob, int restart, double tol, int maxit,
                              int* iters, double* relres, int nworkers);

/* y = A x by direct summation on the device (the matrix of bem_gmres).
 * x, y: n doubles, host or device (same side); they must not alias. */
ifmm_status bem_matvec(const ifmm_tree* t, const ifmm_kernel* k, const double* x, double* y, void* stream);

/* y = A x like bem_matvec, but without allocating any device memory, for callers
 * that cannot call cudaMalloc/cudaFree (code running inside a host framework
 * that owns and sizes the device memory pool, or code that must not trigger the
 * synchronisation an allocation can imply).  The paper has no counterpart: it
 * is a deployment variant of the direct-summation matvec.
 *   - x, y: N doubles in device memory of the current device, caller order,
 *     caller-allocated; they must not alias.  The call only enqueues work on
 *     `stream` and returns; y is ready when the stream reaches that point.
 *   - Scratch is a fixed array in the library's device image (4 MiB, trees of at
 *     most 262,144 points), kept by every GPU that loads the library until the
 *     process exits.  Larger trees are rejected with IFMM_EINVAL.
 *   - The tree must already be resident on the current device: any earlier
 *     ifmm_factor, bem_matvec or bem_gmres on it uploads it (this call never
 *     does, since that would allocate).  Otherwise IFMM_EINVAL.
 *   - The scratch array's device address is looked up (cudaGetSymbolAddress,
 *     which also loads the module holding the array and this call's kernels)
 *     when the tree is first made resident on a device, inside a call that
 *     allocates anyway.  Only if that look-up failed does the first call here
 *     repeat it (and may then load the module); make that first call before
 *     any stream capture.
 *   - All calls share the one scratch array: calls that overlap on the GPU (on
 *     different streams, or from different threads) race and give wrong results.
 *     No part of the scratch needs clearing between calls.
 *   - k->arith selects FP64 or float-pair sums, as for bem_matvec; the FMM
 *     matvec (IFMM_ARITH_FMM) needs its own tables and is refused (IFMM_EINVAL). */
ifmm_status bem_matvec_noalloc(const ifmm_tree* t, const ifmm_kernel* k, const double* x, double* y, void* stream);

/* Rank predictor (the paper's Sec. 5.1 uses a randomized SVD at a prescribed
 * accuracy; here a learned rank sets the width of a randomized range finder).
 * A multilayer perceptron 9 -> 64 -> 64 -> 64 -> 1 with ReLU hidden layers, FP32.
 * Inputs per recompression event: cell centre in [-1,1]^3 (3), block size
 * n_q / 256 (1), level / 10 (1), current rank / 64 (1), fill-in rows / 1024 (1),
 * L1 cell offset to the eliminated neighbour whose fill-ins caused the event / 3
 * (1; 0 at a level start), log10(eps) / 10 (1).  Output: rank / 64.  Weights, row-major W[in][out]:
 *   W1[9][64] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[64][1] b4[1].
 * In IFMM_RANK_LEARNED mode ifmm_factor recompresses an event whose predicted
 * rank k is well below its block width with a randomized range finder of width
 * s = ceil(k) + 8 (Y^T Omega with a +-1 SplitMix64 sketch, orthonormalised;
 * B = Y Q; SVD of B).  The result is accepted when ||Y - B Q^T||_F <=
 * max(eps * sigma_1, 16 u ||Y||_F) (u: unit roundoff of the arithmetic), else the
 * exact pivoted-QR + Jacobi path runs on the same Y.  Counts: ifmm_fact_stats
 * learned_events / learned_sketched / learned_fallbacks. */
#define IFMM_MLP_INPUTS 9
#define IFMM_MLP_NWEIGHTS 9025

/* y[i] = MLP(x[i]) for n feature rows x (n x 9 row-major, host), y (n, host). */
ifmm_status ifmm_mlp_forward(const float* weights, const float* x, int64_t n, float* y, void* stream);

/* Loss L = mean_i (y_i - t_i)^2 / 2 over n rows and its gradient with respect to
 * every weight (IFMM_MLP_NWEIGHTS floats, host), by the library's backward kernels. */
ifmm_status ifmm_mlp_grad(const float* weights, const float* x, const float* t, int64_t n, float* grad, float* loss,
                          void* stream);

/* Trains the MLP on the device: He-uniform initialisation from `seed`
 * (SplitMix64 counter stream), Adam (beta 0.9 / 0.999) with step `lr`, minibatches
 * of `batch` rows in order, `epochs` passes.  weights: out, host; final_loss (may
 * be NULL): L over all rows with the final weights. */
ifmm_status ifmm_mlp_train(const float* x, const float* t, int64_t n, int epochs, int batch, float lr, uint64_t seed,
                           float* weights, float* final_loss, void* stream);

/* Training data from a factorization: the 9 predictor inputs (row-major) and the
 * chosen rank of every recompression event, in the order of ifmm_fact_ranks.
 * features/ranks may be NULL; min(count, cap) rows are written, *count = total. */
ifmm_status ifmm_fact_events(const ifmm_fact* f, float* features, int32_t* ranks, int64_t cap, int64_t* count);

/* Ranks chosen by ifmm_factor, as (level, node, event, rank) quadruples; node is the
 * tree-order node index at that level and event counts that node's recompressions
 * at that level (0 = level start).  Same buffer protocol as ifmm_tree_query. */
ifmm_status ifmm_fact_ranks(const ifmm_fact* f, int32_t* buf, int64_t cap, int64_t* count);

/* Factor statistics as named doubles (timings in seconds, algorithmic flop counts,
 * bytes): writes min(count, cap) values and the full count; ifmm_fact_stat_name
 * gives the name of entry `index` (NULL when out of range).  Families of names:
 * time_* (wall time of the factor and of each level), host_* (host wall time of
 * one phase of the color loop, summed over colors; a suffix _L<level> restricts
 * it to one level; *_wait is time spent waiting on the device), flops_* (the
 * counted work per operation class), bytes_* (device memory of the factor and
 * the solve), learned_* (rank-predictor counts), solve_* (the solve graph's
 * launches and sizes), qrcp_steps (column steps of the pivoted QRs). */
ifmm_status ifmm_fact_stats(const ifmm_fact* f, double* buf, int64_t cap, int64_t* count);
const char* ifmm_fact_stat_name(const ifmm_fact* f, int64_t index);


/* Diagnostic: the binary64 -> binary32 conversion the FP32 kernels use on their
 * FP64 storage (integer operations on the IEEE-754 fields, GB300's FP64 pipe
 * being narrow), applied on the device to n host doubles x scaled by 2^shift:
 * f[i] = x[i] * 2^shift rounded to nearest (ties away from zero; below the
 * binary32 normal range -> signed zero, above it -> infinity), back[i] = f[i] *
 * 2^-shift as a double (exact).  |shift| <= 200, n <= 2^26; host arrays. */
ifmm_status ifmm_convert_check(const double* x, int64_t n, int shift, float* f, double* back);

/* Diagnostic: one C = alpha op(A) op(B) + beta C through the library's batched
 * GEMM in the arithmetic of `precision` (IFMM_PREC_*: FP64 FMA; FP32-accurate
 * 3xTF32 tensor-core MMAs; bfloat16 operands with FP32 accumulation -- the
 * kernels of the factorization's Schur updates), on host arrays, column-major,
 * op(X) = X^T when tX != 0.  m, n, k <= 8192.  Synchronous. */
ifmm_status ifmm_gemm_check(int precision, int m, int n, int k, int ta, int tb, double alpha, const double* A, int lda,
                            const double* B, int ldb, double beta, double* C, int ldc);

/* The Householder QR of the recompression (Algorithm 1's truncated QR of the
 * fill-in blocks, and the QR of the weight stacks), on a host array, through
 * the same kernels and size classes as the factorization (a warp, a CTA, a
 * thread-block cluster, row-chunked reduction or the global-memory kernel, by
 * the block's size).  A is m x n column-major with
 * leading dimension ld >= m (m <= 65536, n <= 1024, ld n <= 2^27), in FP64 or
 * rounded to FP32 as the precision says (IFMM_PREC_FP64 or IFMM_PREC_FP32).
 * On return the leading min(m, n) rows of A hold R (zeros below its diagonal).
 * With pivoted != 0 the columns are pivoted by largest remaining norm and run to
 * completion (no truncation): jpvt[p] is the original index of column p of R
 * and *k the number of steps; jpvt and k are not read otherwise.  Rows of A
 * below R are unspecified.  Synchronous; IFMM_ECUDA without a device. */
ifmm_status ifmm_qr_check(int precision, int pivoted, int m, int n, double* A, int ld, int* jpvt, int* k);

/* The FP64 Gauss-Jordan inverse with partial pivoting of the pivot blocks
 * (Algorithm 1's inverses of Pi_i), on host arrays, through the same size
 * classes as the factorization (one CTA in shared memory, a thread-block
 * cluster, or the batched multi-CTA kernels).  A holds nmat column-major
 * matrices back to back, matrix i of order n[i] (1..4096) with leading
 * dimension n[i]; each is replaced by its inverse.  info[i] = 0, or k + 1 when
 * step k found no nonzero pivot (that matrix is then left partly eliminated).
 * At most 2^28 doubles in all.  Synchronous; IFMM_ECUDA without a device. */
ifmm_status ifmm_inv_check(int nmat, const int* n, double* A, int* info);

/* Measured arithmetic peak of the current GPU in TFLOP/s (no counterpart in the
 * paper: the denominators of the per-phase rooflines).  kind: 0 FP32 FMA, 1 FP64
 * FMA, 2 TF32 warp MMA (m16n8k8), 3 BF16 warp MMA (m16n8k16, FP32 accumulate),
 * 4 FP64 warp MMA (m8n8k4).  Runs register-only dependency chains on 8 CTAs of
 * 256 threads per SM, times the second of two launches with CUDA events on the
 * legacy default stream, and synchronizes.  Allocates one small device buffer. */
ifmm_status ifmm_probe_peak(int kind, double* tflops);

/* Kernel profiling of this process (no counterpart in the paper): ifmm_profile
 * resets the per-kernel counters and, if timing != 0, brackets every later kernel
 * launch (or solve graph launch) with CUDA events on its stream.  Timing adds
 * event records between launches; leave it off for production runs. */
ifmm_status ifmm_profile(int timing);

/* Counter `index` (0..): kernel name, kernels launched so far (a solve graph
 * counts its kernels), and summed event time in ms (0 unless timing).
 * IFMM_EINVAL past the last counter.  Synchronizes with the timed events. */
ifmm_status ifmm_profile_query(int index, const char** name, int64_t* launches, double* ms);

void ifmm_tree_free(ifmm_tree* t);
void ifmm_fact_free(ifmm_fact* f);

/* Message of the last failing call on this thread ("" if none). */
const char* ifmm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* IFMM_H */
