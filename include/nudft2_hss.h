/*
 * nudft2_hss -- direct solver for the 2D type-II inverse NUDFT on one GPU (sm_103a).
 *
 * Problem (Li & Liu, Sec. 1, Eq. 1-2): given M sample points (x_j, y_j) in [0,1)^2 and values
 * f_j, find the coefficients c on the nx-by-ny frequency grid minimising ||A c - f||_2 with
 *     A(j, (kx, ky)) = exp(-2 pi i (kx x_j + ky y_j)),  M >= N = nx * ny,
 * columns ordered lexicographically: index ky + kx * ny, frequencies 0..n-1.
 *
 * Method (Sec. 4.1, Algorithm 1): c = F^{-1} G~_hss^+ f where G~ = A F^{-1} (F = F^x (x) F^y the
 * 2D DFT) is approximated by an HSS matrix built from two 1D HSS approximations through the
 * face-splitting product (Thm. 3.5), recompressed (Sec. 2.2) and factorised by URV (Sec. 2.3).
 *
 * Conventions for every entry point
 *   - Arrays marked d_ are DEVICE pointers (cudaMalloc / torch CUDA tensors) owned by the
 *     caller.  Complex data is interleaved (re, im) complex128 (double2) unless stated.
 *     Matrices of right-hand sides are column major with the given leading dimension.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  All work is
 *     enqueued on it; build and factor synchronise it internally (ranks are read back).
 *   - Return value: NUDFT2_OK or an error code; no exception crosses this interface.  The
 *     message of the last error on the calling thread is returned by nudft2_last_error().
 *   - A handle is not thread safe; distinct handles are independent.
 */
#ifndef NUDFT2_HSS_H
#define NUDFT2_HSS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nudft2_hss_s* nudft2_hss_t;

typedef enum {
  NUDFT2_OK = 0,
  NUDFT2_EINVAL = 1,   /* invalid argument: M < N, bad sizes, points outside [0,1), eps not in (0,1) */
  NUDFT2_ENOMEM = 2,   /* device allocation failed */
  NUDFT2_ECUDA = 3,    /* CUDA runtime error (message in nudft2_last_error) */
  NUDFT2_ERANK = 4,    /* a URV block is rank deficient (fewer rows than eliminated columns) */
  NUDFT2_ETIMEOUT = 5, /* a bounded device wait (tensor-core GEMM pipeline) expired */
  NUDFT2_ESTATE = 6,   /* call out of order (factor before build, solve before factor) */
  NUDFT2_ENOTIMPL = 7  /* operation not available in this build */
} nudft2_status;

typedef enum {
  NUDFT2_FP64 = 0,     /* all HSS work in complex128 */
  NUDFT2_MIXED = 1     /* HSS work in complex64, FP64 iterative refinement with the exact apply */
} nudft2_prec;

typedef enum {
  NUDFT2_FAST_FWD = 0,  /* out (M x nrhs) = G~_hss F in: the HSS forward map (Sec. 4.1, A_fast)   */
  NUDFT2_FAST_ADJ = 1,  /* out (N x nrhs) = (G~_hss F)^* in = F^* G~_hss^* in: the adjoint of
                           FAST_FWD (Sec. 4.1), by the transposed HSS product sweeps            */
  NUDFT2_EXACT_FWD = 2, /* out (M x nrhs) = A in, direct O(MN) sum of Eq. 1 in FP64              */
  NUDFT2_EXACT_ADJ = 3, /* out (N x nrhs) = A^* in, direct O(MN) sum in FP64                     */
  NUDFT2_PINV = 4,      /* out (N x nrhs) = F^{-1} G~_hss^+ in (same as nudft2_hss_solve)         */
  NUDFT2_PINV_ADJ = 5   /* out (M x nrhs) = (F^{-1} G~_hss^+)^* in: the adjoint of PINV, for the
                           backward pass of c = A^+ f (Sec. 4.1 uses the adjoint for LSQR); in
                           MIXED mode refined on A^* out = in with the FP64 exact adjoint        */
} nudft2_op;

typedef struct {
  double eps;          /* HSS tolerance of the recompression (Alg. 1 step 3); 1D factors use eps/10 */
  int levels;          /* depth L of both 1D trees; 0 = derive from leaf                           */
  int leaf;            /* max columns of a product leaf when levels == 0 (e.g. 64 -> 8 x 8)         */
  int prec;            /* nudft2_prec                                                             */
  double refine_tol;   /* MIXED: stop when max relative residual ||f - A c||/||f|| <= refine_tol    */
  int refine_max;      /* MIXED: maximum refinement steps                                          */
  unsigned flags;      /* NUDFT2_FLAG_* bits                                                      */
  int levels_y;        /* depth of T^y when > 0 (then `levels` is the depth of T^x): an unbalanced
                          product tree (Def. 3.3 (2), (3)) with leaves (nx >> levels) x
                          (ny >> levels_y); 0 = both trees have depth `levels`                     */
} nudft2_opts;

/* opts.flags bits */
#define NUDFT2_FLAG_PROFILE 1u   /* time every launch of the main kernel classes with CUDA events */
#define NUDFT2_FLAG_FP64_RESIDUALS 2u   /* MIXED: every refinement residual from the exact FP64 apply
                                           (default: the first; later steps subtract A d of the
                                           O(eps)-small correction d in FP32)               */
#define NUDFT2_FLAG_FADI 4u   /* Alg. 1 step 1 by the route Sec. 3.1 cites: the 1D HSS approximations
                                 by factored ADI on the Sylvester equation of the transformed 1D
                                 matrix (Zolotarev shifts for the two arcs of a block) and the
                                 interpolative decomposition, with nested skeletons; default: the
                                 truncated SVD of each node's kernel-entry block.  EINVAL when eps is
                                 too small for n (more than 64 shifts needed).                    */

/* Accumulated device time of one kernel class (NUDFT2_FLAG_PROFILE), with its algorithmic
 * flop and byte counts summed over launches. */
typedef struct {
  char name[16];
  double ms, flops, bytes;
  int launches;
} nudft2_kstat;

typedef struct {
  int64_t M;
  int nx, ny, levels, prec;
  int max_rank;              /* HSS rank after recompression (r_h of Sec. 5)            */
  int level_rank[16];        /* max basis size per level, level 0 = root               */
  double t_build_ms;         /* t_c: 1D construction + face splitting + recompression  */
  double t_factor_ms;        /* t_f: URV factorization                                 */
  double t_solve_ms;         /* t_s of the last solve (incl. refinement in MIXED)       */
  int refine_iters;          /* refinement steps of the last MIXED solve               */
  double refine_relres;      /* max relative residual after the last MIXED solve       */
  size_t device_bytes;       /* device memory reserved by the handle                   */
  int launches;              /* kernel launches issued by the handle so far            */
  int gemm_tuned;            /* GEMM shape classes the autotuner has measured in this
                                process (kernel choice cached per class)              */
  int solve_graphs;          /* URV solves captured into CUDA graphs (one per RHS count) */
  int solve_graph_failures;  /* captures that failed (those solves run uncaptured)     */
  int solve_replays;         /* solves run by replaying a captured graph               */
  int checkpointed_levels;   /* top levels whose factors are handed back (0 = none)    */
} nudft2_info;

/* Build the HSS approximation of G~ = A F^{-1} (Alg. 1 steps 1-3, Sec. 3 and Sec. 2.2).
 * d_x, d_y: M sample coordinates in [0,1) (copied).  nx, ny: frequency grid, M >= nx*ny.
 * o: options (NULL = defaults: eps 1e-10, leaf 64, FP64).  *out receives the handle.
 * Errors: EINVAL (sizes, eps, points outside [0,1)), ENOMEM, ECUDA. */
nudft2_status nudft2_hss_build(const double* d_x, const double* d_y, int64_t M, int nx, int ny,
                               const nudft2_opts* o, void* stream, nudft2_hss_t* out);

/* URV factorization of the HSS matrix (Alg. 1 step 4, Sec. 2.3).
 * Errors: ESTATE (no build), ERANK (a node has fewer rows than eliminated columns). */
nudft2_status nudft2_hss_factor(nudft2_hss_t h, void* stream);

/* c = F^{-1} G~_hss^+ f (Alg. 1 step 5): URV sweeps then the 2D inverse DFT.
 * d_f: M x nrhs complex128 (ld ldf >= M), point order as given to build.
 * d_c: N x nrhs complex128 (ld ldc >= N), lexicographic ky + kx*ny.
 * MIXED handles refine with the exact residual (opts.refine_tol / refine_max): c += d, d the FP32
 * solve of r = f - A c, until ||r|| / ||f|| <= refine_tol, or, after the first step, until the
 * correction is at most refine_tol ||c|| per column (data with a nonzero least-squares residual).
 * The first residual comes from the exact FP64 apply; later ones are updated as r -= A d with the
 * exact apply of the small correction d in FP32 (its rounding is O(eps u_32) ||f||), unless
 * NUDFT2_FLAG_FP64_RESIDUALS asks for the FP64 apply at every step.  When the residual does not
 * reach refine_tol (data outside the range of A), the stop above is the fixed point of the FP32
 * pseudo-inverse, O(eps) ||r_LS|| away from the least-squares solution; the solve then polishes on
 * the normal equations, c += P P^* A^* r (A^* r in FP64, P the FP32 solve), until the correction
 * is at most refine_tol ||c||: the least-squares solution itself.
 * Errors: ESTATE (not factorised), EINVAL (ld too small, nrhs < 0). */
nudft2_status nudft2_hss_solve(nudft2_hss_t h, const void* d_f, int64_t ldf, int nrhs, void* d_c, int64_t ldc,
                               void* stream);

/* Apply one operator of nudft2_op to nrhs columns: EXACT_FWD/EXACT_ADJ, FAST_FWD and FAST_ADJ
 * need only build; PINV and PINV_ADJ need factor.  Shapes as documented on nudft2_op.
 * Errors: EINVAL (op unknown, ld too small), ESTATE. */
nudft2_status nudft2_hss_apply(nudft2_hss_t h, int op, const void* d_in, int64_t ldi, int nrhs, void* d_out,
                               int64_t ldo, void* stream);

/* Backward pass of the least-squares solution c = A^+ f for a real loss L(c), all complex128
 * device arrays, columns independent right-hand sides:
 *   d_f (M x nrhs, ld ldf)  the data f;  d_c (N x nrhs, ld ldc) its solution (from solve);
 *   d_g (N x nrhs, ld ldg)  the incoming gradient dL/dRe c + i dL/dIm c (torch convention).
 * Outputs (each may be NULL; d_gx and d_gy together):
 *   d_gf (M x nrhs, ld ldgf)  dL/dRe f + i dL/dIm f = lam = (A^+)^* g  (PINV_ADJ);
 *   d_gx, d_gy (M doubles, caller point order)  dL/dx_j, dL/dy_j, summed over the columns:
 *     dL/dx_j = sum_q Re[ -conj(lam_jq) (A_x c)_jq + conj((A_x mu)_jq) r_jq ],
 *   with mu = A^+ lam, r = f - A c, (A_x)_jk = -2 pi i kx A_jk (Golub-Pereyra derivative of a
 *   full-rank least-squares solution; the paper has no gradient).  Products with A are the FP64
 *   exact apply of Eq. 1.  With a MIXED handle mu is the refined solve of lam and the returned
 *   lam is A mu, which puts it in range(A) (the refined adjoint alone meets A^* lam = g but
 *   carries an O(eps) part outside range(A)).  Synchronises the stream.
 * Errors: ESTATE (not factored), EINVAL. */
nudft2_status nudft2_hss_grad(nudft2_hss_t h, const void* d_f, int64_t ldf, const void* d_c, int64_t ldc,
                              const void* d_g, int64_t ldg, int nrhs, void* d_gf, int64_t ldgf, double* d_gx,
                              double* d_gy, void* stream);

/* Many independent problems of uneven sizes (each its own point set, grid, tolerance and
 * precision): build (and, if factor != 0, factor) problem i from d_x[i], d_y[i] (M[i] points),
 * nx[i] x ny[i] frequencies and opts[i] (opts may be NULL: defaults) into out[i].  The problems
 * run concurrently, each on its own handle-owned stream, driven by up to `threads` host threads
 * (<= 0: 8); the kernels of different problems overlap on the GPU.  The paper treats one problem
 * at a time; this is the batched use of the same offline stage (Sec. 4.1).  out[i] is NULL for a
 * problem that failed; status[i] (may be NULL) receives each problem's code.  Returns OK or the
 * first failing problem's code (nudft2_last_error names it).  Synchronises every problem. */
nudft2_status nudft2_hss_build_batched(int count, const double* const* d_x, const double* const* d_y,
                                       const int64_t* M, const int* nx, const int* ny, const nudft2_opts* opts,
                                       int factor, int threads, void* stream, nudft2_hss_t* out,
                                       nudft2_status* status);

/* nudft2_hss_solve for problem i of a batch: d_c[i] (ld ldc[i]) = solution for d_f[i] (ld ldf[i],
 * nrhs[i] columns) with handle h[i], the problems solved concurrently as in build_batched.
 * Distinct entries of h must be distinct handles.  Errors: as nudft2_hss_solve, per problem. */
nudft2_status nudft2_hss_solve_batched(int count, const nudft2_hss_t* h, const void* const* d_f, const int64_t* ldf,
                                       const int* nrhs, void* const* d_c, const int64_t* ldc, int threads,
                                       void* stream, nudft2_status* status);

/* build + factor + solve + free for each problem of a batch, the problems run to completion
 * concurrently on `threads` host threads (each on its own stream; largest problems start first),
 * so that at most `threads` handles hold device memory at a time: the batched offline/online
 * stages of Sec. 4.1 when the factorizations need not outlive the solve.  Problem i: points
 * d_x[i], d_y[i] (M[i]), sizes nx[i] x ny[i], options opts[i] (opts may be NULL), data d_f[i]
 * (M[i] x nrhs[i], ld ldf[i], complex128), solution d_c[i] (N_i x nrhs[i], ld ldc[i], complex128,
 * lexicographic order as for nudft2_hss_solve).  A problem that runs out of device memory while
 * others hold theirs waits for one of them to finish and starts again; alone on the device its
 * ENOMEM stands.  status[i] (may be NULL) receives each problem's code.  Returns OK or the first
 * failing problem's code (nudft2_last_error names it).  Errors: EINVAL, and those of build, factor
 * and solve per problem. */
nudft2_status nudft2_hss_run_batched(int count, const double* const* d_x, const double* const* d_y,
                                     const int64_t* M, const int* nx, const int* ny, const nudft2_opts* opts,
                                     const void* const* d_f, const int64_t* ldf, const int* nrhs, void* const* d_c,
                                     const int64_t* ldc, int threads, void* stream, nudft2_status* status);

/* plsqr: the direct solver as a preconditioner for LSQR (Sec. 4.1, Sec. 5): LSQR (Paige &
 * Saunders) on B c = P f with B = P A and P = F^{-1} G~_hss^+ (one URV solve + 2D inverse DFT, no
 * refinement), B^* = A^* P^* (2D DFT + adjoint URV solve).  A and A^* are the exact FP64 apply of
 * Eq. 1 (this library has no NUFFT).  d_f: M x nrhs, d_c: N x nrhs, complex128, as for solve.
 * Each column stops when its estimated ||P f - B c|| / ||P f|| <= tol, or after maxit
 * iterations.  With a MIXED handle P is applied in FP32, so B is linear only to FP32 level: the
 * LSQR then runs inside an outer defect correction on the exact FP64 residual r = f - A c
 * (LSQR on B x = P r to max(tol, 1e-5), c += x), until ||P r|| <= tol ||P f|| per column.
 * *iters (may be NULL): LSQR iterations of the slowest column, summed over the passes; *relres
 * (may be NULL): the largest ||f - A c|| / ||f|| over the columns (exact apply).  For data in the
 * range of A the result is the least-squares solution; otherwise it differs from it by O(eps)
 * times the least-squares residual (left preconditioning).  Synchronises the stream.
 * Errors: ESTATE (not factored), EINVAL. */
nudft2_status nudft2_hss_plsqr(nudft2_hss_t h, const void* d_f, int64_t ldf, int nrhs, void* d_c, int64_t ldc,
                               double tol, int maxit, int* iters, double* relres, void* stream);

/* Factor store (not in the paper; the reuse of the offline stage across runs, Sec. 4.1).
 * nudft2_hss_save writes a factored handle to the file `path`: a versioned header (the options, M,
 * nx, ny, the tree depths), the points, then every HSS generator and URV factor, entries in the
 * handle's precision (complex128 for FP64, complex64 for MIXED) -- about the handle's device
 * memory (nudft2_hss_info().device_bytes).  Checkpointed levels are recomputed first.  Errors:
 * ESTATE (not factored), EINVAL (file cannot be written), ECUDA.
 * nudft2_hss_load reads such a file into a new factored handle (*out) on which solve, apply, grad
 * and plsqr give the same results as on the saved one; no construction or factorization runs.
 * The header and the points are validated on the host before any device work.  Errors: EINVAL (no
 * such file, not a factor store, another version, truncated or corrupt contents), ENOMEM, ECUDA;
 * *out is NULL on error. */
nudft2_status nudft2_hss_save(nudft2_hss_t h, const char* path);
nudft2_status nudft2_hss_load(const char* path, void* stream, nudft2_hss_t* out);

/* Per-level checkpointing of the URV factors (Sec. 2.3 storage; not in the paper): hand back the
 * device memory of the factors of the top `levels` tree levels and of the root (levels >= L: all
 * of them), keeping the HSS generators and the factors of the levels below.  The next call that
 * needs the factorization (solve, PINV / PINV_ADJ apply, grad, plsqr) recomputes the handed-back
 * levels first, level by level from the kept ones: the same factors, bit for bit, at the cost of
 * factoring those levels again.  The top levels hold most of the factor memory (their blocks are
 * O(sqrt(N)) wide), so this is the memory/time trade of a backward pass that keeps a handle
 * between its forward solve and its adjoint.  Errors: ESTATE (not factored), EINVAL. */
nudft2_status nudft2_hss_checkpoint(nudft2_hss_t h, int levels, void* stream);

/* Statistics of the handle (ranks, stage times, memory).  Errors: EINVAL (NULL). */
nudft2_status nudft2_hss_info(nudft2_hss_t h, nudft2_info* info);

/* Per-class kernel statistics recorded since build (needs NUDFT2_FLAG_PROFILE; synchronises
 * the recorded events).  Writes at most max entries to out and their count to *n.  Classes:
 * gemm (CUDA cores), gemm_tc (tensor cores, operand packing included), qr_panel, jacobi, other,
 * qrcp, and sweep (one URV solve replayed from its CUDA graph; bytes = the factor entries it
 * streams + right-hand sides in and out); in MIXED mode the handle's FP64 work (exact applies of the
 * refinement, DFTs) is listed apart with the suffix "_fp64".
 * Errors: EINVAL (NULL arguments). */
nudft2_status nudft2_hss_kstats(nudft2_hss_t h, nudft2_kstat* out, int max, int* n);

/* Release every device allocation of the handle.  NULL is ignored. */
void nudft2_hss_free(nudft2_hss_t h);

/* Direct O(MN) apply of A (Eq. 1) without building an HSS approximation, in FP64:
 * op = NUDFT2_EXACT_FWD: d_out (M x nrhs, ld ldo >= M) = A d_in (N x nrhs, ld ldi >= N);
 * op = NUDFT2_EXACT_ADJ: d_out (N x nrhs) = A^* d_in (M x nrhs).  Complex128, column major,
 * lexicographic frequency order ky + kx*ny.  Allocates and frees its own workspace.
 * Errors: EINVAL (bad sizes or op), ENOMEM, ECUDA. */
nudft2_status nudft2_exact_apply(const double* d_x, const double* d_y, int64_t M, int nx, int ny, int op,
                                 const void* d_in, int64_t ldi, int nrhs, void* d_out, int64_t ldo, void* stream);

/* Entries of the transformed 1D matrix A^x (F^x)^{-1} (Sec. 2.4, the Cauchy-like kernel
 * Psi(gamma_j, xi_k) = (1/n)((gamma_j/xi_k)^n - 1)/((gamma_j/xi_k) - 1), Psi = 1 at gamma = xi).
 * d_x: M points (device), d_out: M x n complex128 column major (ld M).  Errors: EINVAL. */
nudft2_status nudft2_psi_eval(const double* d_x, int64_t M, int n, void* d_out, void* stream);

/* nudft2_fadi_plan: host only (no device work), for tests of the shift computation of
 * NUDFT2_FLAG_FADI.  The plan of a node of d columns (first column 0) of a 1D matrix with n
 * columns at tolerance eps1: side 0 for its row block G~(J, K^c), side 1 for its column block
 * G~(J^c, K) (Sec. 3.1, the Sylvester equation of the transformed 1D matrix).  Writes the exact
 * columns (*ne entries of ex, <= 65), the J (<= 64) shift positions xa (zeros) and xb (poles) in
 * units of the circle (shift = exp(-2 pi i x)), the (ne + J)^2 mixing matrix C (column major,
 * interleaved re/im doubles) of the candidate basis a^T C, and the bound max|r|/min|r| of the
 * shifts.  All arrays are caller-owned host memory.  Returns 0, or EINVAL for a bad node (d < 1,
 * d >= n) or an eps1 needing more than 64 shifts. */
int nudft2_fadi_plan(int side, int d, int n, double eps1, int* ne, int* J, int* ex, double* xa, double* xb,
                     double* C, double* ratio);

/* nudft2_test_fail_alloc: host-side fault injection for tests (not in the paper).  With k > 0 the
 * k-th device-memory request of the library's arenas from now on fails with ENOMEM, once, on
 * whichever thread makes it; k <= 0 disarms.  Exercises the failure paths (status codes, freeing a
 * handle whose build failed) without touching the GPU. */
void nudft2_test_fail_alloc(long long k);

/* Building blocks, exposed for unit tests of the batched dense kernels.
 * prec: NUDFT2_FP64 (complex128 buffers) or NUDFT2_MIXED (complex64 buffers).
 *
 * nudft2_la_tsvd: truncated SVD of C (r x w) given Ct = C^* (w x r, ld ldct, overwritten):
 * left singular vectors with sigma_i > eps * sigma_1 (the recompression rule of Sec. 2.2) go
 * to d_p (r x min(r,w) capacity, ld ldp), their number to *rank, all min(r,w) sorted singular
 * values to h_sigma (host, double).  Errors: EINVAL. */
nudft2_status nudft2_la_tsvd(int prec, void* d_ct, int64_t w, int64_t r, int64_t ldct, double eps, void* d_p,
                             int64_t ldp, int* rank, double* h_sigma, void* stream);

/* nudft2_la_qr: Householder QR of A (m x n, ld lda) in place (R in the upper trapezoid) and the
 * explicit unitary factor Q (m x m, ld ldq) written to d_q, applying the reflectors panel by panel
 * (grouped = 0) or through the merged 256-column compact-WY blocks (grouped = 1).
 * Errors: EINVAL. */
nudft2_status nudft2_la_qr(int prec, void* d_a, int64_t m, int64_t n, int64_t lda, void* d_q, int64_t ldq,
                           int grouped, void* stream);

/* nudft2_la_qr_apply: Householder QR of A (m x n, ld lda) in place as in nudft2_la_qr, then
 * C <- Q^* C (conj = 1) or C <- Q C (conj = 0) for C (m x s, ld ldc) by the streaming
 * reflector kernels that the URV solve sweeps use (Sec. 2.3), with the 32-column panel factors
 * (grouped = 0) or the merged 256-column blocks (grouped = 1).  s >= 0 (columns are taken in
 * chunks of up to 16).  Synchronises the stream.  Errors: EINVAL. */
nudft2_status nudft2_la_qr_apply(int prec, void* d_a, int64_t m, int64_t n, int64_t lda, void* d_c, int64_t s,
                                 int64_t ldc, int conj, int grouped, void* stream);

/* nudft2_la_gemm: the batched complex GEMM behind every generator product of the construction,
 * factorization and solve:  C_b = alpha op_a(A_b) op_b(B_b) + beta C_b  for b < batch, with
 * X_b = X + b * stride_x (elements).  op: 0 = none, 1 = transpose, 2 = conjugate transpose.
 * All matrices column-major on the device (complex128 for NUDFT2_FP64, complex64 otherwise);
 * op_a(A) is m x k, op_b(B) is k x n (k = 0 allowed: C = beta C; A and B may then be NULL).
 * C must not overlap A or B.  Synchronises the stream.
 * Errors: EINVAL (bad op, size or leading dimension), ECUDA. */
nudft2_status nudft2_la_gemm(int prec, int opa, int opb, int64_t m, int64_t n, int64_t k, double alpha,
                             const void* d_a, int64_t lda, int64_t stride_a, const void* d_b, int64_t ldb,
                             int64_t stride_b, double beta, void* d_c, int64_t ldc, int64_t stride_c, int batch,
                             void* stream);

/* Allocation-free variant of the exact forward apply (NUDFT2_EXACT_FWD of nudft2_exact_apply):
 * d_f (M x nrhs, ld ldf >= M) = A d_c (N x nrhs, ld ldc == N, complex128), in FP64.
 * The paper has no counterpart: this entry point exists for callers that must not allocate
 * device memory while they run -- serving loops that reserve all device memory at start-up,
 * hosts whose own allocator owns the device, and latency-bound paths that cannot pay for
 * cudaMalloc (it may synchronise the device).  It never calls cudaMalloc/cudaFree or any
 * allocating routine; its workspace is one fixed 64 MiB device array inside the library (held
 * by every GPU that loads it, until exit).  Limit: M*(2*nx + ny)*16 bytes must fit in 64 MiB
 * minus 4 KiB (larger sizes return EINVAL); right-hand sides are processed in chunks that fit.
 * The first call on a device looks up the array's address with cudaGetSymbolAddress, so make
 * that first call before any stream capture.  All calls share the array, which keeps the last
 * call's contents: calls that overlap on the GPU race and must be serialised by the caller.
 * The call returns once its work is queued on `stream`; d_f is ready in stream order.
 * Errors: EINVAL (bad sizes, ldc != nx*ny, M or ldf >= 2^31, workspace too small), ECUDA. */
nudft2_status nudft2_exact_fwd_noalloc(const double* d_x, const double* d_y, int64_t M, int nx, int ny,
                                       const void* d_c, int64_t ldc, int nrhs, void* d_f, int64_t ldf, void* stream);

/* Measured FMA throughput of the current GPU in TFLOP/s (2 flops per FMA), for roofline
 * denominators: prec = NUDFT2_MIXED measures the FP32 FFMA pipe, NUDFT2_FP64 the DFMA pipe.  Not part
 * of the paper's method.  Runs a few fixed-length kernels (well under a second) on `stream`, with
 * a small temporary allocation, and synchronises it.  Errors: EINVAL, ECUDA. */
nudft2_status nudft2_peak_fma(int prec, double* tflops, void* stream);

/* Message of the last failing call on this thread ("" if none). */
const char* nudft2_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* NUDFT2_HSS_H */
