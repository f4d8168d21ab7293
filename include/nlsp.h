/*
 * nlsp.h -- C ABI of the GB300 (sm_103a) spectral two-level preconditioned CG
 * library (NeuraLSP, arXiv 2601.20174).
 *
 * The library solves sparse SPD systems A u = f (Sec. 3, Eq. discretized_pde)
 * by preconditioned conjugate gradient (Sec. 4, "Two-grid Solver Evaluation")
 * where every iteration applies the two-level preconditioner of Algorithm 1:
 * weighted-Jacobi pre-smoothing, residual, restriction P^T rho through a dense
 * n x k prolongation P, a k x k Galerkin coarse solve with A_c = P^T A P,
 * prolongation z += P e_c and post-smoothing.  P is the span of the leading k
 * left singular vectors of Jacobi-smoothed random vectors (Sec. 3,
 * "Near-Nullspace Vectors" and "SVD-Centric Construction of Coarse Bases");
 * the exact thin SVD stands in for the paper's learned map f_theta, whose
 * global optima it is (Thm. 1, Cor. 2).
 *
 * Call order (Algorithm 1, setup then apply): nlsp_create ->
 * nlsp_assemble_stencil -> nlsp_build_prolongation (or nlsp_prec_from_basis)
 * -> nlsp_factor_coarse -> nlsp_solve / nlsp_apply_prec -> nlsp_free_* ->
 * nlsp_destroy.
 *
 * Conventions for every entry point:
 *   - Pointers named dev_* are device pointers of the context's device; the
 *     caller owns them, keeps them alive until the enqueued work completes,
 *     and the library never frees them.  Other pointers are host pointers.
 *   - Vectors over the grid are FP64, length n, node order x fastest
 *     (2D: j*N + i; 3D: (l*N + j)*N + i).  Blocks of vectors are column-major
 *     with a leading dimension ld >= n (in elements).
 *   - The library owns nlsp_op / nlsp_prec objects (and the device memory
 *     inside them) until nlsp_free_op / nlsp_free_prec.  An nlsp_prec keeps a
 *     reference to the nlsp_op it was built for; free the prec first.
 *   - All device work is enqueued on the context's stream.  Functions return
 *     after enqueueing, except where "synchronises" is stated.
 *   - Errors are returned as nlsp_status codes; nothing is thrown across the
 *     ABI.  Device-side failures (non-positive pivot, CG breakdown) are
 *     reported through status words that the synchronising calls read.
 *     After NLSP_ERR_CUDA the context should be destroyed.
 *   - Not thread-safe: one host thread per context at a time.
 */
#ifndef NLSP_H_
#define NLSP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define NLSP_API __attribute__((visibility("default")))
#else
#define NLSP_API
#endif

/* Capacity of nlsp_apply_prec_noalloc's static scratch. */
#define NLSP_NOALLOC_MAX_N 262144
#define NLSP_NOALLOC_MAX_RANK 128

typedef struct nlsp_ctx nlsp_ctx;
typedef struct nlsp_op nlsp_op;
typedef struct nlsp_prec nlsp_prec;

typedef enum {
  NLSP_OK = 0,
  NLSP_NOT_CONVERGED = 1,   /* maxit reached; results and info are filled   */
  NLSP_ERR_INVALID = -1,    /* bad argument, size or parameter combination   */
  NLSP_ERR_CUDA = -2,       /* a CUDA runtime call failed                    */
  NLSP_ERR_NOT_SPD = -3,    /* non-positive pivot in the Cholesky of A_c     */
  NLSP_ERR_BREAKDOWN = -4,  /* p^T A p <= 0, r^T z <= 0 or non-finite scalar */
  NLSP_ERR_TIMEOUT = -5,    /* a bounded device wait gave up                 */
  NLSP_ERR_OOM = -6         /* device allocation failed                      */
} nlsp_status;

/* Arithmetic of the preconditioner (outer PCG recurrences are always FP64). */
typedef enum {
  NLSP_FP64 = 0,        /* everything FP64                                   */
  NLSP_MIXED_FP32 = 1,  /* setup and preconditioner FP32 (FP64 reductions),
                           A_c Cholesky and the PCG recurrences FP64         */
  NLSP_MIXED_BF16 = 2,  /* as NLSP_MIXED_FP32, and in the block solver
                           (nlsp_solve_block) the restriction P_r^T rho and
                           the prolongation P_r E run on tensor cores with
                           BF16 operands (P and rho / E rounded to nearest)
                           and FP32 accumulation                             */
  NLSP_MIXED_TF32 = 3   /* the same with TF32 operands                       */
} nlsp_precision;

/* Coefficient layouts for nlsp_assemble_stencil. */
enum {
  NLSP_COEF_CELL_KAPPA = 0,   /* cell-centred diffusion coefficient kappa > 0:
                                 2D (N+1)^2 values [cj][ci], 3D (N+1)^3
                                 values [cl][cj][ci] (x fastest)            */
  NLSP_COEF_CONST_TENSOR = 1  /* constant 2D tensor {a_xx, a_yy, a_xy},
                                 positive definite (9-point stencil)        */
};

/* Algorithm 1 inputs: K test vectors, rank k, weight omega, s1 smoothing
   steps for the samples, nu1 / nu2 pre / post sweeps. */
typedef struct {
  int K;
  int k;
  int s1;
  int nu1;
  int nu2;
  double omega;
  int precision;            /* nlsp_precision */
  unsigned long long seed;  /* S0 stream seed when no S0 is passed */
} nlsp_setup_params;

/* Stream number of the random test vectors S0 in the counter-based generator
   (SplitMix64 counter streams, Box-Muller normals). */
#define NLSP_STREAM_S0 3
/* Stream number of the Gaussian sketch of the randomised-SVD setup. */
#define NLSP_STREAM_SKETCH 11

typedef struct {
  double tol;     /* stop when ||r||_2 <= tol ||b||_2 (recursive residual)  */
  int maxit;      /* iteration cap (>= 1)                                    */
  int flexible;   /* 1: Polak-Ribiere beta; 0: standard; -1: flexible iff
                     the preconditioner is not FP64                         */
  int graph_mode; /* 2: one persistent cooperative kernel per right-hand
                     side runs the whole solve (phases separated by a
                     bounded grid barrier; NLSP_ERR_TIMEOUT if a barrier
                     wait gives up); 1: the loop is one CUDA graph with a
                     device-side while node; 0: graph of one iteration
                     relaunched by the host, checking convergence every
                     few iterations (profilers see each kernel)            */
} nlsp_solve_params;

typedef struct {
  int iterations;      /* products A p taken until the stop test passed     */
  int status;          /* nlsp_status of this right-hand side               */
  double relres;       /* recursive ||r|| / ||b|| at exit                    */
  double true_relres;  /* ||b - A x|| / ||b|| recomputed in FP64 at exit     */
} nlsp_solve_info;

/* Human-readable name of a status code (static string). */
NLSP_API const char* nlsp_status_string(int status);

/* Message of the last failed CUDA runtime call on this host thread (static,
   thread-local string; empty if none). */
NLSP_API const char* nlsp_last_error(void);

/* Creates a context on CUDA device `device`, enqueueing on `cuda_stream`
   (a cudaStream_t, borrowed, not destroyed by the library; NULL = the legacy
   default stream).  Errors: NLSP_ERR_INVALID (no such device),
   NLSP_ERR_CUDA. */
NLSP_API nlsp_status nlsp_create(nlsp_ctx** ctx_out, int device, void* cuda_stream);

/* Replaces the stream that later calls enqueue on (borrowed). */
NLSP_API nlsp_status nlsp_set_stream(nlsp_ctx* ctx, void* cuda_stream);

/* Destroys the context; ops and precs must have been freed.  Synchronises. */
NLSP_API void nlsp_destroy(nlsp_ctx* ctx);

/* ---------------------------------------------------------------------------
 * Operator A (Sec. 3, Eq. discretized_pde; the diffusion / anisotropic PDE
 * families of the Appendix on structured grids, Dirichlet nodes eliminated).
 *   dim = 2, points = 5, layout CELL_KAPPA: -div(kappa grad u), edge weight =
 *       mean kappa of the 2 cells sharing the edge, h = 1/(N+1), A scaled h^-2.
 *   dim = 2, points = 9, layout CONST_TENSOR: -(a_xx u_xx + 2 a_xy u_xy +
 *       a_yy u_yy) with the centred cross difference.
 *   dim = 3, points = 7, layout CELL_KAPPA: edge weight = mean of 4 cells.
 * grid = {N, N, N or 1}: only cubic / square grids (N >= 1).
 * dev_coeffs: device FP64, read during the call (may be freed afterwards).
 * Stores the operator coefficients in FP64 and FP32.  Synchronises.
 * Errors: NLSP_ERR_INVALID (unsupported combination, non-positive diagonal),
 * NLSP_ERR_OOM, NLSP_ERR_CUDA.
 * ------------------------------------------------------------------------- */
NLSP_API nlsp_status nlsp_assemble_stencil(nlsp_ctx* ctx, int dim, const int64_t grid[3], int points,
                                  const double* dev_coeffs, int coeff_layout, nlsp_op** A_out);

/* General sparse SPD operator from compressed sparse rows (Sec. 3, Eq.
   discretized_pde, for any SPD A; the paper's own matrices are P1 finite-
   element stiffness and mass matrices on unstructured meshes, Appendix "FEM
   Dataset Generation").  Row i holds entries dev_val[q] in columns
   dev_col[q] for q in [dev_rowptr[i], dev_rowptr[i+1]); dev_rowptr has n + 1
   entries from 0 to nnz.  Entries of a row need not be sorted; repeated
   (row, column) pairs are summed.  Every row must have a positive diagonal
   (the Jacobi smoother divides by it); A must be symmetric positive definite,
   which is not checked beyond the diagonal.  All three arrays are device
   memory read during the call (they may be freed afterwards).  The library
   stores the diagonal, its inverse and the off-diagonal entries in row
   slices of 32 rows (sliced ELLPACK, each slice as wide as its longest row)
   in FP64 and FP32.  Every entry point that takes an nlsp_op accepts it.
   1 <= n < 2^31, nnz >= n.  Synchronises.  Errors: NLSP_ERR_INVALID (row
   pointers not monotone from 0 to nnz, a column outside [0, n), a missing,
   non-positive or non-finite diagonal, a non-finite entry; message in
   nlsp_last_error), NLSP_ERR_OOM, NLSP_ERR_CUDA. */
NLSP_API nlsp_status nlsp_assemble_csr(nlsp_ctx* ctx, int64_t n, int64_t nnz, const int64_t* dev_rowptr,
                                       const int32_t* dev_col, const double* dev_val, nlsp_op** A_out);

/* Number of unknowns n of the operator. */
NLSP_API int64_t nlsp_op_size(const nlsp_op* A);

/* Y = A X for m columns (FP64).  X is n x m (ldx), Y is n x m (ldy); X and Y
   must not overlap.  Errors: NLSP_ERR_INVALID. */
NLSP_API nlsp_status nlsp_op_apply(nlsp_ctx* ctx, const nlsp_op* A, int m, const double* dev_X, int64_t ldx,
                          double* dev_Y, int64_t ldy);

/* D = diag(A) (Algorithm 1 setup), n values FP64. */
NLSP_API nlsp_status nlsp_op_diagonal(nlsp_ctx* ctx, const nlsp_op* A, double* dev_d);

NLSP_API void nlsp_free_op(nlsp_op* A);

/* ---------------------------------------------------------------------------
 * Setup (Algorithm 1, setup).
 * ------------------------------------------------------------------------- */

/* S = (I - omega D^-1 A)^s1 S0 (Sec. 3, Near-Nullspace Vectors), computed in
   `precision` and returned in FP64.  S0 and S are n x K column-major
   (ld = n) and may be the same buffer.  Errors: NLSP_ERR_INVALID. */
NLSP_API nlsp_status nlsp_smooth_samples(nlsp_ctx* ctx, const nlsp_op* A, int K, int s1, double omega,
                                int precision, const double* dev_S0, double* dev_S);

/* Builds a preconditioner for A from the random test vectors dev_S0 (n x K,
   column-major, ld = n, read during the call; NULL: drawn on the device as
   N(0,1) from the counter-based generator of nlsp_random_normal with
   params->seed and stream NLSP_STREAM_S0, element (i, c) being normal number
   c n + i; the Box-Muller transform is evaluated in the setup precision, so
   NLSP_MIXED_FP32 samples agree with the FP64 stream to a few FP32 ulps):
   smooths them s1 times, takes
   the leading k left singular vectors of S as P (thin SVD via the Gram
   matrix S^T S, a one-sided Jacobi eigensolver (K > 128: on a cluster of
   two CTAs) and, in FP64, iterative refinement), then forms and factors
   A_c = P^T A P for the full rank k (call nlsp_factor_coarse to
   truncate).  Requires 1 <= k <= 128, k <= K <= 256, K <= n,
   nu1 = nu2 >= 1 (PCG needs a symmetric preconditioner) and
   0 < omega < 2.  Synchronises.  Errors: NLSP_ERR_INVALID, NLSP_ERR_NOT_SPD
   (rank-deficient samples), NLSP_ERR_OOM, NLSP_ERR_CUDA. */
NLSP_API nlsp_status nlsp_build_prolongation(nlsp_ctx* ctx, const nlsp_op* A, const nlsp_setup_params* params,
                                    const double* dev_S0, nlsp_prec** M_out);

/* As nlsp_build_prolongation, with the A-weighted spectral basis of the
   Appendix (Galerkin Convergence): the Gram matrix of the smoothed samples is
   S^T A S, so that P = S V_k Sigma_k^-1 satisfies P^T A P = I and A^{1/2} P
   spans the top-k left singular subspace of A^{1/2} S, the coarse space that
   minimises ||A^{1/2} (I - Pi_A(P)) S||_F^2.  The singular values reported
   (nlsp_prec_copy_sigma) are those of A^{1/2} S.  Same arguments and errors,
   except that K <= 128. */
NLSP_API nlsp_status nlsp_build_prolongation_a_weighted(nlsp_ctx* ctx, const nlsp_op* A,
                                                        const nlsp_setup_params* params, const double* dev_S0,
                                                        nlsp_prec** M_out);

/* As nlsp_build_prolongation, with the randomised SVD in place of the exact
   thin SVD (the paper's RandomSVD basis, Sec. 4 baselines; Halko, Martinsson
   and Tropp 2011: randomised range finder with power iterations, then the SVD
   of the small projected matrix): with l = k + oversample columns of a
   Gaussian sketch Omega (K x l), Q = qf(S Omega), power_iters times
   Q = qf(S qf(S^T Q)), then P = Q U_B[:, :k] for the left singular vectors
   U_B of B = Q^T S.  dev_sketch: Omega, FP64 column-major K x l (device,
   read during the call), or NULL to draw it on the device from the
   counter-based generator of nlsp_random_normal with params->seed and stream
   NLSP_STREAM_SKETCH (element (c, j) is normal number j K + c).  The
   singular values reported are those of B (l values, zeros beyond).
   Requires 0 <= oversample, k + oversample <= K <= 128, 0 <= power_iters <=
   16; other arguments and errors as nlsp_build_prolongation (NLSP_ERR_NOT_SPD
   also when S Omega is rank deficient). */
NLSP_API nlsp_status nlsp_build_prolongation_randomized(nlsp_ctx* ctx, const nlsp_op* A,
                                                        const nlsp_setup_params* params, const double* dev_S0,
                                                        int oversample, int power_iters, const double* dev_sketch,
                                                        nlsp_prec** M_out);

/* Builds a preconditioner from a given basis dev_P (n x k column-major,
   ld = n, FP64, read during the call), e.g. the basis a learned map
   produces from the smoothed samples, after its QR layer (Sec. 3 and the
   setup of Algorithm 1).  P need not be orthonormal, only of full column
   rank.
   params->K and params->s1 are ignored.  Factors A_c for rank k.
   Synchronises.  Errors as nlsp_build_prolongation. */
NLSP_API nlsp_status nlsp_prec_from_basis(nlsp_ctx* ctx, const nlsp_op* A, const nlsp_setup_params* params,
                                 const double* dev_P, int k, nlsp_prec** M_out);

/* Draws normals offset .. offset + count - 1 of a counter-based stream into
   dev_out (FP64): the i-th uniform of stream s under seed q is the top 53
   bits of SplitMix64 output i + 1 started at base(q, s) =
   fin(q ^ s * 0xD1B54A32D192ED03 + 0x9E3779B97F4A7C15) (fin = the SplitMix64
   finaliser); normals 2j, 2j+1 are sqrt(-2 log(1 - u_2j)) * (cos, sin)(2 pi
   u_2j+1) (Box-Muller).  This is the definition the host-side input
   generator implements; the random test vectors S0 of Sec. 3 come from it.
   Errors: NLSP_ERR_INVALID. */
NLSP_API nlsp_status nlsp_random_normal(nlsp_ctx* ctx, unsigned long long seed, unsigned long long stream,
                                        unsigned long long offset, int64_t count, double* dev_out);

/* Self-test of the solver's FP64 <-> FP32 conversions, which run on the
   integer pipe (bit operations on the IEEE-754 encodings) because GB300
   executes conversion instructions on its slow FP64 unit.  dev_bits holds n
   64-bit patterns (device memory, read during the call): each is converted
   as an FP64 value to FP32 (round to nearest even) and its low 32 bits as an
   FP32 value to FP64 (exact), and both results are compared bit for bit
   with the hardware conversions (any NaN matches any NaN).  *mismatches (host)
   receives the number of differing results.  Synchronises.  Errors:
   NLSP_ERR_INVALID, NLSP_ERR_CUDA. */
NLSP_API nlsp_status nlsp_check_conversions(nlsp_ctx* ctx, const unsigned long long* dev_bits, int64_t n,
                                            unsigned long long* mismatches);

/* Truncates the coarse space to its first r columns (Algorithm 1 setup:
   P_r = P[:, 1:r], A_c = P_r^T A P_r) and factors A_c = L L^T in FP64.
   1 <= r <= k.  Synchronises.  Errors: NLSP_ERR_INVALID, NLSP_ERR_NOT_SPD. */
NLSP_API nlsp_status nlsp_factor_coarse(nlsp_ctx* ctx, const nlsp_op* A, nlsp_prec* M, int r);

/* Dimensions of a preconditioner: n, built rank k, active rank r, K (0 when
   built from a basis) and precision.  Host pointers, any may be NULL. */
NLSP_API nlsp_status nlsp_prec_dims(const nlsp_prec* M, int64_t* n, int* k, int* r, int* K, int* precision);

/* Copies out P (n x k, column-major, ld = n, FP64; the stored basis,
   converted from FP32 in mixed precision). */
NLSP_API nlsp_status nlsp_prec_copy_basis(nlsp_ctx* ctx, const nlsp_prec* M, double* dev_P);

/* Copies out the singular values sigma_1 >= ... >= sigma_K of S (K values,
   FP64; zeros when built from a basis). */
NLSP_API nlsp_status nlsp_prec_copy_sigma(nlsp_ctx* ctx, const nlsp_prec* M, double* dev_sigma);

/* Copies out A_c (r x r) and its lower Cholesky factor L (r x r), both
   column-major FP64 (either pointer may be NULL). */
NLSP_API nlsp_status nlsp_prec_copy_coarse(nlsp_ctx* ctx, const nlsp_prec* M, double* dev_Ac, double* dev_L);

NLSP_API void nlsp_free_prec(nlsp_prec* M);

/* ---------------------------------------------------------------------------
 * Apply and solve.
 * ------------------------------------------------------------------------- */

/* Z = B R for m columns: one application of the two-level preconditioner
   (Algorithm 1, "Apply preconditioner to residual b").  R, Z FP64, n x m
   (ldr, ldz >= n); must not overlap.  Computed in the prec's precision.
   Errors: NLSP_ERR_INVALID. */
NLSP_API nlsp_status nlsp_apply_prec(nlsp_ctx* ctx, const nlsp_prec* M, int m, const double* dev_R, int64_t ldr,
                            double* dev_Z, int64_t ldz);

/* Same as nlsp_apply_prec, but allocates no device memory: no cudaMalloc,
   cudaFree or allocating library routine is called, and the preconditioner's
   own lazily created solver workspace is not touched.  The paper has no
   counterpart; this exists for callers that cannot allocate while they run:
   code that enqueues work inside its own stream capture (allocation and
   freeing synchronise the device and are not allowed while capturing), and
   applications whose memory pool owns all of device memory under a fixed
   cap.  M itself must have been built beforehand (that does allocate).
   Temporaries live in one static device array, sized for
   n <= NLSP_NOALLOC_MAX_N and a stored basis of k <= NLSP_NOALLOC_MAX_RANK
   columns (the rank M was built with, whatever rank it is truncated to; about
   7 MB, held by every GPU that loads the library until the process exits);
   larger problems return NLSP_ERR_INVALID (message in nlsp_last_error).
   The first call on a device looks up the array's device address (a CUDA
   runtime call, done once per device with that device current): make that
   first call before any stream capture.  All calls share the array and it
   keeps the last call's contents; what must start at zero is cleared on the
   stream by each call.  Calls whose work overlaps on the GPU (different
   streams or contexts of one process) race on the array.
   Errors: NLSP_ERR_INVALID, NLSP_ERR_CUDA. */
NLSP_API nlsp_status nlsp_apply_prec_noalloc(nlsp_ctx* ctx, const nlsp_prec* M, int m, const double* dev_R,
                                             int64_t ldr, double* dev_Z, int64_t ldz);

/* Solves A X = B for m right-hand sides by PCG with the two-level
   preconditioner M (Sec. 4; tolerance on the relative residual, x0 = 0 --
   dev_X is output only).  Columns run independent recurrences; a converged
   column is frozen.  infos: host array of m entries (may be NULL).
   Synchronises.  Returns NLSP_OK when every column converged,
   NLSP_NOT_CONVERGED if one hit maxit, NLSP_ERR_BREAKDOWN if one broke
   down (per-column status in infos), NLSP_ERR_INVALID, NLSP_ERR_CUDA. */
NLSP_API nlsp_status nlsp_solve(nlsp_ctx* ctx, const nlsp_op* A, const nlsp_prec* M, int m, const double* dev_B,
                       int64_t ldb, double* dev_X, int64_t ldx, const nlsp_solve_params* params,
                       nlsp_solve_info* infos);

/* Block PCG: A X = B for m <= 32 right-hand sides advanced together, one
   independent PCG recurrence per column (Sec. 4), so that each
   preconditioner application (Algorithm 1) reads P once for all columns: the
   restriction is the dense product P_r^T rho (r x m) and the prolongation
   P_r E (n x m).  Same arguments, stopping rule and per-column results as
   nlsp_solve (params->graph_mode is ignored); x0 = 0.  Uses the active rank
   r <= 128 of M.  The two products run on tcgen05 tensor cores: with FP32
   inputs split into TF32 high and low parts (three products, FP32 accuracy)
   for NLSP_MIXED_FP32 (restriction only; the prolongation on CUDA cores),
   with BF16 or TF32 operands and FP32 accumulation (both products, from a
   copy of P repacked once per call) for NLSP_MIXED_BF16 / NLSP_MIXED_TF32;
   FP64 preconditioners use CUDA cores.  Allocates its block workspace (about 80 m n bytes) for the
   duration of the call.  Synchronises.  Errors: NLSP_ERR_INVALID,
   NLSP_ERR_CUDA, NLSP_ERR_OOM; per-column NLSP_NOT_CONVERGED /
   NLSP_ERR_BREAKDOWN as nlsp_solve. */
NLSP_API nlsp_status nlsp_solve_block(nlsp_ctx* ctx, const nlsp_op* A, const nlsp_prec* M, int m,
                                      const double* dev_B, int64_t ldb, double* dev_X, int64_t ldx,
                                      const nlsp_solve_params* params, nlsp_solve_info* infos);

/* Block Krylov solve of A X = B for m <= 32 right-hand sides: the columns
   share one search space (the block conjugate gradient of O'Leary 1980, in
   the breakdown-free form of Ji & Li 2017: every iteration the search block
   Z + P beta is re-orthonormalised by a pivoted Cholesky QR that drops the
   directions whose relative pivot is below 1e-14 -- converged columns,
   dependent right-hand sides), preconditioned by the two-level
   preconditioner of Algorithm 1 through the same kernels as
   nlsp_solve_block.  The paper solves each right-hand side by its own PCG;
   this is the block-Krylov alternative.  Arguments and results as
   nlsp_solve_block; infos[c].iterations is the block iteration at which
   column c first met ||r_c|| <= tol ||b_c|| (the block continues until every
   column has).  All block quantities (X, R, P, A P, the Gram matrices and
   small solves) are FP64.  Allocates its workspace for the call.
   Synchronises.  Errors as nlsp_solve_block. */
NLSP_API nlsp_status nlsp_solve_block_cg(nlsp_ctx* ctx, const nlsp_op* A, const nlsp_prec* M, int m,
                                         const double* dev_B, int64_t ldb, double* dev_X, int64_t ldx,
                                         const nlsp_solve_params* params, nlsp_solve_info* infos);

/* Batched solve: instance i solves A_i x_i = b_i by PCG with its own
   preconditioner M[i] (Sec. 4 per instance; the paper solves its instances
   one after another and has no batched counterpart).  One cooperative launch
   of the persistent solver runs every instance on a team of consecutive
   CTAs (one CTA per SM); the team plan is the one nlsp_plan_teams returns
   for the instances' node counts, tiles_per_cta and the device's SM count.
   M: host array of `count` distinct preconditioners of this context, all
   of one stencil kind and one precision.  dev_b, dev_x: host arrays of
   `count` device pointers to FP64 vectors of length n_i; x0 = 0 and x_i is
   output only (must not be b_i).  params: tol, maxit and flexible as in
   nlsp_solve (graph_mode is ignored).  tiles_per_cta: target number of
   128-node tiles per CTA of a team (0: the value nlsp_tune_batched measured
   for a batch of the same sizes on this context, else 16).  infos: host array of `count`
   entries (may be NULL).  Synchronises.  A team barrier gives up after 2 s
   without progress anywhere in the launch (no instance finished an
   iteration), and its instance ends with NLSP_ERR_TIMEOUT.  Returns as nlsp_solve
   (the worst per-instance status), or NLSP_ERR_INVALID, NLSP_ERR_CUDA,
   NLSP_ERR_OOM. */
NLSP_API nlsp_status nlsp_solve_batched(nlsp_ctx* ctx, int count, nlsp_prec* const* M, const double* const* dev_b,
                                        double* const* dev_x, const nlsp_solve_params* params, int tiles_per_cta,
                                        nlsp_solve_info* infos);

/* Autotuner of the batched solver's team size: times one nlsp_solve_batched
   of these instances for each of the `ncand` candidate tiles_per_cta values
   (after one untimed warm-up solve each; CUDA events on the context stream),
   stores the fastest in *best (host) and the times in ms_out[ncand] (host,
   may be NULL), and remembers it in the context for this signature of the
   batch (stencil kind, precision and every instance's node count and active
   rank, in order; the last 8 signatures are kept): later nlsp_solve_batched
   calls with tiles_per_cta = 0 on instances of the same sizes use it.  The
   paper has no counterpart.  dev_x receive the solutions (each solve
   overwrites them).  Arguments as nlsp_solve_batched; candidates >= 1.
   Synchronises.  Errors: NLSP_ERR_INVALID, and any error of the solves. */
NLSP_API nlsp_status nlsp_tune_batched(nlsp_ctx* ctx, int count, nlsp_prec* const* M, const double* const* dev_b,
                                       double* const* dev_x, const nlsp_solve_params* params, const int* candidates,
                                       int ncand, int* best, double* ms_out);

/* The batched solver's team plan (host computation only, no device work).
   Instance i of n[i] nodes (n[i] >= 1) gets team_size[i] =
   clamp(ceil(ceil(n[i] / 128) / tiles_per_cta), 1, min(num_ctas,
   ceil(n[i] / 128))) consecutive CTAs starting at first_cta[i]; start[i] is
   its planned start time in a tile-iteration cost model.  Teams are placed
   largest estimated area first, each in the window of CTAs that frees
   earliest.  Each CTA runs its instances in (start, instance) order, which
   is the same order for every CTA of a team; that is what makes the
   launch free of deadlock.  tiles_per_cta = 0 means 16.  Output arrays
   hold `count` entries.  Errors: NLSP_ERR_INVALID. */
NLSP_API nlsp_status nlsp_plan_teams(int count, const int64_t* n, int num_ctas, int tiles_per_cta, int* first_cta,
                                     int* team_size, double* start);

/* ---------------------------------------------------------------------------
 * Differentiation (the objectives of Sec. 3 and the Appendix).
 * ------------------------------------------------------------------------- */

/* Subspace loss L = ||(I - Q Q^T) B||_F^2 with Q = qf(P_hat), the thin-Q
   factor of P_hat (Sec. 3, the QR layer after the learned map; minimising this residual energy
   maximises the subspace energy, Appendix on the optimality of smooth error
   reduction), and optionally its gradient dL/dP_hat.  P_hat: n x k, B: n x K
   (e.g. the smoothed samples), both FP64 column-major (ld = n), read during
   the call.  precision: NLSP_FP64, or NLSP_MIXED_FP32 for FP32 arithmetic
   with FP64 sums of the k x k / k x K products.  *loss is a host pointer;
   dev_grad (n x k, FP64, ld = n) may be NULL.  k <= 128, K <= 256, P_hat of
   full column rank.  Synchronises.  Errors: NLSP_ERR_INVALID,
   NLSP_ERR_NOT_SPD (P_hat^T P_hat not positive definite), NLSP_ERR_CUDA,
   NLSP_ERR_OOM. */
NLSP_API nlsp_status nlsp_subspace_loss(nlsp_ctx* ctx, int64_t n, int k, int K, int precision,
                                        const double* dev_Phat, const double* dev_B, double* loss, double* dev_grad);

/* Nested subspace loss (NLSS, Sec. 3 "Eq. nlss_loss"): with Q = qf(P_hat)
   and S the n x K sample block, L = (1/k) sum_{l=1..k} (1 - ||Q_{1:l}^T S||_F^2 /
   ||S||_F^2), whose minimum over P_hat is reached by the leading singular
   vectors in order (Thm. 1 / Cor. 2), and optionally dL/dP_hat.  Unlike the
   subspace loss it depends on the order of Q's columns, not only on
   range(P_hat).  Arguments, precision and errors as nlsp_subspace_loss
   (dev_S in place of dev_B). */
NLSP_API nlsp_status nlsp_nlss_loss(nlsp_ctx* ctx, int64_t n, int k, int K, int precision, const double* dev_Phat,
                                    const double* dev_S, double* loss, double* dev_grad);

/* Unrolled-PCG loss L = ||r_T||_2 after exactly T PCG iterations (Sec. 4,
   standard beta, x0 = 0) on A x = b with the two-level preconditioner of
   Algorithm 1 built from the full-rank basis P (A_c = P^T A P, Cholesky;
   nu pre- and post-sweeps of weighted Jacobi with weight omega), and
   optionally dL/dP by reverse mode through the T iterations (the forward
   states are kept as per-iteration checkpoints).  The paper trains with
   subspace objectives only; this loss differentiates the solver itself.
   P: n x k FP64 column-major (ld = n); b: FP64 length n; *loss host;
   dev_grad (n x k, FP64, ld = n) may be NULL.  precision: NLSP_FP64, or
   NLSP_MIXED_FP32 (FP32 preconditioner, FP64 recurrences).  k <= 128,
   1 <= T <= 1000.  Synchronises.  Errors: NLSP_ERR_INVALID,
   NLSP_ERR_NOT_SPD (A_c not positive definite), NLSP_ERR_CUDA,
   NLSP_ERR_OOM. */
NLSP_API nlsp_status nlsp_unrolled_pcg(nlsp_ctx* ctx, const nlsp_op* A, const double* dev_P, int k, int nu,
                                       double omega, int precision, const double* dev_b, int T, double* loss,
                                       double* dev_grad);

/* ---------------------------------------------------------------------------
 * Instrumentation (no counterpart in the paper).
 * ------------------------------------------------------------------------- */

/* Number of kernels this context has enqueued so far (host count, including
   the kernels of every executed PCG graph iteration). */
NLSP_API unsigned long long nlsp_launch_count(const nlsp_ctx* ctx);

/* Enqueues `reps` back-to-back launches of one hot kernel of the
   preconditioner apply on M's internal work vectors (their contents are
   whatever the last apply or solve left; results are discarded), so that a
   caller can time one launch with events recorded on the context stream.
   which: 0 = residual + restriction P_r^T rho (with the coarse solve in its
   last block), 1 = prolongation z += P_r e_c.  Errors: NLSP_ERR_INVALID. */
NLSP_API nlsp_status nlsp_bench_kernel(nlsp_ctx* ctx, const nlsp_prec* M, int which, int reps);

/* Phase timers of the persistent solver (graph_mode 2), accumulated over the
   solves since the last call and then reset: out_ns[2 p] = time CTA 0 spent
   in phase p before its grid barrier, out_ns[2 p + 1] = its wait at that
   barrier, for p = spmv, pre, stored sweeps, restrict, prolong, post, other
   (14 values); then 12 marks inside the phases (time since the previous
   mark or barrier release): spmv totals, spmv nodes, pre totals, pre nodes,
   restrict rho, restrict resident tiles, restrict streamed tiles, restrict
   reduction, prolong coarse solve, prolong resident tiles, prolong streamed
   tiles, post nodes, spmv totals issued, spmv totals finished, restrict stage
   A, restrict stage B, post stage (31 values in all).  Recording is enabled by the environment variable
   NLSP_PHASE_TIMERS=1 when the solver workspace is first created; otherwise
   zeros.  Synchronises. */
NLSP_API nlsp_status nlsp_prec_phase_times(nlsp_ctx* ctx, const nlsp_prec* M, double* out_ns, int count);

#ifdef __cplusplus
}
#endif

#endif /* NLSP_H_ */
