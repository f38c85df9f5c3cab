/*
 * pase.h - C ABI of a GB300 (sm_103a) implementation of the augmented subspace
 * eigensolver of Liao, Liu, Xie and Wang, "PASE: A Massively Parallel Augmented
 * Subspace Eigensolver for Large Scale Eigenvalue Problems" (arXiv 2502.04589).
 *
 * Problem (paper §2.1, §3 Alg. 3 "Require/Ensure"): the nev smallest eigenpairs of the
 * symmetric-definite pencil A_h u = lambda M_h u (M_h is the paper's B_h), given a
 * coarse space V_H subset V_h through an interpolation chain P (the paper's I_H^h; its
 * transpose is the restriction I_h^H) and the coarse pencil (A_H, M_H).
 *
 * One augmented subspace iteration (Alg. 1; Alg. 3 steps 3-6) on the block U [N][m]:
 *   (a) W  = linear solve of A_h w_i = lambda_i M_h u_i from the guess u_i   (pase_linear_solve)
 *   (b) aH = P^T A_h W, bH = P^T M_h W, GA = W^T A_h W, GM = W^T M_h W      (pase_project)
 *   (c) the m smallest pairs of [[A_H, aH],[aH^T, GA]], [[M_H, bH],[bH^T, GM]] (pase_augmented_eig)
 *   (d) U  = P C_H + W C_W                                                  (pase_prolongate)
 * with the residual R = M_h U Lambda - A_h U and the relative residuals
 * ||A u - lambda M u||_2 / (lambda ||M u||_2) feeding (a) and the stopping test (pase_residual).
 *
 * Conventions for every call:
 *  - Return value: PASE_OK (0) or a negative PASE_ERR_* code; no call aborts, traps or
 *    throws.  pase_status_string() names a code; pase_last_error() gives a message.
 *  - Multivectors are dense, row-major ("node-major"): element (i, j) of an [N][m]
 *    block is at p[i*m + j]; the m entries of one node are contiguous.  m is the block
 *    width nev_w (nev plus guard columns) and must be a multiple of 8 and at most 256.
 *  - Pointers to multivectors, lambda and small matrices may be device or host
 *    memory; the library detects which (cudaPointerGetAttributes).  Host inputs are
 *    copied in and host outputs copied back inside the call, on the handle's stream,
 *    through device staging buffers that the handle keeps between calls (they grow to
 *    the largest set of host arguments one call has staged and are freed by
 *    pase_destroy).  A handle must not be used by two host threads at once.
 *  - All device work runs on the CUDA stream given to pase_create; calls return after
 *    the stream has been synchronised, so outputs are ready on return.
 *  - Borrowed inputs are only read during the call.  The handle owns all of its device
 *    memory (pase_setup, pase_reserve) and frees it in pase_destroy.
 */
#ifndef PASE_H
#define PASE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ----------------------------------------------------------------- */
#define PASE_OK 0
#define PASE_ERR_INVALID_ARG (-1)      /* null pointer, bad size, m not a multiple of 8 ...  */
#define PASE_ERR_SHAPE_MISMATCH (-2)   /* matrix shapes do not chain                           */
#define PASE_ERR_PATTERN_MISMATCH (-3) /* A_h and M_h (or A_H, M_H) differ in sparsity pattern */
#define PASE_ERR_NOT_SPD (-4)          /* a Cholesky pivot was not positive                   */
#define PASE_ERR_NAN (-5)              /* a NaN / Inf was produced or given                    */
#define PASE_ERR_NOT_CONVERGED (-6)    /* max_iter reached; outputs are still written          */
#define PASE_ERR_TIMEOUT (-7)          /* a device-side wait exceeded its limit                */
#define PASE_ERR_CUDA (-8)             /* a CUDA runtime call failed                           */
#define PASE_ERR_OUT_OF_MEMORY (-9)    /* device allocation failed                             */
#define PASE_ERR_STATE (-10)           /* call out of order (e.g. solve before setup)          */
#define PASE_ERR_BAD_CSR (-11)         /* row pointers not monotone, column out of range/unsorted */

/* ---- options ------------------------------------------------------------------------ */
#define PASE_PREC_FP64 0  /* every step in FP64                                            */
#define PASE_PREC_MIXED 1 /* step (a) in FP32 storage and arithmetic inside FP64 residual
                             correction (w = u + V32(r64)); (b)-(d) and residuals in FP64  */

#define PASE_SOLVER_VCYCLE 0 /* s V-cycles: damped Jacobi, Galerkin levels, dense coarsest */
#define PASE_SOLVER_CG 1     /* s CG steps per column, column-wise inner products (the block
                                CG of the paper's numerical section, one CG per column)   */
#define PASE_SOLVER_MGCG 2   /* s CG steps per column preconditioned by one V-cycle (robust
                                for rough coefficients); in MIXED precision the V-cycle runs
                                in FP32, the CG recurrences in FP64                           */

typedef struct {
  int precision;       /* PASE_PREC_FP64 (default) or PASE_PREC_MIXED                          */
  int linear_solver;   /* PASE_SOLVER_VCYCLE (default), PASE_SOLVER_CG or PASE_SOLVER_MGCG      */
  int inner_steps;     /* s: V-cycles / CG steps per iteration (default 2)                     */
  int nu1, nu2;        /* damped-Jacobi pre / post sweeps (default 2, 2)                       */
  double omega;        /* Jacobi damping (default 2/3)                                         */
  int coarse_level;    /* level of the P chain that is V_H; -1 (default) = the last level      */
  int max_iter;        /* outer iterations (default 100)                                       */
  int aug_max_iter;    /* inner iterations of the step-(c) block eigensolver (default 60)      */
  double aug_tol;      /* inner relative residual target (default 1e-12)                       */
  int aug_adaptive;    /* 1 (default): inner target max(aug_tol, f x current outer residual),
                          f = aug_factor, made ten times smaller after an iteration whose
                          residual rose (down to aug_factor / 1000) and ten times larger
                          after one that cut it by more than five (up to aug_factor);      
                          0: always aug_tol                                                     */
  int verbose;         /* 0 silent, 1 per-iteration line on stderr, 2 also inner iterations    */
  int use_graphs;      /* 1 (default): inside pase_solve the step-(a) linear solve is captured
                          once into a CUDA graph and replayed (needs a non-NULL stream)        */
  int autotune;        /* 1 (default): pase_reserve times the sparse kernel at a few block
                          sizes for every multigrid matrix and keeps the fastest            */
  int smoother;        /* PASE_SMOOTHER_JACOBI (default) or PASE_SMOOTHER_LEARNED: the fine-
                          level sweeps of the V-cycle use the learned network once
                          pase_set_grid and parameters are given (Jacobi until then)      */
  int split_gemm;      /* 1 (default): the dense products of steps (b) and (d) (Alg. 3 steps
                          4 and 6), the Gram blocks W^T(A_h W), W^T(M_h W) and W C_W
                          (m <= 128, even; wider blocks use the FP64 kernels), run on
                          the BF16 tensor cores with FP64 accuracy (error-free splitting into
                          8-bit digit slices, exact FP32 sums per digit diagonal, 64-bit
                          integer recombination; error a few units of 2^-53 relative to the
                          products of the row and column maxima); 0: FP64 CUDA cores      */
  int stencil;         /* 1 (default): in PASE_PREC_MIXED, every multigrid level whose matrix
                          couples each node only to its 3^d neighbours on an n1^d grid
                          (x-fastest order; Q1 operators and their Galerkin coarse levels)
                          keeps its FP32 values by grid tap, and the FP32 Jacobi sweeps,
                          residuals and products on it run in a structured kernel without
                          column indices; 0: the CSR kernel everywhere                    */
  int post_solve;      /* 0 (default): one linear-solve phase per iteration (Alg. 1);
                          1: the two-solve form of Alg. 3 - after the Rayleigh-Ritz of an
                          iteration that has not converged, a second linear solve
                          A_h u = lambda M_h u-hat from the prolongated u-hat (step 7) feeds
                          the next iteration's step 3; returned vectors are always the
                          Rayleigh-Ritz ones                                              */
  int aug_transform;   /* congruence applied to the augmented pencil before step (c), §4:
                          PASE_AUG_PLAIN (default) none, PASE_AUG_PRECOND_A, _PRECOND_B or
                          _PRECOND_BA (see below)                                        */
  int spmm_df64;       /* 1 (default): the fused fine-level products A_h X, M_h X of step (b)
                          and of the eigen-residual run in double-float arithmetic (each
                          FP64 value as a sum of two FP32 numbers, error-free products and
                          sums on the FP32 pipe; errors a few 2^-48 relative to the row's
                          sum of |a||x|); a block entry above 2^100 or not finite is then
                          reported as PASE_ERR_NAN; 0: FP64 CUDA cores                     */
  int graph_solve;     /* 0 (default): pase_solve runs one outer iteration at a time from the
                          host (a readback of the residual test per iteration; per-phase
                          times in pase_stats); 1: the whole solve - start, outer loop, every
                          step - is recorded once into a CUDA graph whose loops are
                          conditional nodes steered by device-side tests, and replayed with
                          one graph launch per call (no per-phase times).  In both forms
                          step (c) is a recorded graph with its inner loop on the device.
                          pase_solve_batched runs handles that all have graph_solve = 1 as
                          one graph launch                                               */
  int graph_pass_limit; /* 0 (default): every recorded loop may run the passes its test allows
                          (max_iter + 1 outer, aug_max_iter inner); n > 0: at most n passes,
                          after which the loop ends and the call returns PASE_ERR_TIMEOUT
                          (a bound on device-side iteration for callers that want one)   */
  int stencil_columns; /* columns per consumer thread of the structured FP32 kernel: 0
                          (default) the autotuner's choice (4 without it), or 2 / 4 fixed;
                          2 runs twice the threads at half the registers (block widths up
                          to 60)                                                          */
  double aug_factor;   /* the adaptive inner target's factor (default 1e-4), in (0, 1]      */
  int sygv_tridiag;    /* form of the small eigensolver's Householder tridiagonalisation:
                          -1 (default) the autotuner's choice per Rayleigh-Ritz size (without
                          it: one CTA below n = 64, else a cluster of 8 SMs); 0 one CTA;
                          1 a cluster of 8 SMs; 2 a cluster of 16 SMs (8 where the device
                          cannot schedule 16); cluster forms apply from n = 16           */
  int sygv_cholesky;   /* form of its Cholesky factorisation of the Gram matrix: -1 (default)
                          the autotuner's choice (without it: as sygv_tridiag's default);
                          0 one CTA; 1 a cluster of 8 SMs (from n = 16)                  */
} pase_options;

/* Step-(c) variants (§4, Alg. 5).  Each solves the same augmented eigenproblem through the
 * congruence [[I, Z], [0, I]] (eigenvectors mapped back by u_H = u~_H - Z gamma~):
 *   PLAIN       Z = 0;             preconditioner: the block factorisation of A_Hh
 *                                   (coarse V-cycle for A_H^-1, Schur complement of alpha)
 *   PRECOND_A   Z ~ A_H^-1 a_h     (A_Hh becomes block diagonal);  same preconditioner
 *   PRECOND_B   Z ~ B_H^-1 b_h     (B_Hh becomes block diagonal);  block-diagonal
 *                                   preconditioner (coarse V-cycle, alpha~^-1)
 *   PRECOND_BA  PRECOND_B, then the block-factorisation preconditioner of the transformed
 *               A_Hh (the A-type factorisation inside the linear solves)
 * Z comes from a coarse V-cycle (A_H) or Jacobi-preconditioned CG (B_H); the transformed
 * blocks are formed from that Z, so the pencil stays exactly congruent whatever its
 * accuracy. */
#define PASE_AUG_PLAIN 0
#define PASE_AUG_PRECOND_A 1
#define PASE_AUG_PRECOND_B 2
#define PASE_AUG_PRECOND_BA 3

#define PASE_SMOOTHER_JACOBI 0
#define PASE_SMOOTHER_LEARNED 1

/* Per-solve statistics (all times in milliseconds, device-event timed). */
typedef struct {
  int iterations;        /* outer augmented subspace iterations                                */
  int converged;         /* how many of the first nev pairs met tol                            */
  double max_residual;   /* largest relative residual among the first nev                      */
  double solve_ms;       /* whole pase_solve                                                   */
  double phase_ms[5];    /* (a) linear solve, (b) projection, (c) augmented eig, (d) prolongation,
                            residual/convergence                                              */
  int aug_iterations;    /* inner block-eigensolver iterations, summed                         */
  int kernel_launches;   /* library kernels run (those inside replayed graphs included)        */
  int graph_launches;    /* CUDA graph launches issued by the call                            */
} pase_stats;

/* Sparse matrix in CSR (borrowed).  rowptr has nrows+1 entries, rowptr[0] = 0;
 * colind is sorted ascending inside each row.  Values are FP64. */
typedef struct {
  int64_t nrows, ncols, nnz;
  const int64_t* rowptr;
  const int32_t* colind;
  const double* val;
  int on_device; /* 0: the three arrays are host memory, 1: device memory */
} pase_csr;

typedef struct pase_ctx* pase_handle;

/* Fill *opt with the defaults above. */
void pase_default_options(pase_options* opt);

/* Create a handle that runs on `cuda_stream` (a cudaStream_t; NULL = legacy default
 * stream) on the current device.  *opt is copied; NULL means defaults. */
int pase_create(pase_handle* h, const pase_options* opt, void* cuda_stream);

/* Alg. 3 "Require": fine pencil (A_h, M_h), the interpolation chain and the coarse pencil.
 * P[k] (k = 0..n_interp-1) interpolates level k+1 to level k, level 0 being V_h; their
 * product P[0] P[1] ... P[c-1], c = coarse_level, is I_H^h (§3 lets the interpolation be
 * one matrix or a product of several).  Levels below c serve the multigrid solver only.  A_H and
 * M_H live on level c.  A_h and M_h must share one sparsity pattern (as do A_H, M_H).
 * A_H and M_H may both be NULL: the library then forms them as the Galerkin products
 * through the chain (the coarse pencil of nested spaces, computed on the host with
 * OpenMP), which saves the caller forming them for large meshes.
 * Setup validates the CSR arrays, builds the Galerkin multigrid levels
 * A_{k+1} = P[k]^T A_k P[k], the direct interpolation I_H^h and its transpose, a dense
 * inverse of the coarsest multigrid operator, and uploads everything to the device. */
int pase_setup(pase_handle h, const pase_csr* A_h, const pase_csr* M_h, int n_interp,
               const pase_csr* P, const pase_csr* A_H, const pase_csr* M_H);

/* Allocate the workspace for block width m (done implicitly by the calls below). */
int pase_reserve(pase_handle h, int m);

/* Solve for the nev smallest pairs to relative residual tol (Alg. 2 / Alg. 3).
 * U0: the start block [N][m] (m = the block width; row-major) or NULL for the coarse
 * start of Alg. 3 steps 1-2.  A given U0 makes the first iteration skip step (a).
 * m: block width (multiple of 8, >= nev + 1); 0 = nev + max(4, ceil(nev/10)) rounded up to 8.
 * lambda [m] and U [N][m] receive the Ritz values (ascending) and M_h-orthonormal
 * vectors; the first nev are the result.  st may be NULL.
 * Returns PASE_ERR_NOT_CONVERGED (outputs written) if max_iter is reached. */
int pase_solve(pase_handle h, int nev, double tol, int m, const double* U0, double* lambda,
               double* U, pase_stats* st);

/* Many independent problems at once.  The method treats one pencil per call (Alg. 3);
 * solving unrelated pencils side by side has no counterpart in the paper.  When every
 * handle is distinct, set up on the current device and created with graph_solve = 1, the
 * whole batch is one CUDA graph - each problem's recorded solve one branch of it - recorded
 * on the first call, kept by the first handle while the handles, sizes and buffers stay the
 * same, and launched once per call (the branches run concurrently on the GPU).  Otherwise
 * count handles, each set up and best created on its own CUDA stream, are solved
 * concurrently by a pool of host threads so that their kernels overlap on the GPU (handles
 * that share a stream run one after another, largest groups first).  Problem i runs exactly as pase_solve with
 * nev[i], tol[i], m[i] (m NULL or m[i] = 0: the default block width), U0[i] (U0 or U0[i]
 * NULL: coarse start), lambda[i] and U[i]; host or device pointers as in pase_solve.
 * st (may be NULL) receives count stats.  Returns PASE_OK if all converged,
 * PASE_ERR_NOT_CONVERGED if some reached max_iter, else the first other error (the
 * message names the problem); every problem is attempted. */
int pase_solve_batched(pase_handle* hs, int count, const int* nev, const double* tol,
                       const int* m, const double* const* U0, double* const* lambda,
                       double* const* U, pase_stats* st);

/* ---- the steps of one iteration, for callers that drive the loop themselves ---------- */

/* Residual block R = M_h U diag(lambda) - A_h U and relres[j] =
 * ||A u_j - lambda_j M u_j||_2 / (lambda_j ||M u_j||_2).  R may be NULL (norms only). */
int pase_residual(pase_handle h, int m, const double* U, const double* lambda, double* R,
                  double* relres);

/* Step (a): W = U + E where E approximates A_h^-1 R after `inner_steps` V-cycles (or CG /
 * V-cycle-preconditioned CG steps on A_h w = M_h u lambda from w = u), R from
 * pase_residual (R = M_h U diag(lambda) - A_h U, the residual of that system at w = u). */
int pase_linear_solve(pase_handle h, int m, const double* U, const double* lambda,
                      const double* R, double* W);

/* Step (b): aH = P^T A_h W, bH = P^T M_h W ([N_H][m]), GA = W^T A_h W, GM = W^T M_h W ([m][m]). */
int pase_project(pase_handle h, int m, const double* W, double* aH, double* bH, double* GA,
                 double* GM);

/* Step (c): the m smallest pairs of the augmented pencil, B-orthonormal, warm-started
 * at C_H = 0, C_W = I (§3).  Outputs lambda [m], C_H [N_H][m], C_W [m][m].
 * aug_iters (may be NULL) receives the inner iteration count. */
int pase_augmented_eig(pase_handle h, int m, const double* aH, const double* bH,
                       const double* GA, const double* GM, double* lambda, double* C_H,
                       double* C_W, int* aug_iters);

/* Step (d): U = P C_H + W C_W. */
int pase_prolongate(pase_handle h, int m, const double* W, const double* C_H,
                    const double* C_W, double* U);

/* One whole iteration in place: residual of (U, lambda) -> relres (if not NULL), then
 * (a) unless do_linear_solve == 0, (b), (c), (d); U and lambda are overwritten.  nev
 * (1 <= nev <= m) names the wanted pairs: step (c) converges the first
 * nev + (m - nev)/2 columns, to the adaptive inner target when opt.aug_adaptive is set. */
int pase_iterate(pase_handle h, int nev, int m, double* U, double* lambda, int do_linear_solve,
                 double* relres);

/* Fused A_h / M_h product on the fine level: AX = A_h X, MX = M_h X (device pointers,
 * [N][m]).  The hot kernel of steps (b) and the residual; exposed for measurement. */
int pase_spmm_am(pase_handle h, int m, const double* X, double* AX, double* MX);

/* The batch scheme of §5 (Alg. 7) for many eigenpairs: the first nev pairs computed in
 * batches of about k, one batch after the other, each with a block of m columns (its own
 * pairs plus guard columns).
 *   1. the first nev + m pairs of the coarse pencil (A_H, M_H), by a dense solve;
 *   2. batch bounds every k pairs, moved up past coarse eigenvalues within a relative gap
 *      of 1e-3 of their predecessor (no coarse cluster split between batches);
 *   3. per batch, from U = I_H^h u_H and the coarse eigenvalues: (c) the linear solve of the
 *      handle's options, (d) the 2m pairs of the augmented pencil nearest the shift theta
 *      (the midpoint of the batch's coarse eigenvalues), by a dense generalized eigensolve
 *      of the (N_H + m)-sized pencil, (e) the m of them with the largest b-norm component
 *      in span(W) (X GM = C_H^T bH + C_W^T GM, component X(i,:) GM X(i,:)^T), prolongated,
 *      stop when the batch's own pairs meet tol, else (f) the linear solve again from the
 *      new block.
 * The dense step (d) needs N_H + m <= 6400 and nev + 3m <= 1024 unless N_H + m <= 1024.
 * The scheme relies on V_H resolving the pairs of earlier batches (their components grow
 * in the later batches' linear solves): with too coarse a V_H later batches stall.
 * lambda [nev] (ascending within a batch), U [N][nev] (row-major, M-orthonormal within a
 * batch).  Returns PASE_ERR_NOT_CONVERGED (outputs written) when a batch stops at max_iter.
 * st->iterations sums the iterations of all batches. */
int pase_solve_batches(pase_handle h, int nev, int k, int m, double tol, double* lambda, double* U,
                       pase_stats* st);

/* `sweeps` damped-Jacobi sweeps x <- x + omega D^-1 (b - A_h x) on the fine level (the
 * smoother of step (a), Alg. 3 step 3), in the precision the handle smooths in: FP32 for
 * PASE_PREC_MIXED (B and X rounded to FP32 on entry, X returned widened to FP64), FP64
 * otherwise.  B, X: [N][m]; X is updated in place.  For tests and measurement. */
int pase_smooth(pase_handle h, int m, int sweeps, const double* B, double* X);

/* Which form the FP32 fine-level sweeps take: 3 or 2 when the fine matrix was
 * recognised as a grid-neighbour stencil in that many dimensions and the structured
 * kernel serves it (after pase_reserve the autotuner may have chosen the CSR kernel for
 * the level instead), 0 for the CSR kernel. */
int pase_smoother_form(pase_handle h);

/* Residual of a block, for callers that cannot allocate device memory.  Has no
 * counterpart in the paper: it is pase_residual without a handle and without any device
 * allocation, for code that runs under a memory arena owning every device byte, inside
 * another runtime's callbacks that forbid cudaMalloc, or on paths that must not allocate.
 * Computes R = M U diag(lambda) - A U (R may be NULL) and relres[j] =
 * ||A u_j - lambda_j M u_j||_2 / (lambda_j ||M u_j||_2) for an n x n pencil in CSR that
 * shares one pattern (rowptr [n+1], colind [nnz], A_val / M_val [nnz]).
 * Every pointer must be device memory of the current device, or managed memory (no host
 * staging: staging would allocate; a pointer into another GPU's memory is rejected with
 * PASE_ERR_INVALID_ARG); U and R are row-major [n][m] and 16-byte aligned; 8 <= m <= 64, m a multiple of 8 (larger m is
 * rejected with PASE_ERR_INVALID_ARG).  Work is queued on cuda_stream (NULL = legacy
 * default stream) and the call returns without synchronising.
 * Scratch: a fixed 1.19 MiB array in device memory, part of the library image, held by
 * every GPU that loads the library until the process exits.  The first call on each
 * device looks up that array's device address (with that device current) and caches it;
 * make that first call before any stream capture.  All calls on a device share the one
 * array, so calls whose execution overlaps on the GPU (different streams, other host
 * threads) race and give wrong results; serialise them.  Nothing from a previous call
 * is read: each call writes every scratch entry it later reads. */
int pase_residual_noalloc(int64_t n, int m, const int64_t* rowptr, const int32_t* colind,
                          const double* A_val, const double* M_val, const double* U,
                          const double* lambda, double* R, double* relres, void* cuda_stream);

/* Device time of one launch of a hot kernel on the fine level of the set-up problem, for
 * roofline measurement: `reps` back-to-back launches after two warm-up launches, timed
 * with CUDA events on the handle's stream; *ms_per_launch = the average.  Operands are
 * deterministic pseudo-random blocks of width m held in the handle's workspace. */
#define PASE_KERNEL_SPMM_AM_FP64 0  /* fused A_h X, M_h X (FP64)                        */
#define PASE_KERNEL_JACOBI_FP64 1   /* one damped-Jacobi sweep on A_h (FP64)              */
#define PASE_KERNEL_JACOBI_FP32 2   /* the same sweep in FP32 (needs PASE_PREC_MIXED)     */
#define PASE_KERNEL_GRAM_FP64 3     /* W^T Y over N_h rows, symmetric (FP64)               */
#define PASE_KERNEL_PROLONG_FP64 4  /* W C over N_h rows (FP64)                           */
#define PASE_KERNEL_SYGV 5          /* small symmetric-definite eigensolver, n = k = m     */
#define PASE_KERNEL_SYGV3 6         /* the same with n = 3m, k = m (step-(c) Rayleigh-Ritz) */
#define PASE_KERNEL_PROLONG_SPLIT 7 /* W C over N_h rows on the tensor cores (split digits; m <= 128) */
#define PASE_KERNEL_GRAM_SPLIT 8    /* both Gram blocks W^T R, W^T W on the tensor cores (split digits) */
#define PASE_KERNEL_JACOBI_FP32_CSR 9 /* the FP32 sweep in the CSR kernel even on a structured grid  */
#define PASE_KERNEL_FMA_FP64 10     /* FP64 FMA rate: 1216 x 256 threads, 8 independent chains of
                                       4096 FMAs each, 2.04e10 flops per launch, no memory traffic */
#define PASE_KERNEL_SPMM_AM_DF64 11 /* the fused A_h X, M_h X in double-float (split + product)     */
int pase_time_kernel(pase_handle h, int kernel, int m, int reps, double* ms_per_launch);

/* Live timing of one kernel while the handle works (pase_solve, pase_iterate, ...): with
 * kernel = PASE_KERNEL_SPMM_AM_FP64, _JACOBI_FP64 or _JACOBI_FP32, every launch of that
 * kernel on the fine level is bracketed by a pair of CUDA events on the handle's stream
 * (at most 4096 launches between reads; later ones are not timed).  Graph replay of step
 * (a) is suspended while a kernel is selected.  kernel = -1 stops.
 * pase_profile_read waits for the handle's stream, returns the number of timed launches
 * and their summed duration in ms since the last read, and starts a new count. */
int pase_profile_kernel(pase_handle h, int kernel);
int pase_profile_read(pase_handle h, int64_t* launches, double* total_ms);

/* ---- learned fine-level smoother (the paper has no counterpart: a growth item) -------
 * A 3^dim convolutional network, 2 -> 16 -> 16 -> 16 -> 1 channels with ReLU after the
 * first three layers and zero padding, replaces each damped-Jacobi sweep on the fine
 * level of the V-cycle by x <- x + S(b - A x).  Per column: q = D^-1 r, rho = RMS(q),
 * S(r) = rho * net(q / rho, f), f = mean log kappa of the elements around each node.
 * Parameters: one float vector [W1, b1, ..., W4, b4], W_l in [c_out][c_in][tap] order,
 * tap t = sum_k (o_k + 1) 3^k for offsets o in {-1,0,1}^dim (x fastest); the network
 * computes with them rounded to bfloat16 and accumulates in FP32.  Training minimises
 * the squared energy norm of the error left after one step relative to the error before
 * it, (e - S(Ae))^T A (e - S(Ae)) / e^T A e, with Adam on the FP32 master copy.
 * Training uses the handle's workspace: do not interleave it with a solve. */

/* The fine level is the interior-node grid of a uniform n^dim mesh ((n-1)^dim nodes,
 * x fastest; must equal the size of A_h).  log_kappa: n^dim per-element values (host;
 * NULL = all zero).  Call once, after pase_setup. */
int pase_set_grid(pase_handle h, int dim, int n, const double* log_kappa);
/* Number of network parameters P for dim = 2 (5089) or 3 (15169); 0 otherwise. */
int pase_smoother_nparams(int dim);
/* Optimiser state (host memory, 3P + 1 floats): [parameters | Adam first moments |
 * Adam second moments | step count].  get = 1 reads it, get = 0 sets it (setting the
 * parameters enables the learned smoother for PASE_SMOOTHER_LEARNED handles). */
int pase_smoother_state(pase_handle h, float* state, int64_t count, int get);
/* D = S(R) for a residual block R [N][m] (host or device; m a multiple of 8). */
int pase_smoother_apply(pase_handle h, int m, const double* R, double* D);
/* One training step on a batch of 8 columns: E = errors, R = A E ([N][8], host or
 * device).  loss8 (host, 8) receives each column's loss, grad (host, P; may be NULL) the
 * gradient of the batch loss (the mean over the columns) with respect to the rounded
 * parameters; update = 1 also applies one Adam step (lr, beta1, beta2, eps). */
int pase_smoother_step(pase_handle h, const double* E, const double* R, int update, float lr, float beta1,
                       float beta2, float eps, double* loss8, double* grad);
/* Training on samples the solver generates on this handle's problem, on-policy: per
 * step, eight random errors e0 (uniform, seeded), b = A e0, x = 0, then
 * k = (step/4) mod (max_cycles+1) V-cycles with the network being trained, then by
 * step mod 4: nothing more / one pre-smoothing sweep / all pre-sweeps and the coarse-grid
 * correction / that and one post-sweep; the pair is the remaining error e = e0 - x and
 * its residual r = A e.  Afterwards the energy-norm error factor of two V-cycles on fresh
 * errors is measured with the network and with damped Jacobi; if the network is not
 * better, the handle falls back to Jacobi (until new parameters are set).
 * losses (host, 5): mean loss of the first 10 steps, of the last 10 steps, of the damped
 * Jacobi correction on the last 10 steps' samples, and the two V-cycle factors
 * (network, Jacobi). */
typedef struct {
  int steps;
  float lr, beta1, beta2, eps;
  unsigned seed;
  int max_cycles;
} pase_train_options;
void pase_default_train_options(pase_train_options* o);
int pase_train_smoother(pase_handle h, const pase_train_options* o, double* losses);

/* Number of library kernels launched by this handle so far (those run inside replayed
 * CUDA graphs included). */
int64_t pase_kernel_count(pase_handle h);

/* The same count split by how the kernels were issued: *kernels as pase_kernel_count,
 * *kernels_in_graphs of them ran inside graph replays, *graph_launches graph launches were
 * issued; host-issued launch calls = kernels - kernels_in_graphs + graph_launches.  Any
 * pointer may be NULL. */
int pase_launch_counts(pase_handle h, int64_t* kernels, int64_t* kernels_in_graphs, int64_t* graph_launches);

/* Release everything the handle owns.  NULL is accepted. */
int pase_destroy(pase_handle h);

const char* pase_status_string(int code);
/* Message of the last error on this thread (empty if none). */
const char* pase_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PASE_H */
