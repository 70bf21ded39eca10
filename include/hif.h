/*
 * hif.h -- C ABI of the GB300 implementation of the hierarchical interpolative
 * factorization for elliptic differential operators (HIF-DE; Ho & Ying,
 * arXiv:1307.2895).
 *
 * The operator (Eq. 1.1 discretized as in Sections 3.1 and 3.2): on the unit
 * square (dim = 2) or cube (dim = 3) with zero Dirichlet data and an
 * n x n (x n) grid, h = 1/n, unknowns at the N = (n-1)^dim interior nodes,
 *
 *   (1/h^2) sum_e [ a_{j-e/2}(u_j - u_{j-e}) + a_{j+e/2}(u_j - u_{j+e}) ] + b_j u_j = f_j.
 *
 * Unknowns are ordered lexicographically with x fastest.
 *
 * Array arguments:
 *   a_stag  staggered coefficients: ax, ay (, az) concatenated, each block of
 *           n*(n-1)^(dim-1) doubles.  2D: ax[(j2-1)*n + j1] = a((j1+1/2)h, j2 h),
 *           ay[j2*(n-1) + (j1-1)] = a(j1 h, (j2+1/2)h).  3D: ax[((j3-1)*(n-1) +
 *           (j2-1))*n + j1], ay[((j3-1)*n + j2)*(n-1) + (j1-1)],
 *           az[(j3*(n-1) + (j2-1))*(n-1) + (j1-1)].
 *   b       nodal reaction coefficient, N doubles.
 *   vectors N rows x nrhs columns, row-major with row stride ld >= nrhs
 *           (element (i, r) at v[i*ld + r]).
 *
 * Pointers may be host or device memory (any pointer the CUDA runtime does
 * not report as device or managed memory is treated as host memory and is
 * staged through the device).  The caller keeps ownership of every array it
 * passes; arrays are only read (inputs) or written (outputs) during the call.
 * Device work is issued on opts.stream (a cudaStream_t; NULL = legacy default
 * stream) and every call returns after its results are complete.
 *
 * Errors: every call returns an hif_status.  Nothing aborts the process and no
 * device code traps; hif_last_error() gives a message for the last failure on
 * the calling thread.  A handle is not thread-safe.
 */
#ifndef HIF_H
#define HIF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum hif_status {
  HIF_OK = 0,
  HIF_ERR_ARG = 1,       /* invalid argument (grid, sizes, pointers)            */
  HIF_ERR_NOT_SPD = 2,   /* a zero or non-finite pivot in a diagonal block, or a
                            negative one where only Cholesky applies (the tiled
                            elimination of large blocks)                        */
  HIF_ERR_NOCONV = 3,    /* the iteration reached maxit; info is still filled   */
  HIF_ERR_TIMEOUT = 4,   /* a bounded device wait ran out                       */
  HIF_ERR_CUDA = 5,      /* a CUDA runtime call failed                          */
  HIF_ERR_OOM = 6,       /* a device or host allocation failed                  */
  HIF_ERR_HOST = 7       /* another host-side failure (e.g. a thread could not  */
                         /* start); hif_last_error() names it                   */
} hif_status;

/* Variants (Section 5 names): MF = mf2/mf3 (Algorithm 3.1, exact),
 * HIFDE = hifde2/hifde3 (Algorithm 4.1; faces only in 3D), HIFDE3X = hifde3x
 * (Section 4.5, Algorithm 4.2, dim 3 only): after the cells and faces of a
 * level, the edges are skeletonized too (from level 1 on, the paper's rule of
 * thumb read as skipping level 0), and from level 2 on the cells are built
 * algebraically (Voronoi cells of the active DOFs about the cell centers,
 * peeled so that no two are coupled) and the faces and edges are Voronoi
 * groups about their centers; a DOF equidistant to two or more nearest
 * centers joins no group.  Needs n divisible by 2^L; from level 1's edges on
 * the active matrix is held as one dense matrix of the DOFs active at that
 * point (HIF_ERR_ARG if that would exceed 48 GB). */
enum { HIF_VARIANT_MF = 0, HIF_VARIANT_HIFDE = 1, HIF_VARIANT_HIFDE3X = 2 };

/* Diagonal blocks (A_pp of Lemma 2.1, B_rr of Lemma 2.4, the root D) are
 * factored by Cholesky when positive definite; a negative pivot (an
 * indefinite A, e.g. the Helmholtz operator b = -k^2 of Section 5's
 * Examples 3 and 6) makes that block an LDL^T decomposition with 1 x 1
 * pivots in order, D = diag(+-1), in the blocks one thread block factors
 * (every 2D block at the sizes here; 3D blocks below big_cell DOFs) and in
 * the FP64 modes.  F^-1 is then not positive definite: solve with GMRES
 * (hif_set_solver; HIF_SOLVER_AUTO switches on CG's breakdown).
 *
 * Arithmetic of the factorization.  FP64: every block operation in double.
 * MIXED: cell and front blocks, the factor and the apply of F^-1 in float;
 * the root block D is factored in double; the ID's column norms and pivot
 * tests are accumulated in double; diagonal-block Cholesky pivots that fall
 * into FP32 rounding noise are raised (counted in clamped_pivots).
 * FP32_APPLY: the factorization runs in double, the factor is then stored and
 * applied in float.  The CG driver is double(-double) in every mode. */
enum { HIF_PREC_FP64 = 0, HIF_PREC_MIXED = 1, HIF_PREC_FP32_APPLY = 2 };

/* hif_apply modes (Eq. 4.2): y = F x or y = F^-1 x. */
enum { HIF_APPLY_F = 0, HIF_APPLY_FINV = 1 };

typedef struct hif_grid {
  int dim;      /* 2 or 3                                                       */
  int n;        /* grid intervals per axis (N = (n-1)^dim), n >= 4              */
  int leaf;     /* leaf cell width m (Section 3.1: n = 2^L m); 0 -> 8           */
  int variant;  /* HIF_VARIANT_*                                                */
} hif_grid;

/* ID modes (Section 4.3): the pivoted-QR ID of A_{N,c}; or an ID of the
 * Gaussian sketch Phi A_{N,c} with ell = k_hat + oversample rows, accepted only
 * if every column of the residual A_{N,r} - A_{N,s} T has 2-norm at most
 * eps times the largest column 2-norm of A_{N,c} (the quantities the
 * pivoted QR's stopping rule compares, Section 2.2) and k < ell (else the
 * pivoted-QR ID of A_{N,c}), with k_hat = ceil(|c|/2) (RAND) or predicted per
 * front by the rank MLP (LEARNED, opts.rank_model required). */
enum { HIF_ID_QR = 0, HIF_ID_RAND = 1, HIF_ID_LEARNED = 2 };

/* Skeletonization of the fronts (hif_opts.skel).  ID: the interpolative
 * decomposition of Lemma 2.2 (id_mode).  SVD: Section 4.4's optimal low-rank
 * approximation: A_{N,c} = U Sigma V^T, Q_c = diag(V, I); the directions
 * with sigma <= eps sigma_1 are eliminated (Lemma 2.1 against the kept
 * directions) with their interactions dropped, and the k kept directions
 * take the slots of the first k DOFs of c (ascending ids) with interactions
 * A_{N,c} V_2, written over the cells' update matrices.  All fronts of a
 * level take their SVD from the matrix before the level and rotate together
 * (their rotations commute); no rotation when k = 0 or k = |c|.  HIFDE only
 * (not HIFDE3X: the rotated DOFs have no single position), the FP64 and
 * FP32_APPLY precisions, HIF_ID_QR; every front runs the one-block kernel
 * (one-sided Jacobi SVD), whatever its size. */
enum { HIF_SKEL_ID = 0, HIF_SKEL_SVD = 1 };

typedef struct hif_opts {
  int precision;        /* HIF_PREC_*                                           */
  int skip_levels;      /* fractional levels l + 1/2 skipped for l < skip_levels
                           (Section 5: "the first few fractional levels ...")    */
  int id_mode;          /* HIF_ID_*                                             */
  int oversample;       /* sketch rows beyond k_hat (0 -> 10)                    */
  void* stream;         /* cudaStream_t for all device work                     */
  const float* rank_model; /* HIF_ID_LEARNED: HIF_MLP_PARAMS floats (see
                              hif_mlp_train), host or device memory            */
  unsigned long long seed; /* counter-based sketch RNG seed                     */
  int big_cell;         /* cells with at least this many interior DOFs are
                           eliminated by the tiled multi-block kernels (64 x 64
                           tiles, blocked Cholesky, Lemma 2.1), and fronts with
                           at least max(big_cell, 128) DOFs skeletonized by the
                           multi-block front kernels (tiled sketch, residual
                           check and Lemma 2.4 products); 0 -> 192, < 0 ->
                           never.  Same result up to rounding order.           */
  int tensor_cores;     /* HIF_PREC_MIXED: products of the tiled elimination
                           (panel solves, trailing updates, Schur complement)
                           on the tensor cores in TF32 with FP32 accumulation,
                           each operand split into TF32 parts: 0 -> three
                           parts (exact split, about FP32 accuracy), 2 -> two
                           parts (about 2^-21), 1 -> plain TF32, < 0 -> FP32 on
                           the SIMT pipes.  Ignored in the FP64 modes.          */
  int autotune;         /* 0: the first F^-1 application that meets a sweep
                           launch shape (operation, type, right-hand sides,
                           blocks, largest block) times candidate shapes
                           (threads per block, shared-memory staging) on a
                           scratch copy and keeps the fastest, process-wide;
                           < 0: the built-in shapes.                            */
  int edge_start;       /* HIFDE3X: the first level whose edges are
                           skeletonized (Section 4.5's rule of thumb: skip
                           edge skeletonization while it does not pay for the
                           thicker separators it causes): 0 -> level 1, k > 0
                           -> level k (k >= L: no edges, the result is
                           hifde3's), -1 -> level 0.  Ignored otherwise.       */
  int sketch_power;     /* HIF_ID_RAND / LEARNED: power iterations on the
                           sketch, Y = Phi A (A^T A)^q (the end of Section 4.5
                           suggests them for inaccurate sketches), q in 0..2;
                           the sketch's rank rule is then applied at
                           (eps/10)^(2q+1), which must stay well above the
                           FP64 rounding level (q = 1 for eps >= 1e-4).       */
  int deterministic;    /* nonzero: applications of F^-1 and F (and so solves
                           and estimates) are bit-reproducible run to run: the
                           cells' updates of shared boundary DOFs are written
                           per (cell, DOF) and summed per DOF in cell order by
                           a second launch per level, and the multi-block root
                           adds its partial sums in a fixed order, instead of
                           floating-point atomics (about one more launch per
                           cell level and sweep direction).  The factorization
                           of HIF_VARIANT_HIFDE3X's assembled levels still
                           adds with atomics; the other variants' factor-
                           izations are reproducible either way.             */
  long long big_apply;  /* applications of F^-1: blocks with np (np + 2 nq)
                           >= big_apply elements (np eliminated, nq
                           neighbour DOFs) are applied by many thread blocks
                           each, in the pattern of the large root, the others
                           one block each; 0 -> 2^20, < 0 -> never.  Not in
                           the deterministic mode.  Same result up to
                           rounding order.                                   */
  int skel;             /* HIF_SKEL_*: the fronts' low-rank approximation;
                           0 -> HIF_SKEL_ID                                  */
  int two_sided;        /* nonzero: the unsymmetric generalization that the
                           paper's Section 6 sketches.  Diagonal blocks are
                           factored by LU without pivoting (A_pp = L U, L
                           unit lower), giving the two-sided elimination
                           operators R_p = [[L^-T, -A_pp^-T A_qp^T], [0, I]]
                           and S_p = [[U^-1, -A_pp^-1 A_pq], [0, I]] of
                           Lemma 2.1; a front's skeletons and T come from one
                           ID of the stacked [A_{N,c}; A_{c,N}^T] and serve
                           its rows and columns.  The operator is the
                           stencil plus the convection term beta . grad u
                           (central differences, constant beta), so A is
                           unsymmetric when beta != 0.  HIFDE or MF, FP64 or
                           FP32_APPLY, HIF_ID_QR and HIF_SKEL_ID; every block
                           runs the one-block kernels.  hif_solve,
                           hif_matvec and hif_estimate apply the stencil
                           without the convection term: they return
                           HIF_ERR_ARG for a handle with beta != 0.        */
  double beta[3];       /* two_sided: beta per axis (x, y[, z]); must be 0
                           otherwise                                        */
} hif_opts;

typedef struct hif_handle hif_handle;

typedef struct hif_solve_info {
  int iters;            /* inner iterations (CG steps and GMRES Arnoldi steps),
                           all refinement steps                                  */
  int outer;            /* refinement steps                                     */
  int converged;        /* 1 if every column reached tol                        */
  double relres_max;    /* max_r ||b_r - A x_r||_2 / ||b_r||_2 of the
                           double-double iterate x = x_hi + x_lo                 */
  double relres_fp64_max; /* the same for the FP64 iterate x_hi alone           */
  int gmres_iters;      /* of iters, the GMRES Arnoldi steps (0: CG only)        */
} hif_solve_info;

/* Inner solver of hif_solve's refinement steps (Section 5: CG for the SPD
 * systems, GMRES where the preconditioned operator is not SPD). */
enum {
  HIF_SOLVER_AUTO = 0,   /* CG; on a breakdown (r.z <= 0 on a column: F^-1 is
                            not positive definite there, a non-finite
                            residual, or 50 iterations without a new smallest
                            residual) that refinement step and the following
                            ones run flexible GMRES                              */
  HIF_SOLVER_CG = 1,     /* CG only                                              */
  HIF_SOLVER_GMRES = 2   /* flexible GMRES(restart) only                          */
};

typedef struct hif_stats_t {
  int dim, n, levels;          /* L                                              */
  int root_size;               /* |s_L| (Section 5)                              */
  int n_cells, n_fronts;       /* blocks eliminated / skeletonized, all levels   */
  int max_front_rank;          /* largest skeleton size k                        */
  int near_threshold_fronts;   /* fronts with a pivot ratio within 1e-8 of eps   */
  int clamped_pivots;          /* MIXED: Cholesky pivots raised to the floor     */
  int sketched_fronts;         /* fronts whose sketched ID passed the check      */
  int fallback_fronts;         /* fronts that fell back to the pivoted-QR ID     */
  double t_fronts_ms;          /* device time of the front (ID) launches         */
  long long factor_bytes;      /* m_f: bytes of the stored factor                */
  double factor_flops;         /* algorithmic flops of the factorization         */
  double apply_bytes;          /* factor bytes read by one apply of F^-1         */
  double t_factor_ms;          /* device time of the last hif_factor             */
  int negative_pivots;         /* pivots < 0: diagonal blocks of an indefinite A
                                  factored as L D L^T, D = diag(+-1)            */
  double t_wall_ms;            /* host wall time of the last hif_factor          */
  double t_wait_ms;            /* of it, the host blocked on the device (the
                                  per-level read-backs of ranks and skeletons)  */
} hif_stats_t;

/*
 * hif_factor -- Algorithm 3.1 (variant MF) or Algorithm 4.1 (variant HIFDE):
 * for l = 0..L-1, eliminate the interiors of the level-l cells (Lemma 2.1),
 * then skeletonize the strict interiors of the level-l edges (2D) or faces
 * (3D) with an ID of relative precision eps (Lemma 2.4, Section 4.3), and
 * finally factor D = A_L (Cholesky).  eps must be > 0 for HIFDE; it is
 * ignored for MF.  bc_vals must be NULL (zero Dirichlet data; nonzero data
 * belong in the right-hand side: hif_rhs_from_bc).  On success *out owns the factor in
 * device memory; release it with hif_free.
 * Device memory: the factor and the work buffers are stream-ordered
 * allocations from the current device's default memory pool; the library
 * sets that pool to keep up to 8 GB of freed memory for reuse (the
 * factorization allocates and frees per level).
 */
int hif_factor(const hif_grid* grid, const double* a_stag, const double* b,
               const double* bc_vals, double eps, const hif_opts* opts,
               hif_handle** out);

/*
 * hif_apply -- y = F x (mode HIF_APPLY_F) or y = F^-1 x (HIF_APPLY_FINV),
 * with F the generalized LDL^T factorization of Eq. (3.1) / (4.2).
 * x and y: N x nrhs, row stride ld (see above); x and y may alias.
 */
int hif_apply(hif_handle* h, int mode, const double* x, double* y, int nrhs, int ld);

/*
 * hif_solve -- preconditioned CG (Section 5) on A x = rhs with F^-1 as the
 * preconditioner (or GMRES, see hif_set_solver), one independent iteration
 * per column, started from x = 0,
 * until ||rhs_r - A x_r||_2 <= tol ||rhs_r||_2 for every column, or maxit
 * inner iterations.  The iterate is kept in double-double, x = x_hi + x_lo,
 * and the residual is evaluated in double-double from the bond form of the
 * stencil (exact coefficients a n^2): for high-contrast fields the rounding
 * floor of the residual of an FP64 vector lies above 1e-12 (about 2e-10 for a
 * contrast of 1e6 on a 511^2 grid), so the tolerance is certified on x_hi +
 * x_lo.  CG runs in FP64 on corrections (iterative refinement, each step to
 * max(tol ||rhs|| / (2 ||r||), 1e-9) relative).  x receives x_hi; x_lo may be
 * NULL.  info may be NULL.  Returns HIF_ERR_NOCONV if maxit is reached (x
 * then holds the last iterate).  F^-1 is applied eagerly on the first
 * iteration and then replayed from a CUDA graph; the environment variable
 * HIF_NO_GRAPH=1 keeps every application eager (for diagnosis).
 */
int hif_solve(hif_handle* h, const double* rhs, double* x, double* x_lo, int nrhs,
              int ld, double tol, int maxit, hif_solve_info* info);

/*
 * Batches of independent problems (each one a separate HIF-DE, Section 5's
 * workloads at many sizes): hif_factor / hif_solve for problems 0..nprob-1,
 * issued concurrently from up to nthreads host threads (<= 0 -> 8), each
 * problem on its own stream (opts->stream is ignored), so the small launches
 * of different problems overlap on the GPU.  Arrays are indexed by problem;
 * out[p] receives problem p's handle (NULL on failure), infos may be NULL.
 * Returns HIF_OK, or the status of the lowest-numbered failing problem (the
 * other problems still run); hif_last_error() then describes that failure.
 */
int hif_factor_batch(int nprob, const hif_grid* grids, const double* const* a_stag, const double* const* b,
                     const double* eps, const hif_opts* opts, int nthreads, hif_handle** out);
int hif_solve_batch(int nprob, hif_handle* const* hs, const double* const* rhs, double* const* x,
                    const int* nrhs, double tol, int maxit, hif_solve_info* infos, int nthreads);

/* hif_matvec -- y = A x with the stencil of the factored problem (FP64). */
int hif_matvec(hif_handle* h, const double* x, double* y, int nrhs, int ld);

/*
 * hif_rhs_from_bc -- nonzero Dirichlet data.  In the stencil equation of
 * Section 3.1 / 3.2 at an interior node x_j, a neighbour x_k on the boundary
 * contributes -(1/h^2) a_jk u_k with u_k = g_k known; this call moves that term
 * to the right-hand side: rhs[j] += (1/h^2) a_jk g_k for every such pair, per
 * node axis by axis (x, y, z), the lower neighbour before the upper one.
 * Then A x = rhs is the problem with boundary values g (hif_factor with
 * bc_vals = NULL; A does not depend on g).
 * grid: dim and n as for hif_factor (leaf and variant are not read).
 * a_stag: the staggered coefficients of hif_factor.
 * bc_vals: g at every node of the (n+1)^dim grid, coordinates 0..n with x
 *   fastest, nrhs columns with row stride ld; only boundary nodes (a
 *   coordinate 0 or n) are read.
 * rhs: N x nrhs, row stride ld, updated in place.
 * All three in host memory (the work touches only the O(n^(dim-1)) nodes
 * next to the boundary); device pointers give HIF_ERR_ARG.
 * Errors: HIF_ERR_ARG for NULL pointers, dim not 2 or 3, n < 4 or > 32768,
 * nrhs < 1 or ld < nrhs, N > 2^31 - 1.
 */
int hif_rhs_from_bc(const hif_grid* grid, const double* a_stag, const double* bc_vals,
                    double* rhs, int nrhs, int ld);

/* hif_stats -- sizes and counts of the factorization (Section 5 columns). */
/*
 * hif_estimate -- the a posteriori error estimates of Section 5 by power
 * iteration from the start vector x0 (N values, host or device; the paper
 * starts from a uniform random vector), each norm estimate ||op x_k|| with
 * x_{k+1} = op x_k / ||op x_k||, stopped when two successive estimates differ
 * by at most rtol of the newer one (the paper: 1e-2) or after maxit products:
 *   e_a = ||A - F|| / ||A||   (A: the stencil operator in FP64; F applied as
 *                              stored, FP32 in the FP32 apply modes)
 *   e_s = ||I - A F^-1|| = ||(I - F^-1 A)(I - A F^-1)||^(1/2)
 * (A and F are symmetric).  HIF_ERR_ARG: NULL argument, rtol <= 0 or
 * maxit < 1.
 */
int hif_estimate(hif_handle* h, const double* x0, double rtol, int maxit, double* e_a, double* e_s);

/*
 * hif_autotune_table -- the sweep launch shapes chosen so far by the
 * autotuner (hif_opts.autotune), process-wide.  *count receives the number
 * of entries; if out is not NULL, min(cap, count) rows of 9 ints are written:
 * operation (0 up, 1 down), element bytes, right-hand sides, blocks, largest
 * np, largest nq, front flag, then the choice: threads per block (0: built-in)
 * and staging (-1: built-in, 0: off).  HIF_ERR_ARG: NULL count.
 */
int hif_autotune_table(int* out, long long cap, long long* count);

/*
 * hif_set_solver -- the inner solver of later hif_solve calls on h:
 * HIF_SOLVER_* (default AUTO) and the GMRES restart length (0 -> 50,
 * else 2..500).  Flexible GMRES (Saad, 1993) right-preconditioned by F^-1:
 * Arnoldi with classical Gram-Schmidt applied twice, FP64 basis, the
 * preconditioned vectors kept in the factor's apply precision; one GMRES per
 * right-hand side; memory (restart + 1) N nr FP64 + restart N nr values of
 * the apply precision per 16 right-hand sides.  HIF_ERR_ARG: NULL handle,
 * unknown solver, restart out of range.
 */
int hif_set_solver(hif_handle* h, int solver, int restart);

int hif_stats(const hif_handle* h, hif_stats_t* st);

/*
 * hif_structure -- the skeleton structure, for parity checks against the
 * oracle.  Writes int32 records, one per skeletonized front in level order:
 *   level, |c|, k, c[0..|c|-1] (ascending global indices),
 * (level: l for the fronts of level l + 1/2; for HIFDE3X 2l for the faces of
 * level l + 1/3 and 2l + 1 for the edges of level l + 2/3)
 *   s[0..k-1] (skeleton global indices in pivot order)
 * followed by the terminator -1 and then |s_L|.  If buf is NULL or cap is too
 * small, nothing is written; *needed receives the number of int32 required.
 */
int hif_structure(const hif_handle* h, int32_t* buf, long long cap, long long* needed);

/*
 * hif_profile -- event timing of the apply sweeps of F^-1 (the kernels that
 * dominate the solve).  Returns in *out (may be NULL) the summed device time,
 * launch count and algorithmic bytes (factor blocks read + vector rows
 * gathered and written) of the sweep launches recorded since the previous
 * call, resets them, and turns the recording on (enable != 0) or off for
 * later calls on this handle.
 */
typedef struct hif_profile_t {
  double sweep_ms;
  long long sweep_launches;
  double sweep_bytes;
} hif_profile_t;
int hif_profile(hif_handle* h, int enable, hif_profile_t* out);

/* hif_kernel_launches -- kernels launched by this library in this process. */
long long hif_kernel_launches(void);

/*
 * hif_wait_selftest -- exercises one of the library's bounded device waits
 * on an object that nothing completes, with a short bound, and reports it
 * through the same status path as the real wait (no counterpart in the
 * paper; it checks the failure detection of the apply sweeps, the
 * multi-block pivoted QR and the tensor-core Schur update without faulting
 * or hanging the GPU):
 *   which 0: the wait for a bulk copy into shared memory (F^-1 sweeps), a
 *            phase whose bytes are announced and never copied; limit = polls;
 *   which 1: the group barrier of the multi-block QR, one block of a group of
 *            two; limit = polls;
 *   which 2: the wait for tensor-core MMAs, a CTA holding its tensor memory
 *            and issuing no MMA (it frees the memory after the wait gives
 *            up); limit = nanoseconds.
 * limit must lie in 1 .. the production bound (2^26, 2^22 polls; 1e9 ns).
 * Returns HIF_ERR_TIMEOUT with the real wait's message when the wait gave up
 * (the expected outcome), HIF_OK if it completed, HIF_ERR_ARG for a bad
 * which or limit.  Work is issued on stream (NULL: the legacy default
 * stream) and the call returns after it has completed.
 */
int hif_wait_selftest(int which, long long limit, void* stream);

/*
 * hif_residual_norms_noalloc -- rnorm2[r] = ||f_r - A x_r||_2^2 (FP64) for the
 * stencil operator of a grid, computed without allocating any device memory.
 * The paper has no counterpart: this serves callers that cannot call
 * cudaMalloc where they check a solution (inside another library's allocator
 * callback or memory-managed region, or where an allocation must not
 * synchronize the device).  All pointers must be device (or managed) memory:
 * a_stag, b as for hif_factor; f and x are N x nrhs with row stride ld;
 * rnorm2 receives nrhs doubles.  Nothing is staged: a pointer the CUDA
 * runtime does not report as device or managed memory gives HIF_ERR_ARG.  Work is queued on stream (a cudaStream_t, NULL = legacy
 * default stream); the call returns once the kernels are queued.
 * Limits: 1 <= nrhs <= 16 per call (HIF_ERR_ARG otherwise).  The reduction
 * scratch is one fixed 38 KB device array of the library, held by every GPU
 * that loads it until exit and shared by all calls: calls that overlap on the
 * GPU race.  The first call on a device looks up that array's address (with
 * the device current); make it before any stream capture.
 */
int hif_residual_norms_noalloc(int dim, int n, const double* a_stag, const double* b,
                               const double* f, const double* x, int nrhs, int ld,
                               double* rnorm2, void* stream);

/*
 * Rank-prediction MLP (no counterpart in the paper; it sizes the sketch of
 * HIF_ID_LEARNED).  Input: HIF_MLP_FEATURES features per front (level,
 * log2 |c|, log2 |N|, log10 eps, min / max / mean / std / spread of log10 a
 * over the front DOFs' stencil couplings, dim); output: a prediction of
 * log(1 + k).  Three layers of width 64 with ReLU; parameters flat float:
 * W1 (64 x 10) | b1 | W2 (64 x 64) | b2 | W3 (1 x 64) | b3, HIF_MLP_PARAMS
 * floats.  Loss: mean Huber loss (delta 1).  All pointers of these three
 * calls are device pointers; stream may be NULL.
 */
#define HIF_MLP_FEATURES 10
#define HIF_MLP_PARAMS 4929

/* hif_front_log -- features (count x 10 floats), ranks k and sizes |c| of every
 * front of a factorization (the training data of the rank MLP).  Host
 * pointers; nothing is written if cap < count; *count receives the count. */
int hif_front_log(const hif_handle* h, float* feats, int32_t* ranks, int32_t* sizes, long long cap,
                  long long* count);

/* hif_schur_update_f32 -- U_b <- U_b - G_b G_b^T for nb dense FP32 blocks:
 * the Schur complement update of Lemma 2.1 (A_qq - A_qp A_pp^{-1} A_pq with
 * G = A_qp L^{-T}, L L^T = A_pp), on the tensor cores (tcgen05, TF32 inputs,
 * FP32 accumulation).  split = number of TF32 parts each operand value is
 * cut into by repeated round-to-nearest: 3 (exact, six products, about FP32
 * accuracy), 2 (three products, about 2^-21), 1 (plain TF32).  G: nb blocks
 * of m x k, row-major, block b at G + b m k; U: nb blocks of m x m,
 * row-major, block b at U + b m m, overwritten (whole block, both
 * triangles).  Device pointers owned by the caller; work is issued on
 * `stream` (NULL: the default stream) and the call returns after it has
 * completed.  HIF_ERR_ARG: nb, m or k negative, nb > 65535, split not in
 * 1..3, or a NULL pointer with nb m > 0; HIF_ERR_TIMEOUT: a bounded wait for
 * the MMAs ran out. */
int hif_schur_update_f32(int nb, int m, int k, const float* G, float* U, int split, void* stream);

/* hif_mlp_grad -- loss and gradient (mean over the n samples) at params (FP32). */
int hif_mlp_grad(const float* X, const float* target, int n, const float* params, float* grad,
                 float* loss, void* stream);

/* hif_mlp_train -- steps of Adam (lr) on minibatches of `batch` samples taken
 * in a seeded shuffled order; params updated in place; loss_hist (may be
 * NULL) receives the minibatch loss of every step. */
int hif_mlp_train(const float* X, const float* target, int n, float* params, int steps, int batch,
                  float lr, unsigned long long seed, float* loss_hist, void* stream);

/* hif_mlp_predict -- y = MLP(X) with the parameters rounded to BF16, FP32
 * accumulation (the inference used inside hif_factor). */
int hif_mlp_predict(const float* X, int n, const float* params, float* y, void* stream);

/* hif_free -- release the factor (stream-ordered on the handle's stream). */
void hif_free(hif_handle* h);

/* hif_last_error -- message of the last failure on this thread ("" if none). */
const char* hif_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HIF_H */
