/*
 * amgh.h -- C ABI of the GB300 (sm_103a) implementation of AMG preconditioning
 * of the reduced Hessian for linear-quadratic elliptic optimal control
 * (Barker & Draganescu, "Algebraic multigrid preconditioning of the Hessian in
 * PDE-constrained optimization").
 *
 * The problem (Sec. 2, Eq. functional/state): minimise
 *     J(y,u) = 1/2 (y - y_d)^T M_y (y - y_d) + beta/2 u^T M_u u
 * subject to A y = M_yu u, with P1 finite elements on triangles (dim 2) or
 * tetrahedra (dim 3).  State dofs y are the non-Dirichlet vertices in
 * ascending vertex order (m of them); control dofs u are all vertices (n).
 * The library solves the M_u-scaled first-order system (Sec. 5.2, Eq.
 * firstorderpractice)
 *     H u = b,   H = M_yu^T A^-1 M_y A^-1 M_yu + beta M_u,   b = M_yu^T A^-1 M_y y_d,
 * by conjugate gradients preconditioned with the multilevel Hessian
 * preconditioner built from the AMG prolongators (Sec. 3, Algorithm MLAS).
 *
 * Conventions for every call:
 *   - Return value: AMGH_OK (0) or a negative AMGH_ERR_* code; nothing aborts
 *     or throws across this boundary.  amgh_status_string() names a code.
 *   - Vectors named *_dev are caller-owned device pointers (e.g. a torch
 *     tensor's data_ptr()) on the current CUDA device, valid for the problem's
 *     stream (amgh_set_stream); the library never frees them.  Vectors named
 *     *_host are caller-owned host pointers.  Lengths: control vectors n,
 *     state vectors m (both from amgh_query_sizes); blocks of ncols columns
 *     are column-major (column c starts at c*n or c*m).
 *   - The library copies mesh, kappa and y_d into its own device memory at
 *     amgh_problem_create; caller buffers may be freed afterwards.
 *   - Calls enqueue work on the problem's stream and return after it has
 *     completed (they synchronise that stream), unless stated otherwise.
 *   - A problem is not thread-safe; distinct problems on distinct streams are.
 */
#ifndef AMGH_H
#define AMGH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AMGH_OK 0
#define AMGH_ERR_INVALID_ARG (-1)   /* bad pointer, size, option or mesh */
#define AMGH_ERR_NOT_SETUP (-2)     /* amgh_amg_setup has not run */
#define AMGH_ERR_CUDA (-3)          /* a CUDA runtime call failed */
#define AMGH_ERR_OOM (-4)           /* device or host allocation failed */
#define AMGH_ERR_NOT_CONVERGED (-5) /* a CG loop hit its iteration cap */
#define AMGH_ERR_INDEFINITE (-6)    /* p.Ap <= 0 or r.z <= 0 inside a CG loop */
#define AMGH_ERR_NUMERIC (-7)       /* NaN/Inf in a residual norm */
#define AMGH_ERR_TIMEOUT (-8)       /* a bounded device-side wait ran out */

typedef struct amgh_problem amgh_problem; /* opaque, owned by the library */

/* Mesh (Sec. 2: P1 elements).  coords: n_vertices*dim doubles (x fastest);
 * elements: n_elements*(dim+1) 0-based vertex ids; dirichlet: n_vertices
 * bytes, 1 = boundary vertex where y = 0.  on_device = 1: coords, elements,
 * dirichlet and kappa are device pointers; 0: host pointers. */
typedef struct {
    int dim;
    int64_t n_vertices;
    const double *coords;
    int64_t n_elements;
    const int32_t *elements;
    const uint8_t *dirichlet;
    int on_device;
} amgh_mesh;

/* AMG options (Sec. 3.1 smoothed aggregation; Sec. 5.2 usage).
 *  max_levels      cap on AMG levels of each hierarchy (>= 1)
 *  hessian_levels  levels l of the Hessian preconditioner (0 = all, Sec. 5.3)
 *  theta           strength threshold at level 0 (halved per level)
 *  coarse_max      stop coarsening at or below this many rows
 *  smoother        0 = l1-Jacobi, 1 = Chebyshev on D_l1^-1 A over [1/30, 1]
 *  smooth_degree   Jacobi sweeps or Chebyshev degree (1..16)
 *  precision       0 = FP64 everywhere; 1 = FP32 V-cycles, smoothers and
 *                  inner CG with FP64 iterative refinement of every PDE solve;
 *                  2 = FP64 CG for every PDE solve preconditioned by FP32
 *                  V-cycles (FP32 smoothers, transfers and coarse solve)
 *  smooth_prolongator 1 = S = (I - omega D^-1 A) S_hat, 0 = S_hat
 *  coarse_solve    Q_{l-1} on the coarsest Hessian level: 0 = exact, the
 *                  dense inverse of H_{l-1} (the assumption of Sec. 3-4;
 *                  needs at most 4096 control dofs there); 1 = unpreconditioned
 *                  CG on H_{l-1} to the relative residual coarse_tol of the
 *                  solve options (Sec. 5.2 uses 1e-4); 2 = the dense inverse
 *                  where H_{l-1} has at most 4096 dofs, else CG
 *  fuse_coarse     1 = FP32 V-cycles run their levels of at most 32768 rows
 *                  (down to the dense coarsest solve) as one launch on a
 *                  thread-block cluster; 2 = their levels of at most 262144
 *                  rows as one cooperative launch over every SM, phases
 *                  separated by a bounded software grid barrier (a barrier
 *                  that gives up makes the call return AMGH_ERR_TIMEOUT;
 *                  handles from amgh_problem_share, which run concurrently,
 *                  use 0 instead); both give the same result to the bit as
 *                  0 = one launch per smoother step and transfer (the
 *                  default)
 *  autotune        1 = for every state matrix A_l of at least 4096 rows,
 *                  time four back-to-back FP32 Chebyshev steps in each layout
 *                  (SELL-32, or 2..32 lanes per CSR row; L2 flushed first
 *                  for matrices above 32 MB) on this GPU and keep the
 *                  fastest; the choice is remembered per matrix shape for
 *                  the process.  Layouts sum
 *                  a row in different orders, so results may differ in the
 *                  last bits from the default heuristic (0: by mean row
 *                  length), which is reproducible across processes.  On the
 *                  1025^2 L-shape the heuristic's layouts were as fast
 *  aggressive      1 = aggressive first-level coarsening in both hierarchies
 *                  (Sec. 5.1; read for smoothed aggregation): the level-0
 *                  aggregates are aggregated once more on their tentative
 *                  Galerkin matrix S_hat^T A S_hat (strength threshold
 *                  theta/2), and every vertex takes the aggregate of its
 *                  aggregate; the smoothed prolongator is built on the result
 *  geometric       1 = the geometric hierarchy of Sec. 5.4 instead of AMG:
 *                  the mesh must be the structured N x N square grid (vertex
 *                  i + N j, squares split along the (i,j)-(i+1,j+1) diagonal,
 *                  the whole boundary Dirichlet; else INVALID_ARG), and each
 *                  level takes every other grid line (N odd, N >= 5) with P1
 *                  interpolation (weights 1 and 1/2); S_j is its restriction
 *                  to interior vertices; coarse matrices are Galerkin
 *                  products as for AMG (theta, smooth_prolongator and
 *                  aggressive are not used; amgh_get_aggregates is invalid)
 *  matrix_free     1 = on the structured Kuhn cube (see amgh_kuhn_apply;
 *                  else INVALID_ARG) the level-0 smoother steps and residual
 *                  of FP32 V-cycles apply the stiffness matrix-free from the
 *                  element coefficients instead of reading the assembled
 *                  matrix; same operator, different rounding
 *  persistent_cg   1 = the block solver's mass CGs (precisions 1 and 2), and
 *                  the single-column mass CGs of precision 2, run all their
 *                  iterations in one cooperative launch over the GPU
 *                  (grid-stride rows, two bounded software grid barriers per
 *                  iteration; a barrier that gives up makes the call return
 *                  AMGH_ERR_TIMEOUT) instead of graph-replayed kernels;
 *                  handles from amgh_problem_share and the batch runtime's
 *                  handles use 0.  Same arithmetic per row, sums grouped
 *                  differently: results agree with 0 to the CG tolerance, not
 *                  to the bit */
typedef struct {
    int max_levels;
    int hessian_levels;
    double theta;
    int coarse_max;
    int smoother;
    int smooth_degree;
    int precision;
    int smooth_prolongator;
    int coarse_solve;
    int fuse_coarse;
    int autotune;
    int aggressive;
    int geometric;
    int matrix_free;
    int persistent_cg;
} amgh_amg_opts;

/* Solve options (Sec. 5.2-5.3).
 *  tol          outer relative residual ||b - H u|| / ||b||
 *  max_iter     outer CG cap
 *  inner_tol    relative residual of every state/adjoint solve A y = f
 *  mass_tol     relative residual of every mass solve M_{u,j} x = b
 *  precond      0 = none (identity), 1 = multilevel / two-grid (Q_0)
 *  ncols        must be 1 (amgh_solve_block chooses its own block width)
 *  inner_max_iter, mass_max_iter   caps of the inner CG loops
 *  precond_tol  relative residual of the state/adjoint solves of the coarse
 *               Hessians H_j, j >= 1, which occur only inside the
 *               preconditioner (0 = inner_tol; Sec. 5.2 uses 1e-8)
 *  coarse_tol, coarse_max_iter   stopping rule of the coarsest-level CG
 *               (coarse_solve = 1); reaching the cap is not an error, the
 *               iterate is used as it stands
 *  level_fallback  1 = when the outer CG finds the preconditioner indefinite
 *               (possible for small beta, Sec. 3.2; the experiments of
 *               Sec. 5.5-5.6 cut levels for this reason), drop the
 *               coarsest Hessian level and restart from u = 0, down to two
 *               levels (always positive definite); info->fallbacks and
 *               info->hessian_levels record it.  The reduction persists for
 *               later solves of this problem until amgh_amg_setup.  With
 *               coarse_solve = 0 a level whose dense H_{l-1} would exceed
 *               4096 dofs ends the fallback with AMGH_ERR_INDEFINITE; with
 *               coarse_solve = 2 that level is solved by CG instead. */
typedef struct {
    double tol;
    int max_iter;
    double inner_tol;
    double mass_tol;
    int precond;
    int ncols;
    int inner_max_iter;
    int mass_max_iter;
    double precond_tol;
    double coarse_tol;
    int coarse_max_iter;
    int level_fallback;
} amgh_solve_opts;

/* Counters of the last amgh_solve (or since amgh_reset_counters). */
typedef struct {
    int status;
    int outer_iters;
    int64_t hessian_applies; /* fine-level H applies (outer CG + true residual) */
    int64_t inner_iters;     /* all state/adjoint CG iterations, all levels */
    int64_t mass_iters;      /* all mass-matrix CG iterations */
    int64_t refinements;     /* FP64 refinement sweeps (precision = 1) */
    double final_relres;     /* ||b - H u|| / ||b|| recomputed at the end */
    double t_setup_s;
    double t_solve_s;
    int hessian_levels;      /* levels l of the preconditioner at the end */
    int fallbacks;           /* levels dropped by level_fallback */
    int64_t coarse_iters;    /* coarsest-level CG iterations (coarse_solve = 1) */
    double alg_bytes;        /* algorithmic (compulsory) bytes of every kernel the
                                single-column solve phase ran, from sizes: matrix
                                entries and indices, gathered and streamed vectors;
                                the block solver does not count (0) */
} amgh_solve_info;

/* Defaults: max_levels 25, hessian_levels 0, theta 0.08, coarse_max 256,
 * Chebyshev degree 2, precision 0, smoothed prolongator, coarse_solve 0, fuse_coarse 0,
 * autotune 0, aggressive 0, geometric 0, matrix_free 0, persistent_cg 0;
 * tol 1e-8, max_iter 200, inner/mass tol 1e-10, precond 1, ncols 1, caps
 * 1000, precond_tol 0 (= inner_tol), coarse_tol 1e-4, coarse_max_iter 1000,
 * level_fallback 0. */
void amgh_amg_opts_default(amgh_amg_opts *opts);
void amgh_solve_opts_default(amgh_solve_opts *opts);

/* A second handle on a set-up problem: the same assembled matrices, AMG
 * hierarchies and dense coarse inverses, with its own work space, desired
 * state (a copy of the parent's), graphs, counters and stream (initially
 * the parent's; give it another with amgh_set_stream).  Solves and applies
 * on different handles may run at the same time on different streams and
 * host threads.  The parent must outlive its shared handles and must not be
 * set up again while they exist; amgh_amg_setup on a shared handle returns
 * AMGH_ERR_INVALID_ARG.  A level fallback on one handle does not change the
 * others.  Sharing a shared handle shares its parent.  Release with
 * amgh_problem_destroy. */
int amgh_problem_share(amgh_problem *parent, amgh_problem **out);

/* Copy the mesh, per-element kappa (Eq. bilform), beta > 0 and the nodal
 * desired state y_d (n_vertices doubles; on the device iff y_d_on_device) to
 * the device and assemble A, M_y, M_u, M_yu (Sec. 2) there.  Element
 * contributions are summed in ascending element order without fused
 * multiply-add, so the matrices are bit-identical on every run.
 * Errors: INVALID_ARG (dim not 2/3, sizes <= 0, n_vertices or
 * n_elements*(dim+1) >= 2^31, beta <= 0 or infinite, vertex id out of range,
 * degenerate element, no vertex off the Dirichlet boundary), OOM, CUDA.
 * *out is NULL on error. */
int amgh_problem_create(const amgh_mesh *mesh, const double *kappa, double beta,
                        const double *y_d, int y_d_on_device, amgh_problem **out);

/* Replace the desired state (same layout as in amgh_problem_create). */
int amgh_set_yd(amgh_problem *p, const double *y_d, int on_device);

/* Use this cudaStream_t (e.g. torch.cuda.current_stream().cuda_stream) for all
 * later work of the problem; NULL = the legacy default stream. */
int amgh_set_stream(amgh_problem *p, void *cuda_stream);

/* Build the state and control smoothed-aggregation hierarchies (Sec. 3.1,
 * Eq. coarsestiffness/coarsemass) on the device: strength graph, distance-2
 * maximal independent set by splitmix64 priority, aggregates, smoothed
 * prolongators S_j (on A) and P_j (on the all-vertex stiffness), Galerkin
 * products for A, M_y, M_u, M_yu, and the dense coarsest factors.  Aggregates
 * are bit-identical to the sequential definition.  opts NULL = defaults.
 * Errors: INVALID_ARG (bad option, coarsest level above 4096 rows), OOM,
 * INDEFINITE (coarse Hessian not positive definite), CUDA. */
int amgh_amg_setup(amgh_problem *p, const amgh_amg_opts *opts);

/* Set the tolerances used by amgh_hessian_apply / amgh_precond_apply /
 * amgh_rhs / amgh_state_solve / amgh_gradient (inner_tol, mass_tol,
 * precond_tol and the caps; other fields ignored). */
int amgh_set_solve_opts(amgh_problem *p, const amgh_solve_opts *opts);

/* Hu = H u on the finest level (Eq. firstorderpractice): one forward and one
 * adjoint AMG-CG solve (Sec. 5.2).  u_dev, Hu_dev: n*ncols doubles, device,
 * column-major (column c at offset c*n), may not alias.  ncols > 1 runs the
 * block solver: columns in blocks of K = 2, 4 or 8 (the smallest K >= ncols,
 * at most 8), every sparse operator applied to the K columns of a block in
 * one pass, each column with its own inner CG scalars and stopping test; the
 * V-cycles are FP64 for precision 0 and FP32 otherwise.
 * Errors: NOT_SETUP, INVALID_ARG, NOT_CONVERGED, INDEFINITE, NUMERIC, CUDA
 * (for ncols > 1: the first failing column's error). */
int amgh_hessian_apply(amgh_problem *p, const double *u_dev, double *Hu_dev, int ncols);

/* z = Q_0 r, the multilevel Hessian preconditioner in M_u-scaled form
 * (Sec. 3.2 Algorithm MLAS with Eq. twogridinmulti/twogridinmultiactual and
 * the substitution of Sec. 5.2).  r_dev, z_dev: n*ncols doubles, device,
 * column-major; ncols > 1 runs the block solver as amgh_hessian_apply. */
int amgh_precond_apply(amgh_problem *p, const double *r_dev, double *z_dev, int ncols);

/* b = M_yu^T A^-1 M_y y_d (right side of Eq. firstorderpractice); b_dev: n
 * doubles, device. */
int amgh_rhs(amgh_problem *p, double *b_dev);

/* Outer CG on H u = b (Sec. 5.3) from u0 (NULL = 0), to
 * ||r_k|| <= opts->tol ||b||; writes u (n doubles) and, if y_dev is not
 * NULL, the state y = A^-1 M_yu u (m doubles).  All device pointers.
 * info (may be NULL) receives counters and the recomputed relative residual.
 * Errors: as amgh_hessian_apply, plus NOT_CONVERGED for the outer loop. */
int amgh_solve(amgh_problem *p, const double *u0_dev, double *u_dev, double *y_dev,
               const amgh_solve_opts *opts, amgh_solve_info *info);

/* Block solve of the batching pattern: ncols independent control problems on
 * this mesh, one per desired state, each the outer CG of Sec. 5.3 from u = 0
 * to ||b_c - H u_c|| <= opts->tol ||b_c||.  The columns run in blocks of
 * K = 2, 4 or 8 (the smallest K >= ncols, at most 8; a short last block is
 * padded with zero columns): every sparse operator of the outer, inner
 * (state, adjoint, mass) and preconditioner (Algorithm MLAS) work is applied
 * to the K columns of a block in one pass (SpMM), while every column keeps its
 * own CG scalars and stopping tests, so each column is the single-column
 * method.  A failing column (indefinite, non-finite, a cap reached) stops
 * alone; the others continue.  V-cycles are FP64 for precision 0 and FP32
 * otherwise; the problem's own desired state is not changed.
 *   yd_dev   ncols desired states, n_vertices doubles each, column-major,
 *            device
 *   u_dev    ncols controls, n doubles each, column-major, device (output;
 *            a failed column's entries are unspecified)
 *   opts     as amgh_solve (NULL = defaults; ncols must be 1)
 *   info     (may be NULL) counters summed over the columns (outer_iters,
 *            hessian_applies, inner/mass/coarse iterations), final_relres
 *            the largest over the converged columns, status as returned
 * Returns AMGH_OK if every column converged, else the first failing
 * column's error (with level_fallback: after the fallbacks). */
int amgh_solve_block(amgh_problem *p, const double *yd_dev, int ncols, double *u_dev,
                     const amgh_solve_opts *opts, amgh_solve_info *info);

/* Same as amgh_solve with HOST buffers: copies u0 (NULL ok) to the device,
 * solves, copies u (and y if not NULL) back.  This is the end-to-end call. */
int amgh_solve_host(amgh_problem *p, const double *u0_host, double *u_host, double *y_host,
                    const amgh_solve_opts *opts, amgh_solve_info *info);

/* State solve y = A^-1 M_yu u (Sec. 2, Eq. solutionopdef) and, if J_host is not
 * NULL, the reduced cost J(u) (Eq. functional).  u_dev n, y_dev m doubles. */
int amgh_state_solve(amgh_problem *p, const double *u_dev, double *y_dev, double *J_host);

/* Gradient of the reduced cost by the adjoint solve:
 * g = M_yu^T A^-1 M_y (y - y_d) + beta M_u u (= H u - b), with y from
 * amgh_state_solve.  u_dev, g_dev n doubles; y_dev m doubles. */
int amgh_gradient(amgh_problem *p, const double *u_dev, const double *y_dev, double *g_dev);

/* Adjoint of the solution operator K = A^-1 M_yu (Sec. 2, Eq. solutionopdef):
 * g = K^T w = M_yu^T A^-T w for a state-space vector w (m doubles, device);
 * g_dev: n doubles, device.  This is the backward pass of the state solve. */
int amgh_state_adjoint(amgh_problem *p, const double *w_dev, double *g_dev);

/* Level-wise building blocks (for tests and diagnostics).
 * amgh_vcycle: x = V_l b, one symmetric V-cycle on A_l from x = 0.
 * amgh_state_solve_level: A_l y = f by AMG-CG to rel. tolerance tol.
 * amgh_mass_solve: M_{u,l} x = b by Jacobi-CG to the mass tolerance.
 * amgh_hessian_apply_level: H_l v on level l < hessian levels.
 * amgh_precond_apply_level: which = 0: Q_l b; which = 1: R_l b (l < ell-1).
 * All vectors are device pointers of the level's size. */
int amgh_vcycle(amgh_problem *p, int level, const double *b_dev, double *x_dev);
int amgh_state_solve_level(amgh_problem *p, int level, const double *f_dev, double *y_dev,
                           double tol, int64_t *iters);
int amgh_mass_solve(amgh_problem *p, int level, const double *b_dev, double *x_dev,
                    int64_t *iters);
int amgh_hessian_apply_level(amgh_problem *p, int level, const double *v_dev, double *hv_dev);
int amgh_precond_apply_level(amgh_problem *p, int which, int level, const double *b_dev,
                             double *z_dev);

/* Sizes: m, n; number of state levels Ls, control levels Lc, Hessian levels
 * ell; state_sizes / ctrl_sizes receive up to 32 level row counts each
 * (either may be NULL). */
int amgh_query_sizes(const amgh_problem *p, int64_t *m, int64_t *n, int *Ls, int *Lc, int *ell,
                     int64_t *state_sizes, int64_t *ctrl_sizes);

/* Aggregate id of every row of level `level` of hierarchy `hier` (0 = state,
 * 1 = control); agg_host holds that level's row count int32s; *nagg the
 * number of aggregates.  level must be below the hierarchy's last level. */
int amgh_get_aggregates(const amgh_problem *p, int hier, int level, int32_t *agg_host,
                        int32_t *nagg);

/* Copy a level matrix in CSR (sorted columns) to host buffers.
 * which: 0 A, 1 M_y, 2 M_yu, 3 S (level -> level+1), 4 K_N (all-vertex
 * stiffness of the control hierarchy), 5 M_u, 6 P, 7 K_full, 8 M_full.
 * amgh_get_matrix_info gives rows, cols, nnz; amgh_get_matrix fills
 * rowptr (rows+1), col (nnz) and val (nnz). */
int amgh_get_matrix_info(const amgh_problem *p, int which, int level, int64_t *rows,
                         int64_t *cols, int64_t *nnz);
int amgh_get_matrix(const amgh_problem *p, int which, int level, int32_t *rowptr_host,
                    int32_t *col_host, double *val_host);

/* y = A x with the level-0 state stiffness applied matrix-free, for meshes
 * that are the structured Kuhn cube: N^3 vertices at (i,j,k)/(N-1) (vertex
 * i + N j + N^2 k), 6 (N-1)^3 tetrahedra cell by cell, the 6 of a cell in
 * lexicographic order of the axis permutation (a,b,c), each the path
 * o, o+e_a, o+e_a+e_b, o+(1,1,1).  Every such tetrahedron has the P1
 * stiffness kappa_T h/6 tridiag(-1, [1 2 2 1], -1) in path order (Sec. 2),
 * so only kappa is read (no matrix).  The first call checks the mesh (and
 * keeps an FP32 copy of kappa): make it before any stream capture.
 *   prec32  0: x, y double (m each, state order); 1: float
 *   x, y    device vectors of the m states (y = A x, Dirichlet vertices
 *           eliminated as in the assembled A)
 * Errors: INVALID_ARG if the mesh is not such a cube, CUDA.  Works before
 * amgh_amg_setup. */
int amgh_kuhn_apply(amgh_problem *p, int prec32, const void *x_dev, void *y_dev);

/* Two-level approximation numbers of the multilevel analysis (Sec. 4,
 * Assumption with a_j; Sec. 5.1, Tables 1-2), by the power method on the
 * GPU.  With K_j = A_j^-1 M_yu,j, Pi_j = M_u,j+1^-1 P_j^T M_u,j and
 * D_j = K_j - S_j K_j+1 Pi_j on level j:
 *   weighted 0: a~_j = ||D_j||_2 (Eq. aj-tilde), from D_j^T D_j;
 *   weighted 1: a_j = ||M_y,j^1/2 D_j M_u,j^-1/2||_2 (Eq. ajnumerical),
 *               from M_u,j^-1 D_j^T M_y,j D_j in the M_u,j inner product.
 *   level   j, 0 <= j <= min(Ls, Lc) - 2
 *   iters   power iterations (>= 1); each applies D_j and D_j^T (four AMG-CG
 *           state solves and two or three mass solves at the set tolerances)
 *   v0_dev  start vector, n_j doubles on the device (not changed)
 *   est     host: the estimate after `iters` iterations (a lower bound that
 *           increases to the norm)
 * Errors: INVALID_ARG (level, iters, a zero start vector), NOT_SETUP, the
 * solves' statuses. */
int amgh_aj_estimate(amgh_problem *p, int level, int weighted, int iters, const double *v0_dev, double *est);

/* Counters since the last reset (fields as amgh_solve_info). */
int amgh_get_counters(const amgh_problem *p, amgh_solve_info *info);

/* CG iterations since the last reset per level (32 int64 slots each, either
 * may be NULL): inner_host[l] = state/adjoint AMG-CG iterations on level l,
 * mass_host[l] = mass-matrix CG iterations on control level l. */
int amgh_get_level_counters(const amgh_problem *p, int64_t *inner_host, int64_t *mass_host);
int amgh_reset_counters(amgh_problem *p);

/* Kernel timing for roofline reporting: when enabled, CG iterations are
 * launched kernel by kernel (one iteration per host check) instead of as CUDA
 * graphs, and every solve-phase launch of the single-column path is bracketed
 * by CUDA events on the problem's stream and filed under its kernel class
 * (0 .. AMGH_KCLASSES-1; the launches the device skips, the V-cycle of a CG
 * iteration that converged, are not filed).  amgh_kernel_stats returns class
 * 0, the level-0 Chebyshev smoother step (SpMV fused with the smoother
 * update); amgh_kernel_class_stats any class, with its name.  Each returns
 * the number of timed launches, their summed duration in ms, and their
 * summed algorithmic bytes (for a sparse product nnz*(v+i) + v*(rows+cols),
 * v = value bytes, i = index bytes, plus 4*(rows+1) for CSR row pointers;
 * vectors read and written once each).  Enabling or disabling clears them.
 * The events around a launch keep it from overlapping its neighbours, so
 * amgh_kernel_timing_mask times only the classes whose bit is set in mask
 * (bit c = class c; 0 turns timing off), leaving the others to run as usual.
 * Errors: INVALID_ARG for a class out of range. */
#define AMGH_KCLASSES 15
int amgh_kernel_timing(amgh_problem *p, int enable);
int amgh_kernel_timing_mask(amgh_problem *p, unsigned mask);
int amgh_kernel_stats(amgh_problem *p, int64_t *launches, double *ms, double *bytes);
int amgh_kernel_class_stats(amgh_problem *p, int cls, int64_t *launches, double *ms, double *bytes,
                            const char **name);

/* Test hook for the bounded waits (no counterpart in the paper; process-wide,
 * not for production use).
 *   bulk_first_polls  poll limit of the level-0 staged smoother's wait for its
 *                     bulk copies: -1 restores the default, 0 makes every
 *                     block give up at once (its copies still drain under a
 *                     separate, larger limit before the block exits).  A
 *                     block that gives up computes nothing and raises a flag;
 *                     every solve-phase call checks the flag after its work
 *                     and then returns AMGH_ERR_TIMEOUT, whatever else
 *                     happened: all values that call produced are invalid.
 *   mis_round_cap     rounds the aggregation's distance-2 independent-set
 *                     loop may take before amgh_amg_setup returns
 *                     AMGH_ERR_TIMEOUT (-1: the default, n + 1 rounds, which
 *                     always suffice).
 *   prol_row_cap      aggregates a row of the smoothed prolongator may reach
 *                     before its construction moves from the per-thread
 *                     register path to the one-block-per-row path for long
 *                     rows (-1: the default, 256); results are identical.
 * Errors: INVALID_ARG for values below -1, CUDA. */
int amgh_debug_limits(int bulk_first_polls, int mis_round_cap, int prol_row_cap);

/* Batched solves of many independent problems (the batching pattern: many
 * desired states, many meshes of uneven size).  Every (problem, desired
 * state) pair is an independent outer CG.  The batch runtime gives each
 * problem up to `workers` solve slots (default: one per desired state):
 * the problem itself and handles from amgh_problem_share, each with its own
 * non-blocking CUDA stream and host thread, taking every workers-th desired
 * state of that problem; the small, latency-bound coarse-level work of many
 * solves then overlaps on the GPU.  Results are identical to solving each
 * desired state alone on the problem.
 *   probs      nprob distinct problems created by amgh_problem_create on the
 *              current device; the batch borrows them (the caller keeps
 *              ownership and must not use them, nor set them up again, until
 *              amgh_batch_destroy)
 *   amg        options for problems whose hierarchy is not set up (NULL =
 *              defaults); amgh_batch_setup builds all hierarchies concurrently
 * amgh_batch_set_workers: slots per problem (0 = one per desired state).
 * amgh_batch_solve:
 *   yd_dev[p]  device array of ncols[p] desired states of problem p, each of
 *              n_vertices(p) doubles, column-major
 *   u_dev[p]   device array of ncols[p] controls of problem p (n(p) doubles each)
 *   opts       solve options shared by all problems (NULL = defaults)
 *   info       nprob entries (may be NULL): counters summed over the
 *              problem's desired states, t_solve_s the longest slot,
 *              status = the problem's first error
 * Returns AMGH_OK if every solve converged, else the first error in problem
 * order; a failing problem does not stop the others.  The call returns
 * after all work has completed. */
typedef struct amgh_batch amgh_batch;
int amgh_batch_create(amgh_problem *const *probs, int nprob, amgh_batch **out);
int amgh_batch_setup(amgh_batch *b, const amgh_amg_opts *amg);
int amgh_batch_set_workers(amgh_batch *b, int workers);
/* block = 1: every slot solves its desired states (a contiguous share of the
 * problem's columns) with amgh_solve_block instead of one by one, and
 * workers = 0 then means one slot per problem; block = 0 (default) restores
 * the per-column solves.  Errors: INVALID_ARG. */
int amgh_batch_set_block(amgh_batch *b, int block);
int amgh_batch_solve(amgh_batch *b, const double *const *yd_dev, const int *ncols, double *const *u_dev,
                     const amgh_solve_opts *opts, amgh_solve_info *info);
void amgh_batch_destroy(amgh_batch *b);
/* Autotuner of the batch's block width and slot count (no counterpart in the
 * paper; the batching pattern): tries, on the given desired states, one slot
 * per desired state (block 0), then block solves with K = 8, 4 and 2 columns
 * on 8/K slots per problem; each candidate solves the batch once (capturing
 * its graphs) and once more under the host clock, and the fastest stays set
 * for later amgh_batch_solve calls.  Arguments as amgh_batch_solve (opts may
 * use a looser tolerance than the real solves); times (4 doubles, host, may
 * be NULL) receive the candidates' seconds and *choice (may be NULL) the
 * index kept.  Errors: as amgh_batch_solve. */
int amgh_batch_autotune(amgh_batch *b, const double *const *yd_dev, const int *ncols, double *const *u_dev,
                        const amgh_solve_opts *opts, double *times, int *choice);

/* Aggregation of a caller's matrix that allocates no device memory.  The
 * paper has no counterpart: this is a service for callers that cannot call
 * cudaMalloc (a framework's caching allocator owns the memory budget, a hard
 * memory cap, or a latency-critical path that must not allocate or implicitly
 * synchronise).  It returns exactly the level-0 aggregates amgh_amg_setup
 * computes for a matrix with this CSR (strength threshold theta): the
 * distance-2 independent set by splitmix64 priority and phases 1-3.
 *   n              rows, 1 .. 32768 (more: AMGH_ERR_INVALID_ARG)
 *   rowptr_dev, col_dev, val_dev   CSR of a symmetric matrix with sorted
 *                  columns, on the current device; rowptr_dev[0] must be 0
 *                  and rowptr_dev[n] at most 262144 (else AMGH_ERR_INVALID_ARG,
 *                  before any kernel runs)
 *   stream         cudaStream_t to run on (NULL = legacy default stream)
 *   agg_dev        n int32 outputs (device); *nagg_host = number of aggregates
 * Scratch comes from one fixed buffer inside the library (about 5 MB per
 * device that loads it, held until the process exits).  The first call on a
 * device looks up that buffer's device address (make it before any CUDA graph
 * capture).  All calls share the buffer: calls that overlap on the GPU race,
 * so the caller must serialise them.  The call synchronises `stream`. */
int amgh_aggregate_noalloc(int n, const int32_t *rowptr_dev, const int32_t *col_dev,
                           const double *val_dev, double theta, void *stream, int32_t *agg_dev,
                           int32_t *nagg_host);

/* Inverse of a dense symmetric positive definite matrix: the kernel sequence
 * that forms the exact coarsest inverses of the V-cycle (A_{L-1}^-1) and of
 * the Hessian preconditioner (G_{l-1}^-1, Sec. 3.2), exposed on its own.
 * Blocked right-looking Cholesky A = L L^T in 32-wide panels fused with the
 * forward sweep that forms W = L^-1, then A^-1 = W^T W; FP64 throughout.
 *   n          1 .. 4096 (else AMGH_ERR_INVALID_ARG)
 *   a_dev      n x n row-major FP64 on the current device; only the lower
 *              triangle (j <= i) is read, the argument is not modified
 *   inv_dev    n x n row-major FP64 output (device), the full symmetric
 *              inverse; undefined if the call does not return AMGH_OK
 *   stream     cudaStream_t to run on (NULL = legacy default stream)
 *   info       (host, may be NULL) 0, or the 1-based row of the first pivot
 *              that was not positive
 * Errors: INDEFINITE (a pivot <= 0 or not finite: A is not numerically SPD),
 * INVALID_ARG, OOM, CUDA.  Scratch (2 n^2 doubles) is taken from the
 * library's stream-ordered pool; the call synchronises `stream`. */
int amgh_dense_spd_inverse(int n, const double *a_dev, double *inv_dev, void *stream, int *info);

/* The FP64 rate of this GPU, measured: kind 0 = fused multiply-adds on the
 * FP64 pipe (every SM busy, eight independent chains per thread), kind 1 =
 * the FP64 tensor instruction mma.m8n8k4.f64 (four independent accumulators
 * per warp).  *tflops = the rate of one timed launch of about 10 ms after a
 * warm-up.  The dense coarsest-level kernels (amgh_dense_spd_inverse, the
 * coarse Hessian product) are bound by it.  Errors: INVALID_ARG (kind not 0
 * or 1, tflops NULL), OOM, CUDA.  Synchronises `stream`. */
int amgh_fp64_peak(int kind, void *stream, double *tflops);

/* Test hook: the number of polls every software grid barrier wait (the
 * grid-fused V-cycle, the persistent block mass CG) makes before it gives up
 * and the call returns AMGH_ERR_TIMEOUT; -1 restores the default (2^20 polls
 * of about 64 ns).  Process-wide.  Errors: INVALID_ARG below -1, CUDA. */
int amgh_debug_grid_polls(int polls);

/* Number of kernels this library launched since load (all problems). */
int64_t amgh_launch_count(void);

void amgh_problem_destroy(amgh_problem *p);
const char *amgh_status_string(int status);
/* The last CUDA error met inside the library by any host thread (name, code
 * and source location), or "" if none; for diagnosing AMGH_ERR_CUDA.  The
 * string is valid until the calling thread's next call of this function. */
const char *amgh_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* AMGH_H */
