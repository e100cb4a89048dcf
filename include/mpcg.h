/*
 * mpcg.h -- C ABI of the additive-multigrid multipreconditioned CG solver
 * (Kothari, Nestola, Favino, Krause, "Integrating Additive Multigrid with
 * Multipreconditioned Conjugate Gradient Method").
 *
 * The solver computes Algorithm 1 of the paper: every iteration builds the
 * block Z = [z^0 | ... | z^L] of per-level additive multigrid corrections
 * z^l = P_l^L S_l (R_L^l r) (Section 2.2; restriction R = P^T and composite
 * transfers by successive two-level transfers, Section 2.1; damped-Jacobi
 * smoothing S_l^nu on levels l >= 1, Eq. 2; an exact Cholesky solve on the
 * coarsest level), A-orthogonalises it against the last m search blocks,
 * and updates x and r with the energy-optimal coefficients
 * alpha = (P^T A P)^+ P^T r (the step-size formula of Section 2.2 and Eq. 4).
 *
 * Problem class (Section 1): a symmetric positive definite matrix from a Q1
 * finite-element discretisation on a uniform structured grid of the unit
 * square or cube, homogeneous Dirichlet nodes eliminated; scalar unknowns
 * (diffusion) or three displacement components per node (3D elasticity).
 *
 * Conventions for every entry point
 *   - Vectors hold the n unknowns in lexicographic node order, x fastest
 *     (components of a node consecutive for vector problems).
 *   - Pointers named *_dev are CUDA device pointers owned by the caller; the
 *     library never frees them.  mpcg_solve also accepts host pointers for b
 *     and x (pinned or pageable) and stages them through device memory.
 *   - All work is enqueued on the stream given in mpcg_options (0 = legacy
 *     default stream).  Entry points that return results to the host
 *     (iteration counts, histories) synchronise that stream before returning.
 *   - A negative status is an error; mpcg_last_error() returns a message for
 *     the calling thread.  No entry point aborts the process, and no kernel
 *     traps or asserts.
 *   - Thread safety: a hierarchy may be used by one host thread at a time.
 */
#ifndef MPCG_H
#define MPCG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MPCG_OK = 0,
  MPCG_NOT_CONVERGED = 1,  /* maxit reached; x holds the last iterate        */
  MPCG_ERR_ARG = -1,       /* invalid argument (message says which)          */
  MPCG_ERR_CUDA = -2,      /* a CUDA runtime call failed                     */
  MPCG_ERR_NOT_SPD = -3,   /* coarsest operator not positive definite        */
  MPCG_ERR_BREAKDOWN = -4, /* non-finite value, or every search column dropped */
  MPCG_ERR_TIMEOUT = -5,   /* a bounded device-side wait ran out             */
  MPCG_ERR_OOM = -6        /* device allocation failed                       */
} mpcg_status;

enum { MPCG_FORMAT_STENCIL = 0 };
enum { MPCG_SMOOTHER_JACOBI = 0, MPCG_SMOOTHER_SSOR = 1 };
/* Arithmetic of the solve:
 *   MPCG_FP64     FP64 vectors and FP64 arithmetic throughout;
 *   MPCG_MIXED    FP32 bulk with FP64 reductions, pseudo-inverse, coarse
 *                 Cholesky and iterative refinement on the FP64 residual;
 *   MPCG_FP64_DW  FP64 data (b, x, operators) with the bulk in double-word
 *                 arithmetic: every vector entry is a pair of floats
 *                 hi + lo (about 48 significant bits, 8 bytes) computed on
 *                 the FP32 pipe, which GB300 issues 64 times faster than
 *                 FP64; reductions, pseudo-inverse and coarse solve in FP64.
 *                 Results agree with MPCG_FP64 to ~1e-13 relative per step;
 *                 magnitudes must stay within float's exponent range (the
 *                 low word of values below ~1e-30 is flushed). */
enum { MPCG_FP64 = 0, MPCG_MIXED = 1, MPCG_FP64_DW = 2 };

/* Largest supported number of columns (grids, plus an appended column) and
 * window length. */
#define MPCG_MAX_COLS 12
#define MPCG_MAX_WINDOW 16

/*
 * A fine-grid operator in stencil form.
 *   dim        2 or 3
 *   nodes      nodes per side of the grid, boundary included; nodes - 1 (the
 *              elements per side) must be divisible by 2^(levels-1) with at
 *              least 2 elements per side left on the coarsest grid
 *   dofs_per_node
 *              1 (scalar problems such as the diffusion equation of
 *              Section 1), or 3 in 3D (linear elasticity: unknown
 *              i = a + 3 * node is displacement component a of the node)
 *   dirichlet_faces
 *              the faces whose nodes are eliminated (homogeneous Dirichlet):
 *              bit 2a = low face of axis a (x = 0, y = 0, z = 0 for a = 0,1,2),
 *              bit 2a+1 = high face; MPCG_ALL_FACES for all of them.  Nodes
 *              on the other faces are unknowns (natural boundary).  In 2D
 *              the z bits are ignored.  The unknown nodes are numbered
 *              lexicographically, x fastest.
 *   values_dev device array of S * n doubles, S = dofs_per_node * 3^dim,
 *              n the number of unknowns: plane b * 3^dim + s
 *              (s = (dx+1) + 3(dy+1) [+ 9(dz+1)]) holds for every row
 *              unknown (node, a) the coefficient coupling it to the unknown
 *              (node + (dx, dy[, dz]), b).  Couplings to eliminated or
 *              absent nodes must be zero.  The matrix must be symmetric
 *              positive definite.  Read during mg_hierarchy_setup only.
 * The coarse grids keep the same faces; transfers act componentwise, and
 * the smoother of a vector problem is block Jacobi over each node's
 * dofs_per_node x dofs_per_node diagonal block.  Vector problems allow at
 * most 8 grids.
 */
#define MPCG_ALL_FACES 0x3Fu

typedef struct {
  int dim;
  int nodes;
  int format;                 /* MPCG_FORMAT_STENCIL */
  const double* values_dev;
  int dofs_per_node;          /* 1, or 3 (3D) */
  unsigned dirichlet_faces;   /* MPCG_ALL_FACES for the pure Dirichlet problem */
} mg_operator;

/* Solver options.  mpcg_default_options() fills the paper's / the default
 * values: m = 5 (Section 3 uses the last 5 blocks), nu = 2, omega = 2/3,
 * pinv_tau = 1e-12, drop_delta = 1e-10, precision MPCG_FP64,
 * inner_rtol = 3e-3, inner pinv_tau = 1e-6, inner drop_delta = 1e-5,
 * use_graph = 1, sum_columns = 0, smoother = MPCG_SMOOTHER_JACOBI,
 * ssor_omega = 1, vcycle = 0, half_stencil = 1.  The FP32
 * inner solves converge in fewer total iterations when restarted often (the
 * FP64 refinement renews the residual and the search space), hence the
 * loose inner tolerance. */
typedef struct {
  int m;                 /* truncation window: stored search blocks, 1..MPCG_MAX_WINDOW */
  int nu;                /* damped-Jacobi sweeps per level, >= 1 (Eq. 2, c_0 = 0) */
  double omega;          /* Jacobi damping */
  double pinv_tau;       /* eigenvalue cutoff of the scaled pseudo-inverse (FP64 path) */
  double drop_delta;     /* column-drop threshold on A-norm^2 ratios (FP64 path) */
  int precision;         /* MPCG_FP64, MPCG_MIXED or MPCG_FP64_DW (see above) */
  double inner_rtol;     /* MPCG_MIXED: relative tolerance of each FP32 inner solve */
  double inner_pinv_tau; /* MPCG_MIXED: cutoff used inside the FP32 inner solve */
  double inner_drop_delta;
  int max_outer;         /* MPCG_MIXED: maximum refinement steps */
  int use_graph;         /* 1: run each solve as one CUDA graph with a device-side
                            loop; 0: launch the kernels directly (same results) */
  int sum_columns;       /* 1: use the sum of the grids' corrections, B r of Eq. 3,
                            as a single search direction (additive MG as one
                            preconditioner; with m = 1 this is additive-MG PCG,
                            the paper's comparison method); 0: one column per grid */
  int smoother;          /* MPCG_SMOOTHER_JACOBI (damped Jacobi, omega, Eq. 2) or
                            MPCG_SMOOTHER_SSOR: nu multicoloured SSOR steps (relaxation
                            ssor_omega) from zero per grid -- Section 3's smoother */
  double ssor_omega;     /* SSOR relaxation, 0 < ssor_omega < 2 (default 1: symmetric
                            Gauss-Seidel) */
  int vcycle;            /* 1: the multiplicative V(nu, nu) cycle as the single
                            preconditioned direction (with m = 1: the MG(V)-PCG method
                            Section 3 compares against), smoothing with the chosen
                            smoother (nu SSOR steps, or nu damped-Jacobi sweeps, the
                            post-smoothing continuing from the corrected iterate);
                            scalar problems; not with sum_columns */
  int half_stencil;      /* MPCG_MIXED, scalar stencil grids: 1 the FP32 SpMM and
                            smoothing read the stencil's symmetric half (the diagonal
                            and the couplings to the later neighbours, 14 of 27 planes
                            in 3D, 5 of 9 in 2D; a coupling to an earlier neighbour is
                            read as A(i, i - s) = A(i - s, i)); 0 the full stencil.
                            The sums agree where the stored operator is exactly
                            symmetric and differ by rounding where it is not (Galerkin
                            products summed in another order) */
  void* stream;          /* cudaStream_t */
} mpcg_options;

typedef struct mg_hierarchy mg_hierarchy;

/* Fill *opt with the defaults listed above.  Returns MPCG_ERR_ARG on NULL. */
mpcg_status mpcg_default_options(mpcg_options* opt);

/*
 * Build the multilevel hierarchy below A_fine (Section 2.1): `levels` nested
 * grids by uniform coarsening (levels = 1: the fine grid is the coarsest and
 * is solved exactly), bilinear/trilinear prolongations P_j between
 * consecutive grids, restrictions R_j = P_j^T, Galerkin coarse operators
 * A_{j-1} = P_j^T A_j P_j, the damped inverse diagonals, and the dense
 * Cholesky factor of the coarsest operator.  All of it is computed on the
 * device.  The coarsest grid may hold at most 1024 unknowns.
 * On success *out owns device memory until mg_hierarchy_destroy.
 * Errors: MPCG_ERR_ARG (bad sizes, levels too many for the grid),
 * MPCG_ERR_NOT_SPD (coarsest Cholesky failed), MPCG_ERR_OOM, MPCG_ERR_CUDA.
 */
mpcg_status mg_hierarchy_setup(const mg_operator* A_fine, int levels,
                               const mpcg_options* opt, mg_hierarchy** out);

/*
 * Solve A x = b by Algorithm 1 (FP64), or by FP32 inner MPCG solves inside
 * FP64 iterative refinement when opt->precision == MPCG_MIXED.
 *   b, x       n doubles each (device or host memory); x holds x_0 on entry
 *              and the final iterate on return.
 *   rtol       stop when ||b - A x||_2 <= rtol ||b||_2 (recursive residual in
 *              the FP64 path; true FP64 residual in the mixed path)
 *   maxit      maximum number of x updates (inner updates in MIXED)
 *   iters_out  number of x updates performed (may be NULL)
 *   res_hist   host array of >= maxit+1 doubles or NULL: ||r_k||/||b||
 *   alpha_hist host array of >= maxit * ncols doubles or NULL: the alpha
 *              vector of each iteration (FP64 path), ncols = mg_num_columns()
 * Returns MPCG_OK, MPCG_NOT_CONVERGED, or an error.  On MPCG_ERR_BREAKDOWN
 * x holds the last iterate.
 */
mpcg_status mpcg_solve(mg_hierarchy* h, const double* b, double* x, double rtol,
                       int maxit, int* iters_out, double* res_hist, double* alpha_hist);

/*
 * Batches of independent problems on the same grid (each with its own
 * operator): one hierarchy holds all nprob problems and every kernel works on
 * the whole batch (problem index = grid dimension y).  mpcg_solve on such a
 * hierarchy takes b and x as nprob problems of n unknowns back to back,
 * iters_out as nprob ints, res_hist as nprob blocks of maxit+1 doubles and
 * alpha_hist as nprob blocks of maxit*ncols doubles; one graph launch (per
 * refinement step in MPCG_MIXED) runs until every problem has converged,
 * each problem stopping on its own tolerance.  The status is the worst of
 * the problems'.  mg_apply_operator, mg_corrections, mg_get_operator and the
 * learned column take single-problem hierarchies only.
 */
mpcg_status mg_hierarchy_setup_batched(const mg_operator* ops, int nprob, int levels, const mpcg_options* opt,
                                       mg_hierarchy** out);
int mg_num_problems(const mg_hierarchy* h);

/*
 * Algebraic hierarchies (Section 2.1: the nested spaces may come from
 * agglomeration rather than nested meshes; Section 3, Example 2 builds them
 * algebraically).  The grids are built from the fine matrix alone by
 * smoothed aggregation (Vanek, Mandel and Brezina, 1996):
 *   strength   j != i strongly influences i when -a_ij > 0 and
 *              -a_ij >= theta max_{k != i}(-a_ik); i and j are coupled when
 *              either influences the other (positive couplings are weak)
 *   aggregates in index order, an unknown whose strong neighbours are all
 *              free starts an aggregate with them; each remaining unknown
 *              joins the aggregate of its first strong neighbour (ascending
 *              column) placed that way; unknowns without strong neighbours
 *              stay outside every aggregate
 *   transfers  T[i, a] = 1/sqrt(|a|); P = (I - (w/rho) D^-1 A) T with rho =
 *              max_i sum_j |a_ij| / a_ii; R = P^T; A_c = P^T A P
 * until a grid has at most coarse_size unknowns, max_levels grids exist, or
 * an aggregation does not reduce the count.  The setup runs on the host (C++,
 * once per matrix); the solve is the same additive MG-MPCG as for stencil
 * hierarchies, with damped Jacobi (nu sweeps from zero, Eq. 2) on every grid
 * >= 1 with the weight omega_j = min(omega, (4/3) / rho_j), rho_j =
 * max_i sum_k |a_ik| / a_ii on grid j (so that every level correction stays
 * positive definite), the exact coarse solve (at most 1024 unknowns), and every operator
 * and transfer applied by the device in sliced ELLPACK form.  Grid indices
 * follow the paper: 0 is the coarsest, mg_num_levels() - 1 the input matrix.
 * Single problems, scalar unknowns; the V-cycle (vcycle = 1) smooths with
 * damped Jacobi there; the SSOR smoother (its colouring needs grid
 * coordinates), the learned column and the matrix-free operator are not
 * provided for them.
 */
typedef struct {
  int n;                 /* rows = columns, 1 .. 2^30 */
  const int* rowptr;     /* n + 1 offsets into col/val, rowptr[0] = 0 (host) */
  const int* col;        /* column of each entry, ascending within a row (host) */
  const double* val;     /* value of each entry (host) */
} mg_csr;

typedef struct {
  double theta;          /* strength threshold in [0, 1]; default 0.4 */
  double w;              /* prolongator smoothing weight in [0, 2]; 0 = plain aggregation; default 4/3 */
  int max_levels;        /* grids including the finest, 1..MPCG_MAX_COLS; default MPCG_MAX_COLS */
  int coarse_size;       /* stop at <= this many unknowns, 1..1024; default 256 */
} mg_amg_options;

enum { MPCG_AMG_A = 0, MPCG_AMG_P = 1, MPCG_AMG_R = 2 };

mpcg_status mg_amg_default_options(mg_amg_options* amg);

/*
 * Build an algebraic hierarchy for the symmetric positive definite matrix A
 * (host CSR, read during the call only; the matrix must be square with
 * ascending columns, positive diagonal entries and symmetric to 1e-12
 * relative).  amg and opt may be NULL for the defaults; opt->smoother must
 * be MPCG_SMOOTHER_JACOBI.  On success *out owns device
 * memory until mg_hierarchy_destroy; mpcg_solve, mg_corrections,
 * mg_apply_operator and mg_level_size work on it as on a stencil hierarchy
 * (vectors of A.n unknowns in the matrix's order).
 * Errors: MPCG_ERR_ARG (bad matrix or options, coarsest grid above 1024
 * unknowns), MPCG_ERR_NOT_SPD (coarsest Cholesky failed), MPCG_ERR_OOM,
 * MPCG_ERR_CUDA.
 */
mpcg_status mg_hierarchy_setup_algebraic(const mg_csr* A, const mg_amg_options* amg, const mpcg_options* opt,
                                         mg_hierarchy** out);

/*
 * The built hierarchy, for inspection (host copies kept by the handle).
 * mg_amg_aggregates: for grid level >= 1, agg[i] = the unknown of grid
 * level - 1 (the aggregate) that unknown i of grid `level` belongs to, or -1;
 * agg holds mg_level_size(h, level) ints.
 * mg_amg_nnz: entries of A_level (which = MPCG_AMG_A) or of P_level (grid
 * level - 1 -> level, which = MPCG_AMG_P, level >= 1); -1 on bad arguments.
 * mg_amg_get: that matrix in CSR form into host arrays of rows + 1, nnz and
 * nnz entries (rows = mg_level_size(h, level)).
 * Errors: MPCG_ERR_ARG (not an algebraic hierarchy, bad level or pointer).
 */
mpcg_status mg_amg_aggregates(const mg_hierarchy* h, int level, int* agg);
long long mg_amg_nnz(const mg_hierarchy* h, int level, int which);
mpcg_status mg_amg_get(const mg_hierarchy* h, int level, int which, int* rowptr, int* col, double* val);

/*
 * The same smoothed-aggregation setup on the host alone (no device memory,
 * no CUDA call): for inspecting a hierarchy before building a solver.
 * mg_amg_setup_host checks A and amg as mg_hierarchy_setup_algebraic does
 * (amg may be NULL) and builds every grid; the inspection calls take the
 * same arguments as their mg_amg_* counterparts (grid 0 is the coarsest).
 * mg_amg_host_size returns -1 and the others MPCG_ERR_ARG on bad arguments.
 * The handle owns host memory until mg_amg_host_destroy.
 */
typedef struct mg_amg_host mg_amg_host;
mpcg_status mg_amg_setup_host(const mg_csr* A, const mg_amg_options* amg, mg_amg_host** out);
int mg_amg_host_levels(const mg_amg_host* a);
long long mg_amg_host_size(const mg_amg_host* a, int level);
long long mg_amg_host_nnz(const mg_amg_host* a, int level, int which);
mpcg_status mg_amg_host_aggregates(const mg_amg_host* a, int level, int* agg);
mpcg_status mg_amg_host_get(const mg_amg_host* a, int level, int which, int* rowptr, int* col, double* val);
/*
 * The sliced-ELLPACK form the device applies (one warp per slice of 32 / g
 * rows, g = 2^lg lanes per row: the largest power of two <= 32 with
 * g <= mean row length / 6; slot k of lane l of slice s at
 * sptr[s] + 32 k + l, lane l serving row l / g of the slice and its entries
 * l mod g, l mod g + g, ...; padding column 0, value 0) of A_level, P_level
 * or R_level = P_level^T (which = MPCG_AMG_R, level >= 1).
 * mg_amg_host_ell_entries returns the stored entries (padding included), or
 * -1; mg_amg_host_ell writes lg, the slice count, nslices + 1 offsets and
 * that many columns and values.
 */
long long mg_amg_host_ell_entries(const mg_amg_host* a, int level, int which);
mpcg_status mg_amg_host_ell(const mg_amg_host* a, int level, int which, int* lg, int* nslices, int* sptr, int* col,
                            double* val);
void mg_amg_host_destroy(mg_amg_host* a);
/*
 * Problems of uneven size: one batched hierarchy per grid size (nclass of
 * them, preferably each with its own stream in its options), solved
 * concurrently: as one graph launch (mpcg_solve_batched_graph) when every
 * class is a mixed-precision hierarchy with graphs enabled, else from one
 * host thread per class.  b[c], x[c], iters[c] are the arguments of
 * mpcg_solve for class c (iters may be NULL).  Returns the worst status of
 * all problems.
 */
mpcg_status mpcg_solve_batched(mg_hierarchy* const* hs, int nclass, const double* const* b, double* const* x,
                               double rtol, int maxit, int* const* iters);
/*
 * mpcg_solve_batched as ONE CUDA graph launch: every class's whole
 * mixed-precision solve (refinement loop and inner MPCG loop as conditional
 * while nodes, no host round trip) is a root branch of one graph, and the GPU
 * runs the branches concurrently; inputs are packed and results unpacked on
 * hs[0]'s stream around the launch.  The graph is built on the first call and
 * reused while the classes, their graphs, rtol and maxit are unchanged (at
 * most 8 such graphs are cached; destroying a hierarchy drops those holding
 * it).  mpcg_solve_batched takes this path by itself when it applies.
 * Errors: MPCG_ERR_ARG unless every class is a distinct MPCG_MIXED hierarchy
 * with graphs enabled (use_graph) on one device; MPCG_ERR_CUDA if the graph
 * cannot be built; per class as mpcg_solve (the worst status is returned).
 */
mpcg_status mpcg_solve_batched_graph(mg_hierarchy* const* hs, int nclass, const double* const* b,
                                     double* const* x, double rtol, int maxit, int* const* iters);

/* Number of grids and of search columns (grids + appended columns). */
int mg_num_levels(const mg_hierarchy* h);
int mg_num_columns(const mg_hierarchy* h);
/* Interior unknowns of grid `level` (0 = coarsest), or -1. */
long long mg_level_size(const mg_hierarchy* h, int level);

/*
 * Y = A_level X for `ncols` columns (block SpMM of the Section 2.2 update
 * A Z); X_dev, Y_dev are column-major n_level x ncols device arrays.
 */
mpcg_status mg_apply_operator(mg_hierarchy* h, int level, const double* X_dev,
                              double* Y_dev, int ncols);

/*
 * Z = [z^0 | ... | z^J] (Section 2.2): the additive multigrid correction of
 * every grid for the fine residual r, coarse grid first (with the options'
 * smoother).  Z_dev is a column-major n x levels device array.  With
 * vcycle = 1 it is one column instead, the V-cycle B_V r.
 */
mpcg_status mg_corrections(mg_hierarchy* h, const double* r_dev, double* Z_dev);

/*
 * The FP32 arithmetic of the mixed precision's inner solves, for testing it
 * against FP64: mg_apply_operator and mg_corrections with the data rounded to
 * FP32 on entry and the FP32 kernels of the inner iterations (on scalar
 * grids, the stored stencil's symmetric half: the diagonal and the couplings
 * to the lexicographically later neighbours, the others read transposed as
 * A(i, i - s) = A(i - s, i), unless the options set half_stencil = 0).
 * mg_apply_operator_f32 applies the stored stencil even where a matrix-free
 * fine operator is attached (mg_attach_q1_kappa); mg_corrections_f32 smooths
 * as the inner solve does, with that operator on the fine grid when it is
 * attached.  Same arguments and layouts as the
 * FP64 calls; results are returned as doubles.  MPCG_ERR_ARG unless h is a
 * single stencil hierarchy built with precision MPCG_MIXED.
 */
mpcg_status mg_apply_operator_f32(mg_hierarchy* h, int level, const double* X_dev,
                                  double* Y_dev, int ncols);
mpcg_status mg_corrections_f32(mg_hierarchy* h, const double* r_dev, double* Z_dev);

/* Copy grid `level`'s Galerkin operator in the stencil format above into
 * planes_dev (3^dim * n_level doubles, device). */
mpcg_status mg_get_operator(mg_hierarchy* h, int level, double* planes_dev);   /* stencil hierarchies */

/*
 * Measurement support (not part of the method).  Kernel launches are grouped
 * in MPCG_NUM_KERNEL_CLASSES classes named by mpcg_kernel_class_name():
 * pack, residual, init, restrict, coarse_solve, prolong, jacobi, spmm,
 * gram_window, small_beta, orth_update, small_alpha, update_xr, check, aux,
 * net (the learned column) and orth_gram (the Gram partials of the new block
 * in double-word arithmetic, a kernel of its own there).
 *
 * mpcg_solve_profiled runs mpcg_solve with direct kernel launches (no graph)
 * and a CUDA event pair around every launch on the hierarchy's stream; it
 * returns per class the summed device time in ms (class_ms) and the launch
 * count (class_launches), both arrays of MPCG_NUM_KERNEL_CLASSES entries or
 * NULL, and, if trace_cls / trace_ms are not NULL, the class and duration of
 * every launch in launch order (at most trace_cap entries; *trace_len gets
 * the full count).  The numerical result equals that of mpcg_solve.
 * mg_last_launches returns how many kernels the last mpcg_solve or
 * mpcg_solve_profiled call on h executed (graph launches counted per node).
 */
#define MPCG_NUM_KERNEL_CLASSES 17
const char* mpcg_kernel_class_name(int cls);
mpcg_status mpcg_solve_profiled(mg_hierarchy* h, const double* b, double* x, double rtol, int maxit,
                                int* iters_out, double* class_ms, long long* class_launches,
                                int* trace_cls, float* trace_ms, long long trace_cap, long long* trace_len);
long long mg_last_launches(const mg_hierarchy* h);

/*
 * Counters of the last solve on h for problem `problem` of the batch (0 for
 * a single problem), read from the device after the call (synchronises the
 * hierarchy's stream).  out[0] = x updates, out[1] = termination (0 running,
 * 1 converged, 2 maxit, 3 breakdown), out[2] = search columns removed by the
 * drop rule of the singular-Gram remark (Section 2.2) summed over all blocks,
 * out[3] = blocks whose pseudo-inverse (P^T A P)^+ took the eigenvalue path
 * (the Cholesky certificate that every eigenvalue passes the cutoff failed).
 * FP64 path: the whole solve; MPCG_MIXED: the last FP32 inner solve.
 * Errors: MPCG_ERR_ARG (NULL h or out, problem out of range), MPCG_ERR_CUDA.
 */
mpcg_status mg_last_solve_counters(const mg_hierarchy* h, int problem, int* out4);

/*
 * Matrix-free fine operator (an extension: the paper names the combination
 * with a matrix-free strategy as future work, Section 4).  For a scalar
 * hierarchy (2D or 3D, single or batched) whose fine operator is the Q1
 * discretisation of -div(kappa grad u) of Section 1 (kappa constant on each
 * element, isotropic, h = 1/(nodes - 1)), mg_attach_q1_kappa takes the
 * element coefficients kappa_dev (device doubles: for each problem of the
 * batch in turn, (nodes - 1)^dim elements, x fastest) and from then on the
 * FP32 kernels of the mixed-precision inner solves rebuild the fine rows
 * from them (the block SpMM and the fine-grid two-sweep Jacobi) instead of
 * streaming the stored stencil: about 1 instead of 3^dim coefficient words
 * per unknown.  The stored operators stay for setup, the coarse grids and
 * the FP64 refinement residual.  The call checks every coupling between
 * unknowns of the stored FP64 fine stencils against the ones kappa defines
 * (largest difference at most 1e-10 of the largest coefficient) and returns
 * MPCG_ERR_ARG otherwise (and for vector hierarchies); after a refused call
 * the stored operator is in use.  mg_detach_q1_kappa goes back to the stored
 * operator.  Results differ from the stored-operator
 * solve by FP32 rounding only. */
mpcg_status mg_attach_q1_kappa(mg_hierarchy* h, const double* kappa_dev);
mpcg_status mg_detach_q1_kappa(mg_hierarchy* h);

/*
 * Learned search column (an extension beyond the paper; 2D grids).
 * A 3x3 convolutional network N with channels 2 -> 16 -> 16 -> 16 -> 1 (ReLU
 * after the first three, zero padding, no bias; bfloat16 weights and
 * activations, FP32 accumulation) maps the scaled residual r/||r|| and the
 * coefficient channel c = log10(diag A)/3 - mean(...) to an approximate
 * error y.  Once attached, every MPCG iteration appends z = ||r|| y as one
 * more column of Z, which the energy minimisation weights like the others
 * (zero weight, or a dropped column, when it does not help).
 * Parameters: mg_learned_num_params() floats, layer by layer, each layer
 * W[co][ci][ky][kx] (tap (ky, kx) multiplies the input at (x+kx-1, y+ky-1)).
 *
 * Single 3D vector problems (3 unknowns per node, e.g. linear elasticity)
 * take a 3x3x3 network instead: channels 3 -> 16 -> 16 -> 16 -> 3 (ReLU after
 * the first three, zero padding outside the unknown grid, no bias, no
 * coefficient channel; bfloat16 weights and activations, FP32 accumulation)
 * maps the three displacement components of r/||r|| to the three components
 * of y.  Parameters: mg_learned_num_params_of(h) = 16416 floats, layer by
 * layer, each W[co][ci][kz][ky][kx] (tap (kz, ky, kx) multiplies the input
 * at (x+kx-1, y+ky-1, z+kz-1)).  Training batches hold 1..8 pairs.
 */
typedef struct {
  int epochs;        /* passes over the training pairs */
  int batch;         /* pairs per Adam step, 1..MPCG_MAX_COLS (same problem) */
  double lr, beta1, beta2, eps;   /* Adam (Kingma & Ba) */
  unsigned long long seed;        /* shuffling */
} mg_train_opts;

/* Parameter count of the 2D network. */
int mg_learned_num_params(void);
/* Parameter count of h's network (the 2D or the 3D vector one); -1 for NULL. */
int mg_learned_num_params_of(const mg_hierarchy* h);
/* Attach weights (host or device floats, mg_learned_num_params_of(h) of
 * them); mpcg_solve then uses mg_num_levels()+1 columns.  Errors:
 * MPCG_ERR_ARG (scalar 3D or batched problem, wrong count). */
mpcg_status mg_learned_attach(mg_hierarchy* h, const float* params, int nparams);
mpcg_status mg_learned_detach(mg_hierarchy* h);
/* y = N(rhat, c) for nimg images on h's fine grid (device, n floats each,
 * rhat already scaled); needs attached weights. */
mpcg_status mg_learned_forward(mg_hierarchy* h, const float* rhat_dev, float* y_dev, int nimg);
/* mg_learned_forward that also copies the activations out for inspection
 * (the tensor-core inference kernel): acts_dev (device, may be NULL) gets
 * 4 * nimg * n * 16 floats, [layer][image][point][channel], points
 * lexicographic (x fastest); layer 0 holds the two bfloat16 input channels
 * (zero-padded to 16), layers 1-3 the bfloat16 outputs of the first three
 * convolutions after ReLU.  3D vector problems: points are the grid nodes
 * (n / 3 of them), layer 0 holds the three input components. */
mpcg_status mg_learned_forward_acts(mg_hierarchy* h, const float* rhat_dev, float* y_dev, float* acts_dev,
                                   int nimg);
/*
 * One forward and backward pass of the training kernels (no weight update)
 * on nimg (1..MPCG_MAX_COLS; 1..8 for 3D vector problems) pairs (rhat_i,
 * e_i) of problem h (device, n floats each): grad (host or device,
 * mg_learned_num_params_of(h) doubles) gets
 * the gradient of the mean A-angle loss with respect to params (host or
 * device floats, the FP32 master weights; the forward uses their bfloat16
 * rounding); loss (host, may be NULL) the mean loss; acts_dev (device, may
 * be NULL) the training forward's activations in the layout of
 * mg_learned_forward_acts; y_dev (device, may be NULL) the outputs.
 * Errors: MPCG_ERR_ARG, MPCG_ERR_OOM, MPCG_ERR_CUDA.
 */
mpcg_status mg_learned_grad(mg_hierarchy* h, const float* params, const float* rhat_dev, const float* e_dev,
                            int nimg, double* grad, float* acts_dev, float* y_dev, double* loss);
/*
 * Train the network on the GPU: pairs (rhat_i, e_i) of scaled residuals and
 * the matching errors (device, npairs x n floats, compact layout) belonging to
 * problem pair_prob[i] (host ints) among hs[0..nprob-1] (same fine grid).
 * Loss per pair: the A-angle 1 - (e^T A y)^2 / ((e^T A e)(y^T A y)), A in FP32;
 * forward and backward run in the library's kernels, Adam on FP32 master
 * weights.  params (host or device floats) holds the initial weights on entry
 * and the trained ones on return; loss_hist (host, epochs doubles, may be
 * NULL) gets the mean loss of every epoch.
 */
mpcg_status mg_learned_train(mg_hierarchy* const* hs, int nprob, const int* pair_prob, int npairs,
                             const float* rhat_dev, const float* e_dev, const mg_train_opts* opts,
                             float* params, double* loss_hist);

/*
 * Failure-path check of the learned column's tensor-core kernels (no
 * counterpart in the paper).  Every such kernel waits on mbarriers for its
 * MMAs with a bounded number of polls; a wait that runs out makes the kernel
 * let its issued MMAs finish (bounded), free its tensor memory and set an
 * error flag that the calling entry point returns as MPCG_ERR_TIMEOUT (the
 * CUDA context stays usable).  This sets the polls of the first waits on the
 * current device: 0 gives up at once (the failure path runs on every CTA),
 * 4194304 is the default.  Graphs captured earlier read the new value too.
 * Errors: MPCG_ERR_ARG (polls < 0), MPCG_ERR_CUDA.
 */
mpcg_status mg_set_tensor_wait_limit(long long polls);

/* Release everything the hierarchy owns.  NULL is ignored. */
void mg_hierarchy_destroy(mg_hierarchy* h);

/*
 * Y = A X for `ncols` columns (1..MPCG_MAX_COLS), A a fine-grid operator in
 * the mg_operator stencil format (dim, nodes, values_dev), without allocating
 * any device memory.  The paper has no counterpart to this entry point: it is
 * a service for callers that cannot call cudaMalloc -- for example code whose
 * device memory is fully reserved by another framework's pool allocator, or
 * a latency-critical loop that must not call cudaMalloc/cudaFree because
 * cudaFree synchronises the whole device.  It computes what
 * mg_apply_operator computes on the finest grid of a scalar hierarchy whose
 * six faces are all Dirichlet (dofs_per_node = 1, dirichlet_face_mask 0x3F),
 * without needing a hierarchy.
 *   nodes       nodes per side, boundary included; nodes - 1 in [2, 32768]
 *               (any value, as mg_hierarchy_setup accepts)
 *   values_dev  3^dim * n doubles (device), X_dev, Y_dev column-major
 *               n x ncols (device), n = (nodes-2)^dim interior nodes
 *   stream      cudaStream_t; the work is only enqueued on it (the call does
 *               not synchronise), so synchronise before reading Y.
 * Scratch: one static device array of 2^21 doubles (16 MiB) that every GPU
 * which loads the library keeps until the process exits.  A grid needs
 * (3^dim + 2 ncols) * len doubles of it, len ~ (nodes-1)^dim padded;
 * larger requests return MPCG_ERR_ARG with a message naming both sizes
 * (e.g. 3D grids up to 33^3 nodes with 12 columns, 2D grids up to 257^2
 * nodes with 11 columns).
 * The array's device address is looked up with cudaGetSymbolAddress on the
 * first call made in each CUDA context (with that context current) and
 * cached under the context's unique ID; a device reset or another context
 * yields a new ID and therefore a fresh lookup.  Make the first call in a
 * context before any stream capture.  All calls share the one array, and it
 * keeps the last call's contents (the call clears it first): calls whose work
 * overlaps on the GPU (different streams or host threads without ordering)
 * race on it.  A successful call clears mpcg_last_error().
 */
mpcg_status mg_stencil_apply_noalloc(int dim, int nodes, const double* values_dev, const double* X_dev,
                                     double* Y_dev, int ncols, void* stream);

/*
 * Autotuner of the launch shapes (the paper has no counterpart; the
 * kernels' grid shapes otherwise follow fixed rules measured on GB300).
 * Tunables, each keyed by (tunable, arithmetic, grid points incl. padding,
 * problems in the batch, columns):
 *   MG_TUNE_STREAM_BLOCKS  blocks of the streaming block kernels (A-
 *                          orthogonalisation, update, residual) on a grid;
 *   MG_TUNE_SPMM_BLOCKS    blocks of the block SpMM;
 *   MG_TUNE_GRAM_CHUNKS    point chunks per window block of the window Gram;
 *   MG_TUNE_JACOBI_NARROW  1: one point per thread in the Jacobi sweep of a
 *                          grid, 0: a 16-byte vector per thread.
 * Every tuned value is clamped at launch to the range the solver's buffers
 * reserve and to at most 64 FP32 points per thread per partial sum, so no
 * table content can make a launch unsafe or change the accuracy bound.
 *
 * mg_autotune(h, cache_path, timed): for h's finest grid in h's arithmetic
 * (and the Jacobi switch of every scalar grid), times each candidate shape
 * on whole solves of a fixed random right-hand side as they run (graph
 * launch, concurrent multigrid branches; CUDA events around batches of five
 * solves, the best of three batches after a warm-up batch), one shape at a
 * time against the best found so far, and keeps the fastest.  With cache_path (may be NULL) a
 * cache written on this device that holds every key is loaded instead of
 * timing, and the table is written there afterwards.  Changes results only
 * at rounding level (reduction partitions follow the shapes).  Shapes apply
 * to every hierarchy of the process with the same keys; graphs captured
 * before are rebuilt on their next solve.  *timed (may be NULL) gets the
 * number of candidates timed (0 when the cache served).  Synchronises.
 * Errors: MPCG_ERR_ARG (NULL h, unwritable cache), MPCG_ERR_CUDA, or a
 * failed timed solve's status.
 *
 * mg_autotune_load / mg_autotune_save (host only): the JSON cache, tagged
 * with a device name and SM count; a file for another device is refused and
 * loads nothing.  mg_autotune_lookup returns a stored value or -1;
 * mg_autotune_set stores one (clamped at launch like any other);
 * mg_autotune_clear empties the table (the fixed rules apply again).
 */
enum { MG_TUNE_STREAM_BLOCKS = 0, MG_TUNE_SPMM_BLOCKS = 1, MG_TUNE_GRAM_CHUNKS = 2, MG_TUNE_JACOBI_NARROW = 3 };
enum { MG_TUNE_ANY = -1, MG_TUNE_F32 = 0, MG_TUNE_F64 = 1, MG_TUNE_DW = 2 };
mpcg_status mg_autotune(mg_hierarchy* h, const char* cache_path, int* timed);
mpcg_status mg_autotune_load(const char* cache_path, const char* device_name, int sm_count, int* entries);
mpcg_status mg_autotune_save(const char* cache_path, const char* device_name, int sm_count);
int mg_autotune_lookup(int tunable, int kind, long long npts, int nb, int ncols);
void mg_autotune_set(int tunable, int kind, long long npts, int nb, int ncols, int value);
void mg_autotune_clear(void);

/* Message describing the last error on the calling thread ("" if none). */
const char* mpcg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MPCG_H */
