/*
 * hhg.h -- C ABI of the GB300 matrix-free FMG Stokes library.
 *
 * The library solves the discrete Stokes system of Kohl & Ruede,
 * "Textbook efficiency: massively parallel matrix-free multigrid for the
 * Stokes system" (arXiv 2010.13513):
 *
 *     [ A   B^T ] [u]   [f]
 *     [ B   -C  ] [p] = [g],        A = diag(A, A, A)          (Sec. 2, Eq. stokes-discrete)
 *
 * with stabilised P1-P1 (PSPG, Eq. pspg, delta = 1/12) or Taylor-Hood P2-P1
 * elements on a hierarchy of uniformly refined macro meshes (Sec. 2.1),
 * by full multigrid with variable V-cycles (Algorithm 1), an inexact Uzawa
 * smoother (Sec. 3.2, Eqs. uzawa-iteration / uzawa-velocity / uzawa-pressure)
 * and nodal-interpolation transfers (Sec. 3.3).  Every step of the solve
 * runs in the library's own CUDA kernels on one GPU.
 *
 * Conventions shared by all entry points
 * --------------------------------------
 *  - Return value: 0 (HHG_OK) or a negative HHG_E* code.  A human-readable
 *    description of the most recent error of the calling thread is returned
 *    by hhg_last_error().  No entry point aborts the process.
 *  - Handles (hhg_mesh, hhg_problem) are opaque, created and freed by the
 *    library (*_create / *_destroy).
 *  - Device memory: the library never allocates device memory for a
 *    problem.  The caller allocates one workspace of the size reported by
 *    hhg_problem_workspace_bytes() (e.g. as a torch tensor) and binds it with
 *    hhg_problem_bind(); the library owns its contents until the problem is
 *    destroyed, the caller keeps ownership of the allocation.
 *  - Vector arguments "x", "b", "y", "r" are device pointers into caller-owned
 *    buffers laid out as described by hhg_layout(); they are borrowed for the
 *    duration of the call and never freed by the library.  Their element type
 *    is given by the `prec` argument (HHG_FP64: double, HHG_FP32: float).
 *  - Every kernel is issued on the CUDA stream passed to hhg_problem_bind()
 *    and all calls are asynchronous with respect to the host unless they
 *    return host values (norms, statistics), which synchronise that stream.
 *  - Host arrays are "canonical": nodal values in lexicographic order of the
 *    velocity nodes (first index fastest) -- the level-l lattice for P1-P1,
 *    the doubled lattice (the level-(l+1) lattice) for P2-P1 -- and of the
 *    pressure nodes (level-l lattice); a block vector is [u1 | u2 | u3 | p].
 *
 * Supported macro meshes
 * ----------------------
 *  Unions of Kuhn-split cubes: an mx x my x mz box of cubes of side H, each cut
 *  into the 6 tetrahedra around its (0,0,0)-(1,1,1) diagonal.  Bey refinement
 *  of such a macro mesh is the Kuhn (Freudenthal) lattice with spacing
 *  h = H / 2^l on every level, so each field is stored box-shaped and every
 *  macro-cell carries the same constant stencils (Sec. 2.1).  All boundary
 *  faces are Dirichlet for the velocity; the pressure is fixed by its zero
 *  mean (Sec. 2).
 */
#ifndef HHG_H
#define HHG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- codes */
#define HHG_OK          0
#define HHG_EINVAL     -1   /* invalid argument, unsupported mesh or size */
#define HHG_ENOMEM     -2   /* bound workspace too small / host allocation failed */
#define HHG_ECUDA      -3   /* a CUDA runtime call failed */
#define HHG_EDIVERGED  -4   /* residual grew beyond the divergence guard or became NaN */
#define HHG_ETIMEOUT   -5   /* a bounded device-side wait gave up */
#define HHG_EREJECTED  -6   /* learned coarse correction rejected (internal) */
#define HHG_ESTATE     -7   /* call out of order (e.g. before hhg_problem_bind) */

#define HHG_P1P1_PSPG   1   /* stabilised equal order (Sec. 2, Eq. pspg) */
#define HHG_P2P1_TH     2   /* Taylor-Hood, C = 0 */

#define HHG_FP64        0
#define HHG_FP32        1

/* solve precision of a problem */
#define HHG_SOLVE_FP64  0   /* every level in double */
#define HHG_SOLVE_MIXED 1   /* FP32 V-cycles inside FP64 iterative refinement */

/* arithmetic of the mixed solve's refinement residual */
#define HHG_REFINE_FP64 0   /* FP64 rows, rounded to FP32 for the V-cycle          */
#define HHG_REFINE_DF32 1   /* double-float rows (two FP32 numbers per value)      */

/* operators for hhg_apply */
#define HHG_OP_FULL     0   /* y = calA x                                     */
#define HHG_OP_A        1   /* velocity rows: A u_c; pressure rows 0          */
#define HHG_OP_BT       2   /* velocity rows: B^T p                           */
#define HHG_OP_B        3   /* pressure rows: B u                             */
#define HHG_OP_C        4   /* pressure rows: C p                             */
#define HHG_OP_MASS     5   /* consistent mass, all rows incl. boundary       */

/* velocity smoother A_hat (Sec. 3.2) */
#define HHG_AHAT_F      0   /* forward Gauss-Seidel                  */
#define HHG_AHAT_S      1   /* forward + backward Gauss-Seidel       */

typedef struct hhg_mesh hhg_mesh;
typedef struct hhg_problem hhg_problem;
typedef struct hhg_batch hhg_batch;

typedef struct {
    int disc;            /* HHG_P1P1_PSPG or HHG_P2P1_TH                                  */
    int L;               /* finest level                                                  */
    int coarse_level;    /* level of the direct coarse solve (0 = Algorithm 1)            */
    int solve;           /* HHG_SOLVE_FP64 or HHG_SOLVE_MIXED                             */
    double nu_a;         /* viscosity nu = exp(nu_a * z); 0 gives nu = 1                  */
    int pspg_rhs;        /* 1: consistent PSPG load term in g (P1-P1 only)                */
    int error_level;     /* 1: also set up level L+1 for hhg_error_norms                   */
    int nn_hidden;       /* learned coarse correction: hidden width (0 = none)             */
    int nn_samples;      /* training pairs held in the workspace                           */
    int nn_batch;        /* training mini-batch                                            */
} hhg_problem_desc;

typedef struct {
    int level;
    int nx, ny, nz;            /* cells per direction, m * 2^level                          */
    int groups;                /* velocity DoF groups per component: 1 (P1) or 8 (P2)       */
    int sx;                    /* element pitch between j rows of one group array           */
    int64_t sy;                /* element pitch between k planes                            */
    int64_t array_elems;       /* elements of one group array (incl. one halo layer, padded)*/
    int64_t vector_elems;      /* elements of a block vector: (3 * groups + 1) * array_elems */
    int64_t n_velocity_nodes;  /* canonical velocity nodes per component                    */
    int64_t n_pressure_nodes;  /* canonical pressure nodes                                  */
    int64_t n_dofs;            /* 3 * n_velocity_nodes + n_pressure_nodes (incl. Dirichlet) */
    double h;                  /* mesh width of the level                                   */
} hhg_layout_info;

/* The FMG parameter tuple s = (nu_pre, nu_post, nu_inc, kappa, A_hat, xi) of
 * Algorithm 1 / Sec. 5.1 and the pressure relaxation parameter omega^{-1}
 * (S_hat = omega^{-1} M_L). */
typedef struct {
    int nu_pre, nu_post, nu_inc, kappa;
    int ahat;            /* HHG_AHAT_F or HHG_AHAT_S */
    int xi;              /* inner Gauss-Seidel sweeps of the velocity step */
    double omega_inv;
} hhg_params;

typedef struct {
    double wu_model;          /* W(FMG(s)) of the paper's cost model (Sec. 4.2)          */
    double wu_counted;        /* operator-apply equivalents actually executed            */
    double res_u, res_p;      /* final Euclidean residual norms on level L (FP64)        */
    int64_t kernel_launches;  /* kernels issued by the call                              */
} hhg_stats;

/* ------------------------------------------------------------------ errors */
/* Copies the last error message of the calling thread (NUL-terminated). */
int hhg_last_error(char* buf, size_t len);

/* ------------------------------------------------------------------ meshes */
/* Macro mesh T_0 (Sec. 2): nv vertices (xyz, row-major doubles), nt tetrahedra
 * (4 vertex ids each).  Must be a Kuhn-split box of cubes (see above);
 * otherwise HHG_EINVAL.  Arrays are read during the call only. */
int hhg_mesh_create(const double* verts, int nv, const int* tets, int nt, hhg_mesh** out);
/* Same mesh given by its box: mx x my x mz cubes of side H. */
int hhg_mesh_create_box(int mx, int my, int mz, double H, hhg_mesh** out);
int hhg_mesh_destroy(hhg_mesh* mesh);

/* ---------------------------------------------------------------- problems */
/* Level hierarchy coarse_level..L and its constant stencils (Sec. 2.1-2.2,
 * Table 2): element matrices of the 6 Kuhn classes are summed into per-group
 * stencils.  Host-only; no device memory is touched. */
int hhg_problem_create(const hhg_mesh* mesh, const hhg_problem_desc* desc, hhg_problem** out);
int hhg_problem_workspace_bytes(const hhg_problem* pb, size_t* bytes);
/* Binds a device workspace (>= hhg_problem_workspace_bytes, 256-byte aligned)
 * and the CUDA stream (cudaStream_t, 0 = legacy default stream); uploads the
 * stencil and transfer tables, assembles and inverts the bordered coarse
 * system.  Synchronises the stream. */
int hhg_problem_bind(hhg_problem* pb, void* workspace, size_t bytes, void* stream);
int hhg_problem_destroy(hhg_problem* pb);
int hhg_layout(const hhg_problem* pb, int level, hhg_layout_info* info);

/* Canonical host vector -> device layout (and back); halo and padding
 * entries are written as zeros.  Velocity Dirichlet entries are copied as
 * given.  The canonical data cross the bus in one copy (fast from pinned host
 * memory) and are scattered/gathered on the device, staged in the level's
 * scratch vector.  Synchronous (the host buffer may be reused on return).
 * FP32 device vectors need a problem created with HHG_SOLVE_MIXED. */
int hhg_vector_from_host(hhg_problem* pb, int level, int prec, const double* host, void* dev);
int hhg_vector_to_host(hhg_problem* pb, int level, int prec, const void* dev, double* host);

/* Right-hand side of level l (Sec. 2, below Eq. stokes-discrete):
 *   f = M f_h - A w_h (interior velocity rows), g = -B w_h (+ PSPG load),
 * g projected to sum zero.  f_nodal: forcing at the canonical velocity nodes
 * (3 x n_velocity_nodes, component-major); w_nodal: Dirichlet data at the same
 * nodes (only boundary entries are read).  Kept inside the workspace.  Both
 * arrays are copied as they are and placed by a device kernel; synchronous. */
int hhg_set_rhs(hhg_problem* pb, int level, const double* f_nodal, const double* w_nodal);
/* The same for levels l0 .. l1 (f_nodal[l - l0], w_nodal[l - l0] per level):
 * every level's copies and assembly are queued on the problem's stream and
 * the call waits once at the end (instead of once per level).  Synchronous.
 * Every level and pointer is checked before anything is queued: HHG_EINVAL
 * for an empty range, a level outside the hierarchy or a null pointer, and
 * then no level's right-hand side has changed.  If a CUDA call fails after
 * work was queued, the call waits for the queued work before it returns the
 * error (the host buffers are then free; the levels are in an undefined
 * state). */
int hhg_set_rhs_levels(hhg_problem* pb, int l0, int l1, const double* const* f_nodal, const double* const* w_nodal);
/* Device pointer of a library-owned FP64 level vector: 0 = rhs, 1 = boundary
 * lifting w_h, 2 = FMG solution x. */
int hhg_level_vector(hhg_problem* pb, int level, int which, void** dev);

/* ---------------------------------------------------------- hot-path steps */
/* y = Op x on level l (Eq. stokes-discrete blocks); Dirichlet velocity rows
 * of y are 0 except for HHG_OP_MASS.  For HHG_OP_FULL, x must be in lifting
 * form (Dirichlet velocity entries 0, as in every solver vector); the other
 * operators accept any x. */
int hhg_apply(hhg_problem* pb, int level, int op, int prec, const void* x, void* y);
/* r = b - calA x; if norms != NULL, norms[0] = ||r_u||_2, norms[1] = ||r_p||_2
 * (synchronises). */
int hhg_residual(hhg_problem* pb, int level, int prec, const void* x, const void* b, void* r, double* norms);
/* The defect of one refinement step of the mixed solve (HHG_SOLVE_MIXED, a
 * GPU execution choice outside the paper: FP32 V-cycles of Algorithm 1 on the
 * defect of the FP64 iterate), as
 * hhg_fmg_solve computes it: r = fl32(b - calA x) for the full operator of
 * `level`, x and b FP64 device vectors (x in lifting form, 16-byte aligned),
 * r an FP32 device vector.  With HHG_REFINE_DF32 (the default where it
 * applies) every row is a compensated dot product in double-float arithmetic
 * (Ogita, Rump and Oishi's Dot2 on x and the weights split into two FP32
 * numbers each; with a variable viscosity the row's segments scaled by their
 * FP64 factors exp(+-a h k) in the same arithmetic): |r - fl32(b - calA x)|
 * <= 2^-24 |b - calA x| + about (n^2 2^-48 + 2^-46) sum_j |a_ij x_j| for a
 * row of n terms.  With
 * HHG_REFINE_FP64 the rows are FP64 and rounded to FP32.  Overwrites the
 * level's internal FP32 iterate and FP64 scratch vector (x, b and r must not
 * be those).  HHG_EINVAL unless the problem was created with
 * HHG_SOLVE_MIXED. */
int hhg_refinement_residual(hhg_problem* pb, int level, const double* x, const double* b, float* r);
/* Arithmetic of the refinement residual (HHG_REFINE_FP64 or HHG_REFINE_DF32;
 * default HHG_REFINE_DF32, which covers both discretisations with constant
 * or variable viscosity).  Drops the problem's cached graphs when the choice
 * changes; a batch keeps the choice in effect when its graph was recorded.
 * The get call reports the arithmetic in effect. */
int hhg_set_refinement_residual(hhg_problem* pb, int kind);
int hhg_get_refinement_residual(hhg_problem* pb, int* kind);
/* `sweeps` inexact Uzawa iterations (Eq. uzawa-iteration) on x in place. */
int hhg_smooth(hhg_problem* pb, int level, const hhg_params* prm, int sweeps, int prec, void* x, const void* b);
/* r_coarse = I_l^{l-1} r_fine = (I_{l-1}^l)^T r_fine (Sec. 3.3), Dirichlet rows 0. */
int hhg_restrict(hhg_problem* pb, int level, int prec, const void* r_fine, void* r_coarse);
/* x_fine += I_{l-1}^l x_coarse (linear P1 / quadratic P2 interpolation). */
int hhg_prolongate_add(hhg_problem* pb, int level, int prec, const void* x_coarse, void* x_fine);
/* Direct solve on the coarse level, bordered by the mean-pressure constraint. */
int hhg_coarse_solve(hhg_problem* pb, int prec, const void* b, void* x);
/* One VAR-V-CYCLE(l, l, ...) of Algorithm 1 on x in place. */
int hhg_vcycle(hhg_problem* pb, int level, const hhg_params* prm, int prec, void* x, const void* b);
/* FMG of Algorithm 1 with the rhs set by hhg_set_rhs on every level.  Writes
 * the level-L FP64 solution (lifting form: Dirichlet rows 0, p mean zero) to
 * x_out (device, may be NULL to keep it only in the workspace).  stats may be
 * NULL; if given, residual norms are computed (synchronises). */
int hhg_fmg_solve(hhg_problem* pb, const hhg_params* prm, void* x_out, hhg_stats* stats);
/* Per-level autotuner of the launch shapes (threads per block and k planes
 * per thread of the stencil-row kernels, threads per block of the
 * Gauss-Seidel kernels, and the smoother's resident CTA count of
 * hhg_set_level_smoother): every candidate is timed `reps` times with CUDA
 * events on the problem's stream in the precision of the V-cycles, the
 * fastest is kept.  Uses only the library's scratch vectors; cached graphs
 * are dropped.  shapes_out (optional) receives 16 ints per level (coarse ..
 * L): row threads, row k planes, Gauss-Seidel threads (edge groups), resident CTAs,
 * resident threads per CTA, the threads per block of the streaming kernel
 * of the full operator (0 = the plain kernels), the row kernels' sites per
 * thread, the
 * lanes per Gauss-Seidel site of the edge groups and of the vertex colours
 * (tuned apart), and the threads, k planes and sites per thread of the
 * smoother's B^T rows and of its (B, -C) rows (tuned apart from the full
 * operator's), and the Gauss-Seidel threads of the vertex colours.
 * Synchronises. */
int hhg_autotune(hhg_problem* pb, int reps, int* shapes_out);
/* Not in the paper (GPU launch choices): the launch shape of the stencil
 * kernels of one level -- threads per block of the row kernels (64/128/256),
 * k planes per thread (1..64), threads per block of the Gauss-Seidel kernels
 * (64/128/256), and row_tile = 64, 128 or 256 (1 = 128) to evaluate the
 * rows of the full operator (apply, residual) and of the smoother's B^T and
 * (B, -C) residuals, in both precisions, by the streaming kernels with that
 * many threads per block (a block owns 4 x threads positions of the (i, j)
 * plane, stages the planes of its input arrays in shared memory as it marches
 * along k, and loads each line of a thread's stencil footprint once per
 * plane; the grid is one wave of blocks with equal runs of planes; only on
 * levels with nx >= 64, whose pitch sx is a multiple of four; four sites per
 * thread, or two for FP32 with row_sites = 2; 0 = the plain kernels), and
 * row_sites = 1 or 4 sites per thread of the
 * row kernels (4: each warp evaluates four runs of 32 consecutive
 * positions of the padded (i, j) plane, sharing each term's address
 * between the runs; row_tile != 0 takes precedence; sets the FP32
 * and FP64 rows, which hhg_autotune chooses separately), and gs_lanes = 1, 2
 * or 4 lanes per Gauss-Seidel site (the lanes take every gs_lanes-th term
 * of the site's rows and add their sums by shuffles; sets the vertex colours
 * and the edge groups, which hhg_autotune chooses apart; the B^T and
 * (B, -C) rows take this shape too until hhg_autotune gives them their own).  Results agree up to
 * rounding.  Drops cached graphs.  hhg_get_launch_shape writes the six
 * values to shape6 in the same order; its row_sites slot reads 2 when the
 * level's streaming rows (first velocity pass) take 2 sites per thread. */
int hhg_set_launch_shape(hhg_problem* pb, int level, int row_threads, int row_kplanes, int gs_threads, int row_tile,
                         int row_sites, int gs_lanes);
int hhg_get_launch_shape(hhg_problem* pb, int level, int* shape6);

/* Not in the paper (a GPU execution choice): the launch order of the
 * per-phase Gauss-Seidel kernels of `level` (levels whose smoother runs one
 * launch per phase).  order 0: every phase updates the three velocity
 * components; order 1: component by component -- all xi sweeps (forward, and
 * backward for A_s) of u_1, then of u_2, then of u_3, so that one component's
 * group arrays stay in L2 through its sweeps on levels whose vectors exceed
 * L2.  A = diag(A, A, A) (Eq. stokes-discrete) couples no two components, so
 * both orders give the same iterates.  hhg_autotune chooses it by timing;
 * default 0.  Drops cached graphs. */
int hhg_set_level_sweep_order(hhg_problem* pb, int level, int order);
int hhg_get_level_sweep_order(hhg_problem* pb, int level, int* order);

/* ------------------------------------------- learned coarse-grid correction */
/* Not in the paper: a small MLP  y = W3 relu(W2 relu(W1 x + b1) + b2) + b3
 * (hidden width nn_hidden) maps the coarse defect, restricted to the coarse
 * unknowns and scaled to unit norm, to the scaled coarse correction.  It is
 * trained on the GPU by the library's own forward/backward kernels and Adam
 * on pairs (r, Z r) whose targets come from the plain coarse solver Z.  In the
 * V-cycle it replaces the coarse solve only when its residual passes the gate
 * ||b - calA_c x_nn|| <= theta ||b||; otherwise the plain solve runs. */
typedef struct {
    int epochs, batch;
    double lr;
    int n_train;               /* pairs used (<= nn_samples; the rest validates) */
    uint64_t seed;             /* counter-based generator of the random defects */
    int recorded;              /* 1: the defects recorded by hhg_coarse_nn_record come first, random
                                  defects fill the remaining samples; 0: random defects only */
    double smooth_frac;        /* probability of a smooth defect (random low-wavenumber sine modes per
                                  field, like restricted V-cycle residuals); the rest uniform random */
} hhg_nn_cfg;

typedef struct {
    int n;                     /* coarse unknowns (network input/output width)  */
    int64_t n_params;
    double loss_first, loss_last;      /* mean squared error, training set      */
    double val_rel_err;        /* mean ||y - t|| / ||t|| on the validation pairs */
    double train_ms;
} hhg_nn_report;

/* network width n and parameter count of a problem created with nn_hidden > 0 */
int hhg_coarse_nn_size(const hhg_problem* pb, int* n, int64_t* n_params);
/* parameters, flat FP32 [W1 (h x n), b1, W2 (h x h), b2, W3 (n x h), b3],
 * row-major; host arrays */
int hhg_coarse_nn_set_params(hhg_problem* pb, const float* params);
int hhg_coarse_nn_get_params(hhg_problem* pb, float* params);
/* loss and gradients (same flat order) of the mean squared error over a batch
 * X, T (B x n, host, B <= nn_batch) at the current parameters */
int hhg_coarse_nn_grad(hhg_problem* pb, const float* X, const float* T, int B, double* loss, float* grads);
/* trains from the current parameters: nn_samples random unit defects (pressure
 * part with zero lumped-mass mean) from cfg->seed, targets by the plain
 * coarse solve; the last nn_samples - n_train pairs validate.  Synchronises. */
int hhg_coarse_nn_train(hhg_problem* pb, const hhg_nn_cfg* cfg, hhg_nn_report* report);
/* While on, every coarse solve appends its defect (restricted to the coarse
 * unknowns, scaled to unit norm) to the training samples, up to nn_samples
 * (turning it on restarts the count).  *recorded (optional) receives the
 * count.  Drops cached graphs. */
int hhg_coarse_nn_record(hhg_problem* pb, int on, int64_t* recorded);
/* mode 0: plain coarse solve; 1: learned correction gated by theta; 2: learned
 * correction always; 3: no coarse correction at all (2 and 3 are comparison
 * modes for measurements).  Drops cached graphs. */
int hhg_coarse_nn_enable(hhg_problem* pb, int mode, double theta);
/* accepted / rejected learned corrections since the last call (resets) */
int hhg_coarse_nn_counts(hhg_problem* pb, int64_t* accepted, int64_t* rejected);

/* ------------------------------------------------------------------ batches */
/* Not in the paper (many independent problems on one GPU; the paper's
 * ownership of work by primitives, Sec. 2.1, taken across problems).  A batch
 * of n independent problems (each bound, with its rhs set on every level; a
 * problem may belong to one batch at a time).  The handles are borrowed: the
 * problems must outlive the batch.  The batch owns n CUDA streams and
 * events, and (after the first solve) the device copies of the stencil
 * tables and the work-item lists of its merged launches.  Creating the batch
 * gives its problems common launch shapes, so that their kernels can share
 * launches: on each level, every problem of a discretisation takes the
 * launch shape of the one with the most DoFs there; the resident smoother
 * keeps each problem's CTA count and
 * takes the CTA size of the largest problem with that count.  Later
 * hhg_fmg_solve calls of the problems use these shapes too (hhg_autotune or
 * hhg_set_launch_shape change them again). */
int hhg_batch_create(hhg_problem* const* problems, int n, hhg_batch** out);
int hhg_batch_destroy(hhg_batch* batch);
/* FMG (Algorithm 1) of every problem of the batch, params[i] for problem i.
 * The first call (and every call with different parameters) records every
 * problem's kernel sequence without running it, then merges the sequences:
 * the next kernels of all problems that run the same kernel with the same
 * block shape become ONE launch over the flat list of (problem, block) work
 * items, each item with its own problem's arguments; each problem's own
 * order is kept, and the problems share no data, so every problem gets
 * exactly its individual hhg_fmg_solve result.  The problems form cohorts
 * (hhg_batch_set_grouping) whose sequences are merged; each cohort's merged
 * launches form one chain of a CUDA graph, and the cohorts run as parallel
 * branches.  Batches with a problem that uses the learned
 * coarse correction record one graph branch per problem instead.  The graph
 * is launched on `stream` (cudaStream_t, must not be the legacy default
 * stream).  Each problem's solution ends in its workspace
 * (hhg_level_vector(.., L, 2)).  *kernels (optional) receives the kernel
 * count of the graph.  Asynchronous. */
int hhg_batch_fmg_solve(hhg_batch* batch, const hhg_params* params, void* stream, int64_t* kernels);
/* after a solve: *launches = kernels of the batch graph, *problem_kernels =
 * the kernels of the problems' own sequences (their sum over the problems) */
int hhg_batch_launch_counts(const hhg_batch* batch, int64_t* launches, int64_t* problem_kernels);
/* How the batch's sequences are grouped (next solve; drops the cached graph).
 * 0: cohorts of problems whose kernel sequences are the same op for op
 * (discretisation, precision, coarse and finest level, viscosity model,
 * smoothing tuple, resident-smoother CTA counts per level) -- many short
 * chains side by side.  1: cohorts by discretisation, precision, coarse
 * level, viscosity model and smoothing tuple only, whatever the problems'
 * sizes -- fewer, longer chains and fewer launches; the merge aligns the
 * sequences as far as they agree.  2: no merging, one graph branch per
 * problem.  -1 (default): 0 if the cohorts of grouping 0 hold at least four
 * problems each on average, else 2.  HHG_EINVAL otherwise.
 * hhg_batch_get_grouping: the grouping of the current graph (-1 before the
 * first solve). */
int hhg_batch_set_grouping(hhg_batch* batch, int grouping);
int hhg_batch_get_grouping(const hhg_batch* batch, int* grouping);

/* One end-to-end solve from host data: the right-hand sides of every level
 * lc..L from nodal data in host memory (f_nodal[l - lc], w_nodal[l - lc] as
 * for hhg_set_rhs), FMG (Algorithm 1) with params, and the solution in
 * canonical order to x_host (3 n_v + n_p doubles, host; may be null).  The
 * same results as hhg_set_rhs_levels + hhg_fmg_solve + hhg_vector_to_host;
 * the finest level's right-hand side is assembled on a second stream while
 * the FMG stages below it run (when they replay as graphs; the stages then
 * run on an internal stream of the highest priority), so that its host
 * copies and assembly overlap them.  Host buffers in pinned memory let the
 * copies run asynchronously.  Synchronises before returning (the host
 * buffers may then be reused).  *stats optional as for hhg_fmg_solve. */
int hhg_fmg_solve_host(hhg_problem* pb, const hhg_params* params, const double* const* f_nodal,
                       const double* const* w_nodal, double* x_host, hhg_stats* stats);

/* Whether hhg_fmg_solve records its kernel sequence once per parameter tuple
 * as a CUDA graph and replays it (default on).  Graphs are used only when the
 * bound stream is a created stream (not the legacy default stream). */
int hhg_set_graph_mode(hhg_problem* pb, int on);
/* Whether the smoother of the levels that have a resident CTA count (see
 * hhg_set_level_smoother) runs all phases in one launch (default on) or one
 * launch per phase everywhere.  Both give the same iterates. */
int hhg_set_small_level_mode(hhg_problem* pb, int on);
/* Not in the paper (a GPU execution choice, Sec. 3.2's smoother unchanged):
 * the number of CTAs `ctas` (1..16, one thread-block cluster) of `threads`
 * threads (a multiple of 32 in 128..1024; 0 = 1024) that run all phases of
 * the Uzawa smoother of `level` in precision `prec` in one launch with the
 * level's block vector held in their shared memory (a slab of k planes per
 * CTA), or ctas = 0 for one launch per phase.  HHG_EINVAL if the level does
 * not fit (at most 225 KB of slab, residuals and tables per CTA, at least one
 * plane per CTA, the cluster must be schedulable).  Default at bind: the
 * fewest CTAs (<= 8) with at most 8192 lattice sites each, 1024 threads,
 * else 0; hhg_autotune times the choices.  Drops cached graphs.  The iterates
 * agree up to the rounding of the precision (the resident kernel adds the
 * terms of a row in another order). */
int hhg_set_level_smoother(hhg_problem* pb, int level, int prec, int ctas, int threads);
int hhg_get_level_smoother(hhg_problem* pb, int level, int prec, int* ctas, int* threads);
/* omega^{-1}: `iters` power iterations on M_L^{-1}(C + B A_s^{-1} B^T)
 * (Eq. omega-eigenvalue-problem) from the host start vector v0 (canonical
 * pressure order). */
int hhg_estimate_omega(hhg_problem* pb, int level, int iters, const double* v0, double* omega_inv);
/* ||e(x)||_2 of Eq. error: M-norm on level l+1 of x* - I x (x the lifting-form
 * FP64 solution on level l; the boundary values w_h are added), pressures with
 * zero mean.  u_exact / p_exact: exact nodal values on level l+1 (canonical).
 * Needs desc.error_level = 1 and l == L. */
int hhg_error_norms(hhg_problem* pb, int level, const void* x, const double* u_exact,
                    const double* p_exact, double* err_u, double* err_p);

/* ------------------------------------------------- allocation-free utility */
/* Euclidean norms of the two parts of a block vector x (device pointer,
 * element type `prec`): norms[0] = ||x[0 .. n_velocity)||_2 and norms[1] =
 * ||x[n_velocity .. n_velocity + n_pressure)||_2, written to `norms` (device
 * pointer to 2 doubles) on `stream` (cudaStream_t).  With x a residual from
 * hhg_residual and n_velocity = 3 * groups * array_elems, n_pressure =
 * array_elems (hhg_layout), these are the residual norms hhg_residual reports.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory (allocator or pool callbacks, hosts that own
 * every allocation).  It allocates nothing: its partial sums live in a
 * 16 KB __device__ array of the library that every GPU loading the library
 * holds until exit.  Each part may hold at most 2^31 - 1 elements (larger
 * sizes return HHG_EINVAL).  The first call on a device looks the array up
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  The looked-up address belongs to the device's
 * primary context: after a cudaDeviceReset (or anything else that replaces
 * that context) it is stale, and the process must not call this entry point
 * on that device again.  All calls share the array: calls that overlap
 * on the GPU (other streams, other threads) race and must be serialised by
 * the caller.  Every call writes all partial sums it reads, so nothing needs
 * clearing between calls. */
int hhg_block_norms_noalloc(const void* x, int prec, int64_t n_velocity, int64_t n_pressure, double* norms,
                            void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HHG_H */
