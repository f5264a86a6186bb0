/* pkasp.h -- C ABI of the GB300 library for auxiliary-space preconditioned conjugate
 * gradients on P_k Lagrange discretisations of -div(kappa grad u) = f on tetrahedral
 * meshes (Lee, Leng & Zhang, "A Scalable Auxiliary Space Preconditioner for High-Order
 * Finite Element Methods", 2012; Xu's auxiliary space preconditioner B = S_k + Pi B_1 Pi^T).
 *
 * Equations are cited by the paper's consecutive numbering: Eq. (1) the model problem,
 * Eq. (7) the linear system A_h u_h = f_h, Eq. (10) the transfer operators I_P = Pi and
 * I_R = Pi^T; Algorithm 2.1 the two-level method; Remark 2.1 the symmetric (pre- and
 * post-smoothed) form; Sec. 6.1-6.2 the AMG settings and the strength of connection.
 *
 * Conventions for every function:
 *   - Return value: PKASP_OK (0) or a positive error code; pkasp_last_error() then
 *     returns a message for the calling thread. No function aborts the process.
 *   - Ownership: the library owns every pkasp_problem and all device memory it
 *     allocates; pkasp_destroy frees both. The caller owns every array it passes in and
 *     keeps it alive for the duration of the call only (nothing is retained).
 *   - Pointers: arguments named *_host must be host memory; arguments named *_dev must
 *     be device memory of the current device; arguments without a suffix may be either
 *     (the library asks the CUDA driver which, and stages host data itself).
 *   - Streams: every call that launches work takes a cudaStream_t (NULL = legacy
 *     default stream). Calls return after enqueueing unless stated otherwise; calls that
 *     return sizes or statistics synchronise the stream.
 *   - Indices are 0-based. Dense vectors of several right-hand sides are row-major
 *     [n][ld] with column c at offset c (ld >= ncols).
 */
#ifndef PKASP_H
#define PKASP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; declared here so that callers need no CUDA headers. */
typedef struct CUstream_st *pkasp_stream_t;

typedef struct pkasp_problem pkasp_problem;

enum {
    PKASP_OK = 0,
    PKASP_EINVAL = 1,     /* bad argument (size, degree, option value, null pointer) */
    PKASP_EMESH = 2,      /* inverted or degenerate tetrahedron, bad vertex index */
    PKASP_ENOMEM = 3,     /* device or host allocation failed, or a size limit hit */
    PKASP_ENOTCONV = 4,   /* max_iter reached before the tolerance */
    PKASP_EBREAKDOWN = 5, /* p^T A p <= 0 or a zero diagonal: the system is not SPD */
    PKASP_ECUDA = 6,      /* a CUDA runtime call failed */
    PKASP_ESTATE = 7      /* call out of order (e.g. solve before setup) */
};

enum { PKASP_MODE_ADDITIVE = 0, PKASP_MODE_MULTIPLICATIVE = 1, PKASP_MODE_AMG = 2 };
enum { PKASP_SMOOTHER_SGS = 0, PKASP_SMOOTHER_L1JACOBI = 1 };
enum { PKASP_PREC_FP64 = 0, PKASP_PREC_FP32 = 1 };
enum { PKASP_KRYLOV_CG = 0, PKASP_KRYLOV_FGMRES = 1 };
enum { PKASP_SOURCE_NONE = 0, PKASP_SOURCE_SINE = 1, PKASP_SOURCE_NODAL = 2 };
enum { PKASP_MAX_LEVELS = 25, PKASP_MAX_COLS = 64 };

/* Solver options (pkasp_default_options fills the defaults given in brackets). */
typedef struct {
    double theta;         /* strength threshold of Sec. 6.2 [0.25] */
    int mode;             /* PKASP_MODE_*: additive z = S_k r + Pi V(Pi^T r) [additive];
                             multiplicative = Algorithm 2.1 with pre-smoothing (Remark 2.1);
                             AMG = one V-cycle of an AMG hierarchy built on A_h itself, the
                             comparison method of the paper (Sec. 1, Table 1, Sec. 6.2) */
    int smoother;         /* P_k smoother S_k: PKASP_SMOOTHER_* [SGS: one forward and one
                             backward multicolour Gauss-Seidel sweep, Remark 6.1] */
    int level_smoother;   /* AMG level smoother, PKASP_SMOOTHER_* [SGS] */
    int coarse_size;      /* stop coarsening at <= this many rows [256] */
    int max_levels;       /* AMG levels including the coarsest, <= 25 [25] */
    uint64_t seed;        /* seed of the colouring and PMIS hash streams [0] */
    double tol;           /* stop when ||r_k||_2 <= tol ||r_0||_2 [1e-8] */
    int max_iter;         /* [500] */
    int flexible;         /* 1: flexible CG beta (z_new, r_new - r_old)/(z_old, r_old);
                             forced on when precond_precision is FP32 [0] */
    int precond_precision;/* PKASP_PREC_FP64 or PKASP_PREC_FP32: arithmetic of S_k, Pi and
                             the whole AMG hierarchy; SpMV, dots, updates and the
                             convergence test stay FP64 [FP64] */
    int use_graph;        /* 1: each solve runs as one CUDA graph with a device-side
                             while loop; 0: eager launches, host checks every iteration [1] */
    int spmv_threads;     /* threads per row of the fine SpMV and smoother: 4, 8, 16 or
                             32; 0 = pick by mean row length [0] */
    int smoother_layout;  /* fine smoother layout (SGS): 0 = autotuned at setup [0];
                             1 = one launch per colour phase, CSR, lanes fitted per colour;
                             2 = per phase, SELL-32; 3 = per phase, CSR with 2 lanes per
                             row; 4, 8, 16 = per phase, CSR with that many lanes per row;
                             102, 104, 108, 116 = per phase, CSR with 2, 4, 8, 16 lanes and
                             two rows per lane group; 404, 408, 416 = per phase, CSR
                             with 4, 8, 16 lanes per row over a grid of the kernel's
                             resident blocks, each lane group striding over rows and
                             loading the next row's entries during the current row's
                             gathers; -4, -8, -16 = the whole
                             symmetric sweep in one cooperative launch with that many
                             lanes per row.
                             spmv_threads != 0 overrides it with its own lane count. */
    int krylov;           /* outer iteration: PKASP_KRYLOV_CG (CG; flexible CG with the FP32
                             preconditioner) or PKASP_KRYLOV_FGMRES (Saad's flexible GMRES with
                             right preconditioning, the outer method of Sec. 6.2; one
                             right-hand side per call) [CG] */
    int restart;          /* FGMRES restart length m, 1..256 [30] */
    int interp_pmax;      /* AMG interpolation truncation: keep at most this many weights
                             per row (0 = no limit) [0] */
    int interp_trunc;     /* AMG interpolation truncation: drop weights below
                             (interp_trunc / 1000) x the row's largest |w|, 0..999 [0];
                             with either, kept weights are scaled to the row's sum */
    int interp_cc;        /* 1: extended+i+cc interpolation, the form Sec. 1 and Sec. 6.1
                             name: a strong F neighbour k of i adds its strong C points to
                             i's interpolatory set only when k shares no strong C point
                             with i; 0: extended+i [0] */
    int l2_persist;       /* 1: with the FP64 preconditioner and the SGS smoother (additive
                             or multiplicative form), keep the fine smoother's vector
                             (8 n_h bytes) in the L2 persisting set-aside during its
                             colour phases: an access-policy window
                             (persisting hits, streaming misses) on every phase launch.
                             Applied when that vector is at least a quarter of L2 and
                             1.125x it fits the largest set-aside; setup then raises the
                             context's cudaLimitPersistingL2CacheSize to 1.125x the vector
                             if it is lower, and pkasp_destroy resets the persisting lines
                             and restores the limit it found. A cache hint only: results
                             are bitwise the same. 0: never [1] */
} pkasp_options;

/* Problem sizes after assembly and (for the AMG entries) after setup. */
typedef struct {
    int64_t n_h, n_H;       /* P_k and P1 unknowns (Dirichlet nodes removed) */
    int64_t nnz_h, nnz_H, nnz_pi;
    int64_t n_all;          /* all P_k nodes including the boundary */
    int64_t n_tets, n_verts;
    int k;
    int levels;             /* AMG levels (0 before setup) */
    int fine_colours;       /* colours of the A_h graph (0 before setup) */
    int coarse_rows;
    int64_t level_rows[PKASP_MAX_LEVELS];
    int64_t level_nnz[PKASP_MAX_LEVELS];
    int level_colours[PKASP_MAX_LEVELS];
    double op_complexity;   /* sum_l nnz(A_l) / nnz(A_0), A_0 = A_H (A_h in plain AMG
                               mode) (Sec. 6.2, Table 6) */
    double setup_ms, assemble_ms;
    int spmv_layout;        /* autotuned layout of the fine SpMV: 0 = SELL-32 (one thread
                               per row), t > 0 = CSR read by t lanes per row */
    int smoother_layout;    /* same for the fine smoother's colour phases; -1 = CSR with
                               lanes fitted per colour; 100 + t = t lanes, two rows per
                               lane group; 400 + t = t lanes, grid-stride over the resident
                               blocks; -t (t > 1) = the whole symmetric sweep in one
                               cooperative launch, t lanes per row */
    int block_width;        /* columns of the internal multi-RHS blocks (4, 8, 16, 32, 48
                               or 64) of the last solve with ncols > 1; 0 before one */
    int block_group;        /* columns per group of the multi-RHS fine smoother phases,
                               autotuned at the first solve of a width (0 before) */
    int block_lanes;        /* threads per row of those phases (autotuned with it) */
    int64_t l2_persist_bytes; /* bytes of the fine smoother's vector kept in the L2
                               persisting set-aside after setup (options.l2_persist);
                               0: none */
} pkasp_info;

/* Per-solve statistics, filled by pkasp_solve (which synchronises the stream). */
typedef struct {
    int ncols;                          /* columns solved */
    int iters[PKASP_MAX_COLS];          /* PCG iterations per column */
    int status[PKASP_MAX_COLS];         /* PKASP_OK, PKASP_ENOTCONV or PKASP_EBREAKDOWN */
    double true_rel[PKASP_MAX_COLS];    /* ||b - A x|| / ||b - A x0|| at exit */
    double *hist_host;                  /* optional caller buffer [hist_cap][ncols]:
                                           ||r_k||_2 after k iterations (k = 0..iters) */
    int hist_cap;
    int hist_len;                       /* rows written into hist_host */
    int restarts;                       /* true-residual restarts taken (0 or 1) */
    float solve_ms;                     /* device time of the solve (CUDA events) */
    int64_t kernel_launches;            /* kernels of this library run by the solve */
} pkasp_stats;

/* ------------------------------------------------------------------------------------
 * Construction
 * ---------------------------------------------------------------------------------- */

/* Fills *opt with the defaults listed in pkasp_options (the settings of Sec. 6.1-6.2
 * where the paper gives them: theta, one pre- and one post-smoothing sweep). */
void pkasp_default_options(pkasp_options *opt);

/* Message of the last failed call on this thread (always NUL-terminated); library
 * plumbing with no counterpart in the paper. */
int pkasp_last_error(char *buf, size_t n);

/* Builds the P_k problem of Eq. (7) on a conforming tetrahedral mesh: the model problem
 * -div(kappa grad u) = f of Eq. (1) (Sec. 2) in the Lagrange space V_h.
 *   xyz_host   [nv][3] vertex coordinates
 *   tets_host  [nt][4] vertex indices, positively oriented (det > 0)
 *   k          polynomial degree, 1..4 (the paper's V_h = P^{k,0}, Sec. 2)
 *   kappa      [nt] piecewise-constant coefficient, > 0 (host or device)
 *   source     the load f_i = <f, phi_i> of Eq. (7), by a degree 2k+3 Grundmann-Moeller
 *              rule on every element:
 *              PKASP_SOURCE_SINE: f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z);
 *              PKASP_SOURCE_NODAL: the caller's f, given by f_nodal;
 *              PKASP_SOURCE_NONE: zero load (the caller passes its own b to solve).
 *   f_nodal    PKASP_SOURCE_NODAL only (else NULL): [n_all] values of f at every P_k node,
 *              boundary nodes included, in the node numbering below (host or device;
 *              pkasp_nodes_host gives n_all and the node coordinates before assembly).
 *              f is taken as its nodal interpolant f_h = sum_n f_n phi_n, so the load is
 *              b = M f_nodal exactly up to rounding (M the P_k mass matrix; the rule is
 *              exact for f_h phi_i). The library keeps a copy (pkasp_set_kappa reuses it).
 * Dirichlet nodes (those on faces with one adjacent element) are removed (Eq. 1,
 * u = 0 on the boundary). The node numbering is: vertices, then edges sorted by vertex
 * pair (nodes from the lower vertex), then faces sorted by vertex triple (nodes in
 * ascending multi-index order), then element interiors; unknowns keep that order.
 * Assembles A_h (Eq. 7), the P1 matrix A_H of the same mesh and Pi = I_P (Eq. 10) on
 * the device. Errors: EINVAL (sizes, degree, source, f_nodal given without
 * PKASP_SOURCE_NODAL or missing with it), EMESH (det <= 0, index out of range), ENOMEM,
 * ECUDA. On success *out owns everything; release it with pkasp_destroy. */
int pkasp_assemble(const double *xyz_host, int64_t nv, const int32_t *tets_host, int64_t nt,
                   int k, const double *kappa, int source, const double *f_nodal,
                   pkasp_problem **out);

/* Sizes and setup statistics (host struct): n_h = dim V_h with the Dirichlet nodes
 * removed (Sec. 2), n_H = dim of the P1 space V_H, the AMG levels of B_1 (Sec. 6.1) and
 * the operator complexity of Sec. 6.2 / Table 6. No GPU work. */
int pkasp_problem_info(const pkasp_problem *p, pkasp_info *info);

/* Numbering of the unknowns (the nodes x_i^h of V_h, Sec. 2): dof_all_host[n_h] = index
 * among all P_k nodes (the convention of pkasp_assemble) and dof_xyz_host[n_h][3] = node
 * coordinates. Either may be NULL. Host copies; no GPU work. */
int pkasp_get_dofmap(const pkasp_problem *p, int64_t *dof_all_host, double *dof_xyz_host);

/* Copies the assembled load vector f_h (Eq. 7) into b[n_h] (host or device).
 * Synchronises the stream. */
int pkasp_get_rhs(const pkasp_problem *p, double *b, pkasp_stream_t stream);

/* Replaces the coefficient kappa of Eq. (1) [nt] (host or device, > 0) and re-assembles
 * A_h, A_H (Eq. 7) and f_h on the same sparsity pattern, with the source given to
 * pkasp_assemble. Invalidates the setup (call pkasp_setup again). Synchronises. */
int pkasp_set_kappa(pkasp_problem *p, const double *kappa, pkasp_stream_t stream);

/* Builds the preconditioner on the device: Jones-Plassmann colouring of A_h, strength
 * graph (Sec. 6.2), PMIS C/F splitting, extended+i interpolation, Galerkin RAP per level
 * (the relation A_H = I_R A_h I_P of Sec. 2 applied recursively), colourings of every
 * level, the coarsest inverse, and FP32 copies when requested. Synchronises the stream.
 * Errors: EINVAL (options), ENOMEM (coarsest level above 8192 rows), EBREAKDOWN
 * (coarsest matrix not positive definite), ECUDA. */
int pkasp_setup(pkasp_problem *p, const pkasp_options *opt, pkasp_stream_t stream);

/* ------------------------------------------------------------------------------------
 * Solve
 * ---------------------------------------------------------------------------------- */

/* Preconditioned CG on A_h x = b (Eq. 7) with the auxiliary-space preconditioner
 * B = S_k + Pi B_1 Pi^T of Sec. 2 (or the form chosen at setup), for ncols right-hand
 * sides (1..64), columns independent (each converges, stops and is reported on its
 * own). With the FP32 preconditioner the outer iteration is flexible CG. b and x are
 * [n_h][ld] (host or device); x holds the initial guess on entry and the solution on
 * exit. Stops when ||r_k|| <= tol ||r_0|| per column, then checks the true residual and
 * restarts once if it is above tol. Fills *st (may be NULL) and synchronises the stream.
 * Returns PKASP_OK when every column converged, else ENOTCONV or EBREAKDOWN (the
 * per-column status is in *st), or EINVAL/ESTATE/ECUDA. */
int pkasp_solve(pkasp_problem *p, const double *b, double *x, int ncols, int64_t ld,
                pkasp_stats *st, pkasp_stream_t stream);

/* pkasp_solve from the initial guess x0 = 0: x is written, never read (a host x is not
 * uploaded; its columns are zeroed on the device), so a caller that starts from zero
 * moves only b to the device. Same conventions and results as pkasp_solve with a zero x. */
int pkasp_solve_from_zero(pkasp_problem *p, const double *b, double *x, int ncols, int64_t ld,
                          pkasp_stats *st, pkasp_stream_t stream);

/* Adjoint solve A_h^T lambda = g for the gradient of a loss L(u) of the solution of
 * Eq. (7) (g = dL/du; the paper has no adjoint, this is the discrete adjoint of its
 * system). A_h is symmetric, so this is the same operator and preconditioner: lambda
 * holds the initial guess on entry. Same conventions and errors as pkasp_solve. */
int pkasp_solve_adjoint(pkasp_problem *p, const double *g, double *lambda, int ncols,
                        int64_t ld, pkasp_stats *st, pkasp_stream_t stream);

/* Element-wise gradient dL/dkappa_e = -sum_c lambda_{c,e}^T Khat_e u_{c,e}, Khat_e the
 * element matrix of Eq. (7) with kappa_e = 1 (A_h is linear in kappa_e), summed on the
 * device over the ncols (1..64) columns of u and lambda ([n_h][ld] device arrays, column
 * c at offset c, ld >= ncols): the gradient of a loss over a block of solves with one
 * kappa. dkappa_dev [nt] (device) is overwritten. Enqueued on stream. Errors: EINVAL. */
int pkasp_grad_kappa(const pkasp_problem *p, const double *u_dev, const double *lambda_dev,
                     int ncols, int64_t ld, double *dkappa_dev, pkasp_stream_t stream);

/* Frees the problem and all its device memory (synchronises the device first). NULL
 * is accepted. */
int pkasp_destroy(pkasp_problem *p);

/* ------------------------------------------------------------------------------------
 * Operator access (for checks against an independent implementation and for tools).
 * All vectors are device memory of n_h (or n_H) entries.
 * ---------------------------------------------------------------------------------- */

/* y = A_h x (Eq. 7). Enqueued on stream. */
int pkasp_spmv(const pkasp_problem *p, const double *x_dev, double *y_dev, pkasp_stream_t stream);

/* z = B r with the preconditioner of the last pkasp_setup: additive B = S_k + Pi B_1
 * Pi^T (Sec. 2), multiplicative (Algorithm 2.1 with Remark 2.1) or plain AMG on A_h
 * (Sec. 6.2), in FP64 or FP32 arithmetic. Enqueued on stream; ESTATE before setup. */
int pkasp_apply_prec(pkasp_problem *p, const double *r_dev, double *z_dev, pkasp_stream_t stream);

/* z = S_k r from a zero guess: the P_k smoother of Sec. 2 alone (one forward and one
 * backward multicolour Gauss-Seidel sweep, Remark 6.1, or l1-Jacobi). Enqueued. */
int pkasp_apply_smoother(pkasp_problem *p, const double *r_dev, double *z_dev,
                         pkasp_stream_t stream);

/* x = V(b): one AMG V(1,1)-cycle on A_H, the B_1 of Sec. 2 built as in Sec. 6.1
 * (b, x of n_H entries). Enqueued on stream. */
int pkasp_apply_vcycle(pkasp_problem *p, const double *b_dev, double *x_dev,
                       pkasp_stream_t stream);

/* Copies matrix `which` to host CSR arrays (any may be NULL); *nnz_out (may be NULL)
 * receives the entry count. which: 0 A_h (Eq. 7), 1 A_H, 2 Pi (Eq. 10), 3 + 2l AMG
 * level l matrix A_l (Galerkin, Sec. 2 and 6.1),
 * 4 + 2l the interpolation P_l of level l; after pkasp_stokes_setup -1 B, -2 B^T,
 * -3 M_p. Synchronises. ptr is [rows+1]. */
int pkasp_get_matrix(const pkasp_problem *p, int which, int64_t *rows_out, int64_t *cols_out,
                     int64_t *nnz_out, int64_t *ptr_host, int32_t *col_host, double *val_host);

/* ------------------------------------------------------------------------------------
 * Stokes, Taylor-Hood P_k - P_{k-1} (Sec. 5), on the problem's mesh with k >= 2:
 *   F = [A B^T; B 0], A = three copies of A_h (velocity unknowns component-major: entry
 *   c n_h + j is component c of unknown j), B = -div_h with B_{q,(c,j)} = -int psi_q
 *   d_c phi_j, pressure psi_q on every P_{k-1} node of the mesh (node numbering of the
 *   DOF map of degree k-1 without Dirichlet removal; unknowns after the velocity, so a
 *   vector has n = 3 n_h + n_p entries). The preconditioner is the block upper-triangular
 *   Q_t = [A B^T; 0 -S]^{-1} of Eq. (5.4): z_p = -M_p^{-1} r_p by mp_iters steps of CG
 *   with the diagonal of the pressure mass matrix M_p (from zero), then
 *   z_u = B_aux (r_u - B^T z_p) with the problem's auxiliary-space preconditioner per
 *   component. F is singular in the constant pressure; right-hand sides with b_p = 0 are
 *   consistent and the pressure is determined up to a constant.
 * ---------------------------------------------------------------------------------- */

/* Assembles B, B^T and M_p (host, from the mesh; setup work) and allocates the solver.
 * Needs pkasp_setup first (its preconditioner approximates A^{-1}); a later pkasp_setup
 * discards the Stokes data (call this again). Errors: EINVAL (k < 2, mp_iters outside
 * 1..1000), ESTATE, ENOMEM, ECUDA. Synchronises. */
int pkasp_stokes_setup(pkasp_problem *p, int mp_iters, pkasp_stream_t stream);

/* sizes_out[5] = { n_h, n_p, n = 3 n_h + n_p, nnz(B), nnz(M_p) }. */
int pkasp_stokes_sizes(const pkasp_problem *p, int64_t *sizes_out);

/* y = F x and z = Q_t r for device vectors of n entries (enqueued on stream). */
int pkasp_stokes_apply(pkasp_problem *p, const double *x_dev, double *y_dev, pkasp_stream_t stream);
int pkasp_stokes_apply_prec(pkasp_problem *p, const double *r_dev, double *z_dev, pkasp_stream_t stream);

/* FGMRES(options.restart) with Q_t on F x = b (device vectors of n entries; x holds the
 * initial guess), to ||b - F x|| <= tol ||b - F x0|| (options.tol, max_iter), one CUDA
 * graph per solve when use_graph. Fills *st (may be NULL; one column) and synchronises.
 * Returns OK or ENOTCONV (or EINVAL / ESTATE / ECUDA). */
int pkasp_stokes_solve(pkasp_problem *p, const double *b_dev, double *x_dev, pkasp_stats *st,
                       pkasp_stream_t stream);

/* Colouring (colour per row) of A_h (level = -1) or of AMG level l: the multicolour
 * order of the Gauss-Seidel smoothers that replace the hybrid GS of Sec. 6.1; returns
 * the count in *ncolours (may be NULL). Host output; synchronises. */
int pkasp_get_colours(const pkasp_problem *p, int level, int32_t *colour_host, int *ncolours);

/* C/F splitting (+1 C, -1 F; PMIS, Sec. 6.1) and strength flags (Sec. 6.2; one byte
 * per entry of A_l) of AMG level l (not the coarsest). Either may be NULL. Host output;
 * synchronises. */
int pkasp_get_splitting(const pkasp_problem *p, int level, int8_t *cf_host, uint8_t *strong_host);

/* PMIS on a caller-supplied strength graph (De Sterck, Yang & Heys 2006, cited in Sec. 1
 * and 6.1): CSR pattern ptr_dev[n+1], col_dev[nnz] of a structurally symmetric matrix
 * with strong_dev[nnz] flags (1: column j is a strong connection of row i), hash stream
 * `stream_id`; writes cf_dev[n] (+1 C, -1 F). Runs entirely on the device. */
int pkasp_pmis(int64_t n, const int64_t *ptr_dev, const int32_t *col_dev,
               const uint8_t *strong_dev, uint64_t stream_id, int8_t *cf_dev,
               pkasp_stream_t stream);

/* Same splitting as pkasp_pmis, for callers that cannot let a library allocate device
 * memory: processes that hand the whole GPU memory to their own pool at start-up, and
 * code that must not synchronize the device (cudaMalloc and cudaFree do). The paper has
 * no counterpart; this is a deployment variant of pkasp_pmis. It allocates nothing: its
 * scratch is one fixed device array of about 17 MB inside the library, held by every GPU
 * that loads the library until the process exits, and it accepts at most
 * PKASP_NOALLOC_MAX_ROWS rows and PKASP_NOALLOC_MAX_NNZ entries (larger inputs return
 * PKASP_EINVAL before any kernel runs; so do row pointers that do not start at 0 or that
 * decrease, columns outside [0, n), and patterns that are not structurally symmetric
 * with ascending columns). Each call looks up that array's device address on the current
 * device (cudaGetSymbolAddress). Every call shares the one array: calls that overlap on
 * the GPU (from several streams or threads) race and must be serialized by the caller.
 * The output cf_dev[n] is bit-identical to pkasp_pmis for the same inputs (both use the
 * same per-row rules). It synchronizes the stream after every PMIS round (the host reads
 * the count of undecided rows), so it cannot be captured into a CUDA graph. */
enum { PKASP_NOALLOC_MAX_ROWS = 262144, PKASP_NOALLOC_MAX_NNZ = 4194304 };
int pkasp_pmis_noalloc(int64_t n, const int64_t *ptr_dev, const int32_t *col_dev,
                       const uint8_t *strong_dev, uint64_t stream_id, int8_t *cf_dev,
                       pkasp_stream_t stream);

/* ------------------------------------------------------------------------------------
 * Host-only helpers (no GPU needed): the numbering and sparsity patterns that
 * pkasp_assemble builds, for checks and tools.
 * ---------------------------------------------------------------------------------- */

/* Sizes of the DOF map of a mesh (the nodes of V_h, Sec. 2; same arguments and
 * conventions as pkasp_assemble):
 * sizes_out[6] = {n_all, n_h, n_H, nnz(A_h), nnz(A_H), nnz(Pi)}. If the output arrays
 * are non-NULL they are filled: dof_all_host[n_h], elem_dof_host[nt][nloc] (unknown index
 * or -1 per local node, nloc = (k+1)(k+2)(k+3)/6, local nodes = multi-indices m of |m| =
 * k in ascending lexicographic order), ah_ptr_host[n_h+1] / ah_col_host[nnz(A_h)] (the
 * pattern of A_h), pi_ptr_host[n_h+1] / pi_col_host / pi_val_host (I_P of Eq. 10).
 * Call once with NULL arrays to learn the sizes. Errors: EINVAL, EMESH. */
int pkasp_dofmap_host(const double *xyz_host, int64_t nv, const int32_t *tets_host, int64_t nt, int k,
                      int64_t *sizes_out, int64_t *dof_all_host, int32_t *elem_dof_host,
                      int64_t *ah_ptr_host, int32_t *ah_col_host, int64_t *pi_ptr_host,
                      int32_t *pi_col_host, double *pi_val_host);

/* Coordinates of every P_k node of a mesh (same arguments and conventions as
 * pkasp_assemble; Sec. 2): *n_all_out = number of nodes, boundary included; if
 * node_xyz_host is non-NULL it receives [n_all][3] coordinates x = sum_a m_a v_a / k in
 * the node numbering of pkasp_assemble, the order of f_nodal. Host only. Errors:
 * EINVAL, EMESH. */
int pkasp_nodes_host(const double *xyz_host, int64_t nv, const int32_t *tets_host, int64_t nt, int k,
                     int64_t *n_all_out, double *node_xyz_host);

/* The Taylor-Hood P_k - P_{k-1} blocks of Sec. 5 on the host, as pkasp_stokes_setup
 * assembles them (k = 2..4; mesh arguments as pkasp_assemble): sizes_out[4] = {n_h, n_p,
 * nnz(B), nnz(M_p)}. B = -div_h is n_p x 3 n_h (rows: every P_{k-1} node; columns: the
 * velocity unknowns component-major, c n_h + j), M_p the n_p x n_p pressure mass matrix;
 * rows in CSR with ascending columns. Non-NULL arrays are filled: b_ptr[n_p+1],
 * b_col/b_val[nnz(B)], m_ptr[n_p+1], m_col/m_val[nnz(M_p)]. Call once with NULL arrays
 * to learn the sizes. Errors: EINVAL, EMESH. */
int pkasp_stokes_blocks_host(const double *xyz_host, int64_t nv, const int32_t *tets_host, int64_t nt, int k,
                             int64_t *sizes_out, int64_t *b_ptr, int32_t *b_col, double *b_val,
                             int64_t *m_ptr, int32_t *m_col, double *m_val);

/* Reference tensors S[a][b][m][n] = (1/|T|) int_T (d phi_m/d lambda_a)(d phi_n/d lambda_b)
 * of the degree-k Lagrange basis (S_out has 16 nloc^2 entries): the element matrix of
 * Eq. (7) is kappa |T| sum_ab (grad lambda_a . grad lambda_b) S[a][b]. Host only. */
int pkasp_reference_tensors(int k, double *S_out);

/* Measurement aid with no counterpart in the paper: average device time (ms, CUDA
 * events on `stream`) of `reps` back-to-back launches of one hot-path kernel of the
 * current setup: which = 0 fine SpMV, 1 fine smoother
 * (all colour phases of one S_k application), 2 V-cycle, 3 whole preconditioner; on the
 * multi-RHS blocks of the last solve with ncols > 1 (ESTATE before one): 4 blocked SpMM
 * Q = A_h P with its per-column dot (P, Q), 5 blocked fine smoother, 6 blocked
 * preconditioner. The blocked timings overwrite the solve's work blocks and scalars.
 * which = 7: the fine smoother's loads without its colour dependencies (every row of the
 * colour split at once, lower parts then upper parts, the smoother's lanes per row):
 * the memory work of one S_k application with no barrier between colour phases.
 * which = 8: a gather-rate probe, random 8-byte gathers from an n_h vector driven by a
 * streamed index array of min(64M, 8 n_h) entries (scratch allocated for the call);
 * *ms_out then receives NANOSECONDS PER GATHER, the inverse of the GPU's random gather
 * rate from a vector of the size the smoother gathers from. */
int pkasp_time_kernel(pkasp_problem *p, int which, int reps, float *ms_out,
                      pkasp_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* PKASP_H */
