/* pk_oracle.h -- interface of the plain FP64 CPU oracle (test infrastructure only).
 *
 * Only the test-suite, the smoke check and the CPU-baseline leg of the benchmark load
 * this library. It shares no code with the CUDA library.
 */
#ifndef PK_ORACLE_H
#define PK_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ocsr ocsr;
typedef struct oproblem oproblem;

typedef struct {
    double theta;        /* strength threshold (Sec. 6.2), default 0.25 */
    int mode;            /* 0 additive B = S + Pi V Pi^T, 1 multiplicative (Alg. 2.1 + Remark 2.1),
                            2 plain AMG: one V-cycle of the AMG hierarchy of A_h itself */
    int smoother;        /* P_k smoother: 0 multicolour symmetric GS, 1 l1-Jacobi */
    int level_smoother;  /* AMG level smoother: 0 multicolour GS, 1 l1-Jacobi */
    int coarse_size;     /* stop coarsening at or below this many rows */
    int max_levels;      /* AMG levels including the coarsest (<= 25) */
    uint64_t seed;       /* seed of the colouring and PMIS hash streams */
    double tol;          /* relative residual target */
    int max_iter;
    int flexible;        /* 1: flexible CG beta */
    int krylov;          /* outer iteration: 0 CG (FCG when flexible), 1 FGMRES (Sec. 6.2) */
    int restart;         /* FGMRES restart length m */
    int interp_pmax;     /* interpolation truncation: at most this many weights per row (0: no limit) */
    int interp_trunc;    /* interpolation truncation: drop |w| < (interp_trunc / 1000) max|w| */
    int interp_cc;       /* 1: extended+i+cc (an F neighbour sharing a strong C point with i
                            adds no C points of its own); 0: extended+i */
} oopts;

/* problem construction */
oproblem *orc_problem_create(int64_t nv, const double *xyz, int64_t nt, const int32_t *tets,
                             int k, const double *kappa, int source, int dirichlet);
void orc_problem_free(oproblem *p);
void orc_problem_sizes(const oproblem *p, int64_t *out8);
const ocsr *orc_problem_matrix(const oproblem *p, int which); /* 0 A_h, 1 A_H, 2 Pi */
void orc_problem_rhs(const oproblem *p, double *b);
void orc_problem_dofs(const oproblem *p, int64_t *dof_all, double *dof_xyz);
void orc_problem_elem_dofs(const oproblem *p, int32_t *elem_dof);
int orc_set_kappa(oproblem *p, const double *kappa);
int orc_set_source_nodal(oproblem *p, const double *f_all);
void orc_problem_nodes(const oproblem *p, double *xyz_all);

/* CSR access */
void orc_csr_info(const ocsr *a, int64_t *out3);
void orc_csr_copy(const ocsr *a, int64_t *ptr, int32_t *col, double *val);
void orc_csr_free(ocsr *a);
ocsr *orc_csr_new(int64_t nrows, int64_t ncols, int64_t nnz, const int64_t *ptr,
                  const int32_t *col, const double *val);

/* reference element and quadrature */
int orc_nloc(int k);
void orc_ref_nodes(int k, int32_t *m4);
void orc_ref_tensor(int k, double *S);
void orc_basis_eval(int k, const double *lam4, double *phi);
int orc_gm_rule(int s, double *lam, double *w, int cap);
void orc_element_stiffness(int k, const double *x12, double kappa, double *K);

/* graph / AMG pieces on plain CSR */
int orc_colour_jp(int64_t n, const int64_t *ptr, const int32_t *col, uint64_t stream,
                  int32_t *colour);
void orc_strength(const ocsr *a, double theta, uint8_t *strong);
void orc_pmis(const ocsr *a, const uint8_t *strong, uint64_t stream, int8_t *cf);
ocsr *orc_truncate(const ocsr *p, double tf, int pmax);
ocsr *orc_extpi(const ocsr *a, const uint8_t *strong, const int8_t *cf, int cc);
ocsr *orc_transpose(const ocsr *a);
ocsr *orc_spgemm(const ocsr *a, const ocsr *b);
ocsr *orc_rap(const ocsr *a, const ocsr *p);
void orc_spmv(const ocsr *a, const double *x, double *y);
void orc_sgs(const ocsr *a, const int32_t *colour, int ncolour, const double *r, double *z);

/* setup + solve */
int orc_setup(oproblem *p, const oopts *o);
int orc_set_max_iter(oproblem *p, int max_iter);
int orc_levels(const oproblem *p);
const ocsr *orc_level_matrix(const oproblem *p, int l, int which); /* 0 A_l, 1 P_l */
void orc_level_info(const oproblem *p, int l, int64_t *out4);
void orc_level_cf(const oproblem *p, int l, int8_t *cf);
void orc_level_strong(const oproblem *p, int l, uint8_t *strong);
void orc_level_colour(const oproblem *p, int l, int32_t *colour);
void orc_fine_colour(const oproblem *p, int32_t *colour);
void orc_apply_prec(oproblem *p, const double *r, double *z);
void orc_vcycle(oproblem *p, const double *b, double *x);
void orc_smoother(oproblem *p, const double *r, double *z);
/* FGMRES(m) (Saad's flexible GMRES, right preconditioning by orc_apply_prec), classical
 * Gram-Schmidt applied twice per Arnoldi step; hist[k] = the least-squares residual
 * estimate after k inner steps (hist[0] = ||b - A x0||). Called by orc_solve when
 * krylov = 1. */
int orc_fgmres(oproblem *p, const double *b, double *x, double *hist, int hist_cap,
               int *iters_out, double *true_rel_out);
int orc_solve(oproblem *p, const double *b, double *x, double *hist, int hist_cap,
              int *iters_out, double *true_rel_out);
void orc_grad_kappa(const oproblem *p, const double *u, const double *lam, double *g);

/* Stokes, Taylor-Hood P_k - P_{k-1} (Sec. 5): u (degree k, Dirichlet), p (degree k-1,
 * created with dirichlet = 0) on the same mesh; M_p solved by mp_iters diagonal-PCG
 * steps inside the block upper-triangular preconditioner Q_t. */
typedef struct ostokes ostokes;
ostokes *orc_stokes_create(oproblem *u, oproblem *p, int mp_iters);
void orc_stokes_free(ostokes *s);
void orc_stokes_sizes(const ostokes *s, int64_t *out3); /* n_h, n_p, 3 n_h + n_p */
const ocsr *orc_stokes_matrix(const ostokes *s, int which); /* 0 B, 1 B^T, 2 M_p */
void orc_stokes_apply(ostokes *s, const double *x, double *y);
void orc_stokes_prec(ostokes *s, const double *r, double *z);
int orc_stokes_solve(ostokes *s, const double *b, double *x, int restart, double tol, int max_iter,
                     double *hist, int hist_cap, int *iters_out, double *true_rel_out);
double orc_l2_error_sine(const oproblem *p, const double *u);

#ifdef __cplusplus
}
#endif
#endif
