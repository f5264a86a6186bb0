// internal.h -- data structures shared by the translation units of libpkasp.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "pkasp.h"

namespace pk {

// ---------------------------------------------------------------------------------
// Errors: every internal failure throws pk::Error; the C ABI layer converts it into a
// status code and a per-thread message.
// ---------------------------------------------------------------------------------
struct Error {
    int code;
    std::string msg;
};

[[noreturn]] void fail(int code, const std::string &msg);
void cuda_check(cudaError_t e, const char *what, const char *file, int line);
#define PK_CUDA(x) ::pk::cuda_check((x), #x, __FILE__, __LINE__)
// every kernel launch of the library is followed by PK_LAUNCH(), which also counts it
void launched(const char *file, int line);
long long launch_count();
#define PK_LAUNCH() ::pk::launched(__FILE__, __LINE__)

// Device allocation tracked by the owning problem (freed in one place).
struct DevPool {
    std::vector<void *> blocks;
    size_t bytes = 0;
    void *alloc(size_t n);
    void free_all();
    template <class T>
    T *get(size_t count) {
        return static_cast<T *>(alloc(count * sizeof(T)));
    }
};

// CSR matrix in device memory: int64 row pointers, int32 columns (sorted per row).
struct DCSR {
    int64_t n = 0, m = 0, nnz = 0;
    int64_t *ptr = nullptr;
    int32_t *col = nullptr;
    double *val = nullptr;
    float *val32 = nullptr;  // FP32 copy for the mixed-precision preconditioner
};

// I_P with its values as codes. Every entry of I_P is a nodal value m / k (m = 1..k) of
// a P1 basis function at a Lagrange node (Eq. 10), so an entry needs its column and one
// byte: the PCG iteration's prolongation reads a 4-wide row layout (no row pointers) and
// the restriction I_P^T r reads one-byte codes instead of values. Built at assembly.
struct PiCodes {
    int32_t *ell_col = nullptr;    // [n_h][4] columns of the rows of I_P, -1 past a row's end
    uint32_t *ell_code = nullptr;  // [n_h] byte q = code m of entry q of the row (0 past its end)
    uint8_t *t_code = nullptr;     // [nnz] codes of I_P^T, in its CSR order
    double *tab = nullptr;         // [8] tab[m] = m / k (tab[0] = 0)
    float *tab32 = nullptr;        // [8] (float) tab[m]
};

// Host CSR (setup and tests).
struct HCSR {
    int64_t n = 0, m = 0;
    std::vector<int64_t> ptr;
    std::vector<int32_t> col;
    std::vector<double> val;
};

// Rows of a matrix sorted by colour, each split into entries of lower colour (L),
// higher colour (U) and the diagonal. Position p (0..n-1) in colour order holds row
// perm[p]; colour c owns positions off[c]..off[c+1]-1.
struct DSplit {
    int ncol = 0;
    std::vector<int64_t> off;  // host copy of the colour offsets
    int32_t *colour = nullptr; // colour of each row (natural order)
    int32_t *perm = nullptr;
    int64_t *lptr = nullptr, *uptr = nullptr;
    int32_t *lcol = nullptr, *ucol = nullptr;
    double *lval = nullptr, *uval = nullptr, *diag = nullptr;
    double *dinv = nullptr;  // 1 / diag: GB300 runs FP64 at ~2 DFMA per clock per SM, so
    float *dinv32 = nullptr; // the smoother multiplies instead of dividing
    float *lval32 = nullptr, *uval32 = nullptr, *diag32 = nullptr;
    int64_t nnz_l = 0, nnz_u = 0;
    std::vector<int> lmax, umax;  // per colour: longest lower / upper part (host)
    std::vector<int> l90, u90;    // per colour: 90th percentile of those lengths (host)
};

// SELL-32: slices of 32 rows (one thread per row), entries column-major within a slice
// (entry k of slice row r at sptr[slice] + 32 k + r), padded with column -1. perm maps
// a padded position to its row (natural order when null; -1 marks padding rows); coff
// gives each colour's slice range when the rows are colour-sorted.
struct DSell {
    int64_t nslices = 0, npos = 0, nnz_padded = 0;
    int32_t *perm = nullptr;
    int64_t *sptr = nullptr;
    int32_t *swidth = nullptr;
    int32_t *col = nullptr;
    double *val = nullptr;
    float *val32 = nullptr;
    double *diag = nullptr;    // colour split only: the INVERSE diagonal of each position
    float *diag32 = nullptr;
    std::vector<int64_t> coff;
};

struct Level {
    DCSR A;        // level matrix
    DSplit sp;     // colour split of A
    DCSR P, R;     // interpolation to the next level and its transpose
    double *l1 = nullptr;  // row 1-norms
    float *l132 = nullptr;
    int8_t *cf = nullptr;        // C/F splitting (not on the coarsest)
    uint8_t *strong = nullptr;   // strength flags per entry (not on the coarsest)
    // work vectors (FP64 and FP32)
    double *b = nullptr, *x = nullptr, *r = nullptr;
    float *b32 = nullptr, *x32 = nullptr, *r32 = nullptr;
};

struct GmresState;  // gmres.cuh
struct StokesWork;  // stokes.cu

// Scalars of one PCG run (device), per column.
struct PcgState {
    double rho[PKASP_MAX_COLS];
    double alpha[PKASP_MAX_COLS];
    double beta[PKASP_MAX_COLS];
    double rnorm[PKASP_MAX_COLS];
    double r0[PKASP_MAX_COLS];
    int iter[PKASP_MAX_COLS];
    int done[PKASP_MAX_COLS];
    int status[PKASP_MAX_COLS];
    double tnorm[PKASP_MAX_COLS];
    int all_done;
    int ncols;
    int maxit;
    int hist_cap;
    int loops;
    double tol;
};

}  // namespace pk

// ---------------------------------------------------------------------------------
// The problem handle.
// ---------------------------------------------------------------------------------
struct pkasp_problem {
    pk::DevPool pool;       // assembly-lifetime memory
    pk::DevPool setup_pool; // freed and rebuilt by every pkasp_setup
    int device = 0;
    int k = 0, nloc = 0;
    int64_t nv = 0, nt = 0, n_all = 0, nh = 0, nH = 0;
    int source = 0;
    // host copies of the mesh and the DOF map
    std::vector<double> xyz;
    std::vector<int32_t> tets;
    std::vector<int64_t> dof_all;   // [nh]
    std::vector<double> dof_xyz;    // [nh*3]
    std::vector<int32_t> elem_dof;  // [nt*nloc] unknown index or -1
    std::vector<int32_t> elem_vdof; // [nt*4]
    // device mesh data
    double *d_xyz = nullptr, *d_kappa = nullptr;
    int32_t *d_tets = nullptr, *d_elem_dof = nullptr, *d_elem_vdof = nullptr;
    double *d_gfac = nullptr;  // [nt][17]: kappa|T| G_ab (16) and |T|
    double *d_S = nullptr;     // reference tensors [16][nloc][nloc]
    double *d_phiq = nullptr, *d_lamq = nullptr, *d_wq = nullptr;  // load quadrature
    double *d_fall = nullptr;        // PKASP_SOURCE_NODAL: f at every P_k node [n_all]
    int32_t *d_elem_all = nullptr;   // PKASP_SOURCE_NODAL: all-node index [nt*nloc]
    int nq = 0;
    // incidence unknown -> (tet, local) in ascending tet order
    int64_t *d_inc_ptr = nullptr, *d_vinc_ptr = nullptr;
    int32_t *d_inc = nullptr, *d_vinc = nullptr;  // packed tet*64 + local
    // operators
    pk::DCSR Ah, AH, Pi, PiT;
    pk::PiCodes pic;  // I_P and I_P^T with coded values (iteration transfers)
    // L2 persisting window of the fine smoother's vector (options.l2_persist)
    size_t l2_win_bytes = 0;    // window size used by the colour phases (0: none)
    bool l2_raised = false;     // this problem raised the context's persisting limit
    size_t l2_prev_limit = 0;   // the limit found before raising it
    size_t l2_set_limit = 0;    // the limit this problem set
    double *d_b = nullptr;
    double assemble_ms = 0, setup_ms = 0;
    // setup
    bool have_setup = false;
    pkasp_options opt{};
    pk::DSplit fine;      // colour split of A_h
    pk::DSell Asell;      // SELL-32 copy of A_h (natural order)
    pk::DSell fsl, fsu;   // SELL-32 colour-sorted lower / upper parts of A_h
    double *d_l1h = nullptr;
    float *d_l1h32 = nullptr;
    std::vector<pk::Level> lev;
    double *d_cinv = nullptr;  // dense inverse of the coarsest matrix
    float *d_cinv32 = nullptr;
    int64_t nc = 0;
    int64_t *d_fine_off = nullptr;  // device copy of fine.off (persistent smoother)
    unsigned *d_bar = nullptr;      // grid-barrier arrivals / exits of the persistent smoother
    int *d_bar_err = nullptr;       // set when one of its barriers timed out
    int spmv_tpr = 4;   // lanes per row of the fine SpMV (autotuned at setup)
    int fine_tpr = 4;   // lanes per row of the fine smoother phases (autotuned at setup)
    // solve work (sized for ncols = 1 at setup, grown on demand)
    int work_cols = 0;
    double *w_r = nullptr, *w_z = nullptr, *w_p = nullptr, *w_q = nullptr, *w_x = nullptr,
           *w_b = nullptr, *w_zs = nullptr, *w_t = nullptr;
    double *w_rr = nullptr;
    float *w_zs32 = nullptr, *w_t32 = nullptr, *w_rr32 = nullptr;
    cudaStream_t aux_stream = nullptr, cap_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int *d_flag = nullptr;
    double *d_partials = nullptr;
    unsigned int *d_counter = nullptr;
    pk::PcgState *d_state = nullptr;
    double *d_hist = nullptr;
    int hist_cap = 0;
    pk::DevPool work_pool;
    // graph cache
    cudaGraphExec_t graph_exec = nullptr;
    cudaGraph_t graph = nullptr;
    int graph_cols = 0;
    long long g_init = 0, g_body = 0, g_final = 0;  // kernels per graph part
    int64_t graph_ld = 0;
    const void *graph_key_b = nullptr;
    void *graph_key_x = nullptr;
    cudaStream_t graph_stream = nullptr;
    // several right-hand sides: blocks [n][NC] (batched.cu), sized for one width NC
    pk::DevPool bwork_pool;
    int bwork_nc = -1, bwork_hist = 0;
    int bchunk = 0;  // 1 + the autotuned layout of the blocked fine smoother (0: not tuned yet)
    int bgroup_cols = 0, blanes = 0;  // that layout: columns per group, lanes per row
    double *bw_r = nullptr, *bw_z = nullptr, *bw_p = nullptr, *bw_q = nullptr, *bw_b = nullptr,
           *bw_x = nullptr, *bw_zs = nullptr, *bw_t = nullptr, *bw_hist = nullptr;
    float *bw_zs32 = nullptr, *bw_t32 = nullptr, *bw_r32 = nullptr;
    int *bw_mask = nullptr;
    std::vector<double *> bl_b, bl_x, bl_r;  // per level
    std::vector<float *> bl_b32, bl_x32, bl_r32;
    cudaGraphExec_t bgraph_exec = nullptr;
    cudaGraph_t bgraph = nullptr;
    long long bg_init = 0, bg_body = 0, bg_final = 0;
    // FGMRES(m) (gmres.cu): Arnoldi vectors V [(m+1)][n], preconditioned vectors Z [m][n]
    pk::DevPool gm_pool;
    int gm_m = 0;
    double *gm_V = nullptr, *gm_Z = nullptr, *gm_w = nullptr, *gm_vin = nullptr, *gm_zout = nullptr;
    double *gm_H = nullptr, *gm_g = nullptr, *gm_cs = nullptr, *gm_sn = nullptr, *gm_y = nullptr,
           *gm_hc = nullptr, *gm_part = nullptr;
    unsigned *gm_cnt = nullptr;
    pk::GmresState *gm_state = nullptr;
    cudaGraphExec_t gm_graph_exec = nullptr;
    cudaGraph_t gm_graph = nullptr;
    const void *gm_key_b = nullptr;
    void *gm_key_x = nullptr;
    long long gm_g_init = 0, gm_g_body = 0;
    // Taylor-Hood Stokes system (stokes.cpp, stokes.cu), built by pkasp_stokes_setup
    pk::StokesWork *st = nullptr;
    // staging of host arrays [n][ld]
    pk::DevPool stage_pool;
    int64_t stage_elems = 0;
    double *stage_b = nullptr, *stage_x = nullptr;
};

namespace pk {

// ---- host side (mesh.cpp) -------------------------------------------------------
struct HostMesh {
    int k;
    int64_t nv, nt;
    const double *xyz;
    const int32_t *tets;
};
struct DofMap {
    int64_t n_all = 0, nh = 0, nH = 0;
    std::vector<int64_t> dof_all;
    std::vector<double> dof_xyz;
    std::vector<int32_t> elem_dof, elem_vdof;
    std::vector<int32_t> elem_all;  // [nt*nloc] node index before Dirichlet removal
    std::vector<int64_t> inc_ptr, vinc_ptr;
    std::vector<int32_t> inc, vinc;  // tet*64 + local index
    HCSR Ah_pattern, AH_pattern, Pi, PiT;
};
void build_dofmap(const HostMesh &m, DofMap &out);
int nloc_of(int k);
void ref_nodes(int k, std::vector<int> &m4);
void reference_tensors(int k, std::vector<double> &S);          // [16][nloc][nloc]
void gm_rule(int s, std::vector<double> &lam, std::vector<double> &w);
void basis_values(int k, const double *lam, double *phi);

// ---- device side ----------------------------------------------------------------
void assemble_device(pkasp_problem *p, cudaStream_t s);
void assemble_values(pkasp_problem *p, cudaStream_t s);
void setup_device(pkasp_problem *p, cudaStream_t s);
void free_setup(pkasp_problem *p);
int solve_device(pkasp_problem *p, const double *b_dev, double *x_dev, int ncols, int64_t ld,
                 pkasp_stats *st, cudaStream_t s);
void apply_prec(pkasp_problem *p, const double *r, double *z, cudaStream_t s);
void apply_smoother(pkasp_problem *p, const double *r, double *z, cudaStream_t s);
void apply_vcycle(pkasp_problem *p, const double *b, double *x, cudaStream_t s);
void spmv_fine(pkasp_problem *p, const double *x, double *y, cudaStream_t s);
void grad_kappa_device(const pkasp_problem *p, const double *u, const double *lam, int ncols, int64_t ld,
                       double *g, cudaStream_t s);
void pmis_device(int64_t n, const int64_t *ptr, const int32_t *col, const uint8_t *strong,
                 uint64_t stream_id, int8_t *cf, cudaStream_t s);
void pmis_noalloc(int64_t n, const int64_t *ptr, const int32_t *col, const uint8_t *strong, uint64_t stream_id,
                  int8_t *cf, cudaStream_t s);
void ensure_work(pkasp_problem *p, int ncols);
void check_barrier(pkasp_problem *p, cudaStream_t s);
// PCG on several right-hand sides (batched.cu); b and x device arrays [n_h][ld]
int solve_batched(pkasp_problem *p, const double *b, double *x, int ncols, int64_t ld, pkasp_stats *st,
                  cudaStream_t s);
void free_batched(pkasp_problem *p);
float time_batched(pkasp_problem *p, int which, int reps, cudaStream_t s);
// FGMRES(m) outer iteration (gmres.cu); b and x device vectors [n_h]
int solve_gmres(pkasp_problem *p, const double *b, double *x, pkasp_stats *st, cudaStream_t s);
void free_gmres(pkasp_problem *p);
// Stokes (stokes.cpp: patterns of B = -div_h, B^T and the pressure mass matrix, and
// their host values for the host-only entry point; stokes.cu: device assembly of the
// values, operator, block preconditioner, FGMRES)
struct StokesPattern {
    int64_t np = 0;
    int nu = 0, npl = 0;                 // local velocity / pressure nodes
    std::vector<int32_t> elem_p;         // [nt][npl] pressure node of each local node
    std::vector<double> R, Mr;           // reference tensors [4][npl][nu], [npl][npl]
    std::vector<int64_t> iptr, ient;     // pressure node -> (element * 64 + local)
    HCSR B, BT, M;                       // patterns (values empty)
    std::vector<int64_t> bt_src;         // B^T entry o copies B entry bt_src[o]
};
void stokes_patterns(int k, int64_t nv, int64_t nt, const double *xyz, const int32_t *tets, int64_t nh,
                     const int32_t *elem_dof, StokesPattern &P);
// the same from a mesh and its P_k unknown map (elem_dof[nt][nloc(k)]), host only
void stokes_blocks(int k, int64_t nv, int64_t nt, const double *xyz, const int32_t *tets, int64_t nh,
                   const int32_t *elem_dof, HCSR &B, HCSR &BT, HCSR &M, int64_t &np);
void stokes_setup(pkasp_problem *p, int mp_iters, cudaStream_t s);
void stokes_free(pkasp_problem *p);
void stokes_apply(pkasp_problem *p, const double *x, double *y, cudaStream_t s);
void stokes_prec(pkasp_problem *p, const double *r, double *z, cudaStream_t s);
int stokes_solve(pkasp_problem *p, const double *b, double *x, pkasp_stats *st, cudaStream_t s);
const DCSR *stokes_matrix(const pkasp_problem *p, int which);  // -1 B, -2 B^T, -3 M_p
void stokes_sizes(const pkasp_problem *p, int64_t *out5);
float time_kernel(pkasp_problem *p, int which, int reps, cudaStream_t s);

// SELL-32 builders (sell.cu)
void build_sell_natural(DevPool &pool, const DCSR &A, DSell &S, bool want32, cudaStream_t s);
void build_sell_split(DevPool &pool, const DSplit &sp, int64_t n, bool upper, DSell &S, bool want32,
                      cudaStream_t s);

// small device utilities (util.cu)
void to32(const double *x, float *y, int64_t n, cudaStream_t s);
void exclusive_scan(int64_t *d, int64_t n, cudaStream_t s);  // in place, d[n] = total
int64_t read_i64(const int64_t *d, cudaStream_t s);
void dcsr_alloc(DevPool &pool, DCSR &a, int64_t n, int64_t m, int64_t nnz);
void dcsr_upload(DevPool &pool, DCSR &a, const HCSR &h, cudaStream_t s);
void pi_codes_upload(DevPool &pool, const HCSR &Pi, const HCSR &PiT, int k, PiCodes &pc, cudaStream_t s);
void l2_window_release(pkasp_problem *p);
void l2_window_idle(pkasp_problem *p);
void dcsr_download(const DCSR &a, HCSR &h, cudaStream_t s);
void dcsr_make32(DevPool &pool, DCSR &a, cudaStream_t s);

// hash streams of the method's random choices
inline uint64_t stream_colour(uint64_t seed, int m) { return seed * 64 + (uint64_t)m; }
inline uint64_t stream_pmis(uint64_t seed, int l) { return seed * 64 + 32 + (uint64_t)l; }

}  // namespace pk
