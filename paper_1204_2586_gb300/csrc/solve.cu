// solve.cu -- the hot path: preconditioned conjugate gradients on A_h u = f_h (Eq. 7)
// with the auxiliary-space preconditioner
//     additive:       z = S_k r + I_P V(I_R r)
//     multiplicative: Algorithm 2.1 with pre-smoothing (Remark 2.1)
// where S_k is the multicolour symmetric Gauss-Seidel (or l1-Jacobi) smoother on A_h and
// V one V(1,1)-cycle of the P1 AMG hierarchy. The two additive branches are independent
// and run concurrently on two streams (two branches of the captured graph). One PCG
// iteration is a fixed kernel sequence; the whole solve is captured once into a CUDA
// graph whose while-node repeats the iteration until a device-side flag says stop.
#include <type_traits>
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"
#include "kernels.cuh"
#include "persist.cuh"
#include "rowop.cuh"

namespace pk {

void build_split(DevPool &pool, const DCSR &A, uint64_t stream, bool want32, DSplit &sp, cudaStream_t s);
double *row_l1(DevPool &pool, const DCSR &A, cudaStream_t s);
bool coarsen(DevPool &pool, Level &L, double theta, uint64_t pmis_stream, DCSR &Ac, cudaStream_t s,
             double trunc_factor, int pmax, int cc);
void coarse_inverse(DevPool &pool, const DCSR &A, double **inv, cudaStream_t s);

namespace {

// ---------------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------------
// Lanes per row. Short sub-warps keep more rows, and more independent loads per lane,
// in flight: on GB300 four lanes beat sixteen by 1.7x on the P3 matrix (47 entries per
// row). The fine SpMV and the fine smoother are autotuned at setup instead.
int tpr_for(double mean_row) {
    if (mean_row <= 96) return 4;
    return 8;
}
int tpr_of(const DCSR &A) { return tpr_for(A.n > 0 ? (double)A.nnz / (double)A.n : 1.0); }

unsigned rows_grid(int64_t rows, int tpr) {
    int64_t threads = rows * tpr;
    int64_t b = (threads + kBlock - 1) / kBlock;
    return (unsigned)std::max<int64_t>(1, b);
}
unsigned elem_grid(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + kBlock - 1) / kBlock); }

template <typename PT>
__global__ void k_copy_to(int64_t n, const PT *__restrict__ a, double *__restrict__ b) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (double)a[i];
}

template <typename PT>
__global__ void k_to_pt(int64_t n, const double *__restrict__ a, PT *__restrict__ b) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (PT)a[i];
}

template <typename PT>
void to_pt(const double *a, PT *b, int64_t n, cudaStream_t s) {
    k_to_pt<PT><<<elem_grid(n), kBlock, 0, s>>>(n, a, b);
    PK_LAUNCH();
}

#define PK_TPR_SWITCH(tpr, BODY)                 \
    switch (tpr) {                               \
        case 1: { constexpr int TPR = 1; BODY; } break;   \
        case 2: { constexpr int TPR = 2; BODY; } break;   \
        case 4: { constexpr int TPR = 4; BODY; } break;   \
        case 8: { constexpr int TPR = 8; BODY; } break;   \
        case 16: { constexpr int TPR = 16; BODY; } break; \
        default: { constexpr int TPR = 32; BODY; } break; \
    }

template <typename PT> const PT *pick(const double *d, const float *f);
template <> const double *pick<double>(const double *d, const float *) { return d; }
template <> const float *pick<float>(const double *, const float *f) { return f; }
template <typename PT> PT *pickw(double *d, float *f);
template <> double *pickw<double>(double *d, float *) { return d; }
template <> float *pickw<float>(double *, float *f) { return f; }

template <typename PT, typename A_, typename X, typename Y>
void spmv(const DCSR &A, const X *x, Y *y, int tpr, cudaStream_t s) {
    if (A.n == 0) return;
    PK_TPR_SWITCH(tpr, (k_spmv<TPR, A_, PT><<<rows_grid(A.n, TPR), kBlock, 0, s>>>(
                            A.n, A.ptr, A.col, pick<PT>(A.val, A.val32), x, y)));
    PK_LAUNCH();
}

// Launch with programmatic stream serialization (PDL): the kernel may begin while the
// previous kernel on the stream drains; it must call pdl_wait() before reading anything
// an earlier kernel wrote (k_gs_phase does).
// win (optional): an L2 access-policy window for the launch
template <typename... KArgs, typename... Args>
void launch_pdl_w(void (*kern)(KArgs...), unsigned grid, cudaStream_t s, const cudaAccessPolicyWindow *win,
                  Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kBlock);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (win) {
        attr[1].id = cudaLaunchAttributeAccessPolicyWindow;
        attr[1].val.accessPolicyWindow = *win;
        cfg.numAttrs = 2;
    }
    PK_CUDA(cudaLaunchKernelEx(&cfg, kern, args...));
    PK_LAUNCH();
}

template <typename... KArgs, typename... Args>
void launch_pdl(void (*kern)(KArgs...), unsigned grid, cudaStream_t s, Args... args) {
    launch_pdl_w(kern, grid, s, (const cudaAccessPolicyWindow *)nullptr, args...);
}

// a plain launch (no programmatic serialization) with an optional access-policy window
template <typename... KArgs, typename... Args>
void launch_w(void (*kern)(KArgs...), unsigned grid, cudaStream_t s, const cudaAccessPolicyWindow *win,
              Args... args) {
    if (!win) {
        kern<<<grid, kBlock, 0, s>>>(args...);
        PK_LAUNCH();
        return;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kBlock);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeAccessPolicyWindow;
    attr[0].val.accessPolicyWindow = *win;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    PK_CUDA(cudaLaunchKernelEx(&cfg, kern, args...));
    PK_LAUNCH();
}

// Lanes per row for a colour phase whose longest row part has `len` entries: the fewest
// lanes (a power of two, at most 32) for which one batch of loads per lane covers the row.
// A colour phase is latency-bound, and every extra batch is one more DRAM round trip.
int lanes_for(int len) {
    int t = 1;
    while (t < 32 && t * kBatch < len) t <<= 1;
    return t;
}

// Entries per lane and batch for a colour phase with tpr lanes whose row parts mostly
// (90th percentile) have at most `len` entries: the fewest of 2, 4, 8 that cover such a
// row in one batch (else 8); longer rows take further batches.
int batch_for(int tpr, int len) {
    for (int nb : {2, 4, 8})
        if (nb * tpr >= len) return nb;
    return tpr <= 2 ? 16 : 8;  // two lanes per row: up to 32 entries in one batch
}

#define PK_NB_SWITCH(nb, BODY)                           \
    switch (nb) {                                        \
        case 2: { constexpr int NB = 2; BODY; } break;   \
        case 4: { constexpr int NB = 4; BODY; } break;   \
        case 16: { constexpr int NB = 16; BODY; } break; \
        default: { constexpr int NB = 8; BODY; } break;  \
    }

// Grid-stride colour phases (k_gs_phase_gs): at most the kernel's resident blocks (a
// grid of half of them lost on every measured problem). The capacity is taken once per
// kernel variant.
template <auto Kern>
unsigned phase_grid(int64_t rows, int tpr) {
    static int occ = 0, nsm = 0;
    if (occ == 0) {
        int dev = 0, o = 0;
        PK_CUDA(cudaGetDevice(&dev));
        PK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        PK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, Kern, kBlock, 0));
        occ = std::max(1, o);
    }
    return (unsigned)std::min<int64_t>(rows_grid(rows, tpr), (int64_t)nsm * occ);
}
#define PK_TPR3_SWITCH(tpr, BODY)                         \
    switch (tpr) {                                        \
        case 4: { constexpr int TPR = 4; BODY; } break;   \
        case 16: { constexpr int TPR = 16; BODY; } break; \
        default: { constexpr int TPR = 8; BODY; } break;  \
    }
#define PK_NB3_SWITCH(nb, BODY)                          \
    switch (nb) {                                        \
        case 2: { constexpr int NB = 2; BODY; } break;   \
        case 4: { constexpr int NB = 4; BODY; } break;   \
        default: { constexpr int NB = 8; BODY; } break;  \
    }

// colour phases of a forward sweep from zero: y = (D+L)^{-1} r; tpr < 0 picks the lanes
// per colour from the colour's longest lower part
template <typename PT, typename TR>
void gs_forward0(const DSplit &sp, int tpr_fixed, const TR *r, PT *y, cudaStream_t s,
                 const cudaAccessPolicyWindow *win = nullptr) {
    for (int c = 0; c < sp.ncol; ++c) {
        int64_t pb = sp.off[c], pe = sp.off[c + 1];
        if (pe <= pb) continue;
        if (tpr_fixed > 400) {  // grid-stride with prefetch of the next row
            const int tpr = tpr_fixed % 100;
            const int nb = batch_for(tpr, sp.l90[c]);
            PK_TPR3_SWITCH(tpr, PK_NB3_SWITCH(nb, (launch_pdl_w(
                k_gs_phase_gs<TPR, NB, PT, TR, false>,
                phase_grid<k_gs_phase_gs<TPR, NB, PT, TR, false>>(pe - pb, TPR), s, win, pb, pe,
                (const int32_t *)sp.perm, (const int64_t *)sp.lptr, (const int32_t *)sp.lcol,
                pick<PT>(sp.lval, sp.lval32), pick<PT>(sp.dinv, sp.dinv32), r, y))));
            continue;
        }
        const bool two = tpr_fixed > 100;  // two rows per sub-warp
        const int tf = two ? tpr_fixed - 100 : tpr_fixed;
        const int tpr = tf > 0 ? tf : lanes_for(sp.lmax[c]);
        const int nb = batch_for(tpr, sp.l90[c]);
        if (two) {
            PK_TPR_SWITCH(tpr, PK_NB_SWITCH(nb, (launch_pdl_w(k_gs_phase2<TPR, NB, PT, TR, false>,
                                                            rows_grid((pe - pb + 1) / 2, TPR), s, win, pb, pe,
                                                            (const int32_t *)sp.perm, (const int64_t *)sp.lptr,
                                                            (const int32_t *)sp.lcol, pick<PT>(sp.lval, sp.lval32),
                                                            pick<PT>(sp.dinv, sp.dinv32), r, y))));
            continue;
        }
        PK_TPR_SWITCH(tpr, PK_NB_SWITCH(nb, (launch_pdl_w(k_gs_phase<TPR, NB, PT, TR, false>,
                                                        rows_grid(pe - pb, TPR), s, win, pb, pe,
                                                        (const int32_t *)sp.perm, (const int64_t *)sp.lptr,
                                                        (const int32_t *)sp.lcol, pick<PT>(sp.lval, sp.lval32),
                                                        pick<PT>(sp.dinv, sp.dinv32), r, y))));
    }
}

// backward half of the symmetric sweep from zero: y <- y - D^{-1} U y, colours C-1..0
template <typename PT>
void gs_backward0(const DSplit &sp, int tpr_fixed, PT *y, cudaStream_t s,
                  const cudaAccessPolicyWindow *win = nullptr) {
    // the highest colour has no upper part: its phase would leave y unchanged
    for (int c = sp.ncol - 2; c >= 0; --c) {
        int64_t pb = sp.off[c], pe = sp.off[c + 1];
        if (pe <= pb) continue;
        if (tpr_fixed > 400) {
            const int tpr = tpr_fixed % 100;
            const int nb = batch_for(tpr, sp.u90[c]);
            PK_TPR3_SWITCH(tpr, PK_NB3_SWITCH(nb, (launch_pdl_w(
                k_gs_phase_gs<TPR, NB, PT, PT, true>,
                phase_grid<k_gs_phase_gs<TPR, NB, PT, PT, true>>(pe - pb, TPR), s, win, pb, pe,
                (const int32_t *)sp.perm, (const int64_t *)sp.uptr, (const int32_t *)sp.ucol,
                pick<PT>(sp.uval, sp.uval32), pick<PT>(sp.dinv, sp.dinv32), (const PT *)y, y))));
            continue;
        }
        const bool two = tpr_fixed > 100;
        const int tf = two ? tpr_fixed - 100 : tpr_fixed;
        const int tpr = tf > 0 ? tf : lanes_for(sp.umax[c]);
        const int nb = batch_for(tpr, sp.u90[c]);
        if (two) {
            PK_TPR_SWITCH(tpr, PK_NB_SWITCH(nb, (launch_pdl_w(k_gs_phase2<TPR, NB, PT, PT, true>,
                                                            rows_grid((pe - pb + 1) / 2, TPR), s, win, pb, pe,
                                                            (const int32_t *)sp.perm, (const int64_t *)sp.uptr,
                                                            (const int32_t *)sp.ucol, pick<PT>(sp.uval, sp.uval32),
                                                            pick<PT>(sp.dinv, sp.dinv32), (const PT *)y, y))));
            continue;
        }
        PK_TPR_SWITCH(tpr, PK_NB_SWITCH(nb, (launch_pdl_w(k_gs_phase<TPR, NB, PT, PT, true>,
                                                        rows_grid(pe - pb, TPR), s, win, pb, pe,
                                                        (const int32_t *)sp.perm, (const int64_t *)sp.uptr,
                                                        (const int32_t *)sp.ucol, pick<PT>(sp.uval, sp.uval32),
                                                        pick<PT>(sp.dinv, sp.dinv32), (const PT *)y, y))));
    }
}

// full backward GS sweep on A x = b from the current x
template <typename PT>
void gs_backward_full(const DSplit &sp, int tpr_fixed, const PT *b, PT *x, cudaStream_t s,
                      const cudaAccessPolicyWindow *win = nullptr) {
    for (int c = sp.ncol - 1; c >= 0; --c) {
        int64_t pb = sp.off[c], pe = sp.off[c + 1];
        if (pe <= pb) continue;
        const int tpr = tpr_fixed > 0 ? tpr_fixed : lanes_for(std::max(sp.lmax[c], sp.umax[c]));
        const int nb = batch_for(tpr, std::max(sp.l90[c], sp.u90[c]));
        PK_TPR_SWITCH(tpr, PK_NB_SWITCH(nb, (launch_w(k_gs_bwd_full<TPR, NB, PT>, rows_grid(pe - pb, TPR), s, win,
                                                      pb, pe, (const int32_t *)sp.perm, (const int64_t *)sp.lptr,
                                                      (const int32_t *)sp.lcol, pick<PT>(sp.lval, sp.lval32),
                                                      (const int64_t *)sp.uptr, (const int32_t *)sp.ucol,
                                                      pick<PT>(sp.uval, sp.uval32), pick<PT>(sp.diag, sp.diag32),
                                                      b, x))));
    }
}

template <typename PT>
__global__ void k_add_div(int64_t n, const PT *__restrict__ r, const PT *__restrict__ d, PT *__restrict__ x) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] += r[i] / d[i];
}

// ---------------------------------------------------------------------------------
// V(1,1)-cycle on level l (vectors b, x, r of each level)
// ---------------------------------------------------------------------------------
template <typename PT>
PT *lv_b(Level &L) { return pickw<PT>(L.b, L.b32); }
template <typename PT>
PT *lv_x(Level &L) { return pickw<PT>(L.x, L.x32); }
template <typename PT>
PT *lv_r(Level &L) { return pickw<PT>(L.r, L.r32); }

template <typename PT>
void vcycle(pkasp_problem *p, int l, cudaStream_t s, bool pre_done = false);

// b_l = R x (R = I_P^T into level 0, or level l-1's restriction); with l1-Jacobi level
// smoothing on a level that is not the coarsest, the same pass also takes the
// pre-smoothing step from zero, x_l = b_l / l1 (returns true then).
template <typename PT, typename XT>
bool restrict_to(pkasp_problem *p, const DCSR &R, const XT *x, int l, cudaStream_t s) {
    Level &L = p->lev[l];
    const bool fuse = p->opt.level_smoother == PKASP_SMOOTHER_L1JACOBI && l < (int)p->lev.size() - 1;
    if (!fuse || R.n == 0) {
        spmv<PT, PT>(R, x, lv_b<PT>(L), tpr_of(R), s);
        return false;
    }
    if (&R == &p->PiT) {
        // I_P^T with one-byte value codes
        PK_TPR_SWITCH(tpr_of(R), (k_restrict_code_jacobi0<TPR, PT, XT><<<rows_grid(R.n, TPR), kBlock, 0, s>>>(
                                     R.n, R.ptr, R.col, p->pic.t_code, pick<PT>(p->pic.tab, p->pic.tab32), x,
                                     pick<PT>(L.l1, L.l132), lv_b<PT>(L), lv_x<PT>(L))));
        PK_LAUNCH();
        return true;
    }
    PK_TPR_SWITCH(tpr_of(R), (k_restrict_jacobi0<TPR, PT, PT, XT, PT><<<rows_grid(R.n, TPR), kBlock, 0, s>>>(
                                 R.n, R.ptr, R.col, pick<PT>(R.val, R.val32), x, pick<PT>(L.l1, L.l132),
                                 lv_b<PT>(L), lv_x<PT>(L))));
    PK_LAUNCH();
    return true;
}

// V(1,1)-cycle on level l; pre_done: the pre-smoothing step from zero was taken by the
// restriction that produced b_l
template <typename PT>
void vcycle(pkasp_problem *p, int l, cudaStream_t s, bool pre_done) {
    Level &L = p->lev[l];
    const int64_t n = L.A.n;
    if (l == (int)p->lev.size() - 1) {
        k_dense_mv<PT><<<rows_grid(n, 32), kBlock, 0, s>>>(n, pick<PT>(p->d_cinv, p->d_cinv32), lv_b<PT>(L),
                                                          lv_x<PT>(L));
        PK_LAUNCH();
        return;
    }
    const bool jac = p->opt.level_smoother == PKASP_SMOOTHER_L1JACOBI;
    const int ta = tpr_of(L.A), ts = -1;  // lanes per colour phase chosen per colour
    if (jac) {
        if (!pre_done) {
            k_jacobi0<PT, PT><<<elem_grid(n), kBlock, 0, s>>>(n, pick<PT>(L.l1, L.l132), lv_b<PT>(L),
                                                              lv_x<PT>(L));
            PK_LAUNCH();
        }
    } else {
        gs_forward0<PT, PT>(L.sp, ts, lv_b<PT>(L), lv_x<PT>(L), s);
    }
    PK_TPR_SWITCH(ta, (k_residual<TPR, PT, PT, PT><<<rows_grid(n, TPR), kBlock, 0, s>>>(
                          n, L.A.ptr, L.A.col, pick<PT>(L.A.val, L.A.val32), lv_b<PT>(L), lv_x<PT>(L),
                          lv_r<PT>(L))));
    PK_LAUNCH();
    Level &C = p->lev[l + 1];
    const bool pd = restrict_to<PT>(p, L.R, (const PT *)lv_r<PT>(L), l + 1, s);
    vcycle<PT>(p, l + 1, s, pd);
    const int tp = tpr_of(L.P);
    PK_TPR_SWITCH(tp, (k_prolong_inplace<TPR, PT><<<rows_grid(n, TPR), kBlock, 0, s>>>(
                          n, L.P.ptr, L.P.col, pick<PT>(L.P.val, L.P.val32), lv_x<PT>(C), lv_x<PT>(L))));
    PK_LAUNCH();
    if (jac) {
        PK_TPR_SWITCH(ta, (k_residual<TPR, PT, PT, PT><<<rows_grid(n, TPR), kBlock, 0, s>>>(
                              n, L.A.ptr, L.A.col, pick<PT>(L.A.val, L.A.val32), lv_b<PT>(L), lv_x<PT>(L),
                              lv_r<PT>(L))));
        PK_LAUNCH();
        k_add_div<PT><<<elem_grid(n), kBlock, 0, s>>>(n, lv_r<PT>(L), pick<PT>(L.l1, L.l132), lv_x<PT>(L));
        PK_LAUNCH();
    } else {
        gs_backward_full<PT>(L.sp, ts, lv_b<PT>(L), lv_x<PT>(L), s);
    }
}

// the symmetric sweep of the fine split as one cooperative launch (persist.cuh), TPR
// lanes per row, kPersistBlocksPerSm blocks of kPersistBlock threads per SM
constexpr int kPersistBlocksPerSm = 1;

template <int TPR, typename PT, typename TR>
void sgs_persistent(pkasp_problem *p, const TR *r, PT *y, cudaStream_t s) {
    auto kern = k_sgs_persistent<TPR, PT, TR>;
    int occ = 0, sms = 0, dev = 0;
    PK_CUDA(cudaGetDevice(&dev));
    PK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    PK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kPersistBlock, 0));
    if (occ < 1) fail(PKASP_ECUDA, "persistent smoother does not fit on an SM");
    const DSplit &sp = p->fine;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(sms * std::min(occ, kPersistBlocksPerSm)));
    cfg.blockDim = dim3(kPersistBlock);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    PK_CUDA(cudaLaunchKernelEx(&cfg, kern, sp.ncol, (const int64_t *)p->d_fine_off, (const int32_t *)sp.perm,
                               (const int64_t *)sp.lptr, (const int32_t *)sp.lcol, pick<PT>(sp.lval, sp.lval32),
                               (const int64_t *)sp.uptr, (const int32_t *)sp.ucol, pick<PT>(sp.uval, sp.uval32),
                               pick<PT>(sp.dinv, sp.dinv32), r, y, p->d_bar, p->d_bar_err));
    PK_LAUNCH();
}

// reads (and clears) the persistent smoother's barrier-timeout flag; synchronises s
void barrier_status(pkasp_problem *p, cudaStream_t s) {
    if (!p->d_bar_err) return;
    int err = 0;
    PK_CUDA(cudaMemcpyAsync(&err, p->d_bar_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    PK_CUDA(cudaStreamSynchronize(s));
    if (err) {
        PK_CUDA(cudaMemsetAsync(p->d_bar_err, 0, sizeof(int), s));
        PK_CUDA(cudaStreamSynchronize(s));
        fail(PKASP_ECUDA, "the persistent smoother's grid barrier timed out");
    }
}

// the access-policy window that keeps the FP64 fine smoother's vector y in the L2
// set-aside (l2_window_setup); nullptr when there is none
template <typename PT>
const cudaAccessPolicyWindow *smoother_window(const pkasp_problem *p, PT *y, cudaAccessPolicyWindow &win) {
    if (!std::is_same<PT, double>::value || p->l2_win_bytes == 0) return nullptr;
    win = cudaAccessPolicyWindow{};
    win.base_ptr = (void *)y;
    win.num_bytes = p->l2_win_bytes;
    win.hitRatio = 1.0f;
    win.hitProp = cudaAccessPropertyPersisting;
    win.missProp = cudaAccessPropertyStreaming;
    return &win;
}

// S_k r from zero into zs (PT)
template <typename PT>
void smoother(pkasp_problem *p, const double *r, PT *zs, cudaStream_t s) {
    if (p->opt.smoother == PKASP_SMOOTHER_L1JACOBI) {
        k_jacobi0<PT, double><<<elem_grid(p->nh), kBlock, 0, s>>>(p->nh, pick<PT>(p->d_l1h, p->d_l1h32), r, zs);
        PK_LAUNCH();
        return;
    }
    const int ts = p->fine_tpr;
    if (ts < -1) {
        // one cooperative launch for all colour phases, -ts lanes per row
        switch (-ts) {
            case 4: sgs_persistent<4, PT, double>(p, r, zs, s); break;
            case 16: sgs_persistent<16, PT, double>(p, r, zs, s); break;
            default: sgs_persistent<8, PT, double>(p, r, zs, s); break;
        }
        return;
    }
    if (ts == 0) {
        // SELL-32 colour phases: colour c is the slice range [coff[c], coff[c+1])
        const DSell &L = p->fsl, &U = p->fsu;
        const int nc = p->fine.ncol;
        for (int c = 0; c < nc; ++c) {
            const int64_t s0 = L.coff[c], s1 = L.coff[c + 1];
            if (s1 <= s0) continue;
            launch_pdl(k_sell_phase<PT, double, false>, rows_grid((s1 - s0) * 32, 1), s, s0, s1,
                       (const int32_t *)L.perm, (const int64_t *)L.sptr, (const int32_t *)L.swidth,
                       (const int32_t *)L.col, pick<PT>(L.val, L.val32), pick<PT>(L.diag, L.diag32), r, zs);
        }
        // the highest colour has no upper part: its backward phase would leave y as is
        for (int c = nc - 2; c >= 0; --c) {
            const int64_t s0 = U.coff[c], s1 = U.coff[c + 1];
            if (s1 <= s0) continue;
            launch_pdl(k_sell_phase<PT, PT, true>, rows_grid((s1 - s0) * 32, 1), s, s0, s1,
                       (const int32_t *)U.perm, (const int64_t *)U.sptr, (const int32_t *)U.swidth,
                       (const int32_t *)U.col, pick<PT>(U.val, U.val32), pick<PT>(U.diag, U.diag32),
                       (const PT *)zs, zs);
        }
        return;
    }
    cudaAccessPolicyWindow wb;
    const cudaAccessPolicyWindow *win = smoother_window<PT>(p, zs, wb);
    gs_forward0<PT, double>(p->fine, ts, r, zs, s, win);
    gs_backward0<PT>(p->fine, ts, zs, s, win);
}

template <typename PT>
void restrict_vcycle(pkasp_problem *p, const double *r, cudaStream_t s) {
    const bool pd = restrict_to<PT>(p, p->PiT, r, 0, s);
    vcycle<PT>(p, 0, s, pd);
}

// z = B r. tail = false (additive mode only) stops before the last step z = z_s + Pi w:
// the PCG iteration then runs that step inside k_prolong_beta.
template <typename PT>
void precondition(pkasp_problem *p, const double *r, double *z, cudaStream_t s, bool tail = true) {
    PT *zs = pickw<PT>(p->w_zs, p->w_zs32);
    Level &L0 = p->lev[0];
    if (p->opt.mode == PKASP_MODE_AMG) {
        // plain AMG: one V-cycle on the hierarchy of A_h (level 0 is A_h)
        to_pt<PT>(r, lv_b<PT>(L0), p->nh, s);
        vcycle<PT>(p, 0, s);
        k_copy_to<PT><<<elem_grid(p->nh), kBlock, 0, s>>>(p->nh, lv_x<PT>(L0), z);
        PK_LAUNCH();
        return;
    }
    if (p->opt.mode == PKASP_MODE_ADDITIVE) {
        // fork: the V-cycle branch runs on the auxiliary stream, the smoother on s
        PK_CUDA(cudaEventRecord(p->ev_fork, s));
        PK_CUDA(cudaStreamWaitEvent(p->aux_stream, p->ev_fork, 0));
        restrict_vcycle<PT>(p, r, p->aux_stream);
        smoother<PT>(p, r, zs, s);
        PK_CUDA(cudaEventRecord(p->ev_join, p->aux_stream));
        PK_CUDA(cudaStreamWaitEvent(s, p->ev_join, 0));
        if (!tail) return;
        k_prolong_add<PT, double><<<elem_grid(p->nh), kBlock, 0, s>>>(
            p->nh, p->Pi.ptr, p->Pi.col, pick<PT>(p->Pi.val, p->Pi.val32), lv_x<PT>(L0), zs, z);
        PK_LAUNCH();
        return;
    }
    // multiplicative: forward GS (or l1 step) from zero, coarse correction of the new
    // residual, backward GS sweep (or l1 step) from the corrected iterate
    const bool jac = p->opt.smoother == PKASP_SMOOTHER_L1JACOBI;
    // the forward half sweep takes the tuned layout (SELL-32 maps to lanes fitted per
    // colour); the full backward sweep uses the CSR split with one row per lane group
    const int tfw = p->fine_tpr > 0 ? p->fine_tpr : -1;
    const int ts = p->fine_tpr > 0 ? p->fine_tpr % 100 : -1;
    // the residuals read the CSR form (a SELL-32 choice of the autotuner maps to the
    // lanes fitted to the mean row length)
    const int ta = p->spmv_tpr > 0 ? p->spmv_tpr : tpr_of(p->Ah);
    PT *t = pickw<PT>(p->w_t, p->w_t32);
    PT *rr = pickw<PT>(p->w_rr, p->w_rr32);
    if (jac) {
        k_jacobi0<PT, double><<<elem_grid(p->nh), kBlock, 0, s>>>(p->nh, pick<PT>(p->d_l1h, p->d_l1h32), r, zs);
        PK_LAUNCH();
    } else {
        cudaAccessPolicyWindow wb;
        gs_forward0<PT, double>(p->fine, tfw, r, zs, s, smoother_window<PT>(p, zs, wb));
    }
    to_pt<PT>(r, rr, p->nh, s);
    PK_TPR_SWITCH(ta, (k_residual<TPR, PT, PT, PT><<<rows_grid(p->nh, TPR), kBlock, 0, s>>>(
                          p->nh, p->Ah.ptr, p->Ah.col, pick<PT>(p->Ah.val, p->Ah.val32), rr, zs, t)));
    PK_LAUNCH();
    const bool pd = restrict_to<PT>(p, p->PiT, (const PT *)t, 0, s);
    vcycle<PT>(p, 0, s, pd);
    k_prolong_add<PT, PT><<<elem_grid(p->nh), kBlock, 0, s>>>(p->nh, p->Pi.ptr, p->Pi.col,
                                                              pick<PT>(p->Pi.val, p->Pi.val32), lv_x<PT>(L0),
                                                              zs, zs);
    PK_LAUNCH();
    if (jac) {
        PK_TPR_SWITCH(ta, (k_residual<TPR, PT, PT, PT><<<rows_grid(p->nh, TPR), kBlock, 0, s>>>(
                              p->nh, p->Ah.ptr, p->Ah.col, pick<PT>(p->Ah.val, p->Ah.val32), rr, zs, t)));
        PK_LAUNCH();
        k_add_div<PT><<<elem_grid(p->nh), kBlock, 0, s>>>(p->nh, t, pick<PT>(p->d_l1h, p->d_l1h32), zs);
        PK_LAUNCH();
    } else {
        cudaAccessPolicyWindow wb;
        gs_backward_full<PT>(p->fine, ts, (const PT *)rr, zs, s, smoother_window<PT>(p, zs, wb));
    }
    k_copy_to<PT><<<elem_grid(p->nh), kBlock, 0, s>>>(p->nh, zs, z);
    PK_LAUNCH();
}

// ---------------------------------------------------------------------------------
// PCG vector kernels (one right-hand side). Every kernel first reads the stop flag;
// a stopped solve turns every later launch into a no-op, so extra iterations queued
// behind the stop are harmless.
// ---------------------------------------------------------------------------------
enum { ST_RUN = -1 };

__global__ void k_state_reset(PcgState *st, double tol, int maxit, int hist_cap) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    st->iter[0] = 0;
    st->done[0] = 0;
    st->status[0] = ST_RUN;
    st->all_done = 0;
    st->ncols = 1;
    st->tol = tol;
    st->maxit = maxit;
    st->hist_cap = hist_cap;
    st->loops = 0;
    st->r0[0] = 0.0;
}

__global__ void k_state_restart(PcgState *st) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    st->done[0] = 0;
    st->status[0] = ST_RUN;
    st->all_done = 0;
    st->loops = 0;
}

// The fine-operator kernels (one thread or lane group per row, tens of thousands of
// blocks) only write vectors; every dot product and norm is taken by an element-wise
// kernel of kRedGrid blocks (grid_reduce). Each thread of those loads kVec elements
// (i, i + stride, ...) before it computes, and adds its terms in ascending i as a
// one-at-a-time loop would.
constexpr int kVec = 4;

// r = b - A x
template <int TPR>
__global__ void __launch_bounds__(kBlock) k_residual_fine(int64_t n, RowOp A, const double *__restrict__ b,
                                                          const double *__restrict__ x, double *__restrict__ r) {
    for_rows<TPR>(n, A, x, [&](int64_t row, double s) { r[row] = b[row] - s; });
}

// ||v||^2 of the grid, in every thread of the last block (grid_reduce)
__device__ __forceinline__ bool grid_norm2(int64_t n, const double *__restrict__ v, double *partials,
                                           unsigned *counter, double &tot) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double part = 0.0;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += kVec * stride) {
        double t[kVec] = {};
#pragma unroll
        for (int u = 0; u < kVec; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < n) t[u] = v[i];
        }
#pragma unroll
        for (int u = 0; u < kVec; ++u)
            if (i0 + u * stride < n) part += t[u] * t[u];
    }
    double a[1] = {part}, s[1];
    const bool last = grid_reduce<1>(a, partials, counter, s);
    tot = s[0];
    return last;
}

// ||r||; on the first start also r0 and hist[0]
__global__ void __launch_bounds__(kBlock) k_init_norm(int64_t n, const double *__restrict__ r, PcgState *st,
                                                      double *partials, unsigned *counter, double *hist) {
    double tot;
    if (!grid_norm2(n, r, partials, counter, tot) || threadIdx.x != 0) return;
    double rn = sqrt(tot);
    st->rnorm[0] = rn;
    if (st->iter[0] == 0) {
        st->r0[0] = rn;
        if (st->hist_cap > 0) hist[0] = rn;
        if (rn == 0.0) {
            st->done[0] = 1;
            st->status[0] = PKASP_OK;
            st->all_done = 1;
        }
    }
}

// p = z, rho = (r, z)
__global__ void __launch_bounds__(kBlock) k_start(int64_t n, const double *__restrict__ r,
                                                  const double *__restrict__ z, double *__restrict__ p,
                                                  PcgState *st, double *partials, unsigned *counter) {
    if (st->done[0]) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double part = 0.0;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += kVec * stride) {
        double rv[kVec] = {}, zv[kVec] = {};
#pragma unroll
        for (int u = 0; u < kVec; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < n) {
                rv[u] = r[i];
                zv[u] = z[i];
            }
        }
#pragma unroll
        for (int u = 0; u < kVec; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < n) {
                p[i] = zv[u];
                part += rv[u] * zv[u];
            }
        }
    }
    double v[1] = {part}, tot[1];
    if (grid_reduce<1>(v, partials, counter, tot) && threadIdx.x == 0) st->rho[0] = tot[0];
}

// q = A p
template <int TPR>
__global__ void __launch_bounds__(kBlock) k_spmv_q(int64_t n, RowOp A, const double *__restrict__ p,
                                                   double *__restrict__ q, const PcgState *st) {
    if (st->done[0]) return;
    for_rows<TPR>(n, A, p, [&](int64_t row, double s) { q[row] = s; });
}

// alpha = rho / (p, q)
__global__ void __launch_bounds__(kBlock) k_pq_alpha(int64_t n, const double *__restrict__ p,
                                                     const double *__restrict__ q, PcgState *st, double *partials,
                                                     unsigned *counter) {
    if (st->done[0]) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double part = 0.0;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += kVec * stride) {
        double pv[kVec] = {}, qv[kVec] = {};
#pragma unroll
        for (int u = 0; u < kVec; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < n) {
                pv[u] = p[i];
                qv[u] = q[i];
            }
        }
#pragma unroll
        for (int u = 0; u < kVec; ++u)
            if (i0 + u * stride < n) part += pv[u] * qv[u];
    }
    double v[1] = {part}, tot[1];
    if (grid_reduce<1>(v, partials, counter, tot) && threadIdx.x == 0) {
        double pq = tot[0];
        if (!(pq > 0.0)) {
            st->done[0] = 1;
            st->status[0] = PKASP_EBREAKDOWN;
            st->all_done = 1;
        } else {
            st->alpha[0] = st->rho[0] / pq;
        }
    }
}

// x += alpha p, r -= alpha q, ||r||, convergence test
__global__ void __launch_bounds__(kBlock) k_update_xr(int64_t n, double *__restrict__ x, double *__restrict__ r,
                                                      const double *__restrict__ p, const double *__restrict__ q,
                                                      PcgState *st, double *partials, unsigned *counter,
                                                      double *hist) {
    if (st->done[0]) return;
    const double a = st->alpha[0];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double part = 0.0;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += kVec * stride) {
        double xv[kVec] = {}, rv[kVec] = {}, pv[kVec] = {}, qv[kVec] = {};
#pragma unroll
        for (int u = 0; u < kVec; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < n) {
                xv[u] = x[i];
                rv[u] = r[i];
                pv[u] = p[i];
                qv[u] = q[i];
            }
        }
#pragma unroll
        for (int u = 0; u < kVec; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < n) {
                x[i] = xv[u] + a * pv[u];
                double ri = rv[u] - a * qv[u];
                r[i] = ri;
                part += ri * ri;
            }
        }
    }
    double v[1] = {part}, tot[1];
    if (grid_reduce<1>(v, partials, counter, tot) && threadIdx.x == 0) {
        double rn = sqrt(tot[0]);
        int it = st->iter[0] + 1;
        st->iter[0] = it;
        st->rnorm[0] = rn;
        if (it < st->hist_cap) hist[it] = rn;
        if (rn <= st->tol * st->r0[0]) {
            st->done[0] = 1;
            st->status[0] = PKASP_OK;
            st->all_done = 1;
        } else if (it >= st->maxit) {
            st->done[0] = 1;
            st->status[0] = PKASP_ENOTCONV;
            st->all_done = 1;
        }
    }
}

// rho_new = (r, z); beta = rho_new / rho, or -alpha (z, q) / rho for flexible CG
__global__ void __launch_bounds__(kBlock) k_beta(int64_t n, const double *__restrict__ r,
                                                 const double *__restrict__ z, const double *__restrict__ q,
                                                 int flexible, PcgState *st, double *partials, unsigned *counter) {
    if (st->done[0]) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double a0 = 0.0, a1 = 0.0;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += kVec * stride) {
        double rv[kVec] = {}, zv[kVec] = {}, qv[kVec] = {};
#pragma unroll
        for (int u = 0; u < kVec; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < n) {
                rv[u] = r[i];
                zv[u] = z[i];
                qv[u] = q[i];
            }
        }
#pragma unroll
        for (int u = 0; u < kVec; ++u) {
            if (i0 + u * stride < n) {
                a0 += rv[u] * zv[u];
                a1 += zv[u] * qv[u];
            }
        }
    }
    double v[2] = {a0, a1}, tot[2];
    if (grid_reduce<2>(v, partials, counter, tot) && threadIdx.x == 0) {
        double rho = st->rho[0];
        st->beta[0] = flexible ? (-st->alpha[0] * tot[1]) / rho : tot[0] / rho;
        st->rho[0] = tot[0];
    }
}

// The additive preconditioner's last step fused with the beta kernel: z = z_s + Pi w
// (row sums in PT in entry order, then one FP64 add, as k_prolong_add computes them),
// then (r, z) and (z, q) and beta as k_beta, without the round trip of z through memory
// between two kernels. I_P is read in its coded 4-wide layout: one 16-byte load of a
// row's columns and one word of value codes instead of row pointers, columns and
// values.
template <typename PT>
__global__ void __launch_bounds__(kBlock) k_prolong_beta(int64_t n, const int4 *__restrict__ ecol,
                                                             const uint32_t *__restrict__ ecode,
                                                             const PT *__restrict__ tab, const PT *__restrict__ w,
                                                             const PT *__restrict__ zs, const double *__restrict__ r,
                                                             const double *__restrict__ q, double *__restrict__ z,
                                                             int flexible, PcgState *st, double *partials,
                                                             unsigned *counter) {
    if (st->done[0]) return;
    constexpr int V = 2;  // rows in flight per thread (four take 80 registers)
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double a0 = 0.0, a1 = 0.0;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += V * stride) {
        int4 cv[V];
        uint32_t mv[V];
        double zv[V] = {}, rv[V] = {}, qv[V] = {};
#pragma unroll
        for (int u = 0; u < V; ++u) {
            const int64_t i = i0 + u * stride;
            const bool ok = i < n;
            cv[u] = ok ? ecol[i] : make_int4(-1, -1, -1, -1);
            mv[u] = ok ? ecode[i] : 0u;
            if (ok) {
                zv[u] = (double)zs[i];
                rv[u] = r[i];
                qv[u] = q[i];
            }
        }
#pragma unroll
        for (int u = 0; u < V; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < n) {
                const int cc[4] = {cv[u].x, cv[u].y, cv[u].z, cv[u].w};
                PT sv = PT(0);
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const uint32_t m = (mv[u] >> (8 * t)) & 0xffu;
                    if (m) sv += tab[m] * w[cc[t]];
                }
                const double zi = zv[u] + (double)sv;
                z[i] = zi;
                a0 += rv[u] * zi;
                a1 += zi * qv[u];
            }
        }
    }
    double v[2] = {a0, a1}, tot[2];
    if (grid_reduce<2>(v, partials, counter, tot) && threadIdx.x == 0) {
        double rho = st->rho[0];
        st->beta[0] = flexible ? (-st->alpha[0] * tot[1]) / rho : tot[0] / rho;
        st->rho[0] = tot[0];
    }
}

// p = z + beta p
__global__ void __launch_bounds__(kBlock) k_update_p(int64_t n, const double *__restrict__ z, double *__restrict__ p,
                                                     const PcgState *st) {
    if (st->done[0]) return;
    const double b = st->beta[0];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += kVec * stride) {
        double zv[kVec] = {}, pv[kVec] = {};
#pragma unroll
        for (int u = 0; u < kVec; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < n) {
                zv[u] = z[i];
                pv[u] = p[i];
            }
        }
#pragma unroll
        for (int u = 0; u < kVec; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < n) p[i] = zv[u] + b * pv[u];
        }
    }
}

// loop control of the captured while node: continue unless stopped; a safety bound on
// the number of passes stops the loop even if no kernel set the flag
__global__ void k_loop_control(PcgState *st, cudaGraphConditionalHandle h) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int loops = ++st->loops;
    bool go = !st->all_done && loops <= st->maxit + 2;
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

// true residual norm ||t|| (t = b - A x) into st->tnorm
__global__ void __launch_bounds__(kBlock) k_true_norm(int64_t n, const double *__restrict__ t, PcgState *st,
                                                      double *partials, unsigned *counter) {
    double tot;
    if (grid_norm2(n, t, partials, counter, tot) && threadIdx.x == 0) st->tnorm[0] = sqrt(tot);
}

}  // namespace


void l2_window_release(pkasp_problem *p);

// L2 persisting window for the FP64 fine smoother (pkasp_options.l2_persist). The colour
// phases gather the smoother's vector y (8 n_h bytes) once per entry, phase after phase,
// while the matrix streams past it; when y is a sizeable part of L2 the stream evicts it
// and every phase re-reads it from DRAM. Marking y's lines persisting keeps them. Only
// when y is at least a quarter of L2 (smaller vectors stay resident anyway) and the
// set-aside it needs (1.125 x y, measured best against 0.86 x and 1.5 x y) fits the
// device's largest one. The limit is a property of the CUDA context, not of the GPU:
// setup raises it if it is lower, pkasp_destroy restores what it found.
void l2_window_setup(pkasp_problem *p) {
    p->l2_win_bytes = 0;
    const pkasp_options &o = p->opt;
    if (!o.l2_persist || o.precond_precision != PKASP_PREC_FP64 || o.smoother != PKASP_SMOOTHER_SGS ||
        o.mode == PKASP_MODE_AMG) {
        l2_window_release(p);  // give back a set-aside an earlier setup of this problem took
        return;
    }
    // best effort: where the device or the context refuses (no persisting L2, a limit it
    // will not raise), the smoother simply runs without the window
    int dev = 0, l2 = 0, maxp = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&maxp, cudaDevAttrMaxPersistingL2CacheSize, dev) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    const size_t y = sizeof(double) * (size_t)p->nh;
    const size_t mb = size_t(1) << 20;
    const size_t want = (y + y / 8 + mb - 1) / mb * mb;
    if (maxp <= 0 || y < (size_t)l2 / 4 || want > (size_t)maxp) return;
    size_t cur = 0;
    if (cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    if (cur < want) {
        if (cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        size_t got = 0;
        cudaDeviceGetLimit(&got, cudaLimitPersistingL2CacheSize);
        cudaGetLastError();
        if (!p->l2_raised) p->l2_prev_limit = cur;
        p->l2_set_limit = got;
        p->l2_raised = true;
        if (got < y) return;  // granted less than the vector: no window
    }
    p->l2_win_bytes = y;
}

// after a synchronised solve: the smoother vector's lines go back to normal, so that the
// set-aside serves ordinary accesses of whatever runs next (other solves, other problems,
// the caller's kernels); the next S_k marks them persisting again. Never throws.
void l2_window_idle(pkasp_problem *p) {
    if (p->l2_win_bytes == 0) return;
    cudaCtxResetPersistingL2Cache();
    cudaGetLastError();
}

// returns persisting lines to normal and restores the limit this problem raised (if no
// one changed it since); never throws
void l2_window_release(pkasp_problem *p) {
    if (!p->l2_raised) return;
    cudaCtxResetPersistingL2Cache();
    size_t cur = 0;
    if (cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize) == cudaSuccess && cur == p->l2_set_limit)
        cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, p->l2_prev_limit);
    cudaGetLastError();
    p->l2_raised = false;
    p->l2_win_bytes = 0;
}

// ---------------------------------------------------------------------------------
// setup orchestration
// ---------------------------------------------------------------------------------
void free_setup(pkasp_problem *p) {
    free_batched(p);
    free_gmres(p);
    stokes_free(p);  // its solver captured the preconditioner being replaced
    if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    p->graph_exec = nullptr;
    p->graph = nullptr;
    p->graph_key_b = nullptr;
    p->graph_key_x = nullptr;
    p->setup_pool.free_all();
    p->work_pool.free_all();
    p->lev.clear();
    p->fine = DSplit{};
    p->Asell = DSell{};
    p->fsl = DSell{};
    p->fsu = DSell{};
    p->d_l1h = nullptr;
    p->d_l1h32 = nullptr;
    p->d_cinv = nullptr;
    p->d_fine_off = nullptr;
    p->d_bar = nullptr;
    p->d_bar_err = nullptr;
    p->d_cinv32 = nullptr;
    p->work_cols = 0;
    p->have_setup = false;
}

// Lanes-per-row autotuner for the two hot fine-level kernels: every candidate runs a few
// times on the actual matrix (inputs f_h) and the fastest is kept. A fixed
// options.spmv_threads bypasses it.
void autotune(pkasp_problem *p, cudaStream_t s) {
    if (p->opt.spmv_threads) {
        p->spmv_tpr = p->fine_tpr = p->opt.spmv_threads;
        return;
    }
    // a fixed smoother layout: internal code -1 per-colour lanes, 0 SELL-32, t lanes
    // 100 + t (t lanes, two rows per sub-warp) passes through
    const int lay = p->opt.smoother_layout;
    const int fixed_fine = lay == 1 ? -1 : lay == 2 ? 0 : lay == 3 ? 2 : lay;
    cudaEvent_t e0, e1;
    PK_CUDA(cudaEventCreate(&e0));
    PK_CUDA(cudaEventCreate(&e1));
    auto time3 = [&](auto fn) {  // three back-to-back runs
        PK_CUDA(cudaEventRecord(e0, s));
        for (int i = 0; i < 3; ++i) fn();
        PK_CUDA(cudaEventRecord(e1, s));
        PK_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    };
    // Candidates are timed round-robin, three rounds, best round per candidate: the
    // GPU's clock can still be ramping up during setup, and timing candidates one after
    // another would favour the later ones.
    auto tune = [&](const int *cand, int nc, int *slot, auto run) {
        std::vector<float> best(nc, 1e30f);
        for (int k = 0; k < nc; ++k) {
            *slot = cand[k];
            run();  // warm-up (first use of each variant)
        }
        for (int round = 0; round < 3; ++round)
            for (int k = 0; k < nc; ++k) {
                *slot = cand[k];
                best[k] = std::min(best[k], time3(run));
            }
        int pick = 0;
        for (int k = 1; k < nc; ++k)
            if (best[k] < best[pick]) pick = k;
        return cand[pick];
    };
    // 0: SELL-32, one thread per row; t > 0: CSR with t lanes per row; -1 (smoother
    // only): CSR with the lanes of each colour phase fitted to its longest row
    const int cand_spmv[] = {0, 2, 4, 8};
    // 100 + t: t lanes, two rows per sub-warp. The one-launch cooperative sweep (-t) is
    // not a candidate: its grid barrier cost more than a phase launch on every measured
    // problem (P3 32^3, P4 48^3); smoother_layout selects it explicitly.
    // (2 lanes per row, layouts 3 and 102, lost on every measured problem: P3 32^3 FP64
    // 769 vs 467 us; they stay selectable through smoother_layout)
    // 400 + t: t lanes, grid-stride over the resident blocks, the next row's static loads
    // in flight during the current row's gathers.
    const int cand_fine[] = {-1, 0, 4, 8, 16, 104, 108, 116, 404, 408, 416};
    const int pick_spmv = tune(cand_spmv, 4, &p->spmv_tpr, [&] { spmv_fine(p, p->d_b, p->w_q, s); });
    p->spmv_tpr = pick_spmv;
    int pick_fine = -1;
    if (p->opt.smoother == PKASP_SMOOTHER_SGS && p->opt.smoother_layout != 0) {
        pick_fine = fixed_fine;
    } else if (p->opt.smoother == PKASP_SMOOTHER_SGS) {
        if (p->opt.precond_precision == PKASP_PREC_FP32)
            pick_fine = tune(cand_fine, 11, &p->fine_tpr, [&] { smoother<float>(p, p->d_b, p->w_zs32, s); });
        else
            pick_fine = tune(cand_fine, 11, &p->fine_tpr, [&] { smoother<double>(p, p->d_b, p->w_zs, s); });
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p->spmv_tpr = pick_spmv;
    p->fine_tpr = pick_fine;
}

void setup_device(pkasp_problem *p, cudaStream_t s) {
    free_setup(p);
    const pkasp_options &o = p->opt;
    const bool want32 = o.precond_precision == PKASP_PREC_FP32;
    l2_window_setup(p);
    DevPool &pool = p->setup_pool;
    // fine level: colour split of A_h, l1 norms, FP32 copies
    build_split(pool, p->Ah, stream_colour(o.seed, 0), want32, p->fine, s);
    build_sell_natural(pool, p->Ah, p->Asell, false, s);
    build_sell_split(pool, p->fine, p->nh, false, p->fsl, want32, s);
    build_sell_split(pool, p->fine, p->nh, true, p->fsu, want32, s);
    p->d_l1h = row_l1(pool, p->Ah, s);
    if (want32) {
        p->d_l1h32 = pool.get<float>(p->nh);
        to32(p->d_l1h, p->d_l1h32, p->nh, s);
        // FP32 copies of the assembled operators live as long as the problem; they are
        // refreshed here because set_kappa may have changed A_h and A_H
        for (DCSR *M : {&p->Ah, &p->AH, &p->Pi, &p->PiT}) {
            if (!M->val32) dcsr_make32(p->pool, *M, s);
            else to32(M->val, M->val32, M->nnz, s);
        }
    }
    p->spmv_tpr = o.spmv_threads ? o.spmv_threads : tpr_of(p->Ah);
    // P1 hierarchy
    const int maxl = std::max(1, std::min(o.max_levels, (int)PKASP_MAX_LEVELS));
    p->lev.clear();
    p->lev.reserve(maxl);
    p->lev.emplace_back();
    // level 0 aliases an assembled operator owned by the problem: A_H of the auxiliary
    // space, or A_h itself for plain AMG
    const bool amg = o.mode == PKASP_MODE_AMG;
    p->lev[0].A = amg ? p->Ah : p->AH;
    for (int l = 0;; ++l) {
        Level &L = p->lev[l];
        build_split(pool, L.A, stream_colour(o.seed, 1 + l), want32, L.sp, s);
        L.l1 = row_l1(pool, L.A, s);
        if (L.A.n <= o.coarse_size || l + 1 >= maxl) break;
        DCSR Ac;
        if (!coarsen(pool, L, o.theta, stream_pmis(o.seed, l), Ac, s, o.interp_trunc / 1000.0, o.interp_pmax,
                     o.interp_cc))
            break;
        p->lev.emplace_back();
        p->lev[l + 1].A = Ac;
    }
    Level &Lc = p->lev.back();
    p->nc = Lc.A.n;
    coarse_inverse(pool, Lc.A, &p->d_cinv, s);
    // FP32 copies and per-level vectors
    for (size_t l = 0; l < p->lev.size(); ++l) {
        Level &L = p->lev[l];
        const int64_t n = std::max<int64_t>(L.A.n, 1);
        L.b = pool.get<double>(n);
        L.x = pool.get<double>(n);
        L.r = pool.get<double>(n);
        if (want32) {
            L.b32 = pool.get<float>(n);
            L.x32 = pool.get<float>(n);
            L.r32 = pool.get<float>(n);
            if (l > 0) dcsr_make32(pool, L.A, s);
            else L.A.val32 = amg ? p->Ah.val32 : p->AH.val32;
            L.l132 = pool.get<float>(n);
            to32(L.l1, L.l132, L.A.n, s);
            if (L.P.n) {
                dcsr_make32(pool, L.P, s);
                dcsr_make32(pool, L.R, s);
            }
        }
    }
    if (want32) {
        p->d_cinv32 = pool.get<float>(std::max<int64_t>(p->nc * p->nc, 1));
        to32(p->d_cinv, p->d_cinv32, p->nc * p->nc, s);
    }
    if (!p->aux_stream) PK_CUDA(cudaStreamCreateWithFlags(&p->aux_stream, cudaStreamNonBlocking));
    if (!p->cap_stream) PK_CUDA(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
    if (!p->ev_fork) PK_CUDA(cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming));
    if (!p->ev_join) PK_CUDA(cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming));
    ensure_work(p, 1);
    // colour offsets on the device and the grid-barrier state of the persistent smoother
    p->d_fine_off = pool.get<int64_t>(p->fine.off.size());
    PK_CUDA(cudaMemcpyAsync(p->d_fine_off, p->fine.off.data(), sizeof(int64_t) * p->fine.off.size(),
                            cudaMemcpyHostToDevice, s));
    p->d_bar = pool.get<unsigned>(2);
    p->d_bar_err = pool.get<int>(1);
    PK_CUDA(cudaMemsetAsync(p->d_bar, 0, sizeof(unsigned) * 2, s));
    PK_CUDA(cudaMemsetAsync(p->d_bar_err, 0, sizeof(int), s));
    PK_CUDA(cudaStreamSynchronize(s));
    p->have_setup = true;
    autotune(p, s);
}

void ensure_work(pkasp_problem *p, int ncols) {
    if (p->work_cols >= ncols) return;
    p->work_pool.free_all();
    const int64_t n = std::max<int64_t>(p->nh, 1) * ncols;
    DevPool &w = p->work_pool;
    p->w_r = w.get<double>(n);
    p->w_z = w.get<double>(n);
    p->w_p = w.get<double>(n);
    p->w_q = w.get<double>(n);
    p->w_x = w.get<double>(n);
    p->w_b = w.get<double>(n);
    p->w_zs = w.get<double>(n);
    p->w_t = w.get<double>(n);
    p->w_rr = w.get<double>(n);
    p->w_zs32 = w.get<float>(n);
    p->w_t32 = w.get<float>(n);
    p->w_rr32 = w.get<float>(n);
    p->d_partials = w.get<double>((size_t)kRedGrid * 4 * PKASP_MAX_COLS);
    p->d_counter = w.get<unsigned>(4);
    PK_CUDA(cudaMemset(p->d_counter, 0, sizeof(unsigned) * 4));
    p->d_state = w.get<PcgState>(1);
    p->hist_cap = 0;
    p->d_hist = nullptr;
    p->work_cols = ncols;
    if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    p->graph_exec = nullptr;
    p->graph = nullptr;
}

// ---------------------------------------------------------------------------------
// public pieces
// ---------------------------------------------------------------------------------
void spmv_fine(pkasp_problem *p, const double *x, double *y, cudaStream_t s) {
    if (p->spmv_tpr == 0) {
        const DSell &S = p->Asell;
        k_sell_spmv<double, double, double, double><<<elem_grid(p->nh), kBlock, 0, s>>>(
            p->nh, S.sptr, S.swidth, S.col, S.val, x, y);
        PK_LAUNCH();
        return;
    }
    spmv<double, double>(p->Ah, x, y, p->spmv_tpr, s);
}

void apply_prec(pkasp_problem *p, const double *r, double *z, cudaStream_t s) {
    if (p->opt.precond_precision == PKASP_PREC_FP32) precondition<float>(p, r, z, s);
    else precondition<double>(p, r, z, s);
}

void apply_smoother(pkasp_problem *p, const double *r, double *z, cudaStream_t s) {
    if (p->opt.precond_precision == PKASP_PREC_FP32) {
        smoother<float>(p, r, p->w_zs32, s);
        k_copy_to<float><<<elem_grid(p->nh), kBlock, 0, s>>>(p->nh, p->w_zs32, z);
    } else {
        smoother<double>(p, r, z, s);
    }
    PK_LAUNCH();
}

void apply_vcycle(pkasp_problem *p, const double *b, double *x, cudaStream_t s) {
    Level &L0 = p->lev[0];
    const int64_t n = L0.A.n;
    if (p->opt.precond_precision == PKASP_PREC_FP32) {
        to_pt<float>(b, L0.b32, n, s);
        vcycle<float>(p, 0, s);
        k_copy_to<float><<<elem_grid(n), kBlock, 0, s>>>(n, L0.x32, x);
    } else {
        PK_CUDA(cudaMemcpyAsync(L0.b, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        vcycle<double>(p, 0, s);
        PK_CUDA(cudaMemcpyAsync(x, L0.x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    }
    PK_LAUNCH();
}

namespace {


void enqueue_init(pkasp_problem *p, const double *b, double *x, cudaStream_t s) {
    const int tpr = p->spmv_tpr;
    const RowOp A = fine_op(p);
    const unsigned fg = fine_grid(p);
    PK_FMT_SWITCH(tpr, (k_residual_fine<TPR><<<fg, kBlock, 0, s>>>(p->nh, A, b, x, p->w_r)));
    PK_LAUNCH();
    k_init_norm<<<kRedGrid, kBlock, 0, s>>>(p->nh, p->w_r, p->d_state, p->d_partials, p->d_counter, p->d_hist);
    PK_LAUNCH();
    apply_prec(p, p->w_r, p->w_z, s);
    k_start<<<kRedGrid, kBlock, 0, s>>>(p->nh, p->w_r, p->w_z, p->w_p, p->d_state, p->d_partials,
                                              p->d_counter);
    PK_LAUNCH();
}


void enqueue_iteration(pkasp_problem *p, double *x, cudaStream_t s) {
    const int tpr = p->spmv_tpr;
    const RowOp A = fine_op(p);
    const unsigned fg = fine_grid(p);
    PK_FMT_SWITCH(tpr, (k_spmv_q<TPR><<<fg, kBlock, 0, s>>>(p->nh, A, p->w_p, p->w_q, p->d_state)));
    PK_LAUNCH();
    k_pq_alpha<<<kRedGrid, kBlock, 0, s>>>(p->nh, p->w_p, p->w_q, p->d_state, p->d_partials, p->d_counter);
    PK_LAUNCH();
    k_update_xr<<<kRedGrid, kBlock, 0, s>>>(p->nh, x, p->w_r, p->w_p, p->w_q, p->d_state, p->d_partials,
                                                  p->d_counter, p->d_hist);
    PK_LAUNCH();
    const int flex = (p->opt.flexible || p->opt.precond_precision == PKASP_PREC_FP32) ? 1 : 0;
    if (p->opt.mode == PKASP_MODE_ADDITIVE) {
        // additive preconditioner up to z_s and w; z = z_s + Pi w inside the beta kernel
        const PiCodes &pc = p->pic;
        if (p->opt.precond_precision == PKASP_PREC_FP32) {
            precondition<float>(p, p->w_r, p->w_z, s, false);
            k_prolong_beta<float><<<kRedGrid, kBlock, 0, s>>>(
                p->nh, (const int4 *)pc.ell_col, pc.ell_code, pc.tab32, p->lev[0].x32, p->w_zs32, p->w_r, p->w_q,
                p->w_z, flex, p->d_state, p->d_partials, p->d_counter);
        } else {
            precondition<double>(p, p->w_r, p->w_z, s, false);
            k_prolong_beta<double><<<kRedGrid, kBlock, 0, s>>>(
                p->nh, (const int4 *)pc.ell_col, pc.ell_code, pc.tab, p->lev[0].x, p->w_zs, p->w_r, p->w_q,
                p->w_z, flex, p->d_state, p->d_partials, p->d_counter);
        }
    } else {
        apply_prec(p, p->w_r, p->w_z, s);
        k_beta<<<kRedGrid, kBlock, 0, s>>>(p->nh, p->w_r, p->w_z, p->w_q, flex, p->d_state, p->d_partials,
                                                 p->d_counter);
    }
    PK_LAUNCH();
    k_update_p<<<kRedGrid, kBlock, 0, s>>>(p->nh, p->w_z, p->w_p, p->d_state);
    PK_LAUNCH();
}

void enqueue_final(pkasp_problem *p, const double *b, const double *x, cudaStream_t s) {
    const int tpr = p->spmv_tpr;
    const RowOp A = fine_op(p);
    const unsigned fg = fine_grid(p);
    // the residual goes to a work vector the iteration no longer needs
    PK_FMT_SWITCH(tpr, (k_residual_fine<TPR><<<fg, kBlock, 0, s>>>(p->nh, A, b, x, p->w_t)));
    PK_LAUNCH();
    k_true_norm<<<kRedGrid, kBlock, 0, s>>>(p->nh, p->w_t, p->d_state, p->d_partials, p->d_counter);
    PK_LAUNCH();
}

void build_graph(pkasp_problem *p, const double *b, double *x) {
    if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    p->graph_exec = nullptr;
    p->graph = nullptr;
    cudaStream_t cs = p->cap_stream;
    cudaGraph_t g, gi, gf;
    PK_CUDA(cudaGraphCreate(&g, 0));
    // init part
    PK_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    long long c0 = launch_count();
    enqueue_init(p, b, x, cs);
    p->g_init = launch_count() - c0;
    PK_CUDA(cudaStreamEndCapture(cs, &gi));
    cudaGraphNode_t ni, nc, nf;
    PK_CUDA(cudaGraphAddChildGraphNode(&ni, g, nullptr, 0, gi));
    // while loop over iterations
    cudaGraphConditionalHandle h;
    PK_CUDA(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    PK_CUDA(cudaGraphAddNode(&nc, g, &ni, nullptr, 1, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    PK_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    c0 = launch_count();
    enqueue_iteration(p, x, cs);
    k_loop_control<<<1, 32, 0, cs>>>(p->d_state, h);
    PK_LAUNCH();
    p->g_body = launch_count() - c0;
    PK_CUDA(cudaStreamEndCapture(cs, &body));
    // final true residual
    PK_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    c0 = launch_count();
    enqueue_final(p, b, x, cs);
    p->g_final = launch_count() - c0;
    PK_CUDA(cudaStreamEndCapture(cs, &gf));
    PK_CUDA(cudaGraphAddChildGraphNode(&nf, g, &nc, 1, gf));
    PK_CUDA(cudaGraphInstantiate(&p->graph_exec, g, 0));
    cudaGraphDestroy(gi);
    cudaGraphDestroy(gf);
    p->graph = g;
}

}  // namespace

int solve_device(pkasp_problem *p, const double *b, double *x, int ncols, int64_t ld, pkasp_stats *st,
                 cudaStream_t s) {
    if (p->opt.krylov == PKASP_KRYLOV_FGMRES) {
        if (ncols != 1 || ld != 1) fail(PKASP_EINVAL, "FGMRES solves one right-hand side per call");
        return solve_gmres(p, b, x, st, s);
    }
    if (ncols != 1 || ld != 1) return solve_batched(p, b, x, ncols, ld, st, s);
    ensure_work(p, 1);
    const int cap = (st && st->hist_cap > 0) ? st->hist_cap : 1;
    if (cap > p->hist_cap) {
        p->d_hist = p->work_pool.get<double>(cap);
        p->hist_cap = cap;
        if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
        if (p->graph) cudaGraphDestroy(p->graph);
        p->graph_exec = nullptr;
        p->graph = nullptr;
    }
    cudaEvent_t e0, e1;
    PK_CUDA(cudaEventCreate(&e0));
    PK_CUDA(cudaEventCreate(&e1));
    k_state_reset<<<1, 32, 0, s>>>(p->d_state, p->opt.tol, p->opt.max_iter, p->hist_cap);
    PK_LAUNCH();
    PK_CUDA(cudaEventRecord(e0, s));
    const bool use_graph = p->opt.use_graph != 0;
    if (use_graph && (!p->graph_exec || p->graph_key_b != b || p->graph_key_x != x)) {
        PK_CUDA(cudaStreamSynchronize(s));
        build_graph(p, b, x);
        p->graph_key_b = b;
        p->graph_key_x = x;
    }
    PcgState hs;
    int restarts = 0;
    long long launches = 1;  // the state reset
    const long long eager0 = launch_count();
    for (;;) {
        if (use_graph) {
            PK_CUDA(cudaGraphLaunch(p->graph_exec, s));
        } else {
            enqueue_init(p, b, x, s);
            for (int it = 0; it <= p->opt.max_iter + 1; ++it) {
                enqueue_iteration(p, x, s);
                int ad = 0;
                PK_CUDA(cudaMemcpyAsync(&ad, &p->d_state->all_done, sizeof(int), cudaMemcpyDeviceToHost, s));
                PK_CUDA(cudaStreamSynchronize(s));
                if (ad) break;
            }
            enqueue_final(p, b, x, s);
        }
        PK_CUDA(cudaMemcpyAsync(&hs, p->d_state, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
        PK_CUDA(cudaStreamSynchronize(s));
        if (use_graph) launches += p->g_init + (long long)hs.loops * p->g_body + p->g_final;
        const bool conv = hs.status[0] == PKASP_OK;
        if (conv && hs.r0[0] > 0 && hs.tnorm[0] > p->opt.tol * hs.r0[0] && restarts == 0 &&
            hs.iter[0] < p->opt.max_iter) {
            ++restarts;
            k_state_restart<<<1, 32, 0, s>>>(p->d_state);
            PK_LAUNCH();
            continue;
        }
        break;
    }
    PK_CUDA(cudaEventRecord(e1, s));
    PK_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    barrier_status(p, s);
    int status = hs.status[0];
    if (status == ST_RUN) status = PKASP_ENOTCONV;
    if (st) {
        st->ncols = 1;
        st->iters[0] = hs.iter[0];
        st->status[0] = status;
        st->true_rel[0] = hs.r0[0] > 0 ? hs.tnorm[0] / hs.r0[0] : 0.0;
        st->restarts = restarts;
        st->solve_ms = ms;
        st->kernel_launches = use_graph ? launches + restarts : 1 + (launch_count() - eager0);
        st->hist_len = std::min(hs.iter[0] + 1, st->hist_cap);
        if (st->hist_host && st->hist_len > 0)
            PK_CUDA(cudaMemcpy(st->hist_host, p->d_hist, sizeof(double) * st->hist_len, cudaMemcpyDeviceToHost));
    }
    return status;
}

void check_barrier(pkasp_problem *p, cudaStream_t s) { barrier_status(p, s); }

namespace {
// Gather-rate probe: random 8-byte gathers x[idx[j]] driven by a streamed index array,
// eight independent gathers in flight per thread (the access pattern of a sparse row's
// columns without its locality). Not used by a solve.
__global__ void __launch_bounds__(kBlock) k_gather_probe(int64_t m, const int32_t *__restrict__ idx,
                                                         const double *__restrict__ x, double *__restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
    double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = t; i + 7 * st < m; i += 8 * st) {
        int c[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) c[k] = ldst(&idx[i + k * st]);
#pragma unroll
        for (int k = 0; k < 8; ++k) s[k] += x[c[k]];
    }
    double z = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) z += s[k];
    if (z == -1.0) out[0] = z;  // keeps the loads; x is never -1 in a probe
}

// idx[j] = a SplitMix64 hash of j modulo n (the probe's random columns)
__global__ void k_probe_indices(int64_t m, int64_t n, int32_t *__restrict__ idx) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    uint64_t z = 0x5EEDull + ((uint64_t)j + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    idx[j] = (int32_t)(z % (uint64_t)n);
}

}  // namespace

float time_kernel(pkasp_problem *p, int which, int reps, cudaStream_t s) {
    if (reps < 1) reps = 1;
    if (which >= 4 && which <= 6) return time_batched(p, which, reps, s);
    cudaEvent_t e0, e1;
    PK_CUDA(cudaEventCreate(&e0));
    PK_CUDA(cudaEventCreate(&e1));
    int32_t *probe_idx = nullptr;
    const int64_t probe_m = std::min<int64_t>(64ll << 20, 8 * std::max<int64_t>(p->nh, 1));
    if (which == 8) {
        PK_CUDA(cudaMallocAsync((void **)&probe_idx, sizeof(int32_t) * probe_m, s));
        k_probe_indices<<<(unsigned)((probe_m + kBlock - 1) / kBlock), kBlock, 0, s>>>(probe_m, p->nh, probe_idx);
        PK_LAUNCH();
    }
    // inputs: r = f_h in w_r, p-vector = f_h
    PK_CUDA(cudaMemcpyAsync(p->w_r, p->d_b, sizeof(double) * p->nh, cudaMemcpyDeviceToDevice, s));
    PK_CUDA(cudaMemcpyAsync(p->w_p, p->d_b, sizeof(double) * p->nh, cudaMemcpyDeviceToDevice, s));
    auto once = [&]() {
        switch (which) {
            case 0: spmv_fine(p, p->w_p, p->w_q, s); break;
            case 1: {
                if (p->opt.precond_precision == PKASP_PREC_FP32) smoother<float>(p, p->w_r, p->w_zs32, s);
                else smoother<double>(p, p->w_r, p->w_zs, s);
                break;
            }
            case 2: {
                if (p->opt.precond_precision == PKASP_PREC_FP32) restrict_vcycle<float>(p, p->w_r, s);
                else restrict_vcycle<double>(p, p->w_r, s);
                break;
            }
            case 7: {
                // the fine smoother's loads in two dependency-free passes (lower parts, then
                // upper parts) with the smoother's lanes per row
                const DSplit &sp = p->fine;
                const int t = (p->fine_tpr == 8 || p->fine_tpr == 16) ? p->fine_tpr : 4;
                if (p->opt.precond_precision == PKASP_PREC_FP32) {
                    PK_TPR3_SWITCH(t, (k_split_pass<TPR, kBatch, float><<<rows_grid(p->nh, TPR), kBlock, 0, s>>>(
                                          p->nh, sp.perm, sp.lptr, sp.lcol, sp.lval32, sp.dinv32, p->w_zs32, p->w_t32)));
                    PK_LAUNCH();
                    PK_TPR3_SWITCH(t, (k_split_pass<TPR, kBatch, float><<<rows_grid(p->nh, TPR), kBlock, 0, s>>>(
                                          p->nh, sp.perm, sp.uptr, sp.ucol, sp.uval32, sp.dinv32, p->w_zs32, p->w_t32)));
                    PK_LAUNCH();
                } else {
                    PK_TPR3_SWITCH(t, (k_split_pass<TPR, kBatch, double><<<rows_grid(p->nh, TPR), kBlock, 0, s>>>(
                                          p->nh, sp.perm, sp.lptr, sp.lcol, sp.lval, sp.dinv, p->w_p, p->w_t)));
                    PK_LAUNCH();
                    PK_TPR3_SWITCH(t, (k_split_pass<TPR, kBatch, double><<<rows_grid(p->nh, TPR), kBlock, 0, s>>>(
                                          p->nh, sp.perm, sp.uptr, sp.ucol, sp.uval, sp.dinv, p->w_p, p->w_t)));
                    PK_LAUNCH();
                }
                break;
            }
            case 8:
                // random 8-byte gathers from an n_h vector (f_h) by a streamed index array
                k_gather_probe<<<kRedGrid * 4, kBlock, 0, s>>>(probe_m, probe_idx, p->w_p, p->w_t);
                PK_LAUNCH();
                break;
            default: apply_prec(p, p->w_r, p->w_z, s); break;
        }
    };
    for (int i = 0; i < 3; ++i) once();
    PK_CUDA(cudaEventRecord(e0, s));
    for (int i = 0; i < reps; ++i) once();
    PK_CUDA(cudaEventRecord(e1, s));
    PK_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (probe_idx) {
        PK_CUDA(cudaFreeAsync(probe_idx, s));
        PK_CUDA(cudaStreamSynchronize(s));
    }
    // mode 8 reports nanoseconds per gather instead of milliseconds per launch
    if (which == 8) return ms / reps * 1e6f / (float)probe_m;
    return ms / reps;
}

}  // namespace pk
