// stokes.cu -- the Taylor-Hood P_k - P_{k-1} Stokes system of Sec. 5 on the device:
//   F = [A B^T; B 0], A = three copies of the Dirichlet P_k Laplacian A_h (velocity
//   unknowns component-major), B = -div_h (patterns from stokes.cpp, values assembled
//   here), and the block upper
//   triangular preconditioner Q_t = [A B^T; 0 -S]^{-1} of Eq. (5.4) with
//     z_p = -M_p^{-1} r_p   (mp_iters steps of CG with the diagonal of M_p, from zero)
//     z_u = B_aux (r_u - B^T z_p)   (the auxiliary-space preconditioner per component),
//   solved by FGMRES(m) (Sec. 6.3) in one CUDA-graph while loop. The operator kernels
//   take an optional gate (a device flag): the true residual at the end of an FGMRES
//   cycle only runs when the cycle has ended.
#include <algorithm>
#include <cmath>

#include "gmres.cuh"
#include "internal.h"
#include "kernels.cuh"
#include "rowop.cuh"

namespace pk {

struct StokesWork {
    int64_t nh = 0, np = 0, n = 0;
    int mp_iters = 10;
    DevPool pool;
    DCSR B, BT, M;
    double *mdiag = nullptr;
    // preconditioner work
    double *t = nullptr, *rr = nullptr, *zz = nullptr, *pp = nullptr, *qq = nullptr, *xp = nullptr;
    double *scal = nullptr;  // rho, alpha, beta of the inner CG
    // FGMRES
    int m = 0;
    double *V = nullptr, *Z = nullptr, *w = nullptr, *vin = nullptr, *zout = nullptr, *y = nullptr;
    double *H = nullptr, *g = nullptr, *cs = nullptr, *sn = nullptr, *yv = nullptr, *hc = nullptr, *part = nullptr;
    unsigned *cnt = nullptr;
    GmresState *state = nullptr;
    double *hist = nullptr;
    int hist_cap = 0;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    const void *key_b = nullptr;
    void *key_x = nullptr;
    long long g_init = 0, g_body = 0;
};

namespace {

__device__ __forceinline__ bool gated_off(const int *gate) { return gate != nullptr && *gate == 0; }

// first position in col[lo, hi) (ascending) holding a value >= j
__device__ __forceinline__ int64_t ks_lower_bound(const int32_t *col, int64_t lo, int64_t hi, int32_t j) {
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (col[mid] < j) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Values of B = -div_h and M_p, one warp per pressure row q: the row's elements in
// ascending order (incidence iptr/ient), per element its geometry (gradients of the
// barycentric coordinates and volume), then
//   B[q][(c, j)] += -|T| sum_a (grad lambda_a)_c R[a][m][n],  j = elem_dof[t][n],
//   M[q][r']     +=  |T| Mr[m][r],                            r' = elem_p[t][r],
// q being local pressure node m of element t. Within one element every (n, c) and every
// r hits a different entry, so the lanes share an element and the elements follow one
// another (ascending element order per entry, as on the host).
__global__ void ks_assemble_blocks(int64_t np, int64_t nh, int nu, int npl, const double *__restrict__ xyz,
                                   const int32_t *__restrict__ tets, const int32_t *__restrict__ elem_dof,
                                   const int32_t *__restrict__ elem_p, const double *__restrict__ R,
                                   const double *__restrict__ Mr, const int64_t *__restrict__ iptr,
                                   const int64_t *__restrict__ ient, const int64_t *__restrict__ bptr,
                                   const int32_t *__restrict__ bcol, double *__restrict__ bval,
                                   const int64_t *__restrict__ mptr, const int32_t *__restrict__ mcol,
                                   double *__restrict__ mval) {
    const int lane = threadIdx.x & 31;
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= np) return;  // whole warp
    const int64_t b0 = bptr[q], b1 = bptr[q + 1], m0 = mptr[q], m1 = mptr[q + 1];
    for (int64_t x = iptr[q]; x < iptr[q + 1]; ++x) {
        const int64_t t = ient[x] / 64;
        const int m = (int)(ient[x] % 64);
        double X[12];
        for (int v = 0; v < 4; ++v)
            for (int c = 0; c < 3; ++c) X[3 * v + c] = xyz[3 * (int64_t)tets[4 * t + v] + c];
        double J[3][3];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) J[r][c] = X[3 * (c + 1) + r] - X[r];
        const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
        const double inv[3][3] = {{c00 / det, (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det,
                                   (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det},
                                  {c01 / det, (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det,
                                   (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det},
                                  {c02 / det, (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det,
                                   (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det}};
        double g[4][3];
        for (int c = 0; c < 3; ++c) {
            g[1][c] = inv[0][c];
            g[2][c] = inv[1][c];
            g[3][c] = inv[2][c];
            g[0][c] = -(inv[0][c] + inv[1][c] + inv[2][c]);
        }
        const double vol = det / 6.0;
        for (int idx = lane; idx < 3 * nu; idx += 32) {
            const int n = idx / 3, c = idx % 3;
            const int32_t j = elem_dof[t * nu + n];
            if (j < 0) continue;
            double sum = 0.0;
            for (int a = 0; a < 4; ++a) sum += g[a][c] * R[((int64_t)a * npl + m) * nu + n];
            const int32_t col = (int32_t)(c * nh + j);
            const int64_t pos = ks_lower_bound(bcol, b0, b1, col);
            if (pos < b1 && bcol[pos] == col) bval[pos] += -vol * sum;
        }
        for (int r = lane; r < npl; r += 32) {
            const int32_t col = elem_p[t * npl + r];
            const int64_t pos = ks_lower_bound(mcol, m0, m1, col);
            if (pos < m1 && mcol[pos] == col) mval[pos] += vol * Mr[(int64_t)m * npl + r];
        }
        __syncwarp();
    }
}

// one thread per item (no grid-stride loop): blocks to cover n threads
unsigned ks_cover(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + kBlock - 1) / kBlock); }

// B^T values: entry o copies B entry src[o]; diagonal of M_p
__global__ void ks_gather_vals(int64_t n, const int64_t *__restrict__ src, const double *__restrict__ from,
                               double *__restrict__ to) {
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o < n) to[o] = from[src[o]];
}

__global__ void ks_diag(int64_t n, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                        const double *__restrict__ val, double *__restrict__ d) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = 0.0;
    for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e)
        if (col[e] == (int32_t)i) v = val[e];
    d[i] = v;
}

// y_c = A_h x_c for one velocity component
template <int TPR>
__global__ void __launch_bounds__(kBlock) ks_op_u(int64_t n, RowOp A, const double *__restrict__ x,
                                                  double *__restrict__ y, const int *gate) {
    if (gated_off(gate)) return;
    for_rows<TPR>(n, A, x, [&](int64_t row, double s) { y[row] = s; });
}

// y[i] += sum_j T[i][j] x[j] (CSR, one thread per row, entries in column order)
__global__ void ks_add_csr(int64_t n, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                           const double *__restrict__ val, const double *__restrict__ x, double *__restrict__ y,
                           const int *gate) {
    if (gated_off(gate)) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) s += val[e] * x[col[e]];
        y[i] += s;
    }
}

// y = B x_u (8 lanes per pressure row)
__global__ void __launch_bounds__(kBlock) ks_spmv_rows(int64_t n, const int64_t *__restrict__ ptr,
                                                       const int32_t *__restrict__ col,
                                                       const double *__restrict__ val, const double *__restrict__ x,
                                                       double *__restrict__ y, const int *gate) {
    if (gated_off(gate)) return;
    constexpr int TPR = 8;
    const int sub = threadIdx.x & (TPR - 1);
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int rpw = 32 / TPR, sg = (threadIdx.x & 31) / TPR;
    for (int64_t base = warp * rpw; base < n; base += nwarps * rpw) {
        const int64_t row = base + sg;
        const bool ok = row < n;
        const int64_t lo = ok ? ptr[row] : 0, hi = ok ? ptr[row + 1] : 0;
        const double s = row_dot<TPR, double>(lo, hi, sub, col, val, x);
        if (ok && sub == 0) y[row] = s;
    }
}

// ---- inner CG on M_p with the diagonal as preconditioner (device scalars) ----------
// start: r = r_p, z = r / d, p = z, x = 0, rho = (r, z)
__global__ void __launch_bounds__(kBlock) ks_mp_start(int64_t n, const double *__restrict__ rp,
                                                      const double *__restrict__ d, double *rr, double *zz, double *pp,
                                                      double *xp, double *scal, double *partials, unsigned *counter) {
    double part = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double r = rp[i], z = r / d[i];
        rr[i] = r;
        zz[i] = z;
        pp[i] = z;
        xp[i] = 0.0;
        part += r * z;
    }
    double v[1] = {part}, tot[1];
    if (grid_reduce<1>(v, partials, counter, tot) && threadIdx.x == 0) scal[0] = tot[0];
}

// alpha = rho / (p, q) (0 once rho is 0)
__global__ void __launch_bounds__(kBlock) ks_mp_alpha(int64_t n, const double *pp, const double *qq, double *scal,
                                                      double *partials, unsigned *counter) {
    double part = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        part += pp[i] * qq[i];
    double v[1] = {part}, tot[1];
    if (grid_reduce<1>(v, partials, counter, tot) && threadIdx.x == 0)
        scal[1] = scal[0] != 0.0 ? scal[0] / tot[0] : 0.0;
}

// x += alpha p, r -= alpha q, z = r / d; beta = rho_new / rho, rho = rho_new
__global__ void __launch_bounds__(kBlock) ks_mp_update(int64_t n, double *xp, double *rr, double *zz, const double *pp,
                                                       const double *qq, const double *__restrict__ d, double *scal,
                                                       double *partials, unsigned *counter) {
    const double alpha = scal[1];
    double part = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        xp[i] += alpha * pp[i];
        const double r = rr[i] - alpha * qq[i];
        const double z = r / d[i];
        rr[i] = r;
        zz[i] = z;
        part += r * z;
    }
    double v[1] = {part}, tot[1];
    if (grid_reduce<1>(v, partials, counter, tot) && threadIdx.x == 0) {
        scal[2] = scal[0] != 0.0 ? tot[0] / scal[0] : 0.0;
        scal[0] = tot[0];
    }
}

__global__ void ks_mp_p(int64_t n, const double *zz, double *pp, const double *scal) {
    const double beta = scal[2];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        pp[i] = zz[i] + beta * pp[i];
}

// z_p = -x; t = r_u - B^T z_p (one thread per velocity row)
__global__ void ks_neg(int64_t n, const double *x, double *z) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        z[i] = -x[i];
}
__global__ void ks_tsub(int64_t n, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                        const double *__restrict__ val, const double *__restrict__ zp, const double *__restrict__ ru,
                        double *__restrict__ t) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) s += val[e] * zp[col[e]];
        t[i] = ru[i] - s;
    }
}

unsigned grid_for(int64_t n, int per_thread_rows = 1) {
    const int64_t t = (n + per_thread_rows - 1) / per_thread_rows;
    return (unsigned)std::min<int64_t>(152 * 8, std::max<int64_t>(1, (t + kBlock - 1) / kBlock));
}

// y = F x (gate: run only when the flag is set)
void op(pkasp_problem *p, const double *x, double *y, const int *gate, cudaStream_t s) {
    StokesWork &S = *p->st;
    const int64_t nh = S.nh, nu = 3 * nh;
    const RowOp A = fine_op(p);
    for (int c = 0; c < 3; ++c) {
        PK_FMT_SWITCH(p->spmv_tpr, (ks_op_u<TPR><<<fine_grid(p), kBlock, 0, s>>>(nh, A, x + c * nh, y + c * nh,
                                                                                   gate)));
        PK_LAUNCH();
    }
    ks_add_csr<<<grid_for(nu), kBlock, 0, s>>>(nu, S.BT.ptr, S.BT.col, S.BT.val, x + nu, y, gate);
    PK_LAUNCH();
    ks_spmv_rows<<<kRedGrid, kBlock, 0, s>>>(S.np, S.B.ptr, S.B.col, S.B.val, x, y + nu, gate);
    PK_LAUNCH();
}

// z = Q_t r
void prec(pkasp_problem *p, const double *r, double *z, cudaStream_t s) {
    StokesWork &S = *p->st;
    const int64_t nh = S.nh, nu = 3 * nh, np = S.np;
    ks_mp_start<<<kRedGrid, kBlock, 0, s>>>(np, r + nu, S.mdiag, S.rr, S.zz, S.pp, S.xp, S.scal, p->d_partials,
                                            p->d_counter);
    PK_LAUNCH();
    for (int it = 0; it < S.mp_iters; ++it) {
        ks_spmv_rows<<<kRedGrid, kBlock, 0, s>>>(np, S.M.ptr, S.M.col, S.M.val, S.pp, S.qq, nullptr);
        PK_LAUNCH();
        ks_mp_alpha<<<kRedGrid, kBlock, 0, s>>>(np, S.pp, S.qq, S.scal, p->d_partials, p->d_counter);
        PK_LAUNCH();
        ks_mp_update<<<kRedGrid, kBlock, 0, s>>>(np, S.xp, S.rr, S.zz, S.pp, S.qq, S.mdiag, S.scal, p->d_partials,
                                                 p->d_counter);
        PK_LAUNCH();
        ks_mp_p<<<grid_for(np), kBlock, 0, s>>>(np, S.zz, S.pp, S.scal);
        PK_LAUNCH();
    }
    ks_neg<<<grid_for(np), kBlock, 0, s>>>(np, S.xp, z + nu);
    PK_LAUNCH();
    ks_tsub<<<grid_for(nu), kBlock, 0, s>>>(nu, S.BT.ptr, S.BT.col, S.BT.val, z + nu, r, S.t);
    PK_LAUNCH();
    for (int c = 0; c < 3; ++c) apply_prec(p, S.t + c * nh, z + c * nh, s);
}

struct StokesGmres {
    static void init(pkasp_problem *p, const double *b, double *x, cudaStream_t s) {
        StokesWork &S = *p->st;
        op(p, x, S.y, nullptr, s);
        kg_residual_y<<<kRedGrid, kBlock, 0, s>>>(S.n, b, S.y, S.V, S.state, S.g, p->d_partials, p->d_counter, S.hist,
                                                  1);
        PK_LAUNCH();
        kg_scale_v0<<<elem_blocks(S.n), kBlock, 0, s>>>(S.n, S.V, S.vin, S.state);
        PK_LAUNCH();
    }
    static void step(pkasp_problem *p, const double *b, double *x, cudaStream_t s) {
        StokesWork &S = *p->st;
        const int64_t n = S.n;
        prec(p, S.vin, S.zout, s);
        kg_store_z<<<elem_blocks(n), kBlock, 0, s>>>(n, S.zout, S.Z, S.state);
        PK_LAUNCH();
        op(p, S.zout, S.w, nullptr, s);
        const dim3 dg(kDotChunks, S.m + 1);
        for (int pass = 0; pass < 2; ++pass) {
            kg_dots<<<dg, kBlock, 0, s>>>(n, S.V, S.w, S.state, S.part, S.cnt, S.hc, S.H, pass);
            PK_LAUNCH();
            kg_axpy<<<kRedGrid, kBlock, 0, s>>>(n, S.V, S.w, S.state, S.hc, S.H, p->d_partials, p->d_counter, pass);
            PK_LAUNCH();
        }
        kg_scale_next<<<elem_blocks(n), kBlock, 0, s>>>(n, S.V, S.w, S.vin, S.state);
        PK_LAUNCH();
        kg_givens<<<1, 32, 0, s>>>(S.state, S.H, S.cs, S.sn, S.g, S.hist);
        PK_LAUNCH();
        kg_backsolve<<<1, 32, 0, s>>>(S.state, S.H, S.g, S.yv);
        PK_LAUNCH();
        kg_update_x<<<elem_blocks(n), kBlock, 0, s>>>(n, x, S.Z, S.yv, S.state);
        PK_LAUNCH();
        op(p, x, S.y, &S.state->cycle_end, s);
        kg_residual_y<<<kRedGrid, kBlock, 0, s>>>(n, b, S.y, S.V, S.state, S.g, p->d_partials, p->d_counter, S.hist,
                                                  0);
        PK_LAUNCH();
        kg_scale_v0<<<elem_blocks(n), kBlock, 0, s>>>(n, S.V, S.vin, S.state);
        PK_LAUNCH();
    }
    static void build_graph(pkasp_problem *p, const double *b, double *x) {
        StokesWork &S = *p->st;
        if (S.exec) cudaGraphExecDestroy(S.exec);
        if (S.graph) cudaGraphDestroy(S.graph);
        S.exec = nullptr;
        S.graph = nullptr;
        cudaStream_t cs = p->cap_stream;
        cudaGraph_t g, gi;
        PK_CUDA(cudaGraphCreate(&g, 0));
        PK_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        long long c0 = launch_count();
        init(p, b, x, cs);
        S.g_init = launch_count() - c0;
        PK_CUDA(cudaStreamEndCapture(cs, &gi));
        cudaGraphNode_t ni, nc;
        PK_CUDA(cudaGraphAddChildGraphNode(&ni, g, nullptr, 0, gi));
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
        step(p, b, x, cs);
        kg_loop_control<<<1, 32, 0, cs>>>(S.state, h);
        PK_LAUNCH();
        S.g_body = launch_count() - c0;
        PK_CUDA(cudaStreamEndCapture(cs, &body));
        PK_CUDA(cudaGraphInstantiate(&S.exec, g, 0));
        cudaGraphDestroy(gi);
        S.graph = g;
        S.key_b = b;
        S.key_x = x;
    }
};

void ensure_fgmres(StokesWork &S, int m, int hist_cap) {
    if (S.m == m && S.V && S.hist_cap >= hist_cap) return;
    if (S.exec) cudaGraphExecDestroy(S.exec);
    if (S.graph) cudaGraphDestroy(S.graph);
    S.exec = nullptr;
    S.graph = nullptr;
    // the FGMRES arrays live in their own pool so that a new m keeps the operators
    static_assert(sizeof(double) == 8, "");
    DevPool &w = S.pool;
    const int64_t n = std::max<int64_t>(S.n, 1);
    S.V = w.get<double>((size_t)n * (m + 1));
    S.Z = w.get<double>((size_t)n * m);
    S.w = w.get<double>(n);
    S.vin = w.get<double>(n);
    S.zout = w.get<double>(n);
    S.y = w.get<double>(n);
    S.H = w.get<double>((size_t)(m + 1) * m);
    S.g = w.get<double>(m + 1);
    S.cs = w.get<double>(m);
    S.sn = w.get<double>(m);
    S.yv = w.get<double>(m);
    S.hc = w.get<double>(m + 1);
    S.part = w.get<double>((size_t)kDotChunks * (m + 1));
    S.cnt = w.get<unsigned>(m + 1);
    PK_CUDA(cudaMemset(S.cnt, 0, sizeof(unsigned) * (m + 1)));
    S.state = w.get<GmresState>(1);
    S.hist = w.get<double>(std::max(hist_cap, 1));
    S.hist_cap = std::max(hist_cap, 1);
    S.m = m;
}

}  // namespace

void stokes_free(pkasp_problem *p) {
    if (!p->st) return;
    StokesWork &S = *p->st;
    if (S.exec) cudaGraphExecDestroy(S.exec);
    if (S.graph) cudaGraphDestroy(S.graph);
    S.pool.free_all();
    delete p->st;
    p->st = nullptr;
}

void stokes_setup(pkasp_problem *p, int mp_iters, cudaStream_t s) {
    if (p->k < 2) fail(PKASP_EINVAL, "Taylor-Hood elements need k >= 2");
    if (!p->have_setup) fail(PKASP_ESTATE, "pkasp_setup (the velocity preconditioner) must come first");
    if (mp_iters < 1 || mp_iters > 1000) fail(PKASP_EINVAL, "mp_iters must be 1..1000");
    stokes_free(p);
    // patterns and reference tensors on the host (like the A_h pattern), values on the device
    StokesPattern P;
    stokes_patterns(p->k, p->nv, p->nt, p->xyz.data(), p->tets.data(), p->nh, p->elem_dof.data(), P);
    const int64_t np = P.np;
    p->st = new StokesWork();
    StokesWork &S = *p->st;
    S.nh = p->nh;
    S.np = np;
    S.n = 3 * p->nh + np;
    S.mp_iters = mp_iters;
    dcsr_upload(S.pool, S.B, P.B, s);  // values zeroed (pattern only)
    dcsr_upload(S.pool, S.BT, P.BT, s);
    dcsr_upload(S.pool, S.M, P.M, s);
    {
        DevPool tmp;
        try {
            auto up = [&](const auto &v) {
                using T = typename std::decay<decltype(v[0])>::type;
                T *d = tmp.get<T>(std::max<size_t>(v.size(), 1));
                if (!v.empty()) PK_CUDA(cudaMemcpyAsync(d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, s));
                return d;
            };
            const int32_t *d_elem_p = up(P.elem_p);
            const double *d_R = up(P.R);
            const double *d_Mr = up(P.Mr);
            const int64_t *d_iptr = up(P.iptr);
            const int64_t *d_ient = up(P.ient);
            const int64_t *d_src = up(P.bt_src);
            if (np > 0) {
                ks_assemble_blocks<<<ks_cover(np * 32), kBlock, 0, s>>>(
                    np, p->nh, P.nu, P.npl, p->d_xyz, p->d_tets, p->d_elem_dof, d_elem_p, d_R, d_Mr, d_iptr, d_ient,
                    S.B.ptr, S.B.col, S.B.val, S.M.ptr, S.M.col, S.M.val);
                PK_LAUNCH();
            }
            if (S.BT.nnz > 0) {
                ks_gather_vals<<<ks_cover(S.BT.nnz), kBlock, 0, s>>>(S.BT.nnz, d_src, S.B.val, S.BT.val);
                PK_LAUNCH();
            }
            S.mdiag = S.pool.get<double>(std::max<int64_t>(np, 1));
            if (np > 0) {
                ks_diag<<<ks_cover(np), kBlock, 0, s>>>(np, S.M.ptr, S.M.col, S.M.val, S.mdiag);
                PK_LAUNCH();
            }
            PK_CUDA(cudaStreamSynchronize(s));
        } catch (...) {
            cudaStreamSynchronize(s);
            tmp.free_all();
            throw;
        }
        tmp.free_all();
    }
    const int64_t nu = std::max<int64_t>(3 * p->nh, 1), npp = std::max<int64_t>(np, 1);
    S.t = S.pool.get<double>(nu);
    S.rr = S.pool.get<double>(npp);
    S.zz = S.pool.get<double>(npp);
    S.pp = S.pool.get<double>(npp);
    S.qq = S.pool.get<double>(npp);
    S.xp = S.pool.get<double>(npp);
    S.scal = S.pool.get<double>(4);
    PK_CUDA(cudaStreamSynchronize(s));
}

const DCSR *stokes_matrix(const pkasp_problem *p, int which) {
    if (!p->st) return nullptr;
    return which == -1 ? &p->st->B : which == -2 ? &p->st->BT : which == -3 ? &p->st->M : nullptr;
}

void stokes_sizes(const pkasp_problem *p, int64_t *out5) {
    const StokesWork &S = *p->st;
    out5[0] = S.nh;
    out5[1] = S.np;
    out5[2] = S.n;
    out5[3] = S.B.nnz;
    out5[4] = S.M.nnz;
}

void stokes_apply(pkasp_problem *p, const double *x, double *y, cudaStream_t s) {
    if (!p->st) fail(PKASP_ESTATE, "pkasp_stokes_setup first");
    op(p, x, y, nullptr, s);
}

void stokes_prec(pkasp_problem *p, const double *r, double *z, cudaStream_t s) {
    if (!p->st) fail(PKASP_ESTATE, "pkasp_stokes_setup first");
    prec(p, r, z, s);
}

int stokes_solve(pkasp_problem *p, const double *b, double *x, pkasp_stats *st, cudaStream_t s) {
    if (!p->st) fail(PKASP_ESTATE, "pkasp_stokes_setup first");
    StokesWork &S = *p->st;
    ensure_work(p, 1);
    const int m = std::max(1, std::min(p->opt.restart, 256));
    const int cap = (st && st->hist_cap > 0) ? st->hist_cap : 1;
    ensure_fgmres(S, m, cap);
    kg_state_reset<<<1, 32, 0, s>>>(S.state, m, p->opt.tol, p->opt.max_iter, S.hist_cap);
    PK_LAUNCH();
    cudaEvent_t e0, e1;
    PK_CUDA(cudaEventCreate(&e0));
    PK_CUDA(cudaEventCreate(&e1));
    PK_CUDA(cudaEventRecord(e0, s));
    const bool use_graph = p->opt.use_graph != 0;
    if (use_graph && (!S.exec || S.key_b != b || S.key_x != x)) {
        PK_CUDA(cudaStreamSynchronize(s));
        StokesGmres::build_graph(p, b, x);
    }
    const long long eager0 = launch_count();
    if (use_graph) {
        PK_CUDA(cudaGraphLaunch(S.exec, s));
    } else {
        StokesGmres::init(p, b, x, s);
        for (int pass = 0; pass < p->opt.max_iter + p->opt.max_iter / m + 4; ++pass) {
            int done = 0;
            PK_CUDA(cudaMemcpyAsync(&done, &S.state->done, sizeof(int), cudaMemcpyDeviceToHost, s));
            PK_CUDA(cudaStreamSynchronize(s));
            if (done) break;
            StokesGmres::step(p, b, x, s);
        }
    }
    PK_CUDA(cudaEventRecord(e1, s));
    GmresState hs;
    PK_CUDA(cudaMemcpyAsync(&hs, S.state, sizeof(GmresState), cudaMemcpyDeviceToHost, s));
    PK_CUDA(cudaEventSynchronize(e1));
    PK_CUDA(cudaStreamSynchronize(s));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    check_barrier(p, s);
    int status = hs.status < 0 ? PKASP_ENOTCONV : hs.status;
    if (!hs.done) status = PKASP_ENOTCONV;
    if (st) {
        st->ncols = 1;
        st->iters[0] = hs.it;
        st->status[0] = status;
        st->true_rel[0] = hs.r0 > 0 ? hs.tnorm / hs.r0 : 0.0;
        st->restarts = std::max(0, hs.cycles - 1);
        st->solve_ms = ms;
        st->kernel_launches = use_graph ? 1 + S.g_init + (long long)hs.loops * S.g_body : 1 + (launch_count() - eager0);
        st->hist_len = std::min(hs.it + 1, st->hist_cap);
        if (st->hist_host && st->hist_len > 0)
            PK_CUDA(cudaMemcpy(st->hist_host, S.hist, sizeof(double) * st->hist_len, cudaMemcpyDeviceToHost));
    }
    return status;
}

}  // namespace pk
