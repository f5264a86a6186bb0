// gmres.cu -- FGMRES(m), the outer iteration of the paper's experiments (Sec. 6.2):
// Saad's flexible GMRES with right preconditioning by the auxiliary-space preconditioner
// (either form), FP64 Arnoldi vectors, classical Gram-Schmidt applied twice per step.
//
// One Arnoldi step: z_j = B v_j (the preconditioner, on fixed buffers vin -> zout),
// w = A z_j (Z[j] = z_j stored), two passes of h = V^T w, w -= V h, h_{j+1,j} = ||w||,
// v_{j+1} = w / h_{j+1,j}, then the Givens update of the small least-squares problem on
// one thread. The end of a cycle (m steps, convergence of the estimate, or max_iter)
// solves the triangular system, updates x += Z y and recomputes the true residual,
// which either stops the solve or starts the next cycle. Those kernels check a device
// flag and return at once when the cycle goes on, so the whole restarted solve is one
// CUDA-graph while loop with a fixed kernel sequence.
//
// Sums are deterministic: fixed grids, block partials added in block order.
#include <algorithm>
#include <cmath>

#include "gmres.cuh"
#include "internal.h"
#include "kernels.cuh"
#include "rowop.cuh"

namespace pk {
namespace {

// V0 = b - A x and its norm. first: the solve's start (r0, hist[0]); otherwise the
// true residual at the end of a cycle (gated by cycle_end), which decides between
// stopping and the next cycle.
template <int TPR>
__global__ void __launch_bounds__(kBlock) kg_residual(int64_t n, RowOp A, const double *__restrict__ b,
                                                      const double *__restrict__ x, double *__restrict__ v0,
                                                      GmresState *st, double *g, double *partials,
                                                      unsigned *counter, double *hist, int first) {
    if (!first && !st->cycle_end) return;  // the same for every block
    double part = 0.0;
    for_rows<TPR>(n, A, x, [&](int64_t row, double s) {
        const double ri = b[row] - s;
        v0[row] = ri;
        part += ri * ri;
    });
    double v[1] = {part}, tot[1];
    if (grid_reduce<1>(v, partials, counter, tot) && threadIdx.x == 0) {
        const double beta = sqrt(tot[0]);
        st->tnorm = beta;
        st->cycle_end = 0;
        if (first) {
            st->r0 = beta;
            if (st->hist_cap > 0) hist[0] = beta;
        }
        if (beta == 0.0 || beta <= st->tol * st->r0) {
            st->done = 1;
            st->status = PKASP_OK;
        } else if (st->it >= st->maxit) {
            st->done = 1;
            st->status = PKASP_ENOTCONV;
        } else {
            st->beta = beta;
            st->j = 0;
            st->new_cycle = 1;
            st->cycles += 1;
            g[0] = beta;
            for (int i = 1; i <= st->m; ++i) g[i] = 0.0;
        }
    }
}

// w = A z_j, Z[j] = z_j
template <int TPR>
__global__ void __launch_bounds__(kBlock) kg_spmv_w(int64_t n, RowOp A, const double *__restrict__ zout,
                                                    double *__restrict__ w, double *__restrict__ Z, GmresState *st) {
    if (st->done) return;
    const int64_t off = (int64_t)st->j * n;
    for_rows<TPR>(n, A, zout, [&](int64_t row, double s) {
        w[row] = s;
        Z[off + row] = zout[row];
    });
    if (blockIdx.x == 0 && threadIdx.x == 0) st->new_cycle = 0;
}

struct Gmres {
    static void init(pkasp_problem *p, const double *b, double *x, cudaStream_t s) {
        const RowOp A = fine_op(p);
        PK_FMT_SWITCH(p->spmv_tpr, (kg_residual<TPR><<<fine_grid(p), kBlock, 0, s>>>(
                                       p->nh, A, b, x, p->gm_V, p->gm_state, p->gm_g, p->d_partials,
                                       p->d_counter, p->d_hist, 1)));
        PK_LAUNCH();
        kg_scale_v0<<<elem_blocks(p->nh), kBlock, 0, s>>>(p->nh, p->gm_V, p->gm_vin, p->gm_state);
        PK_LAUNCH();
    }
    static void step(pkasp_problem *p, const double *b, double *x, cudaStream_t s) {
        const int64_t n = p->nh;
        const RowOp A = fine_op(p);
        apply_prec(p, p->gm_vin, p->gm_zout, s);
        PK_FMT_SWITCH(p->spmv_tpr, (kg_spmv_w<TPR><<<fine_grid(p), kBlock, 0, s>>>(n, A, p->gm_zout, p->gm_w, p->gm_Z,
                                                                              p->gm_state)));
        PK_LAUNCH();
        const dim3 dg(kDotChunks, p->gm_m + 1);
        for (int pass = 0; pass < 2; ++pass) {
            kg_dots<<<dg, kBlock, 0, s>>>(n, p->gm_V, p->gm_w, p->gm_state, p->gm_part, p->gm_cnt, p->gm_hc,
                                          p->gm_H, pass);
            PK_LAUNCH();
            kg_axpy<<<kRedGrid, kBlock, 0, s>>>(n, p->gm_V, p->gm_w, p->gm_state, p->gm_hc, p->gm_H, p->d_partials,
                                                p->d_counter, pass);
            PK_LAUNCH();
        }
        kg_scale_next<<<elem_blocks(n), kBlock, 0, s>>>(n, p->gm_V, p->gm_w, p->gm_vin, p->gm_state);
        PK_LAUNCH();
        kg_givens<<<1, 32, 0, s>>>(p->gm_state, p->gm_H, p->gm_cs, p->gm_sn, p->gm_g, p->d_hist);
        PK_LAUNCH();
        // end of a cycle (each kernel returns at once otherwise)
        kg_backsolve<<<1, 32, 0, s>>>(p->gm_state, p->gm_H, p->gm_g, p->gm_y);
        PK_LAUNCH();
        kg_update_x<<<elem_blocks(n), kBlock, 0, s>>>(n, x, p->gm_Z, p->gm_y, p->gm_state);
        PK_LAUNCH();
        PK_FMT_SWITCH(p->spmv_tpr, (kg_residual<TPR><<<fine_grid(p), kBlock, 0, s>>>(
                                       n, A, b, x, p->gm_V, p->gm_state, p->gm_g, p->d_partials, p->d_counter,
                                       p->d_hist, 0)));
        PK_LAUNCH();
        kg_scale_v0<<<elem_blocks(n), kBlock, 0, s>>>(n, p->gm_V, p->gm_vin, p->gm_state);
        PK_LAUNCH();
    }
    static void build_graph(pkasp_problem *p, const double *b, double *x) {
        if (p->gm_graph_exec) cudaGraphExecDestroy(p->gm_graph_exec);
        if (p->gm_graph) cudaGraphDestroy(p->gm_graph);
        p->gm_graph_exec = nullptr;
        p->gm_graph = nullptr;
        cudaStream_t cs = p->cap_stream;
        cudaGraph_t g, gi;
        PK_CUDA(cudaGraphCreate(&g, 0));
        PK_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        long long c0 = launch_count();
        init(p, b, x, cs);
        p->gm_g_init = launch_count() - c0;
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
        kg_loop_control<<<1, 32, 0, cs>>>(p->gm_state, h);
        PK_LAUNCH();
        p->gm_g_body = launch_count() - c0;
        PK_CUDA(cudaStreamEndCapture(cs, &body));
        PK_CUDA(cudaGraphInstantiate(&p->gm_graph_exec, g, 0));
        cudaGraphDestroy(gi);
        p->gm_graph = g;
        p->gm_key_b = b;
        p->gm_key_x = x;
    }
};

void ensure_gmres(pkasp_problem *p, int m) {
    if (p->gm_m == m && p->gm_V) return;
    free_gmres(p);
    DevPool &w = p->gm_pool;
    const int64_t n = std::max<int64_t>(p->nh, 1);
    p->gm_V = w.get<double>((size_t)n * (m + 1));
    p->gm_Z = w.get<double>((size_t)n * m);
    p->gm_w = w.get<double>(n);
    p->gm_vin = w.get<double>(n);
    p->gm_zout = w.get<double>(n);
    p->gm_H = w.get<double>((size_t)(m + 1) * m);
    p->gm_g = w.get<double>(m + 1);
    p->gm_cs = w.get<double>(m);
    p->gm_sn = w.get<double>(m);
    p->gm_y = w.get<double>(m);
    p->gm_hc = w.get<double>(m + 1);
    p->gm_part = w.get<double>((size_t)kDotChunks * (m + 1));
    p->gm_cnt = w.get<unsigned>(m + 1);
    PK_CUDA(cudaMemset(p->gm_cnt, 0, sizeof(unsigned) * (m + 1)));
    p->gm_state = w.get<GmresState>(1);
    p->gm_m = m;
}

}  // namespace

void free_gmres(pkasp_problem *p) {
    if (p->gm_graph_exec) cudaGraphExecDestroy(p->gm_graph_exec);
    if (p->gm_graph) cudaGraphDestroy(p->gm_graph);
    p->gm_graph_exec = nullptr;
    p->gm_graph = nullptr;
    p->gm_key_b = nullptr;
    p->gm_key_x = nullptr;
    p->gm_pool.free_all();
    p->gm_V = p->gm_Z = p->gm_w = p->gm_vin = p->gm_zout = nullptr;
    p->gm_state = nullptr;
    p->gm_m = 0;
}

int solve_gmres(pkasp_problem *p, const double *b, double *x, pkasp_stats *st, cudaStream_t s) {
    const int m = p->opt.restart;
    ensure_work(p, 1);
    ensure_gmres(p, m);
    const int cap = (st && st->hist_cap > 0) ? st->hist_cap : 1;
    if (cap > p->hist_cap) {
        p->d_hist = p->work_pool.get<double>(cap);
        p->hist_cap = cap;
        if (p->gm_graph_exec) cudaGraphExecDestroy(p->gm_graph_exec);
        if (p->gm_graph) cudaGraphDestroy(p->gm_graph);
        p->gm_graph_exec = nullptr;
        p->gm_graph = nullptr;
    }
    kg_state_reset<<<1, 32, 0, s>>>(p->gm_state, m, p->opt.tol, p->opt.max_iter, p->hist_cap);
    PK_LAUNCH();
    cudaEvent_t e0, e1;
    PK_CUDA(cudaEventCreate(&e0));
    PK_CUDA(cudaEventCreate(&e1));
    PK_CUDA(cudaEventRecord(e0, s));
    const bool use_graph = p->opt.use_graph != 0;
    if (use_graph && (!p->gm_graph_exec || p->gm_key_b != b || p->gm_key_x != x)) {
        PK_CUDA(cudaStreamSynchronize(s));
        Gmres::build_graph(p, b, x);
    }
    GmresState hs;
    long long launches = 1;
    const long long eager0 = launch_count();
    if (use_graph) {
        PK_CUDA(cudaGraphLaunch(p->gm_graph_exec, s));
    } else {
        Gmres::init(p, b, x, s);
        for (int pass = 0; pass < p->opt.max_iter + p->opt.max_iter / std::max(m, 1) + 4; ++pass) {
            int done = 0;
            PK_CUDA(cudaMemcpyAsync(&done, &p->gm_state->done, sizeof(int), cudaMemcpyDeviceToHost, s));
            PK_CUDA(cudaStreamSynchronize(s));
            if (done) break;
            Gmres::step(p, b, x, s);
        }
    }
    PK_CUDA(cudaEventRecord(e1, s));
    PK_CUDA(cudaMemcpyAsync(&hs, p->gm_state, sizeof(GmresState), cudaMemcpyDeviceToHost, s));
    PK_CUDA(cudaEventSynchronize(e1));
    PK_CUDA(cudaStreamSynchronize(s));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (use_graph) launches += p->gm_g_init + (long long)hs.loops * p->gm_g_body;
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
        st->kernel_launches = use_graph ? launches : 1 + (launch_count() - eager0);
        st->hist_len = std::min(hs.it + 1, st->hist_cap);
        if (st->hist_host && st->hist_len > 0)
            PK_CUDA(cudaMemcpy(st->hist_host, p->d_hist, sizeof(double) * st->hist_len, cudaMemcpyDeviceToHost));
    }
    return status;
}

}  // namespace pk
