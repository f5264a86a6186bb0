// batched.cu -- width dispatch and work memory of the multi-RHS PCG (the kernels and the
// solve loop are in batched_impl.cuh, compiled once per width by batched_w*.cu).
#include <algorithm>

#include "internal.h"

namespace pk {

int solve_block_4(pkasp_problem *p, const double *b, double *x, int ncols, int64_t ld, pkasp_stats *st,
                  cudaStream_t s);
float time_block_4(pkasp_problem *p, int which, int reps, cudaStream_t s);
int solve_block_8(pkasp_problem *p, const double *b, double *x, int ncols, int64_t ld, pkasp_stats *st,
                  cudaStream_t s);
float time_block_8(pkasp_problem *p, int which, int reps, cudaStream_t s);
int solve_block_16(pkasp_problem *p, const double *b, double *x, int ncols, int64_t ld, pkasp_stats *st,
                  cudaStream_t s);
float time_block_16(pkasp_problem *p, int which, int reps, cudaStream_t s);
int solve_block_32(pkasp_problem *p, const double *b, double *x, int ncols, int64_t ld, pkasp_stats *st,
                  cudaStream_t s);
float time_block_32(pkasp_problem *p, int which, int reps, cudaStream_t s);
int solve_block_48(pkasp_problem *p, const double *b, double *x, int ncols, int64_t ld, pkasp_stats *st,
                  cudaStream_t s);
float time_block_48(pkasp_problem *p, int which, int reps, cudaStream_t s);
int solve_block_64(pkasp_problem *p, const double *b, double *x, int ncols, int64_t ld, pkasp_stats *st,
                  cudaStream_t s);
float time_block_64(pkasp_problem *p, int which, int reps, cudaStream_t s);

namespace {

int block_width(int ncols) {
    for (int w : {4, 8, 16, 32, 48, 64})
        if (ncols <= w) return w;
    return -1;
}

}  // namespace

void ensure_batched(pkasp_problem *p, int NC, int hist_entries) {
    if (p->bwork_nc == NC && p->bwork_hist >= hist_entries) return;
    if (p->bgraph_exec) cudaGraphExecDestroy(p->bgraph_exec);
    if (p->bgraph) cudaGraphDestroy(p->bgraph);
    p->bgraph_exec = nullptr;
    p->bgraph = nullptr;
    p->bwork_pool.free_all();
    p->bchunk = 0;
    p->bgroup_cols = p->blanes = 0;
    DevPool &w = p->bwork_pool;
    const int64_t n = std::max<int64_t>(p->nh, 1) * NC;
    p->bw_r = w.get<double>(n);
    p->bw_z = w.get<double>(n);
    p->bw_p = w.get<double>(n);
    p->bw_q = w.get<double>(n);
    p->bw_b = w.get<double>(n);
    p->bw_x = w.get<double>(n);
    p->bw_zs = w.get<double>(n);
    p->bw_zs32 = w.get<float>(n);
    p->bw_t = w.get<double>(n);
    p->bw_t32 = w.get<float>(n);
    p->bw_r32 = w.get<float>(n);
    p->bl_b.assign(p->lev.size(), nullptr);
    p->bl_x.assign(p->lev.size(), nullptr);
    p->bl_r.assign(p->lev.size(), nullptr);
    p->bl_b32.assign(p->lev.size(), nullptr);
    p->bl_x32.assign(p->lev.size(), nullptr);
    p->bl_r32.assign(p->lev.size(), nullptr);
    for (size_t l = 0; l < p->lev.size(); ++l) {
        const int64_t m = std::max<int64_t>(p->lev[l].A.n, 1) * NC;
        p->bl_b[l] = w.get<double>(m);
        p->bl_x[l] = w.get<double>(m);
        p->bl_r[l] = w.get<double>(m);
        p->bl_b32[l] = w.get<float>(m);
        p->bl_x32[l] = w.get<float>(m);
        p->bl_r32[l] = w.get<float>(m);
    }
    p->bw_hist = w.get<double>(std::max(hist_entries, 1));
    p->bw_mask = w.get<int>(PKASP_MAX_COLS);
    p->bwork_nc = NC;
    p->bwork_hist = hist_entries;
}

int solve_batched(pkasp_problem *p, const double *b, double *x, int ncols, int64_t ld, pkasp_stats *st,
                  cudaStream_t s) {
    const int NC = block_width(ncols);
    if (NC < 0) fail(PKASP_EINVAL, "at most 64 right-hand sides per call");
    switch (NC) {
        case 4: return solve_block_4(p, b, x, ncols, ld, st, s);
        case 8: return solve_block_8(p, b, x, ncols, ld, st, s);
        case 16: return solve_block_16(p, b, x, ncols, ld, st, s);
        case 32: return solve_block_32(p, b, x, ncols, ld, st, s);
        case 48: return solve_block_48(p, b, x, ncols, ld, st, s);
        default: return solve_block_64(p, b, x, ncols, ld, st, s);
    }
}

float time_batched(pkasp_problem *p, int which, int reps, cudaStream_t s) {
    if (which > 6) fail(PKASP_EINVAL, "which must be 0..6");
    if (p->bwork_nc <= 0) fail(PKASP_ESTATE, "blocked timings need a solve with ncols > 1 first");
    switch (p->bwork_nc) {
        case 4: return time_block_4(p, which, reps, s);
        case 8: return time_block_8(p, which, reps, s);
        case 16: return time_block_16(p, which, reps, s);
        case 32: return time_block_32(p, which, reps, s);
        case 48: return time_block_48(p, which, reps, s);
        default: return time_block_64(p, which, reps, s);
    }
}

void free_batched(pkasp_problem *p) {
    if (p->bgraph_exec) cudaGraphExecDestroy(p->bgraph_exec);
    if (p->bgraph) cudaGraphDestroy(p->bgraph);
    p->bgraph_exec = nullptr;
    p->bgraph = nullptr;
    p->bwork_pool.free_all();
    p->bwork_nc = -1;
    p->bwork_hist = 0;
    p->bchunk = 0;
    p->bgroup_cols = p->blanes = 0;
}

}  // namespace pk
