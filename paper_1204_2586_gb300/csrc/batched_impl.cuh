// batched_impl.cuh -- PCG for several right-hand sides at once (columns independent).
// Included once per block width by batched_w*.cu (one translation unit per width, so
// the widths compile in parallel); batched.cu holds the width dispatch and the work
// memory.
//
// All vectors are blocks X[n][NC] (row-major, NC columns per row, NC from a fixed set
// of widths; unused columns are zero and marked converged from the start). Every row
// task is a group of W lanes with CPL columns each (NC = W * CPL): the lanes of a task
// read each matrix entry once (the same address: one broadcast load) and gather the
// NC-wide row of X they multiply with as one contiguous access. Scalars (alpha, beta,
// rho, norms, iteration counts, stop flags) are per column; a converged column stops
// changing while the others continue. Reductions over rows are per column, with the
// fixed-grid block-partial scheme of the single-column path (reproducible).
#pragma once

#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"
#include "kernels.cuh"

namespace pk {

// batched.cu: the work blocks of one width (reallocated when the width or the history
// length grows; the tuned layout is reset with them)
void ensure_batched(pkasp_problem *p, int NC, int hist_entries);

namespace {

template <int NC>
struct Tile {
    static constexpr int W = (NC % 32 == 0) ? 32 : (NC % 16 == 0) ? 16 : (NC % 8 == 0) ? 8 : 4;
    static constexpr int CPL = NC / W;
};

template <typename PT> const PT *bpick(const double *d, const float *f);
template <> const double *bpick<double>(const double *d, const float *) { return d; }
template <> const float *bpick<float>(const double *, const float *f) { return f; }
template <typename PT> PT *bpickw(double *d, float *f);
template <> double *bpickw<double>(double *d, float *) { return d; }
template <> float *bpickw<float>(double *, float *f) { return f; }

unsigned tasks_grid(int64_t rows, int W) {
    int64_t t = rows * W;
    return (unsigned)std::max<int64_t>(1, (t + kBlock - 1) / kBlock);
}

// acc[k] = sum_e val[e] * X[col[e]][lane + k*W], entries e in [lo, hi) in ascending
// order, for a task of W lanes with CPL columns each; X has row stride ld and starts at
// the first column of the task's column group
template <int W, int CPL, typename A, typename VT, typename XT>
__device__ __forceinline__ void bdotw(int64_t lo, int64_t hi, const int32_t *__restrict__ col,
                                      const VT *__restrict__ val, const XT *X, int64_t ld, int lane,
                                      A (&acc)[CPL]) {
#pragma unroll
    for (int k = 0; k < CPL; ++k) acc[k] = A(0);
#pragma unroll 4
    for (int64_t e = lo; e < hi; ++e) {
        const int64_t j = __ldg(&col[e]);
        const A a = (A)__ldg(&val[e]);
        const XT *xr = X + j * ld + lane;
#pragma unroll
        for (int k = 0; k < CPL; ++k) acc[k] += a * (A)xr[k * W];
    }
}

// the same for the default task shape of an NC-wide block
template <int NC, typename A, typename VT, typename XT>
__device__ __forceinline__ void bdot(int64_t lo, int64_t hi, const int32_t *__restrict__ col,
                                     const VT *__restrict__ val, const XT *X, int64_t ld, int lane,
                                     A (&acc)[Tile<NC>::CPL]) {
    bdotw<Tile<NC>::W, Tile<NC>::CPL, A>(lo, hi, col, val, X, ld, lane, acc);
}

// Per-column grid reduction: v[q][k] is this lane's partial of quantity q for column
// lane + k*W. The last block to finish writes the totals to out[q*NC + c] (shared)
// and returns true in all its threads.
template <int NC, int NV>
__device__ bool reduce_cols(double (&v)[NV][Tile<NC>::CPL], double *partials, unsigned *counter, double *out) {
    constexpr int W = Tile<NC>::W, CPL = Tile<NC>::CPL, NT = NV * NC;
    __shared__ double sh[NT][kBlock / 32];
    __shared__ int last;
    const int lane32 = threadIdx.x & 31, lane = threadIdx.x % W, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q)
#pragma unroll
        for (int k = 0; k < CPL; ++k) {
            double x = v[q][k];
#pragma unroll
            for (int o = W; o < 32; o <<= 1) x += __shfl_xor_sync(kFull, x, o);
            if (lane32 < W) sh[q * NC + lane + k * W][wid] = x;
        }
    __syncthreads();
    if (threadIdx.x < NT) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += sh[threadIdx.x][w];
        partials[(int64_t)blockIdx.x * NT + threadIdx.x] = s;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned prev = atomicAdd(counter, 1u);
        last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    if (threadIdx.x < NT) {
        double s = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) s += __ldcg(&partials[(int64_t)b * NT + threadIdx.x]);
        out[threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) *counter = 0u;
    return true;
}

// ---------------------------------------------------------------------------------
// PCG vector kernels (FP64)
// ---------------------------------------------------------------------------------
template <int NC>
__global__ void __launch_bounds__(kBlock) kb_init_residual(int64_t n, const int64_t *__restrict__ ptr,
                                                           const int32_t *__restrict__ col,
                                                           const double *__restrict__ val, const double *B,
                                                           const double *X, double *R, float *R32, PcgState *st,
                                                           double *partials, unsigned *counter, double *hist) {
    constexpr int W = Tile<NC>::W, CPL = Tile<NC>::CPL;
    __shared__ double tot[NC];
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x % W;
    const int64_t ntask = ((int64_t)gridDim.x * blockDim.x) / W;
    double v[1][CPL];
#pragma unroll
    for (int k = 0; k < CPL; ++k) v[0][k] = 0.0;
    for (int64_t row = gt / W; row < n; row += ntask) {
        double acc[CPL];
        bdot<NC, double>(ptr[row], ptr[row + 1], col, val, X, NC, lane, acc);
#pragma unroll
        for (int k = 0; k < CPL; ++k) {
            const int64_t o = row * NC + lane + k * W;
            const double r = B[o] - acc[k];
            R[o] = r;
            if (R32) R32[o] = (float)r;
            v[0][k] += r * r;
        }
    }
    if (!reduce_cols<NC, 1>(v, partials, counter, tot)) return;
    // the whole last block continues (uniform branch)
    if (threadIdx.x < NC) {
        const int c = threadIdx.x;
        const double rn = sqrt(tot[c]);
        st->rnorm[c] = rn;
        if (st->iter[c] == 0 && !st->done[c]) {
            st->r0[c] = rn;
            if (st->hist_cap > 0) hist[c] = rn;
            if (rn == 0.0) {
                st->done[c] = 1;
                st->status[c] = PKASP_OK;
            }
        }
    }
    __syncthreads();
    {
        if (threadIdx.x == 0) {
            int all = 1;
            for (int q = 0; q < st->ncols; ++q) all &= st->done[q];
            st->all_done = all;
        }
    }
}

// Q = A P and alpha_c = rho_c / (p_c, q_c) for the columns still running
template <int NC>
__global__ void __launch_bounds__(kBlock) kb_spmv_pq(int64_t n, const int64_t *__restrict__ ptr,
                                                     const int32_t *__restrict__ col, const double *__restrict__ val,
                                                     const double *P, double *Q, PcgState *st, double *partials,
                                                     unsigned *counter) {
    constexpr int W = Tile<NC>::W, CPL = Tile<NC>::CPL;
    __shared__ double tot[NC];
    if (st->all_done) return;
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x % W;
    const int64_t ntask = ((int64_t)gridDim.x * blockDim.x) / W;
    double v[1][CPL];
#pragma unroll
    for (int k = 0; k < CPL; ++k) v[0][k] = 0.0;
    for (int64_t row = gt / W; row < n; row += ntask) {
        double acc[CPL];
        bdot<NC, double>(ptr[row], ptr[row + 1], col, val, P, NC, lane, acc);
#pragma unroll
        for (int k = 0; k < CPL; ++k) {
            const int64_t o = row * NC + lane + k * W;
            Q[o] = acc[k];
            v[0][k] += P[o] * acc[k];
        }
    }
    if (reduce_cols<NC, 1>(v, partials, counter, tot) && threadIdx.x < NC) {
        const int c = threadIdx.x;
        if (!st->done[c]) {
            const double pq = tot[c];
            if (!(pq > 0.0)) {
                st->done[c] = 1;
                st->status[c] = PKASP_EBREAKDOWN;
                st->alpha[c] = 0.0;
            } else {
                st->alpha[c] = st->rho[c] / pq;
            }
        } else {
            st->alpha[c] = 0.0;
        }
    }
}

// ---------------------------------------------------------------------------------
// Element-wise PCG kernels: one thread per element of the [n][NC] block, blocks of
// FlatBT threads (a multiple of NC and of 32), so that every thread keeps one column
// (c = threadIdx.x % NC) through the grid-stride loop and a warp reads 256 contiguous
// bytes. Per-column sums: block partials in fixed order, then the last block.
// ---------------------------------------------------------------------------------
template <int NC>
constexpr int FlatBT = (NC == 48) ? 384 : 256;

template <int NC, int NV>
__device__ bool reduce_flat(const double (&v)[NV], double *partials, unsigned *counter, double *out) {
    constexpr int BT = FlatBT<NC>, NT = NV * NC, RPB = BT / NC;
    __shared__ double sh[NV][BT];
    __shared__ int last;
#pragma unroll
    for (int q = 0; q < NV; ++q) sh[q][threadIdx.x] = v[q];
    __syncthreads();
    if (threadIdx.x < NT) {
        const int q = threadIdx.x / NC, c = threadIdx.x % NC;
        double s = 0.0;
        for (int r = 0; r < RPB; ++r) s += sh[q][r * NC + c];
        partials[(int64_t)blockIdx.x * NT + threadIdx.x] = s;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned prev = atomicAdd(counter, 1u);
        last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    if (threadIdx.x < NT) {
        double s = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) s += __ldcg(&partials[(int64_t)b * NT + threadIdx.x]);
        out[threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) *counter = 0u;
    return true;
}

// Each thread walks its elements t, t+S, t+2S, ... (S = grid stride, a multiple of NC);
// the loops below take four of them per step with all loads issued before any store,
// so a thread keeps four independent loads per stream in flight. Sums still run in
// ascending t per thread.
constexpr int kIlp = 4;

// P = Z and rho_c = (r_c, z_c)
template <int NC>
__global__ void __launch_bounds__(FlatBT<NC>) kb_start(int64_t ne, const double *R, const double *Z, double *P,
                                                         PcgState *st, double *partials, unsigned *counter) {
    constexpr int BT = FlatBT<NC>;
    __shared__ double tot[NC];
    if (st->all_done) return;
    const int64_t S = (int64_t)gridDim.x * BT;
    int64_t t = (int64_t)blockIdx.x * BT + threadIdx.x;
    double v[1] = {0.0};
    for (; t + (kIlp - 1) * S < ne; t += kIlp * S) {
        double z[kIlp], r[kIlp];
#pragma unroll
        for (int u = 0; u < kIlp; ++u) {
            z[u] = Z[t + u * S];
            r[u] = R[t + u * S];
        }
#pragma unroll
        for (int u = 0; u < kIlp; ++u) {
            P[t + u * S] = z[u];
            v[0] += r[u] * z[u];
        }
    }
    for (; t < ne; t += S) {
        const double z = Z[t];
        P[t] = z;
        v[0] += R[t] * z;
    }
    if (reduce_flat<NC, 1>(v, partials, counter, tot) && threadIdx.x < NC) st->rho[threadIdx.x] = tot[threadIdx.x];
}

// X += alpha P, R -= alpha Q per running column (and the FP32 copy of R the
// mixed-precision preconditioner reads); norms; convergence per column
template <int NC>
__global__ void __launch_bounds__(FlatBT<NC>) kb_update_xr(int64_t ne, double *X, double *R, float *R32,
                                                             const double *P, const double *Q, PcgState *st,
                                                             double *partials, unsigned *counter, double *hist) {
    constexpr int BT = FlatBT<NC>;
    __shared__ double tot[NC];
    if (st->all_done) return;
    const int c = threadIdx.x % NC;
    const bool run = !st->done[c];
    const double a = st->alpha[c];
    const int64_t S = (int64_t)gridDim.x * BT;
    int64_t t = (int64_t)blockIdx.x * BT + threadIdx.x;
    double v[1] = {0.0};
    if (run) {
        for (; t + (kIlp - 1) * S < ne; t += kIlp * S) {
            double r[kIlp], q[kIlp], x[kIlp], pp[kIlp];
#pragma unroll
            for (int u = 0; u < kIlp; ++u) {
                r[u] = R[t + u * S];
                q[u] = Q[t + u * S];
                x[u] = X[t + u * S];
                pp[u] = P[t + u * S];
            }
#pragma unroll
            for (int u = 0; u < kIlp; ++u) {
                X[t + u * S] = x[u] + a * pp[u];
                const double rn = r[u] - a * q[u];
                R[t + u * S] = rn;
                if (R32) R32[t + u * S] = (float)rn;
                v[0] += rn * rn;
            }
        }
        for (; t < ne; t += S) {
            X[t] += a * P[t];
            const double rn = R[t] - a * Q[t];
            R[t] = rn;
            if (R32) R32[t] = (float)rn;
            v[0] += rn * rn;
        }
    } else {
        // a converged column: its residual stays as it is (the norm is not used)
        for (; t < ne; t += S) {
            const double r = R[t];
            v[0] += r * r;
        }
    }
    if (!reduce_flat<NC, 1>(v, partials, counter, tot)) return;
    // the whole last block continues (uniform branch)
    if (threadIdx.x < NC) {
        const int cc = threadIdx.x;
        if (!st->done[cc]) {
            const double rn = sqrt(tot[cc]);
            const int it = st->iter[cc] + 1;
            st->iter[cc] = it;
            st->rnorm[cc] = rn;
            if (it < st->hist_cap) hist[(int64_t)it * st->ncols + cc] = rn;
            if (rn <= st->tol * st->r0[cc]) {
                st->done[cc] = 1;
                st->status[cc] = PKASP_OK;
            } else if (it >= st->maxit) {
                st->done[cc] = 1;
                st->status[cc] = PKASP_ENOTCONV;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int all = 1;
        for (int q = 0; q < st->ncols; ++q) all &= st->done[q];
        st->all_done = all;
    }
}

// beta per column (standard or flexible) and rho
template <int NC>
__global__ void __launch_bounds__(FlatBT<NC>) kb_beta(int64_t ne, const double *R, const double *Z,
                                                        const double *Q, int flexible, PcgState *st,
                                                        double *partials, unsigned *counter) {
    constexpr int BT = FlatBT<NC>;
    __shared__ double tot[2 * NC];
    if (st->all_done) return;
    const int64_t S = (int64_t)gridDim.x * BT;
    int64_t t = (int64_t)blockIdx.x * BT + threadIdx.x;
    double v[2] = {0.0, 0.0};
    for (; t + (kIlp - 1) * S < ne; t += kIlp * S) {
        double z[kIlp], r[kIlp], q[kIlp];
#pragma unroll
        for (int u = 0; u < kIlp; ++u) {
            z[u] = Z[t + u * S];
            r[u] = R[t + u * S];
            q[u] = Q[t + u * S];
        }
#pragma unroll
        for (int u = 0; u < kIlp; ++u) {
            v[0] += r[u] * z[u];
            v[1] += z[u] * q[u];
        }
    }
    for (; t < ne; t += S) {
        const double z = Z[t];
        v[0] += R[t] * z;
        v[1] += z * Q[t];
    }
    if (reduce_flat<NC, 2>(v, partials, counter, tot) && threadIdx.x < NC) {
        const int c = threadIdx.x;
        if (!st->done[c]) {
            const double rho = st->rho[c];
            st->beta[c] = flexible ? (-st->alpha[c] * tot[NC + c]) / rho : tot[c] / rho;
            st->rho[c] = tot[c];
        }
    }
}

template <int NC>
__global__ void __launch_bounds__(FlatBT<NC>) kb_update_p(int64_t ne, const double *Z, double *P,
                                                            const PcgState *st) {
    constexpr int BT = FlatBT<NC>;
    if (st->all_done) return;
    const int c = threadIdx.x % NC;
    if (st->done[c]) return;
    const double b = st->beta[c];
    const int64_t S = (int64_t)gridDim.x * BT;
    int64_t t = (int64_t)blockIdx.x * BT + threadIdx.x;
    for (; t + (kIlp - 1) * S < ne; t += kIlp * S) {
        double z[kIlp], pp[kIlp];
#pragma unroll
        for (int u = 0; u < kIlp; ++u) {
            z[u] = Z[t + u * S];
            pp[u] = P[t + u * S];
        }
#pragma unroll
        for (int u = 0; u < kIlp; ++u) P[t + u * S] = z[u] + b * pp[u];
    }
    for (; t < ne; t += S) P[t] = Z[t] + b * P[t];
}

template <int NC>
__global__ void __launch_bounds__(kBlock) kb_true_residual(int64_t n, const int64_t *__restrict__ ptr,
                                                           const int32_t *__restrict__ col,
                                                           const double *__restrict__ val, const double *B,
                                                           const double *X, PcgState *st, double *partials,
                                                           unsigned *counter) {
    constexpr int W = Tile<NC>::W, CPL = Tile<NC>::CPL;
    __shared__ double tot[NC];
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x % W;
    const int64_t ntask = ((int64_t)gridDim.x * blockDim.x) / W;
    double v[1][CPL];
#pragma unroll
    for (int k = 0; k < CPL; ++k) v[0][k] = 0.0;
    for (int64_t row = gt / W; row < n; row += ntask) {
        double acc[CPL];
        bdot<NC, double>(ptr[row], ptr[row + 1], col, val, X, NC, lane, acc);
#pragma unroll
        for (int k = 0; k < CPL; ++k) {
            const double r = B[row * NC + lane + k * W] - acc[k];
            v[0][k] += r * r;
        }
    }
    if (reduce_cols<NC, 1>(v, partials, counter, tot) && threadIdx.x < NC) st->tnorm[threadIdx.x] = sqrt(tot[threadIdx.x]);
}

__global__ void kb_loop_control(PcgState *st, cudaGraphConditionalHandle h) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int loops = ++st->loops;
    bool go = !st->all_done && loops <= st->maxit + 2;
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

__global__ void kb_state_reset(PcgState *st, int ncols, int nc_real, double tol, int maxit, int hist_cap) {
    const int c = threadIdx.x;
    if (blockIdx.x != 0 || c >= PKASP_MAX_COLS) return;
    st->iter[c] = 0;
    st->r0[c] = 0.0;
    st->alpha[c] = st->beta[c] = 0.0;
    // columns beyond the caller's count are padding: converged from the start
    st->done[c] = (c < nc_real) ? 0 : 1;
    st->status[c] = (c < nc_real) ? -1 : PKASP_OK;
    if (c == 0) {
        st->all_done = 0;
        st->ncols = ncols;
        st->tol = tol;
        st->maxit = maxit;
        st->hist_cap = hist_cap;
        st->loops = 0;
    }
}

__global__ void kb_state_restart(PcgState *st, const int *restart_mask) {
    const int c = threadIdx.x;
    if (blockIdx.x != 0 || c >= st->ncols) return;
    if (restart_mask[c]) {
        st->done[c] = 0;
        st->status[c] = -1;
    }
    if (c == 0) {
        st->all_done = 0;
        st->loops = 0;
    }
}

// caller block [n][ld] (ncols used) <-> internal block [n][NC]
__global__ void kb_gather(int64_t n, int ncols, int64_t ld, int NC, const double *src, double *dst) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * NC) return;
    int64_t row = t / NC;
    int c = (int)(t % NC);
    dst[t] = c < ncols ? src[row * ld + c] : 0.0;
}

__global__ void kb_scatter(int64_t n, int ncols, int64_t ld, int NC, const double *src, double *dst) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * NC) return;
    int64_t row = t / NC;
    int c = (int)(t % NC);
    if (c < ncols) dst[row * ld + c] = src[t];
}

// ---------------------------------------------------------------------------------
// Preconditioner kernels on blocks (PT: FP64 or FP32)
// ---------------------------------------------------------------------------------
// Y = A X (CSR), one task per row
template <int NC, typename PT, typename VT, typename XT, typename YT>
__global__ void __launch_bounds__(kBlock) kb_spmv(int64_t n, const int64_t *__restrict__ ptr,
                                                  const int32_t *__restrict__ col, const VT *__restrict__ val,
                                                  const XT *X, YT *Y) {
    constexpr int W = Tile<NC>::W, CPL = Tile<NC>::CPL;
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / W;
    const int lane = threadIdx.x % W;
    if (row >= n) return;
    PT acc[CPL];
    bdot<NC, PT>(ptr[row], ptr[row + 1], col, val, X, NC, lane, acc);
#pragma unroll
    for (int k = 0; k < CPL; ++k) Y[row * NC + lane + k * W] = (YT)acc[k];
}

// R = B - A X
template <int NC, typename PT, typename TB = PT>
__global__ void __launch_bounds__(kBlock) kb_residual(int64_t n, const int64_t *__restrict__ ptr,
                                                      const int32_t *__restrict__ col, const PT *__restrict__ val,
                                                      const TB *B, const PT *X, PT *R) {
    constexpr int W = Tile<NC>::W, CPL = Tile<NC>::CPL;
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / W;
    const int lane = threadIdx.x % W;
    if (row >= n) return;
    PT acc[CPL];
    bdot<NC, PT>(ptr[row], ptr[row + 1], col, val, X, NC, lane, acc);
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
        const int64_t o = row * NC + lane + k * W;
        R[o] = (PT)B[o] - acc[k];
    }
}

template <typename ZT, typename PT>
__global__ void kb_copy(int64_t ne, const PT *src, ZT *dst) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < ne) dst[t] = (ZT)src[t];
}

// X += P XC (interpolation), or Z = ZS + P W (prolongation into the fine block; the
// sum is taken in the preconditioner's precision PT and converted to ZT once)
template <int NC, typename PT, typename ZT>
__global__ void __launch_bounds__(kBlock) kb_prolong(int64_t n, const int64_t *__restrict__ ptr,
                                                     const int32_t *__restrict__ col, const PT *__restrict__ val,
                                                     const PT *XC, const PT *ZS, ZT *Z) {
    constexpr int W = Tile<NC>::W, CPL = Tile<NC>::CPL;
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / W;
    const int lane = threadIdx.x % W;
    if (row >= n) return;
    PT acc[CPL];
    bdot<NC, PT>(ptr[row], ptr[row + 1], col, val, XC, NC, lane, acc);
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
        const int64_t o = row * NC + lane + k * W;
        Z[o] = (ZT)(ZS[o] + acc[k]);
    }
}

// X = D^{-1} B (l1-Jacobi from zero) and X += D^{-1} R
template <int NC, typename PT, typename TB>
__global__ void kb_jacobi0(int64_t n, const PT *__restrict__ d, const TB *B, PT *X) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n * NC) X[t] = (PT)B[t] / d[t / NC];
}
template <int NC, typename PT>
__global__ void kb_add_div(int64_t n, const PT *R, const PT *__restrict__ d, PT *X) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n * NC) X[t] += R[t] / d[t / NC];
}

// X = Ainv B (dense coarsest inverse), one task per row
template <int NC, typename PT>
__global__ void kb_dense(int64_t n, const PT *__restrict__ Ainv, const PT *B, PT *X) {
    constexpr int W = Tile<NC>::W, CPL = Tile<NC>::CPL;
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / W;
    const int lane = threadIdx.x % W;
    if (row >= n) return;
    PT acc[CPL];
#pragma unroll
    for (int k = 0; k < CPL; ++k) acc[k] = PT(0);
    for (int64_t j = 0; j < n; ++j) {
        const PT a = Ainv[row * n + j];
#pragma unroll
        for (int k = 0; k < CPL; ++k) acc[k] += a * B[j * NC + lane + k * W];
    }
#pragma unroll
    for (int k = 0; k < CPL; ++k) X[row * NC + lane + k * W] = acc[k];
}

// colour phase of the symmetric GS from zero on a group of CH columns of blocks with
// row stride ld (R and Y point at the group's first column), W lanes per row, column
// lane + k*W of the group in lane `lane` (PDL: the static loads come first):
//   BACK = false: Y_i = (R_i - sum_L a_ij Y_j) * dinv_i ;  BACK = true: Y_i -= (sum_U a_ij Y_j) * dinv_i
template <int CH, int W, typename PT, bool BACK>
__global__ void __launch_bounds__(kBlock) kb_gs_phase(int64_t pb, int64_t pe, const int32_t *__restrict__ perm,
                                                      const int64_t *__restrict__ xptr,
                                                      const int32_t *__restrict__ xcol,
                                                      const PT *__restrict__ xval, const PT *__restrict__ dinv,
                                                      const PT *R, PT *Y, int64_t ld) {
    static_assert(CH % W == 0 && 32 % W == 0, "lanes must divide the group and the warp");
    constexpr int CPL = CH / W;
    pdl_trigger();
    const int64_t p = pb + ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / W;
    const int lane = threadIdx.x % W;
    const bool ok = p < pe;
    const int32_t i = ok ? perm[p] : 0;
    const PT di = ok ? dinv[p] : PT(1);
    const int64_t lo = ok ? xptr[p] : 0, hi = ok ? xptr[p + 1] : 0;
    pdl_wait();
    if (!ok) return;
    PT acc[CPL];
    bdotw<W, CPL, PT>(lo, hi, xcol, xval, (const PT *)Y, ld, lane, acc);
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
        const int64_t o = (int64_t)i * ld + lane + k * W;
        Y[o] = BACK ? Y[o] - acc[k] * di : (R[o] - acc[k]) * di;
    }
}

// full backward GS sweep phase from the current X (level and multiplicative post-smoother)
template <int NC, typename PT, typename TB>
__global__ void __launch_bounds__(kBlock) kb_gs_full(int64_t pb, int64_t pe, const int32_t *__restrict__ perm,
                                                     const int64_t *__restrict__ lptr, const int32_t *__restrict__ lcol,
                                                     const PT *__restrict__ lval, const int64_t *__restrict__ uptr,
                                                     const int32_t *__restrict__ ucol, const PT *__restrict__ uval,
                                                     const PT *__restrict__ diag, const TB *B, PT *X) {
    constexpr int W = Tile<NC>::W, CPL = Tile<NC>::CPL;
    const int64_t p = pb + ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / W;
    const int lane = threadIdx.x % W;
    if (p >= pe) return;
    const int32_t i = perm[p];
    PT sl[CPL], su[CPL];
    bdot<NC, PT>(lptr[p], lptr[p + 1], lcol, lval, (const PT *)X, NC, lane, sl);
    bdot<NC, PT>(uptr[p], uptr[p + 1], ucol, uval, (const PT *)X, NC, lane, su);
    const PT d = diag[p];
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
        const int64_t o = (int64_t)i * NC + lane + k * W;
        X[o] = ((PT)B[o] - sl[k] - su[k]) / d;
    }
}

template <typename... KArgs, typename... Args>
void blaunch_pdl(void (*kern)(KArgs...), unsigned grid, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kBlock);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    PK_CUDA(cudaLaunchKernelEx(&cfg, kern, args...));
    PK_LAUNCH();
}

// ---------------------------------------------------------------------------------
// host-side drivers for one block width NC
// ---------------------------------------------------------------------------------
template <int NC>
struct Batched {
    static constexpr int W = Tile<NC>::W;

    // symmetric GS phases from zero over column groups of CH columns, W lanes per row:
    // every phase of a group reads the group's columns of Y, so a group small enough to
    // stay in L2 saves the re-reads from HBM that a full-width block costs on a large
    // fine level; fewer lanes per row put more rows (and loads) in flight per SM
    template <int CH, int WL, typename PT>
    static void gs_sym_group(const DSplit &sp, const PT *r, PT *y, bool backward, cudaStream_t s) {
        for (int c0 = 0; c0 < NC; c0 += CH) {
            const PT *rg = r + c0;
            PT *yg = y + c0;
            for (int c = 0; c < sp.ncol; ++c) {
                const int64_t pb = sp.off[c], pe = sp.off[c + 1];
                if (pe <= pb) continue;
                blaunch_pdl(kb_gs_phase<CH, WL, PT, false>, tasks_grid(pe - pb, WL), s, pb, pe,
                            (const int32_t *)sp.perm, (const int64_t *)sp.lptr, (const int32_t *)sp.lcol,
                            bpick<PT>(sp.lval, sp.lval32), bpick<PT>(sp.dinv, sp.dinv32), rg, yg, (int64_t)NC);
            }
            if (!backward) continue;
            for (int c = sp.ncol - 2; c >= 0; --c) {
                const int64_t pb = sp.off[c], pe = sp.off[c + 1];
                if (pe <= pb) continue;
                blaunch_pdl(kb_gs_phase<CH, WL, PT, true>, tasks_grid(pe - pb, WL), s, pb, pe,
                            (const int32_t *)sp.perm, (const int64_t *)sp.uptr, (const int32_t *)sp.ucol,
                            bpick<PT>(sp.uval, sp.uval32), bpick<PT>(sp.dinv, sp.dinv32), (const PT *)yg, yg,
                            (int64_t)NC);
            }
        }
    }
    // the layouts the autotuner tries: (group columns, lanes per row)
    static constexpr int kLayouts = 6;
    static constexpr int layout_ch(int k) { return k < 2 ? NC : (k < 4 ? 16 : 8); }
    static constexpr int layout_w(int k) {
        return k == 0 ? Tile<NC>::W : k == 1 ? (Tile<NC>::W > 2 ? Tile<NC>::W / 2 : 2) : k == 2 ? 16 : k == 3 ? 8
                                                                                          : k == 4 ? 8 : 4;
    }
    static constexpr bool layout_ok(int k) {
        return NC % layout_ch(k) == 0 && layout_ch(k) % layout_w(k) == 0 && (k < 2 || layout_ch(k) < NC);
    }
    template <int K, typename PT>
    static void gs_layout(const DSplit &sp, const PT *r, PT *y, bool backward, cudaStream_t s) {
        if constexpr (layout_ok(K)) gs_sym_group<layout_ch(K), layout_w(K), PT>(sp, r, y, backward, s);
        else fail(PKASP_EINVAL, "smoother layout not available for this block width");
    }
    // layout k of the list above (0: full width, the default lanes)
    template <typename PT>
    static void gs_sym(const DSplit &sp, const PT *r, PT *y, bool backward, int k, cudaStream_t s) {
        switch (k) {
            case 1: gs_layout<1, PT>(sp, r, y, backward, s); break;
            case 2: gs_layout<2, PT>(sp, r, y, backward, s); break;
            case 3: gs_layout<3, PT>(sp, r, y, backward, s); break;
            case 4: gs_layout<4, PT>(sp, r, y, backward, s); break;
            case 5: gs_layout<5, PT>(sp, r, y, backward, s); break;
            default: gs_layout<0, PT>(sp, r, y, backward, s); break;
        }
    }
    template <typename PT, typename TB>
    static void gs_full(const DSplit &sp, const TB *b, PT *x, cudaStream_t s) {
        for (int c = sp.ncol - 1; c >= 0; --c) {
            const int64_t pb = sp.off[c], pe = sp.off[c + 1];
            if (pe <= pb) continue;
            kb_gs_full<NC, PT, TB><<<tasks_grid(pe - pb, W), kBlock, 0, s>>>(
                pb, pe, sp.perm, sp.lptr, sp.lcol, bpick<PT>(sp.lval, sp.lval32), sp.uptr, sp.ucol,
                bpick<PT>(sp.uval, sp.uval32), bpick<PT>(sp.diag, sp.diag32), b, x);
            PK_LAUNCH();
        }
    }
    template <typename PT, typename XT, typename YT>
    static void spmv(const DCSR &A, const XT *x, YT *y, cudaStream_t s) {
        if (A.n == 0) return;
        kb_spmv<NC, PT, PT, XT, YT><<<tasks_grid(A.n, W), kBlock, 0, s>>>(A.n, A.ptr, A.col,
                                                                           bpick<PT>(A.val, A.val32), x, y);
        PK_LAUNCH();
    }

    template <typename PT>
    static void vcycle(pkasp_problem *p, int l, cudaStream_t s) {
        Level &L = p->lev[l];
        const int64_t n = L.A.n;
        PT *b = bpickw<PT>(p->bl_b[l], p->bl_b32[l]);
        PT *x = bpickw<PT>(p->bl_x[l], p->bl_x32[l]);
        PT *r = bpickw<PT>(p->bl_r[l], p->bl_r32[l]);
        if (l == (int)p->lev.size() - 1) {
            kb_dense<NC, PT><<<tasks_grid(n, W), kBlock, 0, s>>>(n, bpick<PT>(p->d_cinv, p->d_cinv32), b, x);
            PK_LAUNCH();
            return;
        }
        const bool jac = p->opt.level_smoother == PKASP_SMOOTHER_L1JACOBI;
        const int64_t ne = n * NC;
        if (jac) {
            kb_jacobi0<NC, PT, PT><<<(unsigned)((ne + kBlock - 1) / kBlock), kBlock, 0, s>>>(
                n, bpick<PT>(L.l1, L.l132), b, x);
            PK_LAUNCH();
        } else {
            gs_sym<PT>(L.sp, b, x, false, 0, s);
        }
        kb_residual<NC, PT><<<tasks_grid(n, W), kBlock, 0, s>>>(n, L.A.ptr, L.A.col, bpick<PT>(L.A.val, L.A.val32),
                                                                b, x, r);
        PK_LAUNCH();
        PT *bc = bpickw<PT>(p->bl_b[l + 1], p->bl_b32[l + 1]);
        spmv<PT, PT, PT>(L.R, r, bc, s);
        vcycle<PT>(p, l + 1, s);
        PT *xc = bpickw<PT>(p->bl_x[l + 1], p->bl_x32[l + 1]);
        kb_prolong<NC, PT, PT><<<tasks_grid(n, W), kBlock, 0, s>>>(n, L.P.ptr, L.P.col, bpick<PT>(L.P.val, L.P.val32),
                                                                   xc, x, x);
        PK_LAUNCH();
        if (jac) {
            kb_residual<NC, PT><<<tasks_grid(n, W), kBlock, 0, s>>>(n, L.A.ptr, L.A.col,
                                                                    bpick<PT>(L.A.val, L.A.val32), b, x, r);
            PK_LAUNCH();
            kb_add_div<NC, PT><<<(unsigned)((ne + kBlock - 1) / kBlock), kBlock, 0, s>>>(n, r, bpick<PT>(L.l1, L.l132),
                                                                                         x);
            PK_LAUNCH();
        } else {
            gs_full<PT, PT>(L.sp, b, x, s);
        }
    }

    // multiplicative form: pre-smooth from zero, coarse correction of the new residual,
    // post-smooth from the corrected iterate
    template <typename PT>
    static void multiplicative(pkasp_problem *p, const PT *R, double *Z, cudaStream_t s) {
        PT *zs = bpickw<PT>(p->bw_zs, p->bw_zs32);
        PT *t = bpickw<PT>(p->bw_t, p->bw_t32);
        const int64_t nh = p->nh, ne = nh * NC;
        const unsigned eg = (unsigned)((ne + kBlock - 1) / kBlock);
        const bool jac = p->opt.smoother == PKASP_SMOOTHER_L1JACOBI;
        const PT *ahv = bpick<PT>(p->Ah.val, p->Ah.val32);
        if (jac) {
            kb_jacobi0<NC, PT, PT><<<eg, kBlock, 0, s>>>(nh, bpick<PT>(p->d_l1h, p->d_l1h32), R, zs);
            PK_LAUNCH();
        } else {
            gs_sym<PT>(p->fine, R, zs, false, p->bchunk - 1, s);
        }
        kb_residual<NC, PT, PT><<<tasks_grid(nh, W), kBlock, 0, s>>>(nh, p->Ah.ptr, p->Ah.col, ahv, R, zs, t);
        PK_LAUNCH();
        spmv<PT, PT, PT>(p->PiT, t, bpickw<PT>(p->bl_b[0], p->bl_b32[0]), s);
        vcycle<PT>(p, 0, s);
        PT *x0 = bpickw<PT>(p->bl_x[0], p->bl_x32[0]);
        kb_prolong<NC, PT, PT><<<tasks_grid(nh, W), kBlock, 0, s>>>(nh, p->Pi.ptr, p->Pi.col,
                                                                    bpick<PT>(p->Pi.val, p->Pi.val32), x0, zs, zs);
        PK_LAUNCH();
        if (jac) {
            kb_residual<NC, PT, PT><<<tasks_grid(nh, W), kBlock, 0, s>>>(nh, p->Ah.ptr, p->Ah.col, ahv, R, zs, t);
            PK_LAUNCH();
            kb_add_div<NC, PT><<<eg, kBlock, 0, s>>>(nh, t, bpick<PT>(p->d_l1h, p->d_l1h32), zs);
            PK_LAUNCH();
        } else {
            gs_full<PT, PT>(p->fine, R, zs, s);
        }
        kb_copy<double, PT><<<eg, kBlock, 0, s>>>(ne, zs, Z);
        PK_LAUNCH();
    }

    // Z = B R; R in the preconditioner's precision PT, Z in FP64; the additive form runs
    // its two branches on two streams
    template <typename PT>
    static void precondition(pkasp_problem *p, const PT *R, double *Z, cudaStream_t s) {
        if (p->opt.mode == PKASP_MODE_AMG) {
            // plain AMG: one V-cycle on the hierarchy of A_h (level 0 is A_h)
            const int64_t ne = p->nh * NC;
            const unsigned eg = (unsigned)((ne + kBlock - 1) / kBlock);
            kb_copy<PT, PT><<<eg, kBlock, 0, s>>>(ne, R, bpickw<PT>(p->bl_b[0], p->bl_b32[0]));
            PK_LAUNCH();
            vcycle<PT>(p, 0, s);
            kb_copy<double, PT><<<eg, kBlock, 0, s>>>(ne, bpickw<PT>(p->bl_x[0], p->bl_x32[0]), Z);
            PK_LAUNCH();
            return;
        }
        if (p->opt.mode != PKASP_MODE_ADDITIVE) return multiplicative<PT>(p, R, Z, s);
        PT *zs = bpickw<PT>(p->bw_zs, p->bw_zs32);
        PK_CUDA(cudaEventRecord(p->ev_fork, s));
        PK_CUDA(cudaStreamWaitEvent(p->aux_stream, p->ev_fork, 0));
        // V-cycle branch
        PT *b0 = bpickw<PT>(p->bl_b[0], p->bl_b32[0]);
        spmv<PT, PT, PT>(p->PiT, R, b0, p->aux_stream);
        vcycle<PT>(p, 0, p->aux_stream);
        // smoother branch
        const int64_t nh = p->nh, ne = nh * NC;
        if (p->opt.smoother == PKASP_SMOOTHER_L1JACOBI) {
            kb_jacobi0<NC, PT, PT><<<(unsigned)((ne + kBlock - 1) / kBlock), kBlock, 0, s>>>(
                nh, bpick<PT>(p->d_l1h, p->d_l1h32), R, zs);
            PK_LAUNCH();
        } else {
            gs_sym<PT>(p->fine, R, zs, true, p->bchunk - 1, s);
        }
        PK_CUDA(cudaEventRecord(p->ev_join, p->aux_stream));
        PK_CUDA(cudaStreamWaitEvent(s, p->ev_join, 0));
        PT *x0 = bpickw<PT>(p->bl_x[0], p->bl_x32[0]);
        kb_prolong<NC, PT, double><<<tasks_grid(nh, W), kBlock, 0, s>>>(nh, p->Pi.ptr, p->Pi.col,
                                                                        bpick<PT>(p->Pi.val, p->Pi.val32), x0, zs, Z);
        PK_LAUNCH();
    }

    // the autotuner of the fine smoother's layout (column group width, lanes per row):
    // times one symmetric sweep per candidate. Results are the same bits for every
    // layout: each column's sums run over the same entries in the same order. Returns
    // 1 + the index of the fastest layout.
    static int tune_group(pkasp_problem *p, cudaStream_t s) {
        if (p->opt.smoother == PKASP_SMOOTHER_L1JACOBI) return 1;
        int best = 0;
        float best_ms = 1e30f;
        const bool f32 = p->opt.precond_precision == PKASP_PREC_FP32;
        PK_CUDA(cudaMemsetAsync(p->bw_r, 0, sizeof(double) * p->nh * NC, s));
        PK_CUDA(cudaMemsetAsync(p->bw_r32, 0, sizeof(float) * p->nh * NC, s));
        cudaEvent_t e0, e1;
        PK_CUDA(cudaEventCreate(&e0));
        PK_CUDA(cudaEventCreate(&e1));
        const bool ok[kLayouts] = {layout_ok(0), layout_ok(1), layout_ok(2), layout_ok(3), layout_ok(4), layout_ok(5)};
        auto once = [&](int k) {
            if (f32) gs_sym<float>(p->fine, p->bw_r32, p->bw_zs32, true, k, s);
            else gs_sym<double>(p->fine, p->bw_r, p->bw_zs, true, k, s);
        };
        // round-robin rounds (the clock may still be ramping up), best round per layout
        float ms_best[kLayouts];
        for (int k = 0; k < kLayouts; ++k) {
            ms_best[k] = 1e30f;
            if (ok[k]) once(k);
        }
        for (int round = 0; round < 3; ++round)
            for (int k = 0; k < kLayouts; ++k) {
                if (!ok[k]) continue;
                PK_CUDA(cudaEventRecord(e0, s));
                for (int r = 0; r < 2; ++r) once(k);
                PK_CUDA(cudaEventRecord(e1, s));
                PK_CUDA(cudaEventSynchronize(e1));
                float ms = 0;
                PK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                ms_best[k] = std::min(ms_best[k], ms);
            }
        for (int k = 0; k < kLayouts; ++k)
            if (ok[k] && ms_best[k] < best_ms) {
                best_ms = ms_best[k];
                best = k;
            }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return best + 1;
    }

    // device time of one blocked operation on the work blocks (input: the last RHS block)
    static float time_op(pkasp_problem *p, int which, int reps, cudaStream_t s) {
        kb_state_reset<<<1, PKASP_MAX_COLS, 0, s>>>(p->d_state, NC, NC, p->opt.tol, p->opt.max_iter, 1);
        PK_LAUNCH();
        PK_CUDA(cudaMemcpyAsync(p->bw_p, p->bw_b, sizeof(double) * p->nh * NC, cudaMemcpyDeviceToDevice, s));
        const bool f32 = p->opt.precond_precision == PKASP_PREC_FP32;
        const int64_t ne = p->nh * NC;
        kb_copy<float, double><<<(unsigned)((ne + kBlock - 1) / kBlock), kBlock, 0, s>>>(ne, p->bw_b, p->bw_r32);
        PK_LAUNCH();
        auto once = [&]() {
            if (which == 4) {
                kb_spmv_pq<NC><<<kRedGrid, kBlock, 0, s>>>(p->nh, p->Ah.ptr, p->Ah.col, p->Ah.val, p->bw_p,
                                                           p->bw_q, p->d_state, p->d_partials, p->d_counter);
                PK_LAUNCH();
            } else if (which == 5) {
                if (f32) gs_sym<float>(p->fine, p->bw_r32, p->bw_zs32, true, p->bchunk - 1, s);
                else gs_sym<double>(p->fine, p->bw_b, p->bw_zs, true, p->bchunk - 1, s);
            } else {
                prec(p, p->bw_b, p->bw_z, s);
            }
        };
        for (int i = 0; i < 3; ++i) once();
        cudaEvent_t e0, e1;
        PK_CUDA(cudaEventCreate(&e0));
        PK_CUDA(cudaEventCreate(&e1));
        PK_CUDA(cudaEventRecord(e0, s));
        for (int i = 0; i < reps; ++i) once();
        PK_CUDA(cudaEventRecord(e1, s));
        PK_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return ms / reps;
    }

    // Z = B R: the FP32 preconditioner reads the FP32 copy of R in bw_r32 (written by the
    // kernel that produced R), the FP64 one reads R itself
    static void prec(pkasp_problem *p, const double *R, double *Z, cudaStream_t s) {
        if (p->opt.precond_precision == PKASP_PREC_FP32) precondition<float>(p, p->bw_r32, Z, s);
        else precondition<double>(p, R, Z, s);
    }
    static float *r32_out(pkasp_problem *p) {
        return p->opt.precond_precision == PKASP_PREC_FP32 ? p->bw_r32 : nullptr;
    }

    static void init(pkasp_problem *p, const double *B, double *X, cudaStream_t s) {
        kb_init_residual<NC><<<kRedGrid, kBlock, 0, s>>>(p->nh, p->Ah.ptr, p->Ah.col, p->Ah.val, B, X, p->bw_r,
                                                         r32_out(p), p->d_state, p->d_partials, p->d_counter,
                                                         p->d_hist);
        PK_LAUNCH();
        prec(p, p->bw_r, p->bw_z, s);
        kb_start<NC><<<kRedGrid, FlatBT<NC>, 0, s>>>(p->nh * NC, p->bw_r, p->bw_z, p->bw_p, p->d_state,
                                                     p->d_partials, p->d_counter);
        PK_LAUNCH();
    }

    static void iteration(pkasp_problem *p, double *X, cudaStream_t s) {
        kb_spmv_pq<NC><<<kRedGrid, kBlock, 0, s>>>(p->nh, p->Ah.ptr, p->Ah.col, p->Ah.val, p->bw_p, p->bw_q,
                                                   p->d_state, p->d_partials, p->d_counter);
        PK_LAUNCH();
        kb_update_xr<NC><<<kRedGrid, FlatBT<NC>, 0, s>>>(p->nh * NC, X, p->bw_r, r32_out(p), p->bw_p, p->bw_q,
                                                         p->d_state, p->d_partials, p->d_counter, p->d_hist);
        PK_LAUNCH();
        prec(p, p->bw_r, p->bw_z, s);
        const int flex = (p->opt.flexible || p->opt.precond_precision == PKASP_PREC_FP32) ? 1 : 0;
        kb_beta<NC><<<kRedGrid, FlatBT<NC>, 0, s>>>(p->nh * NC, p->bw_r, p->bw_z, p->bw_q, flex, p->d_state,
                                                    p->d_partials, p->d_counter);
        PK_LAUNCH();
        kb_update_p<NC><<<kRedGrid, FlatBT<NC>, 0, s>>>(p->nh * NC, p->bw_z, p->bw_p, p->d_state);
        PK_LAUNCH();
    }

    static void final_(pkasp_problem *p, const double *B, const double *X, cudaStream_t s) {
        kb_true_residual<NC><<<kRedGrid, kBlock, 0, s>>>(p->nh, p->Ah.ptr, p->Ah.col, p->Ah.val, B, X, p->d_state,
                                                         p->d_partials, p->d_counter);
        PK_LAUNCH();
    }

    static void build_graph(pkasp_problem *p, const double *B, double *X) {
        if (p->bgraph_exec) cudaGraphExecDestroy(p->bgraph_exec);
        if (p->bgraph) cudaGraphDestroy(p->bgraph);
        p->bgraph_exec = nullptr;
        p->bgraph = nullptr;
        cudaStream_t cs = p->cap_stream;
        cudaGraph_t g, gi, gf;
        PK_CUDA(cudaGraphCreate(&g, 0));
        PK_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        long long c0 = launch_count();
        init(p, B, X, cs);
        p->bg_init = launch_count() - c0;
        PK_CUDA(cudaStreamEndCapture(cs, &gi));
        cudaGraphNode_t ni, nc, nf;
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
        iteration(p, X, cs);
        kb_loop_control<<<1, 32, 0, cs>>>(p->d_state, h);
        PK_LAUNCH();
        p->bg_body = launch_count() - c0;
        PK_CUDA(cudaStreamEndCapture(cs, &body));
        PK_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        c0 = launch_count();
        final_(p, B, X, cs);
        p->bg_final = launch_count() - c0;
        PK_CUDA(cudaStreamEndCapture(cs, &gf));
        PK_CUDA(cudaGraphAddChildGraphNode(&nf, g, &nc, 1, gf));
        PK_CUDA(cudaGraphInstantiate(&p->bgraph_exec, g, 0));
        cudaGraphDestroy(gi);
        cudaGraphDestroy(gf);
        p->bgraph = g;
    }
};

template <int NC>
int solve_nc(pkasp_problem *p, const double *b, double *x, int ncols, int64_t ld, pkasp_stats *st, cudaStream_t s) {
    const int hist_rows = (st && st->hist_cap > 0) ? st->hist_cap : 1;
    ensure_batched(p, NC, hist_rows * NC);
    if (p->bchunk == 0) {
        p->bchunk = Batched<NC>::tune_group(p, s);
        p->bgroup_cols = Batched<NC>::layout_ch(p->bchunk - 1);
        p->blanes = Batched<NC>::layout_w(p->bchunk - 1);
    }
    const int64_t n = p->nh, ne = n * NC;
    const unsigned eg = (unsigned)((ne + kBlock - 1) / kBlock);
    kb_gather<<<eg, kBlock, 0, s>>>(n, ncols, ld, NC, b, p->bw_b);
    PK_LAUNCH();
    kb_gather<<<eg, kBlock, 0, s>>>(n, ncols, ld, NC, x, p->bw_x);
    PK_LAUNCH();
    double *saved_hist = p->d_hist;
    p->d_hist = p->bw_hist;
    kb_state_reset<<<1, PKASP_MAX_COLS, 0, s>>>(p->d_state, NC, ncols, p->opt.tol, p->opt.max_iter, hist_rows);
    PK_LAUNCH();
    cudaEvent_t e0, e1;
    PK_CUDA(cudaEventCreate(&e0));
    PK_CUDA(cudaEventCreate(&e1));
    PK_CUDA(cudaEventRecord(e0, s));
    const bool use_graph = p->opt.use_graph != 0;
    if (use_graph && !p->bgraph_exec) {
        PK_CUDA(cudaStreamSynchronize(s));
        Batched<NC>::build_graph(p, p->bw_b, p->bw_x);
    }
    long long launches = 4;  // two gathers, the state reset, the scatter
    const long long eager0 = launch_count();
    PcgState hs;
    int restarts = 0;
    for (;;) {
        if (use_graph) {
            PK_CUDA(cudaGraphLaunch(p->bgraph_exec, s));
        } else {
            Batched<NC>::init(p, p->bw_b, p->bw_x, s);
            for (int it = 0; it <= p->opt.max_iter + 1; ++it) {
                Batched<NC>::iteration(p, p->bw_x, s);
                int ad = 0;
                PK_CUDA(cudaMemcpyAsync(&ad, &p->d_state->all_done, sizeof(int), cudaMemcpyDeviceToHost, s));
                PK_CUDA(cudaStreamSynchronize(s));
                if (ad) break;
            }
            Batched<NC>::final_(p, p->bw_b, p->bw_x, s);
        }
        PK_CUDA(cudaMemcpyAsync(&hs, p->d_state, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
        PK_CUDA(cudaStreamSynchronize(s));
        if (use_graph) launches += p->bg_init + (long long)hs.loops * p->bg_body + p->bg_final;
        // one restart for the columns whose true residual is above the tolerance
        int mask[PKASP_MAX_COLS] = {0};
        bool any = false;
        for (int c = 0; c < ncols; ++c)
            if (hs.status[c] == PKASP_OK && hs.r0[c] > 0 && hs.tnorm[c] > p->opt.tol * hs.r0[c] &&
                hs.iter[c] < p->opt.max_iter) {
                mask[c] = 1;
                any = true;
            }
        if (any && restarts == 0) {
            ++restarts;
            PK_CUDA(cudaMemcpyAsync(p->bw_mask, mask, sizeof(mask), cudaMemcpyHostToDevice, s));
            kb_state_restart<<<1, PKASP_MAX_COLS, 0, s>>>(p->d_state, p->bw_mask);
            PK_LAUNCH();
            ++launches;
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
    kb_scatter<<<eg, kBlock, 0, s>>>(n, ncols, ld, NC, p->bw_x, x);
    PK_LAUNCH();
    p->d_hist = saved_hist;
    int rc = PKASP_OK;
    for (int c = 0; c < ncols; ++c) {
        int stc = hs.status[c] < 0 ? PKASP_ENOTCONV : hs.status[c];
        if (stc != PKASP_OK && rc == PKASP_OK) rc = stc;
    }
    if (st) {
        st->ncols = ncols;
        int maxit = 0;
        for (int c = 0; c < ncols; ++c) {
            st->iters[c] = hs.iter[c];
            st->status[c] = hs.status[c] < 0 ? PKASP_ENOTCONV : hs.status[c];
            st->true_rel[c] = hs.r0[c] > 0 ? hs.tnorm[c] / hs.r0[c] : 0.0;
            maxit = std::max(maxit, hs.iter[c]);
        }
        st->restarts = restarts;
        st->solve_ms = ms;
        st->kernel_launches = use_graph ? launches : 3 + (launch_count() - eager0);
        st->hist_len = std::min(maxit + 1, st->hist_cap);
        if (st->hist_host && st->hist_len > 0) {
            // device history is [row][NC]; the caller's buffer is [row][ncols]
            std::vector<double> h((size_t)st->hist_len * NC);
            PK_CUDA(cudaMemcpy(h.data(), p->bw_hist, sizeof(double) * h.size(), cudaMemcpyDeviceToHost));
            for (int r = 0; r < st->hist_len; ++r)
                for (int c = 0; c < ncols; ++c)
                    st->hist_host[(size_t)r * ncols + c] = (r <= hs.iter[c]) ? h[(size_t)r * NC + c] : 0.0;
        }
    }
    return rc;
}

}  // namespace
}  // namespace pk

// the two entry points of one block width, defined in that width's translation unit
#define PK_BATCHED_WIDTH(NC)                                                                         \
    namespace pk {                                                                                   \
    int solve_block_##NC(pkasp_problem *p, const double *b, double *x, int ncols, int64_t ld,        \
                         pkasp_stats *st, cudaStream_t s) {                                          \
        return solve_nc<NC>(p, b, x, ncols, ld, st, s);                                              \
    }                                                                                                \
    float time_block_##NC(pkasp_problem *p, int which, int reps, cudaStream_t s) {                   \
        return Batched<NC>::time_op(p, which, reps, s);                                              \
    }                                                                                                \
    }
