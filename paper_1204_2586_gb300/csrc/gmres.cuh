// gmres.cuh -- the parts of FGMRES(m) that do not depend on the operator: the state,
// classical Gram-Schmidt twice per step (chunked dots summed in fixed order, then the
// multi-vector update), the scaling of the next Arnoldi vector, the Givens update on
// one thread, the end-of-cycle triangular solve and update of x, the restart decision
// from a true residual b - y with y = A x supplied by the caller, and the loop control
// of the CUDA-graph while loop. gmres.cu (the Poisson system) and stokes.cu (the Stokes
// system) build their solvers from these.
#pragma once

#include <algorithm>
#include <cmath>

#include "internal.h"
#include "kernels.cuh"

namespace pk {

struct GmresState {
    int j;          // current Arnoldi step of the cycle (0-based)
    int k;          // steps of the cycle that just ended
    int it;         // inner steps over all cycles
    int done;       // 1: stop
    int status;     // PKASP_OK / PKASP_ENOTCONV
    int cycle_end;  // 1: the cycle ended, run the end-of-cycle kernels
    int new_cycle;  // 1: V0 holds an unnormalised residual to start a cycle from
    int cycles;     // cycles started
    int loops;      // while-loop passes
    int maxit, m, hist_cap, maxloops;
    double r0, beta, tol, tnorm, hn;
};

namespace {

constexpr int kDotChunks = 152 * 2;  // row chunks of the Gram-Schmidt dot products

// hc_i = (w, v_i) for i <= j: block (c, i) adds rows of chunk c; the last block of
// column i adds the chunk partials in chunk order, then H(i, j) gets hc_i (pass 0) or
// hc_i added (pass 1)
__global__ void __launch_bounds__(kBlock) kg_dots(int64_t n, const double *__restrict__ V,
                                                  const double *__restrict__ w, GmresState *st, double *part,
                                                  unsigned *cnt, double *hc, double *H, int pass) {
    const int i = blockIdx.y;
    if (st->done || i > st->j) return;
    const int m = st->m, j = st->j;
    const int64_t L = (n + gridDim.x - 1) / gridDim.x;
    const int64_t lo = (int64_t)blockIdx.x * L, hi = min(n, lo + L);
    const double *vi = V + (int64_t)i * n;
    double s = 0.0;
    for (int64_t q = lo + threadIdx.x; q < hi; q += blockDim.x) s += w[q] * vi[q];
    __shared__ double sh[kBlock / 32];
    __shared__ int last;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int k = 0; k < kBlock / 32; ++k) b += sh[k];
        part[(int64_t)i * gridDim.x + blockIdx.x] = b;
        __threadfence();
        const unsigned prev = atomicAdd(&cnt[i], 1u);
        last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    // the chunk partials, summed by the whole block in a fixed tree (thread t adds chunks
    // t, t + blockDim, ... in order; then warps, then the warp sums in order)
    __threadfence();
    double t = 0.0;
    for (unsigned c = threadIdx.x; c < gridDim.x; c += blockDim.x) t += __ldcg(&part[(int64_t)i * gridDim.x + c]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double u = 0.0;
        for (int k = 0; k < kBlock / 32; ++k) u += sh[k];
        hc[i] = u;
        if (pass == 0) H[i * m + j] = u;
        else H[i * m + j] += u;
        cnt[i] = 0u;
    }
}

// w -= sum_{i <= j} hc_i v_i (in ascending i); with norm: ||w|| into H(j+1, j)
__global__ void __launch_bounds__(kBlock) kg_axpy(int64_t n, const double *__restrict__ V, double *__restrict__ w,
                                                  GmresState *st, const double *__restrict__ hc, double *H,
                                                  double *partials, unsigned *counter, int norm) {
    if (st->done) return;
    const int j = st->j;
    double part = 0.0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        double x = w[q];
#pragma unroll 4
        for (int i = 0; i <= j; ++i) x -= hc[i] * V[(int64_t)i * n + q];
        w[q] = x;
        part += x * x;
    }
    if (!norm) return;
    double v[1] = {part}, tot[1];
    if (grid_reduce<1>(v, partials, counter, tot) && threadIdx.x == 0) {
        const double hn = sqrt(tot[0]);
        st->hn = hn;
        H[(j + 1) * st->m + j] = hn;
    }
}

// v_{j+1} = w / h_{j+1,j}, also into the preconditioner's input buffer
__global__ void kg_scale_next(int64_t n, double *V, const double *__restrict__ w, double *vin, const GmresState *st) {
    if (st->done || !(st->hn > 0.0)) return;
    const double s = 1.0 / st->hn;
    double *vn = V + (int64_t)(st->j + 1) * n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = w[i] * s;
        vn[i] = v;
        vin[i] = v;
    }
}

// Givens update of column j, the residual estimate, the end-of-cycle decision
__global__ void kg_givens(GmresState *st, double *H, double *cs, double *sn, double *g, double *hist) {
    if (threadIdx.x != 0 || blockIdx.x != 0 || st->done) return;
    const int m = st->m, j = st->j;
    for (int i = 0; i < j; ++i) {
        const double a = H[i * m + j], c = H[(i + 1) * m + j];
        H[i * m + j] = cs[i] * a + sn[i] * c;
        H[(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
    }
    const double a = H[j * m + j], c = H[(j + 1) * m + j];
    const double d = sqrt(a * a + c * c);
    cs[j] = d > 0.0 ? a / d : 1.0;
    sn[j] = d > 0.0 ? c / d : 0.0;
    H[j * m + j] = d;
    H[(j + 1) * m + j] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    const int it = ++st->it;
    const double est = fabs(g[j + 1]);
    if (it < st->hist_cap) hist[it] = est;
    if (est <= st->tol * st->r0 || st->hn == 0.0 || j + 1 == m || it >= st->maxit) {
        st->cycle_end = 1;
        st->k = j + 1;
    } else {
        st->j = j + 1;
    }
}

// y = H(1:k,1:k)^{-1} g(1:k)
__global__ void kg_backsolve(const GmresState *st, const double *H, const double *g, double *y) {
    if (threadIdx.x != 0 || blockIdx.x != 0 || !st->cycle_end) return;
    const int m = st->m, k = st->k;
    for (int i = k - 1; i >= 0; --i) {
        double s = g[i];
        for (int l = i + 1; l < k; ++l) s -= H[i * m + l] * y[l];
        y[i] = s / H[i * m + i];
    }
}

// x += sum_{l < k} y_l z_l (ascending l)
__global__ void kg_update_x(int64_t n, double *x, const double *__restrict__ Z, const double *__restrict__ y,
                            const GmresState *st) {
    if (!st->cycle_end) return;
    const int k = st->k;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        double xv = x[q];
        for (int l = 0; l < k; ++l) xv += y[l] * Z[(int64_t)l * n + q];
        x[q] = xv;
    }
}

__global__ void kg_state_reset(GmresState *st, int m, double tol, int maxit, int hist_cap) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    st->j = st->k = st->it = 0;
    st->done = 0;
    st->status = -1;
    st->cycle_end = st->new_cycle = 0;
    st->cycles = st->loops = 0;
    st->m = m;
    st->tol = tol;
    st->maxit = maxit;
    st->hist_cap = hist_cap;
    // every pass of the loop is an Arnoldi step; each cycle adds one pass at most
    st->maxloops = maxit + maxit / (m > 1 ? m : 1) + 4;
    st->r0 = st->beta = st->tnorm = st->hn = 0.0;
}

__global__ void kg_loop_control(GmresState *st, cudaGraphConditionalHandle h) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int loops = ++st->loops;
    const bool go = !st->done && loops <= st->maxloops;
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

unsigned elem_blocks(int64_t n) { return (unsigned)std::min<int64_t>(152 * 8, std::max<int64_t>(1, (n + kBlock - 1) / kBlock)); }

// v0 = b - y (y = A x computed by the caller) and its norm. first: the solve's start
// (r0, hist[0]); otherwise the true residual at the end of a cycle (gated by
// cycle_end), which decides between stopping and the next cycle.
__global__ void __launch_bounds__(kBlock) kg_residual_y(int64_t n, const double *__restrict__ b,
                                                        const double *__restrict__ y, double *__restrict__ v0,
                                                        GmresState *st, double *g, double *partials,
                                                        unsigned *counter, double *hist, int first) {
    if (!first && !st->cycle_end) return;  // the same for every block
    double part = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double ri = b[i] - y[i];
        v0[i] = ri;
        part += ri * ri;
    }
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

// start of a cycle: v_0 = r / beta, also into the preconditioner's input buffer
__global__ void kg_scale_v0(int64_t n, double *v0, double *vin, const GmresState *st) {
    if (!st->new_cycle) return;
    const double s = 1.0 / st->beta;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = v0[i] * s;
        v0[i] = v;
        vin[i] = v;
    }
}

// Z[j] = zout (the preconditioned vector of step j); also clears new_cycle
__global__ void kg_store_z(int64_t n, const double *__restrict__ zout, double *__restrict__ Z, GmresState *st) {
    if (st->done) return;
    const int64_t off = (int64_t)st->j * n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        Z[off + i] = zout[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) st->new_cycle = 0;
}

}  // namespace
}  // namespace pk
