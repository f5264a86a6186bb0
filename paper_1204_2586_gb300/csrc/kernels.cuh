// kernels.cuh -- hot-path kernels of one PCG iteration: CSR SpMV, the colour phases of
// the multicolour Gauss-Seidel smoothers, l1-Jacobi, the transfer operators I_P / I_R
// (Eq. 10), the dense coarsest solve and the fused PCG vector updates.
//
// Rows are processed by sub-warps of TPR lanes (TPR in {4, 8, 16, 32}): the lanes of a
// sub-warp stride over the row's entries, so the column and value loads of consecutive
// lanes are coalesced, and the partial sums meet in a fixed xor-shuffle tree. Every
// reduction uses a fixed grid and a fixed summation tree, so results are bitwise
// reproducible from run to run.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace pk {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kBlock = 256;
constexpr int kRedGrid = 152 * 4;  // fixed grid of the reduction kernels

template <typename T>
__device__ __forceinline__ T ldg(const T *p) {
    return __ldg(p);
}

// Matrix entries are read once per application and streamed: loads marked evict-first
// (ld.global.cs) keep them from pushing the gathered vector out of L2, which the colour
// phases and the SpMV read many times.
template <typename T>
__device__ __forceinline__ T ldst(const T *p) {
    return __ldcs(p);
}

// sum over the TPR lanes of a sub-warp (every lane of the warp must call this)
template <int TPR, typename A>
__device__ __forceinline__ A subwarp_sum(A v) {
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Entries per batch: a lane issues the column and value loads of kBatch entries (as
// predicated loads) before the first dependent gather of x, so the whole batch's memory
// traffic is in flight at once. Small colour phases are latency-bound and need this.
constexpr int kBatch = 8;

// sum_{e in [lo,hi)} val[e] * x[col[e]] accumulated in A by the lanes of a sub-warp,
// lane `sub` adding entries lo+sub, lo+sub+TPR, ... in that order
template <int TPR, typename A, typename VT, typename XT, int NB = kBatch>
__device__ __forceinline__ A row_dot(int64_t lo, int64_t hi, int sub, const int32_t *__restrict__ col,
                                     const VT *__restrict__ val, const XT *__restrict__ x) {
    A acc = A(0);
    for (int64_t base = lo + sub; base < hi; base += NB * TPR) {
        int c[NB];
        A v[NB];
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            const int64_t e = base + (int64_t)k * TPR;
            const bool ok = e < hi;
            c[k] = ok ? ldg(&col[e]) : -1;
            v[k] = ok ? (A)ldg(&val[e]) : A(0);
        }
#pragma unroll
        for (int k = 0; k < NB; ++k)
            if (c[k] >= 0) acc += v[k] * (A)ldg(&x[c[k]]);
    }
    return subwarp_sum<TPR>(acc);
}

// ---------------------------------------------------------------------------------
// Deterministic reductions. The order of every addition is fixed by the grid alone,
// never by timing.
//  - strided_sum: thread t of a block adds a[lo + t], a[lo + t + blockDim], ... below
//    hi in that order (loads issued eight at a time).
//  - block_partials: a warp shuffle tree, then the block's warps in order, into
//    partials[block].
//  - grid_reduce: the last block to arrive (fence and atomic counter) adds the block
//    partials with strided_sum and a block tree.
// The PCG's reductions run in element-wise kernels of kRedGrid blocks. GB300 issues one
// warp-wide FP64 instruction per 16 cycles per SM, so a shuffle tree of doubles at the
// end of every warp of a one-row-per-thread SpMV (5 adds per 32 rows) costs about as
// much as streaming the operand vectors once more: the PCG's fine SpMV writes q only,
// and the dot products read their vectors in a kernel of their own. FGMRES's residual
// and the Stokes operator (off the headline path) still reduce inside their full-grid
// kernels.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ double strided_sum(const double *a, int64_t lo, int64_t hi, int stride_nv, int q) {
    constexpr int U = 8;
    const int64_t bd = blockDim.x;
    double x = 0.0;
    for (int64_t b0 = lo + threadIdx.x; b0 < hi; b0 += U * bd) {
        double t[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t b = b0 + u * bd;
            t[u] = b < hi ? __ldcg(&a[b * stride_nv + q]) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (b0 + u * bd < hi) x += t[u];
    }
    return x;
}

template <int NV>
__device__ __forceinline__ void block_partials(double (&v)[NV], double *partials) {
    __shared__ double sh[NV][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double x = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
        if (lane == 0) sh[q][wid] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += sh[q][w];
            partials[(int64_t)blockIdx.x * NV + q] = s;
        }
    }
}

template <int NV>
__device__ __forceinline__ bool grid_reduce(double (&v)[NV], double *partials, unsigned *counter,
                                            double (&tot)[NV]) {
    __shared__ double sh[NV][32];
    __shared__ int last;
    block_partials<NV>(v, partials);
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned prev = atomicAdd(counter, 1u);
        last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double x = strided_sum(partials, 0, gridDim.x, NV, q);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
        if (lane == 0) sh[q][wid] = x;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += sh[q][w];
        tot[q] = s;
    }
    if (threadIdx.x == 0) *counter = 0u;
    return true;
}

// ---------------------------------------------------------------------------------
// Plain CSR SpMV y = A x (transfer operators, level residual parts)
// ---------------------------------------------------------------------------------
template <int TPR, typename A, typename VT, typename XT, typename YT>
__global__ void __launch_bounds__(kBlock) k_spmv(int64_t n, const int64_t *__restrict__ ptr,
                                                 const int32_t *__restrict__ col, const VT *__restrict__ val,
                                                 const XT *__restrict__ x, YT *__restrict__ y) {
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t row = gt / TPR;
    const int sub = threadIdx.x & (TPR - 1);
    const bool ok = row < n;
    int64_t lo = ok ? ptr[row] : 0, hi = ok ? ptr[row + 1] : 0;
    A s = row_dot<TPR, A>(lo, hi, sub, col, val, x);
    if (ok && sub == 0) y[row] = (YT)s;
}

// Restriction fused with the l1-Jacobi pre-smoothing step from zero of the level it
// feeds: b = R x (as k_spmv) and x_c = b / l1 (as k_jacobi0) in one pass, bitwise the two
// kernels' results.
template <int TPR, typename A, typename VT, typename XT, typename PT>
__global__ void __launch_bounds__(kBlock) k_restrict_jacobi0(int64_t n, const int64_t *__restrict__ ptr,
                                                             const int32_t *__restrict__ col,
                                                             const VT *__restrict__ val, const XT *__restrict__ x,
                                                             const PT *__restrict__ l1, PT *__restrict__ b,
                                                             PT *__restrict__ xc) {
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t row = gt / TPR;
    const int sub = threadIdx.x & (TPR - 1);
    const bool ok = row < n;
    int64_t lo = ok ? ptr[row] : 0, hi = ok ? ptr[row + 1] : 0;
    A s = row_dot<TPR, A>(lo, hi, sub, col, val, x);
    if (ok && sub == 0) {
        const PT bi = (PT)s;
        b[row] = bi;
        xc[row] = bi / l1[row];
    }
}

// b = I_P^T x with I_P^T's values given by one-byte codes (value tab[code]), fused like
// k_restrict_jacobi0 with the level's first l1-Jacobi step xc = b / l1; the same lanes,
// batches and order of additions as row_dot, so the result equals k_restrict_jacobi0's
template <int TPR, typename PT, typename XT>
__global__ void __launch_bounds__(kBlock) k_restrict_code_jacobi0(int64_t n, const int64_t *__restrict__ ptr,
                                                                  const int32_t *__restrict__ col,
                                                                  const uint8_t *__restrict__ code,
                                                                  const PT *__restrict__ tab,
                                                                  const XT *__restrict__ x,
                                                                  const PT *__restrict__ l1, PT *__restrict__ b,
                                                                  PT *__restrict__ xc) {
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t row = gt / TPR;
    const int sub = threadIdx.x & (TPR - 1);
    const bool ok = row < n;
    const int64_t lo = ok ? ptr[row] : 0, hi = ok ? ptr[row + 1] : 0;
    PT acc = PT(0);
    for (int64_t base = lo + sub; base < hi; base += kBatch * TPR) {
        int c[kBatch];
        PT v[kBatch];
#pragma unroll
        for (int k = 0; k < kBatch; ++k) {
            const int64_t e = base + (int64_t)k * TPR;
            const bool in = e < hi;
            c[k] = in ? ldg(&col[e]) : -1;
            v[k] = in ? ldg(&tab[ldg(&code[e])]) : PT(0);
        }
#pragma unroll
        for (int k = 0; k < kBatch; ++k)
            if (c[k] >= 0) acc += v[k] * (PT)ldg(&x[c[k]]);
    }
    acc = subwarp_sum<TPR>(acc);
    if (ok && sub == 0) {
        b[row] = acc;
        xc[row] = acc / l1[row];
    }
}

// r = b - A x
template <int TPR, typename A, typename VT, typename T>
__global__ void __launch_bounds__(kBlock) k_residual(int64_t n, const int64_t *__restrict__ ptr,
                                                     const int32_t *__restrict__ col, const VT *__restrict__ val,
                                                     const T *__restrict__ b, const T *__restrict__ x,
                                                     T *__restrict__ r) {
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t row = gt / TPR;
    const int sub = threadIdx.x & (TPR - 1);
    const bool ok = row < n;
    int64_t lo = ok ? ptr[row] : 0, hi = ok ? ptr[row + 1] : 0;
    const A bi = (ok && sub == 0) ? (A)b[row] : A(0);
    A s = row_dot<TPR, A>(lo, hi, sub, col, val, x);
    if (ok && sub == 0) r[row] = (T)(bi - s);
}

// ---------------------------------------------------------------------------------
// Multicolour Gauss-Seidel colour phases on a colour split (positions p in [pb, pe)
// hold row perm[p]; L/U hold the entries of lower/higher colour).
// forward from zero:   y_i = (r_i - sum_L a_ij y_j) / a_ii
// backward from there: y_i = y_i - (sum_U a_ij y_j) / a_ii
// backward full sweep: x_i = (b_i - sum_L a_ij x_j - sum_U a_ij x_j) / a_ii
// ---------------------------------------------------------------------------------
template <int TPR, typename PT, typename TR>
__global__ void __launch_bounds__(kBlock) k_gs_fwd0(int64_t pb, int64_t pe, const int32_t *__restrict__ perm,
                                                    const int64_t *__restrict__ lptr, const int32_t *__restrict__ lcol,
                                                    const PT *__restrict__ lval, const PT *__restrict__ diag,
                                                    const TR *__restrict__ r, PT *y) {
    // every per-row load that does not depend on the row sum is issued first, so the
    // phase costs one round trip for them plus the entry loads and gathers
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t p = pb + gt / TPR;
    const int sub = threadIdx.x & (TPR - 1);
    const bool ok = p < pe;
    const bool lead = ok && sub == 0;
    const int32_t i = lead ? perm[p] : 0;
    const PT d = lead ? diag[p] : PT(1);
    int64_t lo = ok ? lptr[p] : 0, hi = ok ? lptr[p + 1] : 0;
    const PT ri = lead ? (PT)r[i] : PT(0);
    PT s = row_dot<TPR, PT>(lo, hi, sub, lcol, lval, (const PT *)y);
    if (lead) y[i] = (ri - s) / d;
}

// Programmatic dependent launch (sm_90+): a kernel launched with programmatic stream
// serialization may start while its predecessor is still running. It lets its own
// successor launch at once, loads the data no kernel of the solve writes (the matrix),
// then waits until the predecessor has finished and its writes are visible before it
// touches any vector. Without the launch attribute both instructions are no-ops.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// One colour phase of the symmetric Gauss-Seidel sweep from zero (CSR colour split):
//   BACK = false: y_i = (r_i - sum_L a_ij y_j) / a_ii
//   BACK = true:  y_i = y_i - (sum_U a_ij y_j) / a_ii
// Static loads (position, bounds, diagonal, first batch of the row's entries) happen
// before the dependency wait, so they overlap the previous phase. A lane takes NB
// entries per batch (entries sub, sub + TPR, ...): NB is fitted to the colour's longest
// row part, because every FMA slot of a batch is issued whether its entry exists or not
// and GB300's FP64 pipe is narrow. Lane `sub` adds its entries in ascending order for
// every NB, so the result does not depend on NB.
template <int TPR, int NB, typename PT, typename TR, bool BACK>
__global__ void __launch_bounds__(kBlock) k_gs_phase(int64_t pb, int64_t pe, const int32_t *__restrict__ perm,
                                                     const int64_t *__restrict__ xptr, const int32_t *__restrict__ xcol,
                                                     const PT *__restrict__ xval, const PT *__restrict__ dinv,
                                                     const TR *r, PT *y) {
    pdl_trigger();
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t p = pb + gt / TPR;
    const int sub = threadIdx.x & (TPR - 1);
    const bool ok = p < pe;
    const bool lead = ok && sub == 0;
    const int32_t i = lead ? perm[p] : 0;
    const PT di = lead ? dinv[p] : PT(1);
    const int64_t lo = ok ? xptr[p] : 0, hi = ok ? xptr[p + 1] : 0;
    int c[NB];
    PT v[NB];
    const int64_t b0 = lo + sub;
#pragma unroll
    for (int k = 0; k < NB; ++k) {
        const int64_t e = b0 + (int64_t)k * TPR;
        const bool in = e < hi;
        c[k] = in ? ldst(&xcol[e]) : -1;
        v[k] = in ? ldst(&xval[e]) : PT(0);
    }
    // entries of the warp's busiest lane: FMA slots past it are skipped by a warp-uniform
    // branch (an issued FP64 slot costs the same whether a lane uses it or not)
    const unsigned mine = hi > b0 ? (unsigned)((hi - b0 + TPR - 1) / TPR) : 0u;
    const int wmax = (int)__reduce_max_sync(kFull, mine);
    pdl_wait();
    PT own = PT(0);
    if (lead) own = BACK ? y[i] : (PT)r[i];
    PT acc = PT(0);
#pragma unroll
    for (int k = 0; k < NB; ++k)
        if (k < wmax && c[k] >= 0) acc += v[k] * y[c[k]];
    for (int k0 = NB; k0 < wmax; k0 += NB) {
        const int64_t base = b0 + (int64_t)k0 * TPR;
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            const int64_t e = base + (int64_t)k * TPR;
            const bool in = e < hi;
            c[k] = in ? ldst(&xcol[e]) : -1;
            v[k] = in ? ldst(&xval[e]) : PT(0);
        }
#pragma unroll
        for (int k = 0; k < NB; ++k)
            if (k0 + k < wmax && c[k] >= 0) acc += v[k] * y[c[k]];
    }
    acc = subwarp_sum<TPR>(acc);
    if (lead) y[i] = BACK ? own - acc * di : (own - acc) * di;
}

// The loads of a colour phase without its dependency: every position of [0, n) at
// once, out[i] = dinv_i * sum_part a_ij x_j with x read-only (a measurement of the
// smoother's memory work without the barriers between colours; not used by a solve).
template <int TPR, int NB, typename PT>
__global__ void __launch_bounds__(kBlock) k_split_pass(int64_t n, const int32_t *__restrict__ perm,
                                                       const int64_t *__restrict__ xptr,
                                                       const int32_t *__restrict__ xcol,
                                                       const PT *__restrict__ xval, const PT *__restrict__ dinv,
                                                       const PT *__restrict__ x, PT *__restrict__ out) {
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t p = gt / TPR;
    const int sub = threadIdx.x & (TPR - 1);
    const bool ok = p < n;
    const int64_t lo = ok ? xptr[p] : 0, hi = ok ? xptr[p + 1] : 0;
    PT acc = PT(0);
    for (int64_t base = lo + sub; base < hi; base += (int64_t)NB * TPR) {
        int c[NB];
        PT v[NB];
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            const int64_t e = base + (int64_t)k * TPR;
            const bool in = e < hi;
            c[k] = in ? ldst(&xcol[e]) : -1;
            v[k] = in ? ldst(&xval[e]) : PT(0);
        }
#pragma unroll
        for (int k = 0; k < NB; ++k)
            if (c[k] >= 0) acc += v[k] * x[c[k]];
    }
    acc = subwarp_sum<TPR>(acc);
    if (ok && sub == 0) out[perm[p]] = acc * dinv[p];
}

// The same phase over a capped grid: sub-warp g takes rows pb + g, pb + g + nsub, ...
// (nsub sub-warps in the grid) and loads the next row's position, diagonal and first
// batch of entries while the current row's gathers are in flight, with the bounds of
// the row after that one step further ahead. Each row's sum is formed exactly as in
// k_gs_phase<TPR, NB> (bitwise the same result). The grid is at most the blocks that
// are resident at once, so on phases of several waves no block waits for a slot and
// every lane group keeps a row's loads in flight behind the current one.
// The loop runs while the warp's first sub-warp has a row, so every lane of the warp
// reaches the shuffles; a sub-warp past the end takes no entries and stores nothing.
template <int TPR, int NB, typename PT>
__device__ __forceinline__ void gs_row_static(int64_t q, bool ok, bool lead, int sub, int64_t lo, int64_t hi,
                                              const int32_t *__restrict__ perm, const int32_t *__restrict__ xcol,
                                              const PT *__restrict__ xval, const PT *__restrict__ dinv,
                                              int32_t &i, PT &di, int (&c)[NB], PT (&v)[NB]) {
    i = (ok && lead) ? perm[q] : 0;
    di = (ok && lead) ? dinv[q] : PT(1);
    const int64_t b0 = lo + sub;
#pragma unroll
    for (int k = 0; k < NB; ++k) {
        const int64_t e = b0 + (int64_t)k * TPR;
        const bool in = e < hi;
        c[k] = in ? ldst(&xcol[e]) : -1;
        v[k] = in ? ldst(&xval[e]) : PT(0);
    }
}

template <int TPR, int NB, typename PT, typename TR, bool BACK>
__global__ void __launch_bounds__(kBlock) k_gs_phase_gs(int64_t pb, int64_t pe, const int32_t *__restrict__ perm,
                                                        const int64_t *__restrict__ xptr,
                                                        const int32_t *__restrict__ xcol,
                                                        const PT *__restrict__ xval, const PT *__restrict__ dinv,
                                                        const TR *r, PT *y) {
    pdl_trigger();
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nsub = (int64_t)gridDim.x * blockDim.x / TPR;
    const int sub = threadIdx.x & (TPR - 1);
    const bool lead = sub == 0;
    int64_t p = pb + gt / TPR;
    int64_t pw = pb + (gt & ~(int64_t)31) / TPR;  // the warp's first sub-warp's row
    bool ok = p < pe;
    int64_t lo = ok ? xptr[p] : 0, hi = ok ? xptr[p + 1] : 0;
    int32_t i;
    PT di;
    int c[NB];
    PT v[NB];
    gs_row_static<TPR, NB, PT>(p, ok, lead, sub, lo, hi, perm, xcol, xval, dinv, i, di, c, v);
    int64_t pn = p + nsub;
    int64_t lon = pn < pe ? xptr[pn] : 0, hin = pn < pe ? xptr[pn + 1] : 0;
    pdl_wait();
    while (pw < pe) {
        // next row: static loads now, consumed in the next pass
        const bool okn = pn < pe;
        int32_t i_n;
        PT di_n;
        int cn[NB];
        PT vn[NB];
        gs_row_static<TPR, NB, PT>(pn, okn, lead, sub, lon, hin, perm, xcol, xval, dinv, i_n, di_n, cn, vn);
        const int64_t pnn = pn + nsub;
        const int64_t lonn = pnn < pe ? xptr[pnn] : 0, hinn = pnn < pe ? xptr[pnn + 1] : 0;
        // this row
        PT own = PT(0);
        if (ok && lead) own = BACK ? y[i] : (PT)r[i];
        PT acc = PT(0);
#pragma unroll
        for (int k = 0; k < NB; ++k)
            if (c[k] >= 0) acc += v[k] * y[c[k]];
        for (int64_t base = lo + sub + (int64_t)NB * TPR; base < hi; base += (int64_t)NB * TPR) {
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                const int64_t e = base + (int64_t)k * TPR;
                const bool in = e < hi;
                c[k] = in ? ldst(&xcol[e]) : -1;
                v[k] = in ? ldst(&xval[e]) : PT(0);
            }
#pragma unroll
            for (int k = 0; k < NB; ++k)
                if (c[k] >= 0) acc += v[k] * y[c[k]];
        }
        acc = subwarp_sum<TPR>(acc);
        if (ok && lead) y[i] = BACK ? own - acc * di : (own - acc) * di;
        // advance
        p = pn;
        pw += nsub;
        ok = okn;
        i = i_n;
        di = di_n;
        lo = lon;
        hi = hin;
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            c[k] = cn[k];
            v[k] = vn[k];
        }
        pn = pnn;
        lon = lonn;
        hin = hinn;
    }
}

// The same phase with two rows per sub-warp: rows p and p + half of the colour (no edge
// joins two rows of one colour, so neither reads the other's result). Both rows' loads
// are issued before either row's gathers, doubling the loads in flight per lane for
// phases that are bound by load latency. Each row's sum is formed exactly as above.
template <int TPR, int NB, typename PT, typename TR, bool BACK>
__global__ void __launch_bounds__(kBlock) k_gs_phase2(int64_t pb, int64_t pe, const int32_t *__restrict__ perm,
                                                      const int64_t *__restrict__ xptr,
                                                      const int32_t *__restrict__ xcol, const PT *__restrict__ xval,
                                                      const PT *__restrict__ dinv, const TR *r, PT *y) {
    pdl_trigger();
    const int64_t half = (pe - pb + 1) / 2;
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t p0 = pb + gt / TPR;
    const int sub = threadIdx.x & (TPR - 1);
    int64_t pr[2] = {p0, p0 + half};
    bool ok[2], lead[2];
    int32_t i[2];
    PT di[2];
    int64_t lo[2], hi[2];
    int c[2][NB];
    PT v[2][NB];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        ok[q] = (q == 0 ? pr[0] < pb + half : pr[1] < pe);
        lead[q] = ok[q] && sub == 0;
        i[q] = lead[q] ? perm[pr[q]] : 0;
        di[q] = lead[q] ? dinv[pr[q]] : PT(1);
        lo[q] = ok[q] ? xptr[pr[q]] : 0;
        hi[q] = ok[q] ? xptr[pr[q] + 1] : 0;
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            const int64_t e = lo[q] + sub + (int64_t)k * TPR;
            const bool in = e < hi[q];
            c[q][k] = in ? ldst(&xcol[e]) : -1;
            v[q][k] = in ? ldst(&xval[e]) : PT(0);
        }
    }
    pdl_wait();
    PT own[2], acc[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        own[q] = PT(0);
        if (lead[q]) own[q] = BACK ? y[i[q]] : (PT)r[i[q]];
        acc[q] = PT(0);
    }
    PT x[2][NB];
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int k = 0; k < NB; ++k) x[q][k] = c[q][k] >= 0 ? y[c[q][k]] : PT(0);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
#pragma unroll
        for (int k = 0; k < NB; ++k)
            if (c[q][k] >= 0) acc[q] += v[q][k] * x[q][k];
        for (int64_t base = lo[q] + sub + (int64_t)NB * TPR; base < hi[q]; base += (int64_t)NB * TPR) {
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                const int64_t e = base + (int64_t)k * TPR;
                const bool in = e < hi[q];
                c[q][k] = in ? ldst(&xcol[e]) : -1;
                v[q][k] = in ? ldst(&xval[e]) : PT(0);
            }
#pragma unroll
            for (int k = 0; k < NB; ++k)
                if (c[q][k] >= 0) acc[q] += v[q][k] * y[c[q][k]];
        }
        acc[q] = subwarp_sum<TPR>(acc[q]);
    }
#pragma unroll
    for (int q = 0; q < 2; ++q)
        if (lead[q]) y[i[q]] = BACK ? own[q] - acc[q] * di[q] : (own[q] - acc[q]) * di[q];
}

template <int TPR, typename PT>
__global__ void __launch_bounds__(kBlock) k_gs_bwd0(int64_t pb, int64_t pe, const int32_t *__restrict__ perm,
                                                    const int64_t *__restrict__ uptr, const int32_t *__restrict__ ucol,
                                                    const PT *__restrict__ uval, const PT *__restrict__ diag,
                                                    PT *y) {
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t p = pb + gt / TPR;
    const int sub = threadIdx.x & (TPR - 1);
    const bool ok = p < pe;
    const bool lead = ok && sub == 0;
    const int32_t i = lead ? perm[p] : 0;
    const PT d = lead ? diag[p] : PT(1);
    int64_t lo = ok ? uptr[p] : 0, hi = ok ? uptr[p + 1] : 0;
    const PT yi = lead ? y[i] : PT(0);
    PT s = row_dot<TPR, PT>(lo, hi, sub, ucol, uval, (const PT *)y);
    if (lead) y[i] = yi - s / d;
}

template <int TPR, int NB, typename PT>
__global__ void __launch_bounds__(kBlock) k_gs_bwd_full(int64_t pb, int64_t pe, const int32_t *__restrict__ perm,
                                                        const int64_t *__restrict__ lptr, const int32_t *__restrict__ lcol,
                                                        const PT *__restrict__ lval, const int64_t *__restrict__ uptr,
                                                        const int32_t *__restrict__ ucol, const PT *__restrict__ uval,
                                                        const PT *__restrict__ diag, const PT *__restrict__ b,
                                                        PT *x) {
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t p = pb + gt / TPR;
    const int sub = threadIdx.x & (TPR - 1);
    const bool ok = p < pe;
    const bool lead = ok && sub == 0;
    const int32_t i = lead ? perm[p] : 0;
    const PT d = lead ? diag[p] : PT(1);
    const int64_t llo = ok ? lptr[p] : 0, lhi = ok ? lptr[p + 1] : 0;
    const int64_t ulo = ok ? uptr[p] : 0, uhi = ok ? uptr[p + 1] : 0;
    const PT bi = lead ? b[i] : PT(0);
    PT sl = row_dot<TPR, PT, PT, PT, NB>(llo, lhi, sub, lcol, lval, (const PT *)x);
    PT su = row_dot<TPR, PT, PT, PT, NB>(ulo, uhi, sub, ucol, uval, (const PT *)x);
    if (lead) x[i] = (bi - sl - su) / d;
}

// l1-Jacobi: x = r / d (from zero) and x += (b - A x) / d
template <typename PT, typename TR>
__global__ void k_jacobi0(int64_t n, const PT *__restrict__ d, const TR *__restrict__ r, PT *__restrict__ x) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = (PT)r[i] / d[i];
}

template <int TPR, typename PT>
__global__ void __launch_bounds__(kBlock) k_jacobi_step(int64_t n, const int64_t *__restrict__ ptr,
                                                        const int32_t *__restrict__ col, const PT *__restrict__ val,
                                                        const PT *__restrict__ d, const PT *__restrict__ b,
                                                        const PT *__restrict__ xin, PT *__restrict__ xout) {
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t row = gt / TPR;
    const int sub = threadIdx.x & (TPR - 1);
    const bool ok = row < n;
    int64_t lo = ok ? ptr[row] : 0, hi = ok ? ptr[row + 1] : 0;
    PT s = row_dot<TPR, PT>(lo, hi, sub, col, val, xin);
    if (ok && sub == 0) xout[row] = xin[row] + (b[row] - s) / d[row];
}

// z_i = zs_i + sum_j Pi_ij w_j (I_P has at most 4 entries per row: one thread per row)
template <typename PT, typename ZT>
__global__ void k_prolong_add(int64_t n, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                              const PT *__restrict__ val, const PT *__restrict__ w, const PT *zs, ZT *z) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    PT s = PT(0);
    for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) s += val[e] * w[col[e]];
    z[i] = (ZT)zs[i] + (ZT)s;
}

// x_i += sum_j P_ij xc_j
template <int TPR, typename PT>
__global__ void __launch_bounds__(kBlock) k_prolong_inplace(int64_t n, const int64_t *__restrict__ ptr,
                                                            const int32_t *__restrict__ col,
                                                            const PT *__restrict__ val, const PT *__restrict__ xc,
                                                            PT *__restrict__ x) {
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t row = gt / TPR;
    const int sub = threadIdx.x & (TPR - 1);
    const bool ok = row < n;
    int64_t lo = ok ? ptr[row] : 0, hi = ok ? ptr[row + 1] : 0;
    const PT xi = (ok && sub == 0) ? x[row] : PT(0);
    PT s = row_dot<TPR, PT>(lo, hi, sub, col, val, xc);
    if (ok && sub == 0) x[row] = xi + s;
}

// x = Ainv b for the dense inverse of the coarsest matrix (one warp per row)
template <typename PT>
__global__ void k_dense_mv(int64_t n, const PT *__restrict__ Ainv, const PT *__restrict__ b, PT *__restrict__ x) {
    const int lane = threadIdx.x & 31;
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= n) return;  // whole warp leaves together
    PT s = PT(0);
    for (int64_t j = lane; j < n; j += 32) s += Ainv[row * n + j] * b[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if (lane == 0) x[row] = s;
}

// ---------------------------------------------------------------------------------
// SELL-32 kernels: one thread per row; a warp is one slice, so every column and value
// load of the warp is one contiguous access. Padding entries carry column -1.
// ---------------------------------------------------------------------------------
template <typename A, typename VT, typename XT>
__device__ __forceinline__ A sell_dot(int64_t base, int w, const int32_t *__restrict__ col,
                                      const VT *__restrict__ val, const XT *x) {
    A acc = A(0);
    for (int k0 = 0; k0 < w; k0 += kBatch) {
        int c[kBatch];
        A v[kBatch];
#pragma unroll
        for (int k = 0; k < kBatch; ++k) {
            const int64_t e = base + 32 * (int64_t)(k0 + k);
            const bool ok = k0 + k < w;
            c[k] = ok ? ldst(&col[e]) : -1;
            v[k] = ok ? (A)ldst(&val[e]) : A(0);
        }
#pragma unroll
        for (int k = 0; k < kBatch; ++k)
            if (c[k] >= 0) acc += v[k] * (A)x[c[k]];
    }
    return acc;
}

// y = A x, rows in natural order
template <typename A, typename VT, typename XT, typename YT>
__global__ void __launch_bounds__(kBlock) k_sell_spmv(int64_t n, const int64_t *__restrict__ sptr,
                                                      const int32_t *__restrict__ sw, const int32_t *__restrict__ col,
                                                      const VT *__restrict__ val, const XT *__restrict__ x,
                                                      YT *__restrict__ y) {
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n) return;
    const int64_t s = row >> 5;
    y[row] = (YT)sell_dot<A>(sptr[s] + (row & 31), sw[s], col, val, x);
}

// One colour phase of the symmetric Gauss-Seidel sweep from zero over the SELL-32 slices
// [s0, s1) of a colour-sorted split, one thread per row (no reduction across lanes):
//   BACK = false: y_i = (r_i - sum_L a_ij y_j) * dinv_i
//   BACK = true:  y_i = y_i - (sum_U a_ij y_j) * dinv_i
// Padding positions (perm < 0) only carry column -1 entries. Launched with PDL: static
// loads before the dependency wait.
template <typename PT, typename TR, bool BACK>
__global__ void __launch_bounds__(kBlock) k_sell_phase(int64_t s0, int64_t s1, const int32_t *__restrict__ perm,
                                                       const int64_t *__restrict__ sptr, const int32_t *__restrict__ sw,
                                                       const int32_t *__restrict__ col, const PT *__restrict__ val,
                                                       const PT *__restrict__ dinv, const TR *r, PT *y) {
    pdl_trigger();
    const int64_t q = s0 * 32 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= s1 * 32) return;
    const int64_t s = q >> 5;
    const int32_t i = perm[q];
    const int64_t base = sptr[s] + (q & 31);
    const int w = sw[s];
    const PT di = dinv[q];
    int c[kBatch];
    PT v[kBatch];
#pragma unroll
    for (int k = 0; k < kBatch; ++k) {
        const bool in = k < w;
        c[k] = in ? ldst(&col[base + 32 * (int64_t)k]) : -1;
        v[k] = in ? ldst(&val[base + 32 * (int64_t)k]) : PT(0);
    }
    pdl_wait();
    PT own = PT(0);
    if (i >= 0) own = BACK ? y[i] : (PT)r[i];
    PT acc = PT(0);
#pragma unroll
    for (int k = 0; k < kBatch; ++k)
        if (c[k] >= 0) acc += v[k] * y[c[k]];
    for (int k0 = kBatch; k0 < w; k0 += kBatch) {
#pragma unroll
        for (int k = 0; k < kBatch; ++k) {
            const bool in = k0 + k < w;
            c[k] = in ? ldst(&col[base + 32 * (int64_t)(k0 + k)]) : -1;
            v[k] = in ? ldst(&val[base + 32 * (int64_t)(k0 + k)]) : PT(0);
        }
#pragma unroll
        for (int k = 0; k < kBatch; ++k)
            if (c[k] >= 0) acc += v[k] * y[c[k]];
    }
    if (i >= 0) y[i] = BACK ? own - acc * di : (own - acc) * di;
}

}  // namespace pk
