// persist.cuh -- the symmetric multicolour Gauss-Seidel sweep from zero (S_k of the
// additive preconditioner B = S_k + Pi B_1 Pi^T) as ONE cooperative launch.
//
// The phase-per-launch form pays a launch, a dependency resolution and a pipeline drain
// per colour; on a 857k-row P3 matrix each phase does only ~2 us of memory work. Here
// the grid stays resident and the colours are separated by a grid-wide barrier. The
// barrier spins with a bound: a block that waits more than kBarrierSpins polls sets the
// error flag, every block then leaves its loops and the host reports the failure (no
// wait in this kernel is unbounded).
//
// A row written in one phase is read by other SMs in later phases. Those reads are
// plain (coherent, not read-only-path) loads issued after the barrier's acquire, which
// the PTX memory model orders after the writers' release: the barrier's arrival is a
// fence plus an atomic, its exit an acquire load and a CTA barrier. Matrix data and r
// are read-only during the kernel and use the read-only path.
#pragma once

#include "kernels.cuh"

namespace pk {

constexpr unsigned kBarrierSpins = 1u << 20;  // polls of >= 32 ns each: >= 34 ms per barrier
// one block per SM: the barrier's cost grows with the number of arriving blocks
constexpr int kPersistBlock = 1024;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier of a cooperative launch. `arrive` counts arrivals over the whole
// launch; barrier number m (1, 2, ...) completes when it reaches m * gridDim.x. Returns
// false in every thread of the block once any block has given up.
__device__ __forceinline__ bool grid_barrier(unsigned *arrive, unsigned target, int *err) {
    __shared__ int good;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();  // this block's writes of the phase, before the arrival
        atomicAdd(arrive, 1u);
        unsigned spins = 0;
        while (ld_acquire_u32(arrive) < target) {
            if (*(volatile int *)err) {
                ok = 0;
                break;
            }
            if (++spins > kBarrierSpins) {
                atomicExch(err, 1);
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
        good = ok;
    }
    __syncthreads();
    return good != 0;
}

// sum over a row part read by the TPR lanes of a sub-warp (x written in this launch:
// plain loads, never the read-only path)
template <int TPR, typename A, typename VT>
__device__ __forceinline__ A row_dot_l2(int64_t lo, int64_t hi, int sub, const int32_t *__restrict__ col,
                                        const VT *__restrict__ val, const A *x) {
    A acc = A(0);
    for (int64_t base = lo + sub; base < hi; base += kBatch * TPR) {
        int c[kBatch];
        A v[kBatch];
#pragma unroll
        for (int k = 0; k < kBatch; ++k) {
            const int64_t e = base + (int64_t)k * TPR;
            const bool ok = e < hi;
            c[k] = ok ? ldg(&col[e]) : -1;
            v[k] = ok ? (A)ldg(&val[e]) : A(0);
        }
#pragma unroll
        for (int k = 0; k < kBatch; ++k)
            if (c[k] >= 0) acc += v[k] * x[c[k]];
    }
    return subwarp_sum<TPR>(acc);
}

// y = S r for the colour split (off: device colour offsets, ncol + 1 entries):
//   forward, colours 0..C-1:  y_i = (r_i - sum_L a_ij y_j) * dinv_i
//   backward, colours C-2..0: y_i = y_i - (sum_U a_ij y_j) * dinv_i
// Each sub-warp of TPR lanes takes rows task, task + ntask, ... of a colour; the loop
// trip count is the same for every lane of the grid (shuffles need the whole warp).
// bar[0] counts barrier arrivals, bar[1] exits; the last block to exit zeroes both.
template <int TPR, typename PT, typename TR>
__global__ void __launch_bounds__(kPersistBlock, 1) k_sgs_persistent(int ncol, const int64_t *__restrict__ off,
                                                           const int32_t *__restrict__ perm,
                                                           const int64_t *__restrict__ lptr,
                                                           const int32_t *__restrict__ lcol,
                                                           const PT *__restrict__ lval,
                                                           const int64_t *__restrict__ uptr,
                                                           const int32_t *__restrict__ ucol,
                                                           const PT *__restrict__ uval, const PT *__restrict__ dinv,
                                                           const TR *__restrict__ r, PT *y, unsigned *bar, int *err) {
    const int64_t ntask = ((int64_t)gridDim.x * blockDim.x) / TPR;
    const int64_t task = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / TPR;
    const int sub = threadIdx.x & (TPR - 1);
    unsigned phase = 0;
    bool go = true;
    for (int c = 0; c < ncol && go; ++c) {
        const int64_t pb = off[c], pe = off[c + 1];
        for (int64_t base = pb; base < pe; base += ntask) {
            const int64_t p = base + task;
            const bool ok = p < pe;
            const bool lead = ok && sub == 0;
            const int32_t i = lead ? perm[p] : 0;
            const PT di = lead ? dinv[p] : PT(1);
            const int64_t lo = ok ? lptr[p] : 0, hi = ok ? lptr[p + 1] : 0;
            const PT acc = row_dot_l2<TPR, PT>(lo, hi, sub, lcol, lval, y);
            if (lead) y[i] = ((PT)r[i] - acc) * di;
        }
        go = grid_barrier(&bar[0], (++phase) * gridDim.x, err);
    }
    for (int c = ncol - 2; c >= 0 && go; --c) {
        const int64_t pb = off[c], pe = off[c + 1];
        for (int64_t base = pb; base < pe; base += ntask) {
            const int64_t p = base + task;
            const bool ok = p < pe;
            const bool lead = ok && sub == 0;
            const int32_t i = lead ? perm[p] : 0;
            const PT di = lead ? dinv[p] : PT(1);
            const int64_t lo = ok ? uptr[p] : 0, hi = ok ? uptr[p + 1] : 0;
            const PT own = lead ? y[i] : PT(0);
            const PT acc = row_dot_l2<TPR, PT>(lo, hi, sub, ucol, uval, y);
            if (lead) y[i] = own - acc * di;
        }
        if (c > 0) go = grid_barrier(&bar[0], (++phase) * gridDim.x, err);
    }
    // the last block out resets the counters for the next launch on this stream
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&bar[1], 1u);
        if (prev == gridDim.x - 1) {
            bar[0] = 0u;
            bar[1] = 0u;
            __threadfence();
        }
    }
}

}  // namespace pk
