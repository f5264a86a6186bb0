// rowop.cuh -- the fine operator A_h as the fused Krylov kernels (PCG in solve.cu,
// FGMRES in gmres.cu) read it: the layout the setup's autotuner picked.
#pragma once

#include "kernels.cuh"

namespace pk {

// The fine operator A_h as the fused PCG kernels see it: CSR rows read by sub-warps of
// TPR lanes (TPR > 0), or SELL-32 slices read one thread per row (TPR == 0; ptr then
// holds the slice pointers and sw the slice widths).
struct RowOp {
    const int64_t *ptr;
    const int32_t *col;
    const double *val;
    const int32_t *sw;
};

inline RowOp fine_op(const pkasp_problem *p) {
    if (p->spmv_tpr == 0) return RowOp{p->Asell.sptr, p->Asell.col, p->Asell.val, p->Asell.swidth};
    return RowOp{p->Ah.ptr, p->Ah.col, p->Ah.val, nullptr};
}

// Grid of the kernels that read A_h through for_rows (some of them reduce one value
// with grid_reduce): a thread (SELL-32) or sub-warp (CSR) per row, as in the plain
// SpMV, up to the capacity of the partials buffer (kRedGrid * 4 * PKASP_MAX_COLS
// values). A grid of kRedGrid blocks striding over the rows left the SpMV at about 1.5x
// the plain one's time.
inline unsigned fine_grid(const pkasp_problem *p) {
    const int64_t threads = p->nh * (p->spmv_tpr > 0 ? p->spmv_tpr : 1);
    const int64_t g = std::max<int64_t>(1, (threads + kBlock - 1) / kBlock);
    return (unsigned)std::min<int64_t>(g, (int64_t)kRedGrid * 4 * PKASP_MAX_COLS);
}

// f(row, (A x)_row) for every row, grid-stride; every lane of a warp runs the same
// number of trips (the shuffles of the CSR form need the whole warp)
template <int TPR, class F>
__device__ __forceinline__ void for_rows(int64_t n, const RowOp &A, const double *x, F f) {
    if constexpr (TPR == 0) {
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n; row += stride) {
            const int64_t s = row >> 5;
            f(row, sell_dot<double>(A.ptr[s] + (row & 31), A.sw[s], A.col, A.val, x));
        }
    } else {
        const int sub = threadIdx.x & (TPR - 1);
        const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
        const int rpw = 32 / TPR, sg = (threadIdx.x & 31) / TPR;
        for (int64_t base = warp * rpw; base < n; base += nwarps * rpw) {
            const int64_t row = base + sg;
            const bool ok = row < n;
            int64_t lo = ok ? A.ptr[row] : 0, hi = ok ? A.ptr[row + 1] : 0;
            double s = row_dot<TPR, double>(lo, hi, sub, A.col, A.val, x);
            if (ok && sub == 0) f(row, s);
        }
    }
}

// kernel template dispatch on the fine SpMV layout (0 = SELL-32, t = CSR with t lanes)
#define PK_FMT_SWITCH(tpr, BODY)                          \
    switch (tpr) {                                        \
        case 0: { constexpr int TPR = 0; BODY; } break;   \
        case 2: { constexpr int TPR = 2; BODY; } break;   \
        case 4: { constexpr int TPR = 4; BODY; } break;   \
        case 8: { constexpr int TPR = 8; BODY; } break;   \
        case 16: { constexpr int TPR = 16; BODY; } break; \
        default: { constexpr int TPR = 32; BODY; } break; \
    }

}  // namespace pk
