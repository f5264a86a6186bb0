// sell.cu -- SELL-32 copies of the fine-level operators for the hot kernels.
//
// A slice is 32 consecutive rows (one warp, one thread per row); its entries are
// stored column-major (entry k of the slice's row r at sptr[slice] + 32 k + r) and
// padded to the slice's longest row with column -1. Every load of a warp is then one
// contiguous 128-byte (columns) or 256-byte (FP64 values) access.
//
//  * natural order: the rows of A_h as numbered (the numbering already groups rows of
//    equal length: vertex, edge, face and interior nodes);
//  * colour split: for each colour of the multicolour Gauss-Seidel, the rows of that
//    colour sorted by decreasing length of their lower (or upper) part and padded to a
//    whole number of slices, so a colour phase is a contiguous range of slices.
#include <algorithm>
#include <numeric>

#include "internal.h"

namespace pk {
namespace {

unsigned blocks_for(int64_t n, int per) {
    int64_t b = (n + per - 1) / per;
    return (unsigned)std::max<int64_t>(1, b);
}

__global__ void k_slice_width(int64_t n, int64_t nslices, const int64_t *__restrict__ ptr,
                              int32_t *__restrict__ width) {
    int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (s >= nslices) return;  // whole warp
    int64_t row = s * 32 + lane;
    int len = row < n ? (int)(ptr[row + 1] - ptr[row]) : 0;
    for (int o = 16; o > 0; o >>= 1) len = max(len, __shfl_xor_sync(0xffffffffu, len, o));
    if (lane == 0) width[s] = len;
}

__global__ void k_sell_fill_natural(int64_t n, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                                    const double *__restrict__ val, const int64_t *__restrict__ sptr,
                                    const int32_t *__restrict__ width, int32_t *__restrict__ scol,
                                    double *__restrict__ sval) {
    int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t s = row >> 5;
    int lane = (int)(row & 31);
    int64_t nslices = (n + 31) / 32;
    if (s >= nslices) return;
    int w = width[s];
    int64_t base = sptr[s] + lane;
    int64_t lo = row < n ? ptr[row] : 0, len = row < n ? ptr[row + 1] - lo : 0;
    for (int k = 0; k < w; ++k) {
        bool real = k < len;
        scol[base + 32 * (int64_t)k] = real ? col[lo + k] : -1;
        sval[base + 32 * (int64_t)k] = real ? val[lo + k] : 0.0;
    }
}

// padded position q of a colour-split SELL takes the entries of CSR-split position
// src[q] (or none when src[q] < 0)
__global__ void k_sell_fill_split(int64_t nq, const int64_t *__restrict__ src, const int64_t *__restrict__ xptr,
                                  const int32_t *__restrict__ xcol, const double *__restrict__ xval,
                                  const double *__restrict__ xdiag, const int64_t *__restrict__ sptr,
                                  const int32_t *__restrict__ width, int32_t *__restrict__ scol,
                                  double *__restrict__ sval, double *__restrict__ sdiag) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    int64_t s = q >> 5;
    int lane = (int)(q & 31);
    int w = width[s];
    int64_t base = sptr[s] + lane;
    int64_t p = src[q];
    int64_t lo = p >= 0 ? xptr[p] : 0, len = p >= 0 ? xptr[p + 1] - lo : 0;
    for (int k = 0; k < w; ++k) {
        bool real = k < len;
        scol[base + 32 * (int64_t)k] = real ? xcol[lo + k] : -1;
        sval[base + 32 * (int64_t)k] = real ? xval[lo + k] : 0.0;
    }
    sdiag[q] = p >= 0 ? xdiag[p] : 1.0;
}

}  // namespace

void build_sell_natural(DevPool &pool, const DCSR &A, DSell &S, bool want32, cudaStream_t s) {
    const int64_t n = A.n, ns = (n + 31) / 32;
    S = DSell{};
    S.nslices = ns;
    S.npos = ns * 32;
    S.swidth = pool.get<int32_t>(ns > 0 ? ns : 1);
    if (ns > 0) {
        k_slice_width<<<blocks_for(ns * 32, 256), 256, 0, s>>>(n, ns, A.ptr, S.swidth);
        PK_LAUNCH();
    }
    std::vector<int32_t> w(ns);
    PK_CUDA(cudaMemcpyAsync(w.data(), S.swidth, sizeof(int32_t) * ns, cudaMemcpyDeviceToHost, s));
    PK_CUDA(cudaStreamSynchronize(s));
    std::vector<int64_t> sp(ns + 1, 0);
    for (int64_t i = 0; i < ns; ++i) sp[i + 1] = sp[i] + 32 * (int64_t)w[i];
    S.nnz_padded = sp[ns];
    S.sptr = pool.get<int64_t>(ns + 1);
    PK_CUDA(cudaMemcpyAsync(S.sptr, sp.data(), sizeof(int64_t) * (ns + 1), cudaMemcpyHostToDevice, s));
    S.col = pool.get<int32_t>(S.nnz_padded > 0 ? S.nnz_padded : 1);
    S.val = pool.get<double>(S.nnz_padded > 0 ? S.nnz_padded : 1);
    if (ns > 0) {
        k_sell_fill_natural<<<blocks_for(ns * 32, 256), 256, 0, s>>>(n, A.ptr, A.col, A.val, S.sptr, S.swidth,
                                                                     S.col, S.val);
        PK_LAUNCH();
    }
    if (want32) {
        S.val32 = pool.get<float>(S.nnz_padded > 0 ? S.nnz_padded : 1);
        to32(S.val, S.val32, S.nnz_padded, s);
    }
    PK_CUDA(cudaStreamSynchronize(s));
}

// upper = false: the lower (earlier colour) parts; true: the upper parts
void build_sell_split(DevPool &pool, const DSplit &sp, int64_t n, bool upper, DSell &S, bool want32,
                      cudaStream_t s) {
    S = DSell{};
    const int64_t *xptr = upper ? sp.uptr : sp.lptr;
    std::vector<int64_t> hp(n + 1);
    std::vector<int32_t> perm(n);
    PK_CUDA(cudaMemcpyAsync(hp.data(), xptr, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, s));
    PK_CUDA(cudaMemcpyAsync(perm.data(), sp.perm, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    PK_CUDA(cudaStreamSynchronize(s));
    // per colour: positions sorted by decreasing part length (ties by position), padded
    std::vector<int64_t> src;   // padded position -> CSR-split position or -1
    std::vector<int32_t> row;   // padded position -> row or -1
    std::vector<int32_t> width; // per slice
    S.coff.assign(sp.ncol + 1, 0);
    std::vector<int64_t> order;
    for (int c = 0; c < sp.ncol; ++c) {
        const int64_t pb = sp.off[c], pe = sp.off[c + 1];
        order.resize(pe - pb);
        std::iota(order.begin(), order.end(), pb);
        std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
            return (hp[a + 1] - hp[a]) > (hp[b + 1] - hp[b]);
        });
        const int64_t m = (int64_t)order.size(), padded = (m + 31) / 32 * 32;
        for (int64_t q = 0; q < padded; ++q) {
            if (q < m) {
                src.push_back(order[q]);
                row.push_back(perm[order[q]]);
            } else {
                src.push_back(-1);
                row.push_back(-1);
            }
            if (q % 32 == 0) width.push_back(q < m ? (int32_t)(hp[order[q] + 1] - hp[order[q]]) : 0);
        }
        S.coff[c + 1] = (int64_t)width.size();
    }
    const int64_t ns = (int64_t)width.size();
    S.nslices = ns;
    S.npos = ns * 32;
    std::vector<int64_t> spt(ns + 1, 0);
    for (int64_t i = 0; i < ns; ++i) spt[i + 1] = spt[i] + 32 * (int64_t)width[i];
    S.nnz_padded = spt[ns];
    S.perm = pool.get<int32_t>(S.npos > 0 ? S.npos : 1);
    S.swidth = pool.get<int32_t>(ns > 0 ? ns : 1);
    S.sptr = pool.get<int64_t>(ns + 1);
    S.col = pool.get<int32_t>(S.nnz_padded > 0 ? S.nnz_padded : 1);
    S.val = pool.get<double>(S.nnz_padded > 0 ? S.nnz_padded : 1);
    S.diag = pool.get<double>(S.npos > 0 ? S.npos : 1);
    DevPool tmp;
    try {
        int64_t *dsrc = tmp.get<int64_t>(S.npos > 0 ? S.npos : 1);
        PK_CUDA(cudaMemcpyAsync(S.perm, row.data(), sizeof(int32_t) * S.npos, cudaMemcpyHostToDevice, s));
        PK_CUDA(cudaMemcpyAsync(S.swidth, width.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, s));
        PK_CUDA(cudaMemcpyAsync(S.sptr, spt.data(), sizeof(int64_t) * (ns + 1), cudaMemcpyHostToDevice, s));
        PK_CUDA(cudaMemcpyAsync(dsrc, src.data(), sizeof(int64_t) * S.npos, cudaMemcpyHostToDevice, s));
        if (S.npos > 0) {
            k_sell_fill_split<<<blocks_for(S.npos, 256), 256, 0, s>>>(
                S.npos, dsrc, xptr, upper ? sp.ucol : sp.lcol, upper ? sp.uval : sp.lval, sp.dinv, S.sptr,
                S.swidth, S.col, S.val, S.diag);
            PK_LAUNCH();
        }
        if (want32) {
            S.val32 = pool.get<float>(S.nnz_padded > 0 ? S.nnz_padded : 1);
            S.diag32 = pool.get<float>(S.npos > 0 ? S.npos : 1);
            to32(S.val, S.val32, S.nnz_padded, s);
            to32(S.diag, S.diag32, S.npos, s);
        }
        PK_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
        cudaStreamSynchronize(s);
        tmp.free_all();
        throw;
    }
    tmp.free_all();
}

}  // namespace pk
