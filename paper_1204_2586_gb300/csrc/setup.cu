// setup.cu -- device-side construction of the auxiliary-space preconditioner:
//   * Jones-Plassmann colouring of a matrix graph and the colour split used by the
//     multicolour Gauss-Seidel smoothers (the paper's hybrid GS of Sec. 6.1 replaced by
//     a GS that parallelises over colours);
//   * the P1 algebraic multigrid hierarchy on A_H (Step 1 of Algorithm 2.1 solved by one
//     AMG cycle, Remark 2.1): strength of connection (Sec. 6.2), PMIS coarsening and
//     extended+i interpolation (cited in Sec. 1 and 6.1), Galerkin products P^T A P
//     (the relation A_H = I_R A_h I_P of Sec. 2 applied level by level) and a dense
//     inverse of the coarsest matrix.
// Everything that decides an integer (colours, strength, C/F) is computed from the same
// FP64 values by integer-exact rules, so it is reproducible; floating-point sums run in a
// fixed order per entry (one thread or one warp per row, no atomics on values).
#include <algorithm>
#include <cstring>

#include "internal.h"
#include "pmis.cuh"

namespace pk {

void to32(const double *x, float *y, int64_t n, cudaStream_t s);

namespace {

unsigned blocks_for(int64_t n, int per) {
    int64_t b = (n + per - 1) / per;
    return (unsigned)std::max<int64_t>(1, b);
}


// ---------------------------------------------------------------------------------
// Jones-Plassmann colouring: priority (hash, -index); each round the local maxima among
// uncoloured vertices take the smallest colour unused by already coloured neighbours.
// ---------------------------------------------------------------------------------
__global__ void k_jp_pick(int64_t n, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                          uint64_t stream, const int32_t *__restrict__ colour, uint8_t *__restrict__ pick) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (colour[i] >= 0) {
        pick[i] = 0;
        return;
    }
    // largest-degree-first priority (degree, hash, -index); the degree counts the
    // off-diagonal entries of the row (rows are sorted, so the diagonal appears once)
    const uint64_t hi = splitmix64(stream, (uint64_t)i);
    const int64_t lo_i = ptr[i], hi_i = ptr[i + 1];
    int64_t di = hi_i - lo_i;
    for (int64_t e = lo_i; e < hi_i; ++e) di -= (col[e] == i);
    uint8_t best = 1;
    for (int64_t e = lo_i; e < hi_i; ++e) {
        int32_t j = col[e];
        if (j == i || colour[j] >= 0) continue;
        int64_t dj = ptr[j + 1] - ptr[j];
        for (int64_t f = ptr[j]; f < ptr[j + 1]; ++f) dj -= (col[f] == j);
        bool i_wins;
        if (di != dj) i_wins = di > dj;
        else {
            uint64_t hj = splitmix64(stream, (uint64_t)j);
            i_wins = (hi != hj) ? (hi > hj) : (i < j);
        }
        if (!i_wins) {
            best = 0;
            break;
        }
    }
    pick[i] = best;
}

__global__ void k_jp_assign(int64_t n, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                            int32_t *__restrict__ colour, const uint8_t *__restrict__ pick,
                            unsigned long long *__restrict__ ncoloured, int *__restrict__ maxcol) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !pick[i]) return;
    int base = 0, c = -1;
    while (c < 0) {
        unsigned long long used = 0ull;
        for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) {
            int32_t j = col[e];
            if (j == i || pick[j]) continue;
            int cj = colour[j] - base;
            if (cj >= 0 && cj < 64) used |= 1ull << cj;
        }
        if (~used != 0ull) c = base + __ffsll((long long)~used) - 1;
        else base += 64;
    }
    colour[i] = c;
    atomicAdd(ncoloured, 1ull);
    atomicMax(maxcol, c + 1);
}

// ---------------------------------------------------------------------------------
// Colour split
// ---------------------------------------------------------------------------------
__global__ void k_split_count(int64_t n, const int32_t *__restrict__ perm, const int64_t *__restrict__ ptr,
                              const int32_t *__restrict__ col, const int32_t *__restrict__ colour,
                              int64_t *__restrict__ lcnt, int64_t *__restrict__ ucnt) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int32_t i = perm[p];
    int ci = colour[i];
    int64_t l = 0, u = 0;
    for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) {
        int32_t j = col[e];
        if (j == i) continue;
        if (colour[j] < ci) ++l;
        else ++u;  // a proper colouring leaves no equal colours off the diagonal
    }
    lcnt[p] = l;
    ucnt[p] = u;
}

__global__ void k_split_fill(int64_t n, const int32_t *__restrict__ perm, const int64_t *__restrict__ ptr,
                             const int32_t *__restrict__ col, const double *__restrict__ val,
                             const int32_t *__restrict__ colour, const int64_t *__restrict__ lptr,
                             const int64_t *__restrict__ uptr, int32_t *__restrict__ lcol,
                             double *__restrict__ lval, int32_t *__restrict__ ucol, double *__restrict__ uval,
                             double *__restrict__ diag, double *__restrict__ dinv, int *__restrict__ bad) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int32_t i = perm[p];
    int ci = colour[i];
    int64_t lo = lptr[p], uo = uptr[p];
    double d = 0.0;
    for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) {
        int32_t j = col[e];
        if (j == i) {
            d = val[e];
            continue;
        }
        if (colour[j] == ci) atomicExch(bad, 2);
        if (colour[j] < ci) {
            lcol[lo] = j;
            lval[lo++] = val[e];
        } else {
            ucol[uo] = j;
            uval[uo++] = val[e];
        }
    }
    if (d == 0.0) atomicExch(bad, 1);
    diag[p] = d;
    dinv[p] = d != 0.0 ? 1.0 / d : 0.0;
}

__global__ void k_l1norm(int64_t n, const int64_t *__restrict__ ptr, const double *__restrict__ val,
                         double *__restrict__ l1) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) s += fabs(val[e]);
    l1[i] = s;
}

// ---------------------------------------------------------------------------------
// Strength of connection (Sec. 6.2): j strong for i iff j != i and
// -a_ij > theta * max_{k != i}(-a_ik); no strong entries if that maximum is <= 0.
// ---------------------------------------------------------------------------------
__global__ void k_strength(int64_t n, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                           const double *__restrict__ val, double theta, uint8_t *__restrict__ strong) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double mx = 0.0;
    bool have = false;
    for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) {
        if (col[e] == i) continue;
        double v = -val[e];
        if (!have || v > mx) mx = v;
        have = true;
    }
    const double thr = __dmul_rn(theta, mx);
    for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) {
        uint8_t s = 0;
        if (have && mx > 0.0 && col[e] != i) s = (-val[e] > thr) ? 1 : 0;
        strong[e] = s;
    }
}

// ---------------------------------------------------------------------------------
// PMIS (De Sterck, Yang & Heys 2006), one thread per row; the per-row rules are in
// pmis.cuh (shared with the fixed-scratch entry point).
// ---------------------------------------------------------------------------------
__global__ void k_mirror(int64_t n, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                         int64_t *__restrict__ mirror, int *__restrict__ bad) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) pmis_mirror_row<int64_t>(i, n, ptr, col, mirror, bad);
}

__global__ void k_pmis_init(int64_t n, const int64_t *__restrict__ ptr, const int64_t *__restrict__ mirror,
                            const uint8_t *__restrict__ strong, int64_t *__restrict__ mu,
                            int8_t *__restrict__ cf, unsigned long long *__restrict__ undecided) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && pmis_init_row<int64_t>(i, ptr, mirror, strong, mu, cf)) atomicAdd(undecided, 1ull);
}

__global__ void k_pmis_select(int64_t n, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                              const int64_t *__restrict__ mirror, const uint8_t *__restrict__ strong,
                              const int64_t *__restrict__ mu, uint64_t stream, const int8_t *__restrict__ cf,
                              uint8_t *__restrict__ newc) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) newc[i] = pmis_select_row<int64_t>(i, ptr, col, mirror, strong, mu, stream, cf);
}

__global__ void k_pmis_commit(int64_t n, const uint8_t *__restrict__ newc, int8_t *__restrict__ cf) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && newc[i]) cf[i] = 1;
}

__global__ void k_pmis_mark_f(int64_t n, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                              const uint8_t *__restrict__ strong, const uint8_t *__restrict__ newc,
                              int8_t *__restrict__ cf, unsigned long long *__restrict__ undecided) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && pmis_mark_row(i, ptr, col, strong, newc, cf)) atomicAdd(undecided, 1ull);
}

__global__ void k_flag_c(int64_t n, const int8_t *__restrict__ cf, int64_t *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (cf[i] == 1) ? 1 : 0;
}

// ---------------------------------------------------------------------------------
// Extended+i interpolation (De Sterck, Falgout, Nolting & Yang 2008), no truncation; a
// strong F neighbour k with zero denominator is lumped into the diagonal. With cc = 1
// (extended+i+cc, the form Sec. 1 and Sec. 6.1 name) a strong F neighbour k that shares
// a strong C point with i adds none of its own C points to the interpolatory set; the
// weights then follow from the same formula over that smaller set.
// ---------------------------------------------------------------------------------
__global__ void k_extpi_ub(int64_t n, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                           const uint8_t *__restrict__ strong, const int8_t *__restrict__ cf,
                           int64_t *__restrict__ ub) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (cf[i] == 1) {
        ub[i] = 1;
        return;
    }
    int64_t s = 0;
    for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) {
        if (!strong[e]) continue;
        int32_t k = col[e];
        s += 1;
        if (cf[k] == -1) s += ptr[k + 1] - ptr[k];
    }
    ub[i] = s;
}

__device__ void sort_unique_i32(int32_t *a, int64_t &m) {
    // insertion sort (rows are short), then drop duplicates
    for (int64_t x = 1; x < m; ++x) {
        int32_t v = a[x];
        int64_t y = x - 1;
        while (y >= 0 && a[y] > v) {
            a[y + 1] = a[y];
            --y;
        }
        a[y + 1] = v;
    }
    int64_t u = 0;
    for (int64_t x = 0; x < m; ++x)
        if (x == 0 || a[x] != a[x - 1]) a[u++] = a[x];
    m = u;
}

// 1 when k has a strong C point that is also a strong C point of i
__device__ bool shares_strong_c(const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                                const uint8_t *__restrict__ strong, const int8_t *__restrict__ cf, int64_t i,
                                int32_t k) {
    for (int64_t f = ptr[k]; f < ptr[k + 1]; ++f) {
        if (!strong[f] || cf[col[f]] != 1) continue;
        for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e)
            if (strong[e] && col[e] == col[f]) return true;
    }
    return false;
}

__global__ void k_extpi_hat(int64_t n, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                            const uint8_t *__restrict__ strong, const int8_t *__restrict__ cf,
                            const int64_t *__restrict__ ub_off, int32_t *__restrict__ scratch,
                            int64_t *__restrict__ cnt, int cc) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (cf[i] == 1) {
        cnt[i] = 1;
        return;
    }
    int32_t *h = scratch + ub_off[i];
    int64_t m = 0;
    for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) {
        if (!strong[e]) continue;
        int32_t k = col[e];
        if (cf[k] == 1) h[m++] = k;
        else if (!cc || !shares_strong_c(ptr, col, strong, cf, i, k))
            for (int64_t f = ptr[k]; f < ptr[k + 1]; ++f)
                if (strong[f] && cf[col[f]] == 1) h[m++] = col[f];
    }
    sort_unique_i32(h, m);
    cnt[i] = m;
}

__device__ __forceinline__ double abar(double akl, double akk) {
    if (akk > 0.0) return akl < 0.0 ? akl : 0.0;
    if (akk < 0.0) return akl > 0.0 ? akl : 0.0;
    return akl;
}

__device__ __forceinline__ int64_t find_sorted(const int32_t *h, int64_t m, int32_t v) {
    int64_t lo = 0, hi = m;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (h[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return (lo < m && h[lo] == v) ? lo : -1;
}

__global__ void k_extpi_fill(int64_t n, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                             const double *__restrict__ val, const uint8_t *__restrict__ strong,
                             const int8_t *__restrict__ cf, const int64_t *__restrict__ cidx,
                             const int64_t *__restrict__ ub_off, const int32_t *__restrict__ scratch,
                             const int64_t *__restrict__ pptr, int32_t *__restrict__ pcol,
                             double *__restrict__ pval) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t o = pptr[i];
    if (cf[i] == 1) {
        pcol[o] = (int32_t)cidx[i];
        pval[o] = 1.0;
        return;
    }
    const int64_t m = pptr[i + 1] - o;
    if (m == 0) return;
    const int32_t *h = scratch + ub_off[i];
    double *w = pval + o;
    for (int64_t q = 0; q < m; ++q) {
        w[q] = 0.0;
        pcol[o + q] = (int32_t)cidx[h[q]];
    }
    double aii = 0.0;
    for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e)
        if (col[e] == i) aii = val[e];
    double diag = aii;
    for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) {
        int32_t j = col[e];
        if (j == i) continue;
        int64_t q = find_sorted(h, m, j);
        if (q >= 0) w[q] = val[e];
        else if (!strong[e]) diag = __dadd_rn(diag, val[e]);
    }
    for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) {
        if (!strong[e]) continue;
        int32_t k = col[e];
        if (cf[k] != -1) continue;
        const double aik = val[e];
        double akk = 0.0;
        for (int64_t f = ptr[k]; f < ptr[k + 1]; ++f)
            if (col[f] == k) akk = val[f];
        double d = 0.0;
        for (int64_t f = ptr[k]; f < ptr[k + 1]; ++f) {
            int32_t l = col[f];
            if (l == k) continue;
            if (l == i || find_sorted(h, m, l) >= 0) d = __dadd_rn(d, abar(val[f], akk));
        }
        if (d == 0.0) {
            diag = __dadd_rn(diag, aik);
            continue;
        }
        for (int64_t f = ptr[k]; f < ptr[k + 1]; ++f) {
            int32_t l = col[f];
            if (l == k) continue;
            double t = __ddiv_rn(__dmul_rn(aik, abar(val[f], akk)), d);
            if (l == i) diag = __dadd_rn(diag, t);
            else {
                int64_t q = find_sorted(h, m, l);
                if (q >= 0) w[q] = __dadd_rn(w[q], t);
            }
        }
    }
    for (int64_t q = 0; q < m; ++q) w[q] = __ddiv_rn(-w[q], diag);
}

// ---------------------------------------------------------------------------------
// Transpose (R = P^T): count, scan, scatter, then sort every row of R by column.
// ---------------------------------------------------------------------------------
__global__ void k_count_cols(int64_t nnz, const int32_t *__restrict__ col, unsigned long long *__restrict__ cnt) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nnz) atomicAdd(&cnt[col[e]], 1ull);
}

__global__ void k_transpose_scatter(int64_t n, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                                    const double *__restrict__ val, unsigned long long *__restrict__ fill,
                                    int32_t *__restrict__ tcol, double *__restrict__ tval) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) {
        unsigned long long q = atomicAdd(&fill[col[e]], 1ull);
        tcol[q] = (int32_t)i;
        tval[q] = val[e];
    }
}

__global__ void k_sort_rows(int64_t n, const int64_t *__restrict__ ptr, int32_t *__restrict__ col,
                            double *__restrict__ val) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t lo = ptr[i], hi = ptr[i + 1];
    for (int64_t x = lo + 1; x < hi; ++x) {
        int32_t c = col[x];
        double v = val[x];
        int64_t y = x - 1;
        while (y >= lo && col[y] > c) {
            col[y + 1] = col[y];
            val[y + 1] = val[y];
            --y;
        }
        col[y + 1] = c;
        val[y + 1] = v;
    }
}

// ---------------------------------------------------------------------------------
// SpGEMM C = A B, one thread per row: the candidate columns are collected in a private
// scratch slice, heap-sorted and de-duplicated (symbolic phase); the numeric phase adds
// the products in the order of A's row then B's row (a fixed order per entry).
// ---------------------------------------------------------------------------------
__global__ void k_gemm_ub(int64_t n, const int64_t *__restrict__ aptr, const int32_t *__restrict__ acol,
                          const int64_t *__restrict__ bptr, int64_t *__restrict__ ub) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t s = 0;
    for (int64_t e = aptr[i]; e < aptr[i + 1]; ++e) s += bptr[acol[e] + 1] - bptr[acol[e]];
    ub[i] = s;
}

__device__ void heap_sort_i32(int32_t *a, int64_t m) {
    auto sift = [&](int64_t root, int64_t end) {
        while (2 * root + 1 < end) {
            int64_t c = 2 * root + 1;
            if (c + 1 < end && a[c + 1] > a[c]) ++c;
            if (a[root] >= a[c]) return;
            int32_t t = a[root];
            a[root] = a[c];
            a[c] = t;
            root = c;
        }
    };
    for (int64_t s = m / 2 - 1; s >= 0; --s) sift(s, m);
    for (int64_t end = m - 1; end > 0; --end) {
        int32_t t = a[0];
        a[0] = a[end];
        a[end] = t;
        sift(0, end);
    }
}

__global__ void k_gemm_symbolic(int64_t n, const int64_t *__restrict__ aptr, const int32_t *__restrict__ acol,
                                const int64_t *__restrict__ bptr, const int32_t *__restrict__ bcol,
                                const int64_t *__restrict__ ub_off, int32_t *__restrict__ scratch,
                                int64_t *__restrict__ cnt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t *h = scratch + ub_off[i];
    int64_t m = 0;
    for (int64_t e = aptr[i]; e < aptr[i + 1]; ++e) {
        int32_t k = acol[e];
        for (int64_t f = bptr[k]; f < bptr[k + 1]; ++f) h[m++] = bcol[f];
    }
    heap_sort_i32(h, m);
    int64_t u = 0;
    for (int64_t x = 0; x < m; ++x)
        if (x == 0 || h[x] != h[x - 1]) h[u++] = h[x];
    cnt[i] = u;
}

__global__ void k_gemm_numeric(int64_t n, const int64_t *__restrict__ aptr, const int32_t *__restrict__ acol,
                               const double *__restrict__ aval, const int64_t *__restrict__ bptr,
                               const int32_t *__restrict__ bcol, const double *__restrict__ bval,
                               const int64_t *__restrict__ ub_off, const int32_t *__restrict__ scratch,
                               const int64_t *__restrict__ cptr, int32_t *__restrict__ ccol,
                               double *__restrict__ cval) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t lo = cptr[i], hi = cptr[i + 1];
    const int32_t *h = scratch + ub_off[i];
    for (int64_t q = lo; q < hi; ++q) {
        ccol[q] = h[q - lo];
        cval[q] = 0.0;
    }
    for (int64_t e = aptr[i]; e < aptr[i + 1]; ++e) {
        int32_t k = acol[e];
        double a = aval[e];
        for (int64_t f = bptr[k]; f < bptr[k + 1]; ++f) {
            int64_t q = lower_bound_col(ccol, lo, hi, bcol[f]);
            if (q < hi) cval[q] = __dadd_rn(cval[q], __dmul_rn(a, bval[f]));
        }
    }
}

// ---------------------------------------------------------------------------------
// Coarsest level: dense Cholesky factor and explicit inverse (one block).
// ---------------------------------------------------------------------------------
__global__ void k_csr_to_dense(int64_t n, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                               const double *__restrict__ val, double *__restrict__ D) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int64_t j = 0; j < n; ++j) D[i * n + j] = 0.0;
    for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) D[i * n + col[e]] = val[e];
}

__global__ void k_cholesky_inverse(int64_t n, double *__restrict__ L, double *__restrict__ Ainv,
                                   int *__restrict__ bad) {
    __shared__ double piv;
    // right-looking is not needed: column j uses the finished columns q < j
    for (int64_t j = 0; j < n; ++j) {
        if (threadIdx.x == 0) {
            double s = L[j * n + j];
            for (int64_t q = 0; q < j; ++q) s -= L[j * n + q] * L[j * n + q];
            if (!(s > 0.0)) {
                atomicExch(bad, 1);
                s = 1.0;
            }
            piv = sqrt(s);
            L[j * n + j] = piv;
        }
        __syncthreads();
        for (int64_t i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
            double t = L[i * n + j];
            for (int64_t q = 0; q < j; ++q) t -= L[i * n + q] * L[j * n + q];
            L[i * n + j] = t / piv;
        }
        __syncthreads();
    }
    // column c of A^{-1}: solve L y = e_c, then L^T x = y (x stored in Ainv column c)
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
        for (int64_t i = 0; i < n; ++i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int64_t q = c; q < i; ++q) s -= L[i * n + q] * Ainv[q * n + c];
            Ainv[i * n + c] = (i < c) ? 0.0 : s / L[i * n + i];
        }
        for (int64_t i = n - 1; i >= 0; --i) {
            double s = Ainv[i * n + c];
            for (int64_t q = i + 1; q < n; ++q) s -= L[q * n + i] * Ainv[q * n + c];
            Ainv[i * n + c] = s / L[i * n + i];
        }
    }
}

// ---------------------------------------------------------------------------------
// host drivers
// ---------------------------------------------------------------------------------
int jp_colour(int64_t n, const int64_t *ptr, const int32_t *col, uint64_t stream, int32_t *colour,
              DevPool &tmp, cudaStream_t s) {
    uint8_t *pick = tmp.get<uint8_t>(n);
    unsigned long long *cnt = tmp.get<unsigned long long>(1);
    int *maxc = tmp.get<int>(1);
    PK_CUDA(cudaMemsetAsync(colour, 0xff, sizeof(int32_t) * n, s));
    PK_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
    PK_CUDA(cudaMemsetAsync(maxc, 0, sizeof(int), s));
    unsigned long long done = 0;
    int rounds = 0;
    while ((int64_t)done < n) {
        for (int r = 0; r < 4; ++r) {
            k_jp_pick<<<blocks_for(n, 256), 256, 0, s>>>(n, ptr, col, stream, colour, pick);
            PK_LAUNCH();
            k_jp_assign<<<blocks_for(n, 256), 256, 0, s>>>(n, ptr, col, colour, pick, cnt, maxc);
            PK_LAUNCH();
        }
        PK_CUDA(cudaMemcpyAsync(&done, cnt, sizeof(done), cudaMemcpyDeviceToHost, s));
        PK_CUDA(cudaStreamSynchronize(s));
        rounds += 4;
        if (rounds > 4 * (n + 8)) fail(PKASP_ECUDA, "colouring did not terminate");
    }
    int h = 0;
    PK_CUDA(cudaMemcpyAsync(&h, maxc, sizeof(int), cudaMemcpyDeviceToHost, s));
    PK_CUDA(cudaStreamSynchronize(s));
    return h;
}

}  // namespace

// Colour split of A for the multicolour Gauss-Seidel sweeps.
void build_split(DevPool &pool, const DCSR &A, uint64_t stream, bool want32, DSplit &sp, cudaStream_t s) {
    DevPool tmp;
    try {
        const int64_t n = A.n;
        sp.colour = pool.get<int32_t>(n > 0 ? n : 1);
        sp.ncol = n > 0 ? jp_colour(n, A.ptr, A.col, stream, sp.colour, tmp, s) : 0;
        // stable counting sort of the rows by colour (host: n small integers)
        std::vector<int32_t> hc(n);
        PK_CUDA(cudaMemcpyAsync(hc.data(), sp.colour, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
        PK_CUDA(cudaStreamSynchronize(s));
        sp.off.assign(sp.ncol + 1, 0);
        for (int32_t c : hc) sp.off[c + 1]++;
        for (int c = 0; c < sp.ncol; ++c) sp.off[c + 1] += sp.off[c];
        std::vector<int64_t> fill(sp.off.begin(), sp.off.end() - 1);
        std::vector<int32_t> perm(n);
        for (int64_t i = 0; i < n; ++i) perm[fill[hc[i]]++] = (int32_t)i;
        sp.perm = pool.get<int32_t>(n > 0 ? n : 1);
        PK_CUDA(cudaMemcpyAsync(sp.perm, perm.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
        sp.lptr = pool.get<int64_t>(n + 1);
        sp.uptr = pool.get<int64_t>(n + 1);
        if (n > 0) {
            k_split_count<<<blocks_for(n, 256), 256, 0, s>>>(n, sp.perm, A.ptr, A.col, sp.colour, sp.lptr, sp.uptr);
            PK_LAUNCH();
        }
        exclusive_scan(sp.lptr, n, s);
        exclusive_scan(sp.uptr, n, s);
        sp.nnz_l = read_i64(sp.lptr + n, s);
        sp.nnz_u = read_i64(sp.uptr + n, s);
        {
            // longest lower/upper part of each colour: it fixes the lanes per row of that
            // colour's phase (one batch of loads per lane covers the whole row)
            std::vector<int64_t> hl(n + 1), hu(n + 1);
            PK_CUDA(cudaMemcpyAsync(hl.data(), sp.lptr, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, s));
            PK_CUDA(cudaMemcpyAsync(hu.data(), sp.uptr, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, s));
            PK_CUDA(cudaStreamSynchronize(s));
            sp.lmax.assign(sp.ncol, 0);
            sp.umax.assign(sp.ncol, 0);
            sp.l90.assign(sp.ncol, 0);
            sp.u90.assign(sp.ncol, 0);
            std::vector<int> ll, ul;
            for (int c = 0; c < sp.ncol; ++c) {
                ll.clear();
                ul.clear();
                for (int64_t q = sp.off[c]; q < sp.off[c + 1]; ++q) {
                    ll.push_back((int)(hl[q + 1] - hl[q]));
                    ul.push_back((int)(hu[q + 1] - hu[q]));
                    sp.lmax[c] = std::max<int>(sp.lmax[c], ll.back());
                    sp.umax[c] = std::max<int>(sp.umax[c], ul.back());
                }
                // 90th percentile: the length one batch of loads should cover
                if (!ll.empty()) {
                    const size_t k = (ll.size() * 9) / 10;
                    std::nth_element(ll.begin(), ll.begin() + k, ll.end());
                    std::nth_element(ul.begin(), ul.begin() + k, ul.end());
                    sp.l90[c] = ll[k];
                    sp.u90[c] = ul[k];
                }
            }
        }
        sp.lcol = pool.get<int32_t>(sp.nnz_l > 0 ? sp.nnz_l : 1);
        sp.lval = pool.get<double>(sp.nnz_l > 0 ? sp.nnz_l : 1);
        sp.ucol = pool.get<int32_t>(sp.nnz_u > 0 ? sp.nnz_u : 1);
        sp.uval = pool.get<double>(sp.nnz_u > 0 ? sp.nnz_u : 1);
        sp.diag = pool.get<double>(n > 0 ? n : 1);
        sp.dinv = pool.get<double>(n > 0 ? n : 1);
        int *bad = tmp.get<int>(1);
        PK_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
        if (n > 0) {
            k_split_fill<<<blocks_for(n, 256), 256, 0, s>>>(n, sp.perm, A.ptr, A.col, A.val, sp.colour, sp.lptr,
                                                            sp.uptr, sp.lcol, sp.lval, sp.ucol, sp.uval, sp.diag,
                                                            sp.dinv, bad);
            PK_LAUNCH();
        }
        int hb = 0;
        PK_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
        PK_CUDA(cudaStreamSynchronize(s));
        if (hb == 1) fail(PKASP_EBREAKDOWN, "zero diagonal entry in a smoothed matrix");
        if (hb == 2) fail(PKASP_ECUDA, "colouring left two neighbours with the same colour");
        if (want32) {
            sp.lval32 = pool.get<float>(sp.nnz_l > 0 ? sp.nnz_l : 1);
            sp.uval32 = pool.get<float>(sp.nnz_u > 0 ? sp.nnz_u : 1);
            sp.diag32 = pool.get<float>(n > 0 ? n : 1);
            sp.dinv32 = pool.get<float>(n > 0 ? n : 1);
            to32(sp.lval, sp.lval32, sp.nnz_l, s);
            to32(sp.uval, sp.uval32, sp.nnz_u, s);
            to32(sp.diag, sp.diag32, n, s);
            to32(sp.dinv, sp.dinv32, n, s);
        }
        PK_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
        cudaStreamSynchronize(s);
        tmp.free_all();
        throw;
    }
    tmp.free_all();
}

double *row_l1(DevPool &pool, const DCSR &A, cudaStream_t s) {
    double *l1 = pool.get<double>(A.n > 0 ? A.n : 1);
    if (A.n > 0) {
        k_l1norm<<<blocks_for(A.n, 256), 256, 0, s>>>(A.n, A.ptr, A.val, l1);
        PK_LAUNCH();
    }
    return l1;
}

// C = A B on the device (A: n x k, B: k x m)
void spgemm(DevPool &pool, const DCSR &A, const DCSR &B, DCSR &C, cudaStream_t s) {
    const int64_t n = A.n;
    DevPool tmp;
    try {
        int64_t *ub = tmp.get<int64_t>(n + 1);
        if (n > 0) {
            k_gemm_ub<<<blocks_for(n, 256), 256, 0, s>>>(n, A.ptr, A.col, B.ptr, ub);
            PK_LAUNCH();
        }
        exclusive_scan(ub, n, s);
        int64_t tot = read_i64(ub + n, s);
        if (tot > ((int64_t)1 << 31)) fail(PKASP_ENOMEM, "Galerkin product scratch above 2^31 entries");
        int32_t *scr = tmp.get<int32_t>(tot > 0 ? tot : 1);
        int64_t *cnt = tmp.get<int64_t>(n + 1);
        if (n > 0) {
            k_gemm_symbolic<<<blocks_for(n, 128), 128, 0, s>>>(n, A.ptr, A.col, B.ptr, B.col, ub, scr, cnt);
            PK_LAUNCH();
        }
        exclusive_scan(cnt, n, s);
        int64_t nnz = read_i64(cnt + n, s);
        dcsr_alloc(pool, C, n, B.m, nnz);
        PK_CUDA(cudaMemcpyAsync(C.ptr, cnt, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToDevice, s));
        if (n > 0) {
            k_gemm_numeric<<<blocks_for(n, 128), 128, 0, s>>>(n, A.ptr, A.col, A.val, B.ptr, B.col, B.val, ub, scr,
                                                             C.ptr, C.col, C.val);
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

void transpose(DevPool &pool, const DCSR &A, DCSR &T, cudaStream_t s) {
    DevPool tmp;
    try {
        const int64_t m = A.m;
        unsigned long long *cnt = tmp.get<unsigned long long>(m + 1);
        PK_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * (m + 1), s));
        if (A.nnz > 0) {
            k_count_cols<<<blocks_for(A.nnz, 256), 256, 0, s>>>(A.nnz, A.col, cnt);
            PK_LAUNCH();
        }
        static_assert(sizeof(unsigned long long) == sizeof(int64_t), "scan type");
        exclusive_scan(reinterpret_cast<int64_t *>(cnt), m, s);
        dcsr_alloc(pool, T, m, A.n, A.nnz);
        PK_CUDA(cudaMemcpyAsync(T.ptr, cnt, sizeof(int64_t) * (m + 1), cudaMemcpyDeviceToDevice, s));
        if (A.n > 0) {
            k_transpose_scatter<<<blocks_for(A.n, 256), 256, 0, s>>>(A.n, A.ptr, A.col, A.val, cnt, T.col, T.val);
            PK_LAUNCH();
        }
        if (m > 0) {
            k_sort_rows<<<blocks_for(m, 128), 128, 0, s>>>(m, T.ptr, T.col, T.val);
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

// PMIS on a structurally symmetric pattern with given strength flags.
void pmis_run(int64_t n, const int64_t *ptr, const int32_t *col, const uint8_t *strong, uint64_t stream,
              int8_t *cf, cudaStream_t s) {
    DevPool tmp;
    try {
        int64_t nnz = read_i64(ptr + n, s);
        int64_t *mirror = tmp.get<int64_t>(nnz > 0 ? nnz : 1);
        int64_t *mu = tmp.get<int64_t>(n > 0 ? n : 1);
        uint8_t *newc = tmp.get<uint8_t>(n > 0 ? n : 1);
        int *bad = tmp.get<int>(1);
        unsigned long long *und = tmp.get<unsigned long long>(1);
        PK_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
        PK_CUDA(cudaMemsetAsync(und, 0, sizeof(unsigned long long), s));
        if (n > 0) {
            k_mirror<<<blocks_for(n, 256), 256, 0, s>>>(n, ptr, col, mirror, bad);
            PK_LAUNCH();
            k_pmis_init<<<blocks_for(n, 256), 256, 0, s>>>(n, ptr, mirror, strong, mu, cf, und);
            PK_LAUNCH();
        }
        int hb = 0;
        unsigned long long left = 0;
        PK_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
        PK_CUDA(cudaMemcpyAsync(&left, und, sizeof(left), cudaMemcpyDeviceToHost, s));
        PK_CUDA(cudaStreamSynchronize(s));
        if (hb == 2) fail(PKASP_EINVAL, "PMIS: a column index lies outside [0, n)");
        if (hb) fail(PKASP_EINVAL, "PMIS needs a structurally symmetric pattern with ascending columns in every row");
        int rounds = 0;
        while (left > 0) {
            PK_CUDA(cudaMemsetAsync(und, 0, sizeof(unsigned long long), s));
            k_pmis_select<<<blocks_for(n, 256), 256, 0, s>>>(n, ptr, col, mirror, strong, mu, stream, cf, newc);
            PK_LAUNCH();
            k_pmis_commit<<<blocks_for(n, 256), 256, 0, s>>>(n, newc, cf);
            PK_LAUNCH();
            k_pmis_mark_f<<<blocks_for(n, 256), 256, 0, s>>>(n, ptr, col, strong, newc, cf, und);
            PK_LAUNCH();
            PK_CUDA(cudaMemcpyAsync(&left, und, sizeof(left), cudaMemcpyDeviceToHost, s));
            PK_CUDA(cudaStreamSynchronize(s));
            if (++rounds > n + 8) fail(PKASP_ECUDA, "PMIS did not terminate");
        }
    } catch (...) {
        cudaStreamSynchronize(s);
        tmp.free_all();
        throw;
    }
    tmp.free_all();
}

void pmis_device(int64_t n, const int64_t *ptr, const int32_t *col, const uint8_t *strong, uint64_t stream_id,
                 int8_t *cf, cudaStream_t s) {
    pmis_run(n, ptr, col, strong, stream_id, cf, s);
}

// One coarsening step on level L: strength, PMIS, ext+i P, R = P^T, A_c = R (A P).
// Returns false when PMIS keeps no point or every point (the level becomes the coarsest).
// ---------------------------------------------------------------------------------
// Interpolation truncation (optional): in every row drop |w| < tf * max|w|, keep the
// pmax largest |w| of the rest (ties: the lower column), scale the kept weights to the
// row's original sum. One thread per row; kept entries stay in column order.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ bool trunc_keep(const int32_t *col, const double *val, int64_t lo, int64_t hi,
                                           int64_t e, double cut, int pmax) {
    const double a = fabs(val[e]);
    if (a < cut) return false;
    if (pmax <= 0) return true;
    int rank = 0;  // candidates ahead of e: larger |w|, or equal |w| and a lower column
    for (int64_t f = lo; f < hi; ++f) {
        const double b = fabs(val[f]);
        if (b < cut || f == e) continue;
        if (b > a || (b == a && col[f] < col[e])) ++rank;
    }
    return rank < pmax;
}

__global__ void k_trunc_count(int64_t n, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                              const double *__restrict__ val, double tf, int pmax, int64_t *__restrict__ cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t lo = ptr[i], hi = ptr[i + 1];
    double mx = 0.0;
    for (int64_t e = lo; e < hi; ++e) mx = fmax(mx, fabs(val[e]));
    const double cut = tf > 0.0 ? tf * mx : -1.0;
    int64_t c = 0;
    for (int64_t e = lo; e < hi; ++e) c += trunc_keep(col, val, lo, hi, e, cut, pmax);
    cnt[i] = c;
}

__global__ void k_trunc_fill(int64_t n, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                             const double *__restrict__ val, double tf, int pmax, const int64_t *__restrict__ optr,
                             int32_t *__restrict__ ocol, double *__restrict__ oval) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t lo = ptr[i], hi = ptr[i + 1];
    double mx = 0.0, sum = 0.0;
    for (int64_t e = lo; e < hi; ++e) {
        mx = fmax(mx, fabs(val[e]));
        sum += val[e];
    }
    const double cut = tf > 0.0 ? tf * mx : -1.0;
    int64_t o = optr[i];
    double kept = 0.0;
    for (int64_t e = lo; e < hi; ++e)
        if (trunc_keep(col, val, lo, hi, e, cut, pmax)) {
            ocol[o] = col[e];
            oval[o] = val[e];
            kept += val[e];
            ++o;
        }
    if (o - optr[i] < hi - lo && kept != 0.0) {
        const double scale = sum / kept;
        for (int64_t q = optr[i]; q < o; ++q) oval[q] *= scale;
    }
}

bool coarsen(DevPool &pool, Level &L, double theta, uint64_t pmis_stream, DCSR &Ac, cudaStream_t s,
             double trunc_factor, int pmax, int cc) {
    const DCSR &A = L.A;
    const int64_t n = A.n;
    L.strong = pool.get<uint8_t>(A.nnz > 0 ? A.nnz : 1);
    L.cf = pool.get<int8_t>(n > 0 ? n : 1);
    k_strength<<<blocks_for(n, 256), 256, 0, s>>>(n, A.ptr, A.col, A.val, theta, L.strong);
    PK_LAUNCH();
    pmis_run(n, A.ptr, A.col, L.strong, pmis_stream, L.cf, s);
    DevPool tmp;
    bool ok = true;
    try {
        int64_t *cidx = tmp.get<int64_t>(n + 1);
        k_flag_c<<<blocks_for(n, 256), 256, 0, s>>>(n, L.cf, cidx);
        PK_LAUNCH();
        exclusive_scan(cidx, n, s);
        const int64_t nc = read_i64(cidx + n, s);
        if (nc == 0 || nc == n) {
            ok = false;
        } else {
            int64_t *ub = tmp.get<int64_t>(n + 1);
            k_extpi_ub<<<blocks_for(n, 256), 256, 0, s>>>(n, A.ptr, A.col, L.strong, L.cf, ub);
            PK_LAUNCH();
            exclusive_scan(ub, n, s);
            int64_t tot = read_i64(ub + n, s);
            if (tot > ((int64_t)1 << 31)) fail(PKASP_ENOMEM, "interpolation scratch above 2^31 entries");
            int32_t *scr = tmp.get<int32_t>(tot > 0 ? tot : 1);
            int64_t *cnt = tmp.get<int64_t>(n + 1);
            k_extpi_hat<<<blocks_for(n, 128), 128, 0, s>>>(n, A.ptr, A.col, L.strong, L.cf, ub, scr, cnt, cc);
            PK_LAUNCH();
            exclusive_scan(cnt, n, s);
            int64_t pnnz = read_i64(cnt + n, s);
            const bool trunc = trunc_factor > 0.0 || pmax > 0;
            DCSR full;  // ext+i before truncation (scratch when truncating)
            dcsr_alloc(trunc ? tmp : pool, full, n, nc, pnnz);
            PK_CUDA(cudaMemcpyAsync(full.ptr, cnt, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToDevice, s));
            k_extpi_fill<<<blocks_for(n, 128), 128, 0, s>>>(n, A.ptr, A.col, A.val, L.strong, L.cf, cidx, ub, scr,
                                                            full.ptr, full.col, full.val);
            PK_LAUNCH();
            if (trunc) {
                int64_t *tc = tmp.get<int64_t>(n + 1);
                k_trunc_count<<<blocks_for(n, 256), 256, 0, s>>>(n, full.ptr, full.col, full.val, trunc_factor, pmax,
                                                                 tc);
                PK_LAUNCH();
                exclusive_scan(tc, n, s);
                const int64_t tnnz = read_i64(tc + n, s);
                dcsr_alloc(pool, L.P, n, nc, tnnz);
                PK_CUDA(cudaMemcpyAsync(L.P.ptr, tc, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToDevice, s));
                k_trunc_fill<<<blocks_for(n, 256), 256, 0, s>>>(n, full.ptr, full.col, full.val, trunc_factor, pmax,
                                                                L.P.ptr, L.P.col, L.P.val);
                PK_LAUNCH();
            } else {
                L.P = full;
            }
            PK_CUDA(cudaStreamSynchronize(s));
            transpose(pool, L.P, L.R, s);
            DCSR AP;
            DevPool aptmp;
            try {
                spgemm(aptmp, A, L.P, AP, s);
                spgemm(pool, L.R, AP, Ac, s);
            } catch (...) {
                cudaStreamSynchronize(s);
                aptmp.free_all();
                throw;
            }
            aptmp.free_all();
        }
        PK_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
        cudaStreamSynchronize(s);
        tmp.free_all();
        throw;
    }
    tmp.free_all();
    return ok;
}

// Dense inverse of the coarsest matrix.
void coarse_inverse(DevPool &pool, const DCSR &A, double **inv, cudaStream_t s) {
    const int64_t n = A.n;
    if (n > 8192) fail(PKASP_ENOMEM, "coarsest level has more than 8192 rows; raise max_levels or coarse_size");
    DevPool tmp;
    try {
        double *L = tmp.get<double>(n * n > 0 ? n * n : 1);
        *inv = pool.get<double>(n * n > 0 ? n * n : 1);
        int *bad = tmp.get<int>(1);
        PK_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
        if (n > 0) {
            k_csr_to_dense<<<blocks_for(n, 128), 128, 0, s>>>(n, A.ptr, A.col, A.val, L);
            PK_LAUNCH();
            k_cholesky_inverse<<<1, 1024, 0, s>>>(n, L, *inv, bad);
            PK_LAUNCH();
        }
        int hb = 0;
        PK_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
        PK_CUDA(cudaStreamSynchronize(s));
        if (hb) fail(PKASP_EBREAKDOWN, "coarsest AMG matrix is not positive definite");
    } catch (...) {
        cudaStreamSynchronize(s);
        tmp.free_all();
        throw;
    }
    tmp.free_all();
}

}  // namespace pk
