// pmis.cuh -- the per-row rules of the PMIS C/F splitting (De Sterck, Yang & Heys 2006,
// the coarsening named in Sec. 1 and Sec. 6.1), shared by the allocating setup path
// (setup.cu) and the fixed-scratch entry point (noalloc.cu) so that both take the same
// decisions bit for bit. Index type I is the width of the mirror and measure arrays.
//
//   measure of row i: (mu_i, hash(stream, i), i) compared lexicographically, mu_i =
//     |S_i^T| (rows that depend strongly on i); the hash is SplitMix64 (Steele, Lea &
//     Flood 2014), the published constants and finaliser;
//   rows with no strong connection in either direction start as F;
//   each round, an undecided row whose measure beats every undecided neighbour in
//     S_i u S_i^T becomes C; then every undecided row with a strong dependency on a new
//     C row becomes F.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pk {

__device__ __forceinline__ uint64_t splitmix64(uint64_t stream, uint64_t i) {
    uint64_t z = stream + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// first position in col[lo, hi) (ascending) holding a value >= j
__device__ __forceinline__ int64_t lower_bound_col(const int32_t *col, int64_t lo, int64_t hi, int32_t j) {
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (col[mid] < j) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// mirror[e] = position of (j, i) for the entries e = (i, j) of row i. Sets *bad = 1 when
// a row's pattern has no transposed entry (not structurally symmetric, or columns not
// ascending) and *bad = 2 for a column outside [0, n); such entries mirror themselves and
// read nothing out of range.
template <typename I>
__device__ __forceinline__ void pmis_mirror_row(int64_t i, int64_t n, const int64_t *__restrict__ ptr,
                                                const int32_t *__restrict__ col, I *__restrict__ mirror,
                                                int *__restrict__ bad) {
    for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) {
        const int32_t j = col[e];
        if (j < 0 || (int64_t)j >= n) {
            atomicExch(bad, 2);
            mirror[e] = (I)e;
            continue;
        }
        const int64_t q = lower_bound_col(col, ptr[j], ptr[j + 1], (int32_t)i);
        if (q >= ptr[j + 1] || col[q] != (int32_t)i) {
            atomicCAS(bad, 0, 1);
            mirror[e] = (I)e;
        } else {
            mirror[e] = (I)q;
        }
    }
}

// initial state of row i: mu_i and C/F/undecided (0); returns true when undecided
template <typename I>
__device__ __forceinline__ bool pmis_init_row(int64_t i, const int64_t *__restrict__ ptr,
                                              const I *__restrict__ mirror, const uint8_t *__restrict__ strong,
                                              I *__restrict__ mu, int8_t *__restrict__ cf) {
    I m = 0, d = 0;
    for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) {
        d += strong[e];
        m += strong[mirror[e]];
    }
    mu[i] = m;
    const int8_t c = (d == 0 && m == 0) ? (int8_t)-1 : (int8_t)0;
    cf[i] = c;
    return c == 0;
}

template <typename I>
__device__ __forceinline__ bool pmis_beats(I mi, uint64_t hi, int64_t i, I mj, uint64_t hj, int64_t j) {
    if (mi != mj) return mi > mj;
    if (hi != hj) return hi > hj;
    return i > j;
}

// 1 when undecided row i beats every undecided neighbour in S_i u S_i^T
template <typename I>
__device__ __forceinline__ uint8_t pmis_select_row(int64_t i, const int64_t *__restrict__ ptr,
                                                   const int32_t *__restrict__ col, const I *__restrict__ mirror,
                                                   const uint8_t *__restrict__ strong, const I *__restrict__ mu,
                                                   uint64_t stream, const int8_t *__restrict__ cf) {
    if (cf[i] != 0) return 0;
    const uint64_t hi = splitmix64(stream, (uint64_t)i);
    const I mi = mu[i];
    for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) {
        const int32_t j = col[e];
        if (j == i || cf[j] != 0) continue;
        if (!strong[e] && !strong[mirror[e]]) continue;
        if (!pmis_beats<I>(mi, hi, i, mu[j], splitmix64(stream, (uint64_t)j), j)) return 0;
    }
    return 1;
}

// after the new C rows are committed: an undecided row with a strong dependency on a
// new C row becomes F; returns true when row i is still undecided
__device__ __forceinline__ bool pmis_mark_row(int64_t i, const int64_t *__restrict__ ptr,
                                              const int32_t *__restrict__ col, const uint8_t *__restrict__ strong,
                                              const uint8_t *__restrict__ newc, int8_t *__restrict__ cf) {
    if (cf[i] != 0) return false;
    for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e)
        if (strong[e] && newc[col[e]]) {
            cf[i] = -1;
            return false;
        }
    return true;
}

}  // namespace pk
