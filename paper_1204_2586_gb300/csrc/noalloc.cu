// noalloc.cu -- PMIS C/F splitting without any device allocation.
//
// pkasp_pmis() obtains its scratch (mirror index, measures, round flags) from
// cudaMalloc. Some callers cannot let a library allocate: processes that reserve the
// whole GPU memory for their own pool up front, and code that must not synchronize the
// device (cudaMalloc and cudaFree synchronize). pkasp_pmis_noalloc() computes the same
// splitting with its scratch in one file-scope device array of fixed size, which every
// GPU that loads this library holds until the process exits.
#include <cstring>
#include <mutex>

#include "internal.h"

namespace {

constexpr int64_t kMaxRows = PKASP_NOALLOC_MAX_ROWS;
constexpr int64_t kMaxNnz = PKASP_NOALLOC_MAX_NNZ;
constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
// layout: mirror int32[kMaxNnz] | measure int32[kMaxRows] | new-C flags u8[kMaxRows] |
//         error flag int | undecided counter u64
constexpr size_t kOffMirror = 0;
constexpr size_t kOffMu = align256(kOffMirror + sizeof(int32_t) * kMaxNnz);
constexpr size_t kOffNewc = align256(kOffMu + sizeof(int32_t) * kMaxRows);
constexpr size_t kOffBad = align256(kOffNewc + sizeof(uint8_t) * kMaxRows);
constexpr size_t kOffUnd = align256(kOffBad + sizeof(int));
constexpr size_t kScratchBytes = align256(kOffUnd + sizeof(unsigned long long));

static __device__ __align__(256) unsigned char g_pmis_scratch[kScratchBytes];

// device address of g_pmis_scratch, looked up once per device (the name itself is only
// a host-side stand-in in host code)
std::mutex g_mu;
void *g_addr[64] = {nullptr};

void *scratch_address() {
    int dev = 0;
    PK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) pk::fail(PKASP_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_pmis_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            pk::fail(PKASP_ECUDA, std::string("cudaGetSymbolAddress of the PMIS scratch failed: ") +
                                      cudaGetErrorString(e));
        }
        g_addr[dev] = p;
    }
    return g_addr[dev];
}

unsigned blocks_for(int64_t n) { return (unsigned)((n + 255) / 256 > 0 ? (n + 255) / 256 : 1); }

__device__ __forceinline__ uint64_t mix64(uint64_t stream, uint64_t i) {
    uint64_t z = stream + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_na_mirror(int64_t n, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                            int32_t *__restrict__ mirror, int *__restrict__ bad) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) {
        const int32_t j = col[e];
        int64_t lo = ptr[j], hi = ptr[j + 1];
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (col[mid] < (int32_t)i) lo = mid + 1;
            else hi = mid;
        }
        if (lo >= ptr[j + 1] || col[lo] != (int32_t)i) {
            atomicExch(bad, 1);
            mirror[e] = (int32_t)e;
        } else {
            mirror[e] = (int32_t)lo;
        }
    }
}

__global__ void k_na_init(int64_t n, const int64_t *__restrict__ ptr, const int32_t *__restrict__ mirror,
                          const uint8_t *__restrict__ strong, int32_t *__restrict__ mu, int8_t *__restrict__ cf,
                          unsigned long long *__restrict__ und) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t m = 0, d = 0;
    for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) {
        d += strong[e];
        m += strong[mirror[e]];
    }
    mu[i] = m;
    const int8_t c = (d == 0 && m == 0) ? (int8_t)-1 : (int8_t)0;
    cf[i] = c;
    if (c == 0) atomicAdd(und, 1ull);
}

__device__ __forceinline__ bool beats(int32_t mi, uint64_t hi, int64_t i, int32_t mj, uint64_t hj, int64_t j) {
    if (mi != mj) return mi > mj;
    if (hi != hj) return hi > hj;
    return i > j;
}

__global__ void k_na_select(int64_t n, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                            const int32_t *__restrict__ mirror, const uint8_t *__restrict__ strong,
                            const int32_t *__restrict__ mu, uint64_t stream, const int8_t *__restrict__ cf,
                            uint8_t *__restrict__ newc) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint8_t sel = 0;
    if (cf[i] == 0) {
        sel = 1;
        const uint64_t hi = mix64(stream, (uint64_t)i);
        for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) {
            const int32_t j = col[e];
            if (j == i || cf[j] != 0) continue;
            if (!strong[e] && !strong[mirror[e]]) continue;
            if (!beats(mu[i], hi, i, mu[j], mix64(stream, (uint64_t)j), j)) {
                sel = 0;
                break;
            }
        }
    }
    newc[i] = sel;
}

__global__ void k_na_commit(int64_t n, const uint8_t *__restrict__ newc, int8_t *__restrict__ cf) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && newc[i]) cf[i] = 1;
}

__global__ void k_na_mark(int64_t n, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                          const uint8_t *__restrict__ strong, const uint8_t *__restrict__ newc,
                          int8_t *__restrict__ cf, unsigned long long *__restrict__ und) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || cf[i] != 0) return;
    for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e)
        if (strong[e] && newc[col[e]]) {
            cf[i] = -1;
            return;
        }
    atomicAdd(und, 1ull);
}

}  // namespace

namespace pk {

void pmis_noalloc(int64_t n, const int64_t *ptr, const int32_t *col, const uint8_t *strong, uint64_t stream_id,
                  int8_t *cf, cudaStream_t s) {
    if (n > kMaxRows)
        fail(PKASP_EINVAL, "pkasp_pmis_noalloc: " + std::to_string(n) + " rows exceed the fixed scratch limit of " +
                               std::to_string(kMaxRows));
    unsigned char *base = static_cast<unsigned char *>(scratch_address());
    int64_t nnz = 0;
    PK_CUDA(cudaMemcpyAsync(&nnz, ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    PK_CUDA(cudaStreamSynchronize(s));
    if (nnz > kMaxNnz)
        fail(PKASP_EINVAL, "pkasp_pmis_noalloc: " + std::to_string(nnz) +
                               " entries exceed the fixed scratch limit of " + std::to_string(kMaxNnz));
    if (n == 0) return;
    int32_t *mirror = reinterpret_cast<int32_t *>(base + kOffMirror);
    int32_t *mu = reinterpret_cast<int32_t *>(base + kOffMu);
    uint8_t *newc = base + kOffNewc;
    int *bad = reinterpret_cast<int *>(base + kOffBad);
    unsigned long long *und = reinterpret_cast<unsigned long long *>(base + kOffUnd);
    // the array keeps the previous call's contents: clear the two counters
    PK_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    PK_CUDA(cudaMemsetAsync(und, 0, sizeof(unsigned long long), s));
    k_na_mirror<<<blocks_for(n), 256, 0, s>>>(n, ptr, col, mirror, bad);
    PK_LAUNCH();
    k_na_init<<<blocks_for(n), 256, 0, s>>>(n, ptr, mirror, strong, mu, cf, und);
    PK_LAUNCH();
    int hb = 0;
    unsigned long long left = 0;
    PK_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    PK_CUDA(cudaMemcpyAsync(&left, und, sizeof(left), cudaMemcpyDeviceToHost, s));
    PK_CUDA(cudaStreamSynchronize(s));
    if (hb) fail(PKASP_EINVAL, "pkasp_pmis_noalloc needs a structurally symmetric matrix");
    int64_t rounds = 0;
    while (left > 0) {
        PK_CUDA(cudaMemsetAsync(und, 0, sizeof(unsigned long long), s));
        k_na_select<<<blocks_for(n), 256, 0, s>>>(n, ptr, col, mirror, strong, mu, stream_id, cf, newc);
        PK_LAUNCH();
        k_na_commit<<<blocks_for(n), 256, 0, s>>>(n, newc, cf);
        PK_LAUNCH();
        k_na_mark<<<blocks_for(n), 256, 0, s>>>(n, ptr, col, strong, newc, cf, und);
        PK_LAUNCH();
        PK_CUDA(cudaMemcpyAsync(&left, und, sizeof(left), cudaMemcpyDeviceToHost, s));
        PK_CUDA(cudaStreamSynchronize(s));
        if (++rounds > n + 8) fail(PKASP_ECUDA, "PMIS did not terminate");
    }
}

}  // namespace pk
