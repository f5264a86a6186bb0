// noalloc.cu -- PMIS C/F splitting without any device allocation.
//
// pkasp_pmis() obtains its scratch (mirror index, measures, round flags) from
// cudaMalloc. Some callers cannot let a library allocate: processes that reserve the
// whole GPU memory for their own pool up front, and code that must not synchronize the
// device (cudaMalloc and cudaFree synchronize). pkasp_pmis_noalloc() computes the same
// splitting with its scratch in one file-scope device array of fixed size, which every
// GPU that loads this library holds until the process exits.
#include <cstring>

#include "internal.h"
#include "pmis.cuh"

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

// Device address of g_pmis_scratch on the current device. In host code the array's
// name is only a host-side stand-in, so the address is looked up with
// cudaGetSymbolAddress on every call: the lookup is cheap next to the per-round
// synchronisations, and it stays right if the device's context was reset and the module
// loaded again at another address.
void *scratch_address() {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_pmis_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        pk::fail(PKASP_ECUDA, std::string("cudaGetSymbolAddress of the PMIS scratch failed: ") +
                                  cudaGetErrorString(e));
    }
    return p;
}

unsigned blocks_for(int64_t n) { return (unsigned)((n + 255) / 256 > 0 ? (n + 255) / 256 : 1); }

// Row pointers must start at 0 and never decrease: the mirror pass writes one scratch
// slot per entry, so a malformed ptr must not reach it (sets *bad = 3).
__global__ void k_na_check_ptr(int64_t n, const int64_t *__restrict__ ptr, int *__restrict__ bad) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    if ((i == 0 && ptr[0] != 0) || (i > 0 && ptr[i] < ptr[i - 1])) atomicExch(bad, 3);
}

// the per-row rules are those of pkasp_pmis (pmis.cuh), with 32-bit mirror and measure
// arrays to keep the fixed scratch small
__global__ void k_na_mirror(int64_t n, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                            int32_t *__restrict__ mirror, int *__restrict__ bad) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) pk::pmis_mirror_row<int32_t>(i, n, ptr, col, mirror, bad);
}

__global__ void k_na_init(int64_t n, const int64_t *__restrict__ ptr, const int32_t *__restrict__ mirror,
                          const uint8_t *__restrict__ strong, int32_t *__restrict__ mu, int8_t *__restrict__ cf,
                          unsigned long long *__restrict__ und) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && pk::pmis_init_row<int32_t>(i, ptr, mirror, strong, mu, cf)) atomicAdd(und, 1ull);
}

__global__ void k_na_select(int64_t n, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                            const int32_t *__restrict__ mirror, const uint8_t *__restrict__ strong,
                            const int32_t *__restrict__ mu, uint64_t stream, const int8_t *__restrict__ cf,
                            uint8_t *__restrict__ newc) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) newc[i] = pk::pmis_select_row<int32_t>(i, ptr, col, mirror, strong, mu, stream, cf);
}

__global__ void k_na_commit(int64_t n, const uint8_t *__restrict__ newc, int8_t *__restrict__ cf) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && newc[i]) cf[i] = 1;
}

__global__ void k_na_mark(int64_t n, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                          const uint8_t *__restrict__ strong, const uint8_t *__restrict__ newc,
                          int8_t *__restrict__ cf, unsigned long long *__restrict__ und) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && pk::pmis_mark_row(i, ptr, col, strong, newc, cf)) atomicAdd(und, 1ull);
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
    if (nnz < 0) fail(PKASP_EINVAL, "pkasp_pmis_noalloc: ptr[n] is negative");
    if (n == 0) return;
    int32_t *mirror = reinterpret_cast<int32_t *>(base + kOffMirror);
    int32_t *mu = reinterpret_cast<int32_t *>(base + kOffMu);
    uint8_t *newc = base + kOffNewc;
    int *bad = reinterpret_cast<int *>(base + kOffBad);
    unsigned long long *und = reinterpret_cast<unsigned long long *>(base + kOffUnd);
    // the array keeps the previous call's contents: clear the two counters
    PK_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    PK_CUDA(cudaMemsetAsync(und, 0, sizeof(unsigned long long), s));
    {
        k_na_check_ptr<<<blocks_for(n + 1), 256, 0, s>>>(n, ptr, bad);
        PK_LAUNCH();
        int hp = 0;
        PK_CUDA(cudaMemcpyAsync(&hp, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
        PK_CUDA(cudaStreamSynchronize(s));
        if (hp) fail(PKASP_EINVAL, "pkasp_pmis_noalloc: ptr must start at 0 and never decrease");
    }
    k_na_mirror<<<blocks_for(n), 256, 0, s>>>(n, ptr, col, mirror, bad);
    PK_LAUNCH();
    k_na_init<<<blocks_for(n), 256, 0, s>>>(n, ptr, mirror, strong, mu, cf, und);
    PK_LAUNCH();
    int hb = 0;
    unsigned long long left = 0;
    PK_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    PK_CUDA(cudaMemcpyAsync(&left, und, sizeof(left), cudaMemcpyDeviceToHost, s));
    PK_CUDA(cudaStreamSynchronize(s));
    if (hb == 2) fail(PKASP_EINVAL, "pkasp_pmis_noalloc: a column index lies outside [0, n)");
    if (hb) fail(PKASP_EINVAL, "pkasp_pmis_noalloc needs a structurally symmetric pattern with ascending columns "
                               "in every row");
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
