// util.cu -- errors, the device allocation pool, an exclusive scan and CSR transfers.
#include <atomic>
#include <cstdio>
#include <cstring>

#include "internal.h"

namespace pk {

void fail(int code, const std::string &msg) { throw Error{code, msg}; }

void cuda_check(cudaError_t e, const char *what, const char *file, int line) {
    if (e == cudaSuccess) return;
    char buf[512];
    snprintf(buf, sizeof(buf), "%s failed at %s:%d: %s", what, file, line, cudaGetErrorString(e));
    int code = (e == cudaErrorMemoryAllocation) ? PKASP_ENOMEM : PKASP_ECUDA;
    throw Error{code, buf};
}

static std::atomic<long long> g_launches{0};

void launched(const char *file, int line) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    cuda_check(cudaGetLastError(), "kernel launch", file, line);
}

long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

void *DevPool::alloc(size_t n) {
    void *p = nullptr;
    if (n == 0) n = 16;
    n = (n + 255) & ~(size_t)255;
    cudaError_t e = cudaMalloc(&p, n);
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(PKASP_ENOMEM, "cudaMalloc of " + std::to_string(n) + " bytes failed");
    }
    blocks.push_back(p);
    bytes += n;
    return p;
}

void DevPool::free_all() {
    for (void *p : blocks) cudaFree(p);
    blocks.clear();
    bytes = 0;
}

// ---------------------------------------------------------------------------------
// Exclusive scan of int64 in place, with the total written to d[n]: each block scans
// 4 * 256 consecutive entries, the block totals are scanned recursively, then added.
// ---------------------------------------------------------------------------------
namespace {
constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void k_scan_tile(int64_t *d, int64_t n, int64_t *tile_sums) {
    __shared__ int64_t warp_tot[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t run = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        int64_t i = base + q;
        v[q] = (i < n) ? d[i] : 0;
        int64_t t = v[q];
        v[q] = run;  // exclusive within the thread
        run += t;
    }
    // inclusive scan of the thread totals within the warp
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t inc = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int64_t w = (lane < kScanThreads / 32) ? warp_tot[lane] : 0;
        int64_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = wi - w;  // exclusive warp offsets
        if (lane == kScanThreads / 32 - 1) tile_sums[blockIdx.x] = wi;
    }
    __syncthreads();
    const int64_t off = warp_tot[wid] + (inc - run);
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        int64_t i = base + q;
        if (i < n) d[i] = v[q] + off;
    }
}

__global__ void k_scan_add(int64_t *d, int64_t n, const int64_t *tile_off) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) d[i] += tile_off[i / kScanTile];
}

void scan_rec(int64_t *d, int64_t n, cudaStream_t s, int64_t *total_out_dev) {
    int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    int64_t *sums = nullptr;
    PK_CUDA(cudaMallocAsync((void **)&sums, sizeof(int64_t) * (ntiles + 1), s));
    k_scan_tile<<<(unsigned)ntiles, kScanThreads, 0, s>>>(d, n, sums);
    PK_LAUNCH();
    if (ntiles > 1) {
        // sums[0..ntiles) -> exclusive offsets, sums[ntiles] = total
        scan_rec(sums, ntiles, s, sums + ntiles);
        k_scan_add<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d, n, sums);
        PK_LAUNCH();
        PK_CUDA(cudaMemcpyAsync(total_out_dev, sums + ntiles, sizeof(int64_t),
                                cudaMemcpyDeviceToDevice, s));
    } else {
        PK_CUDA(cudaMemcpyAsync(total_out_dev, sums, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    }
    PK_CUDA(cudaFreeAsync(sums, s));
}
}  // namespace

void exclusive_scan(int64_t *d, int64_t n, cudaStream_t s) {
    if (n <= 0) {
        PK_CUDA(cudaMemsetAsync(d, 0, sizeof(int64_t), s));
        return;
    }
    scan_rec(d, n, s, d + n);
}

int64_t read_i64(const int64_t *d, cudaStream_t s) {
    int64_t v = 0;
    PK_CUDA(cudaMemcpyAsync(&v, d, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    PK_CUDA(cudaStreamSynchronize(s));
    return v;
}

void dcsr_alloc(DevPool &pool, DCSR &a, int64_t n, int64_t m, int64_t nnz) {
    a.n = n;
    a.m = m;
    a.nnz = nnz;
    a.ptr = pool.get<int64_t>(n + 1);
    a.col = pool.get<int32_t>(nnz > 0 ? nnz : 1);
    a.val = pool.get<double>(nnz > 0 ? nnz : 1);
    a.val32 = nullptr;
}

void dcsr_upload(DevPool &pool, DCSR &a, const HCSR &h, cudaStream_t s) {
    int64_t nnz = h.ptr.empty() ? 0 : h.ptr.back();
    dcsr_alloc(pool, a, h.n, h.m, nnz);
    PK_CUDA(cudaMemcpyAsync(a.ptr, h.ptr.data(), sizeof(int64_t) * (h.n + 1), cudaMemcpyHostToDevice, s));
    if (nnz > 0) {
        PK_CUDA(cudaMemcpyAsync(a.col, h.col.data(), sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, s));
        if (!h.val.empty())
            PK_CUDA(cudaMemcpyAsync(a.val, h.val.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice, s));
        else
            PK_CUDA(cudaMemsetAsync(a.val, 0, sizeof(double) * nnz, s));
    }
    PK_CUDA(cudaStreamSynchronize(s));  // host vectors may go out of scope
}

void pi_codes_upload(DevPool &pool, const HCSR &Pi, const HCSR &PiT, int k, PiCodes &pc, cudaStream_t s) {
    pc = PiCodes();
    // every entry of I_P is m / k by construction (mesh.cpp); anything else is a bug
    auto bad = [](const char *what) { fail(PKASP_EMESH, std::string("I_P: ") + what); };
    if (k < 1 || k > 7) bad("degree outside 1..7");
    auto code_of = [k](double v) -> int {
        for (int m = 1; m <= k; ++m)
            if (v == (double)m / k) return m;
        return -1;
    };
    const int64_t n = Pi.n;
    std::vector<int32_t> ec((size_t)4 * n, -1);
    std::vector<uint32_t> ecode((size_t)n, 0u);
    for (int64_t i = 0; i < n; ++i) {
        const int64_t lo = Pi.ptr[i], hi = Pi.ptr[i + 1];
        if (hi - lo > 4) bad("a row with more than 4 entries");
        for (int64_t e = lo; e < hi; ++e) {
            const int m = code_of(Pi.val[e]);
            if (m < 0) bad("an entry that is not m / k");
            ec[(size_t)4 * i + (e - lo)] = Pi.col[e];
            ecode[i] |= (uint32_t)m << (8 * (e - lo));
        }
    }
    std::vector<uint8_t> tc(PiT.val.size());
    for (size_t e = 0; e < tc.size(); ++e) {
        const int m = code_of(PiT.val[e]);
        if (m < 0) bad("an entry of the transpose that is not m / k");
        tc[e] = (uint8_t)m;
    }
    double tab[8];
    float tab32[8];
    for (int m = 0; m < 8; ++m) {
        tab[m] = (m >= 1 && m <= k) ? (double)m / k : 0.0;
        tab32[m] = (float)tab[m];
    }
    pc.ell_col = pool.get<int32_t>((size_t)4 * std::max<int64_t>(n, 1));
    pc.ell_code = pool.get<uint32_t>(std::max<int64_t>(n, 1));
    pc.t_code = pool.get<uint8_t>(std::max<size_t>(tc.size(), 1));
    pc.tab = pool.get<double>(8);
    pc.tab32 = pool.get<float>(8);
    if (n > 0) {
        PK_CUDA(cudaMemcpyAsync(pc.ell_col, ec.data(), sizeof(int32_t) * ec.size(), cudaMemcpyHostToDevice, s));
        PK_CUDA(cudaMemcpyAsync(pc.ell_code, ecode.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice, s));
    }
    if (!tc.empty()) PK_CUDA(cudaMemcpyAsync(pc.t_code, tc.data(), tc.size(), cudaMemcpyHostToDevice, s));
    PK_CUDA(cudaMemcpyAsync(pc.tab, tab, sizeof(tab), cudaMemcpyHostToDevice, s));
    PK_CUDA(cudaMemcpyAsync(pc.tab32, tab32, sizeof(tab32), cudaMemcpyHostToDevice, s));
    PK_CUDA(cudaStreamSynchronize(s));  // host vectors go out of scope
}

void dcsr_download(const DCSR &a, HCSR &h, cudaStream_t s) {
    h.n = a.n;
    h.m = a.m;
    h.ptr.resize(a.n + 1);
    h.col.resize(a.nnz);
    h.val.resize(a.nnz);
    PK_CUDA(cudaMemcpyAsync(h.ptr.data(), a.ptr, sizeof(int64_t) * (a.n + 1), cudaMemcpyDeviceToHost, s));
    if (a.nnz > 0) {
        PK_CUDA(cudaMemcpyAsync(h.col.data(), a.col, sizeof(int32_t) * a.nnz, cudaMemcpyDeviceToHost, s));
        PK_CUDA(cudaMemcpyAsync(h.val.data(), a.val, sizeof(double) * a.nnz, cudaMemcpyDeviceToHost, s));
    }
    PK_CUDA(cudaStreamSynchronize(s));
}

namespace {
__global__ void k_to32(const double *__restrict__ x, float *__restrict__ y, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (float)x[i];
}
}  // namespace

void to32(const double *x, float *y, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_to32<<<(unsigned)blocks, 256, 0, s>>>(x, y, n);
    PK_LAUNCH();
}

void dcsr_make32(DevPool &pool, DCSR &a, cudaStream_t s) {
    a.val32 = pool.get<float>(a.nnz > 0 ? a.nnz : 1);
    to32(a.val, a.val32, a.nnz, s);
}

}  // namespace pk
