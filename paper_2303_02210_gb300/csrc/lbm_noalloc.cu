// Allocation-free front heights: a variant of the observer's front-height
// reduction for callers that cannot allocate device memory, for example a
// host whose device memory is entirely reserved by another allocator (a
// framework's caching pool), or a latency-bound loop that must not wait on
// the allocator. Its cross-block scratch (one
// partial result per block and a completion counter) is a file-scope device
// array that every GPU loading this library holds until the process exits.
#include <atomic>
#include <cstdio>
#include <mutex>

#include "../../include/lbm.h"
#include "lbm_common.cuh"

namespace lbm {

constexpr int NOALLOC_TPB = 256;                  // 8 warps, one 32-column mask word each
constexpr int NOALLOC_WARPS = NOALLOC_TPB / 32;
constexpr int NOALLOC_MAX_BLOCKS = 128;           // W <= 128 * 8 * 32 = 32768 columns

struct NoallocPartial {
    long long s1, s2;
};

struct NoallocScratch {
    unsigned int done;      // blocks finished; zeroed before every launch
    unsigned int pad[63];
    NoallocPartial part[NOALLOC_MAX_BLOCKS];
};

static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

// One warp per 32-column word of the mask: h(x) = 1 + highest set row, read
// 32 rows per pass with one ballot per column; per-block sums; the last block
// to finish adds the partials in block order and writes hbar and the Eq. 6
// width w = sqrt(W S2 - S1^2) / W.
__global__ void __launch_bounds__(NOALLOC_TPB)
    k_front_noalloc(const uint32_t *__restrict__ mask, int W, int H, int MW, int32_t *__restrict__ heights,
                    double *__restrict__ stats, NoallocScratch *scr)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __shared__ long long s_a[NOALLOC_WARPS], s_b[NOALLOC_WARPS];
    __shared__ int s_last;
    long long S1 = 0, S2 = 0;
    const int m = blockIdx.x * NOALLOC_WARPS + warp;
    if (m < MW) {
        const int x = m * 32 + lane;
        unsigned pending = __ballot_sync(0xffffffffu, x < W);
        int h = 0;
        for (int yb = H - 1; yb >= 0 && pending; yb -= 32) {
            const int y = yb - lane;
            const unsigned word = y >= 0 ? mask[(long long)y * MW + m] : 0u;
            unsigned any = word;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) any |= __shfl_xor_sync(0xffffffffu, any, o);
            unsigned todo = pending & any;
            while (todo) {
                const int c = __ffs(todo) - 1;
                todo &= todo - 1;
                const unsigned b = __ballot_sync(0xffffffffu, (word >> c) & 1u);
                if (lane == c) h = yb - (__ffs(b) - 1) + 1;
                pending &= ~(1u << c);
            }
        }
        if (x < W) {
            heights[x] = h;
            S1 += h;
            S2 += (long long)h * h;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        S1 += __shfl_xor_sync(0xffffffffu, S1, o);
        S2 += __shfl_xor_sync(0xffffffffu, S2, o);
    }
    if (lane == 0) {
        s_a[warp] = S1;
        s_b[warp] = S2;
    }
    __syncthreads();
    if (tid == 0) {
        NoallocPartial p{0, 0};
        for (int i = 0; i < NOALLOC_WARPS; ++i) {
            p.s1 += s_a[i];
            p.s2 += s_b[i];
        }
        scr->part[blockIdx.x] = p;
        __threadfence();
        s_last = atomicAdd(&scr->done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last || tid != 0) return;
    __threadfence();
    const volatile NoallocPartial *vp = scr->part;
    long long a = 0, b = 0;
    for (int i = 0; i < (int)gridDim.x; ++i) {
        a += vp[i].s1;
        b += vp[i].s2;
    }
    stats[0] = (double)a / (double)W;
    stats[1] = sqrt((double)((long long)W * b - a * a)) / (double)W;
}

// Device address of the scratch array, looked up once per device (with that
// device current) by the first call made there. Host threads may make their
// first calls concurrently: the lookup runs under a mutex and the address is
// published through an atomic pointer, so every later call only loads it.
static std::atomic<void *> g_scratch_addr[64];
static std::mutex g_scratch_lock;

static cudaError_t scratch_address(int dev, NoallocScratch **out)
{
    void *p = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (!p) {
        std::lock_guard<std::mutex> guard(g_scratch_lock);
        p = g_scratch_addr[dev].load(std::memory_order_relaxed);
        if (!p) {
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return e;
            g_scratch_addr[dev].store(p, std::memory_order_release);
        }
    }
    *out = (NoallocScratch *)p;
    return cudaSuccess;
}

} // namespace lbm

using namespace lbm;

extern "C" int lbm_front_heights_noalloc(const uint32_t *mask_dev, int32_t width, int32_t height,
                                         int32_t *heights_dev, double *stats_dev, void *stream)
{
    if (!mask_dev || !heights_dev || !stats_dev) return LBM_ERR_INVALID_ARG;
    if (width < 1 || height < 1 || width > LBM_NOALLOC_MAX_WIDTH || height > 32768) return LBM_ERR_INVALID_ARG;
    const int MW = (width + 31) / 32;
    const int blocks = (MW + NOALLOC_WARPS - 1) / NOALLOC_WARPS;
    if (blocks > NOALLOC_MAX_BLOCKS) return LBM_ERR_INVALID_ARG;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return lbm_record_cuda_error(e);
    if (dev < 0 || dev >= 64) return LBM_ERR_INVALID_ARG;
    NoallocScratch *scr = nullptr;
    e = scratch_address(dev, &scr);
    if (e != cudaSuccess) return lbm_record_cuda_error(e);
    cudaStream_t s = (cudaStream_t)stream;
    // the completion counter must start at zero; the partials are overwritten
    e = cudaMemsetAsync(&scr->done, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return lbm_record_cuda_error(e);
    k_front_noalloc<<<blocks, NOALLOC_TPB, 0, s>>>(mask_dev, width, height, MW, heights_dev, stats_dev, scr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return lbm_record_cuda_error(e);
    return LBM_OK;
}
