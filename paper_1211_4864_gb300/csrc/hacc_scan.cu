// Deterministic exclusive prefix sum of int32 counts (reduce-then-scan).
// Used for cell starts, task offsets and radix-sort digit offsets.
#include <atomic>

#include "hacc_common.cuh"

namespace hacc {

namespace {

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;  // 4096

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t &excl, int32_t *warp_tot)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int32_t wt = lane < SCAN_THREADS / 32 ? warp_tot[lane] : 0;
        int32_t wi = wt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < SCAN_THREADS / 32) warp_tot[lane] = wi - wt;  // exclusive warp offsets
        if (lane == SCAN_THREADS / 32 - 1) warp_tot[SCAN_THREADS / 32] = wi;
    }
    __syncthreads();
    excl = warp_tot[warp] + incl - v;
    int32_t total = warp_tot[SCAN_THREADS / 32];
    __syncthreads();
    return total;
}

// Per tile: sum of its items.
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const int32_t *__restrict__ in, int64_t n,
                                                              int32_t *__restrict__ partial)
{
    __shared__ int32_t warp_tot[SCAN_THREADS / 32 + 1];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + (int64_t)k * SCAN_THREADS + threadIdx.x;
        if (i < n) s += in[i];
    }
    int32_t excl;
    int32_t total = block_exclusive_scan(s, excl, warp_tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

// Per tile: exclusive scan plus the tile's offset; optionally out[n] = total.
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tiles(const int32_t *__restrict__ in, int64_t n,
                                                             const int32_t *__restrict__ tile_off,
                                                             int32_t *__restrict__ out, int write_total)
{
    __shared__ int32_t buf[SCAN_TILE];
    __shared__ int32_t warp_tot[SCAN_THREADS / 32 + 1];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + (int64_t)k * SCAN_THREADS + threadIdx.x;
        buf[k * SCAN_THREADS + threadIdx.x] = i < n ? in[i] : 0;
    }
    __syncthreads();
    int32_t v[SCAN_ITEMS];
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = buf[threadIdx.x * SCAN_ITEMS + k];
        s += v[k];
    }
    int32_t excl;
    int32_t total = block_exclusive_scan(s, excl, warp_tot);
    int32_t off = (tile_off ? tile_off[blockIdx.x] : 0) + excl;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        buf[threadIdx.x * SCAN_ITEMS + k] = off;
        off += v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + (int64_t)k * SCAN_THREADS + threadIdx.x;
        if (i < n) out[i] = buf[k * SCAN_THREADS + threadIdx.x];
    }
    if (write_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0)
        out[n] = (tile_off ? tile_off[blockIdx.x] : 0) + total;
}

int64_t ntiles(int64_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE; }

}  // namespace

size_t scan_workspace_bytes(int64_t n)
{
    size_t bytes = 0;
    while (n > SCAN_TILE) {
        int64_t nb = ntiles(n);
        bytes += round_up((size_t)(nb + 1) * sizeof(int32_t), 256) * 2;
        n = nb;
    }
    return bytes + 256;
}

// Recursive reduce-then-scan; ws holds (partials, scanned partials) per level.
static int scan_level(const int32_t *in, int32_t *out, int64_t n, int write_total, char *ws,
                      cudaStream_t st)
{
    if (n <= SCAN_TILE) {
        k_scan_tiles<<<1, SCAN_THREADS, 0, st>>>(in, n, nullptr, out, write_total);
        HACC_LAUNCH_CHECK();
        return HACC_OK;
    }
    int64_t nb = ntiles(n);
    size_t lvl = round_up((size_t)(nb + 1) * sizeof(int32_t), 256);
    int32_t *partial = reinterpret_cast<int32_t *>(ws);
    int32_t *scanned = reinterpret_cast<int32_t *>(ws + lvl);
    k_scan_reduce<<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, n, partial);
    HACC_LAUNCH_CHECK();
    int rc = scan_level(partial, scanned, nb, 0, ws + 2 * lvl, st);
    if (rc) return rc;
    k_scan_tiles<<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, n, scanned, out, write_total);
    HACC_LAUNCH_CHECK();
    return HACC_OK;
}

int scan_exclusive_i32(const int32_t *in, int32_t *out, int64_t n, void *ws, cudaStream_t st)
{
    if (n <= 0) return HACC_OK;
    return scan_level(in, out, n, 1, reinterpret_cast<char *>(ws), st);
}

static std::atomic<uint64_t> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

uint64_t launches() { return g_launches.load(std::memory_order_relaxed); }

int num_sms()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    return sms > 0 ? sms : 1;
}

}  // namespace hacc

extern "C" uint64_t hacc_kernel_launches(void) { return hacc::launches(); }
