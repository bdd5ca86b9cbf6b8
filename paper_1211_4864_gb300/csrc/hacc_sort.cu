// Stable LSD radix sort of indices by int32 key (sort_index_stable): the
// task order of the list builders (hacc_lists.cu, hacc_rcb.cu) sorts the
// tasks by cost class with it.  Each pass: a digit histogram per tile of 4096
// keys (digit-major), its exclusive scan, and a stable scatter that ranks the
// tile's keys per warp (match masks, per-warp counters) and stores it in
// digit order.
#include "hacc_common.cuh"

namespace hacc {
namespace {

constexpr int RADIX_BITS = 10;  // sort_index_stable: 1024 digits per pass
constexpr int RADIX = 1 << RADIX_BITS;
constexpr int R_THREADS = 256;
constexpr int R_WARPS = R_THREADS / 32;
constexpr int R_ITEMS = 16;
constexpr int R_TILE = R_THREADS * R_ITEMS;  // 4096 keys per block

// Radix pass, step 1: digit histogram of each 4096-key tile, digit-major.
__global__ void __launch_bounds__(R_THREADS)
k_radix_hist(const int32_t *__restrict__ keys, int64_t N, int shift, int nblk, int32_t *__restrict__ hist)
{
    __shared__ int32_t cnt[RADIX];
    for (int d = threadIdx.x; d < RADIX; d += R_THREADS) cnt[d] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * R_TILE;
#pragma unroll 4
    for (int k = 0; k < R_ITEMS; ++k) {
        int64_t i = base + (int64_t)k * R_THREADS + threadIdx.x;
        if (i < N) atomicAdd(&cnt[((uint32_t)keys[i] >> shift) & (RADIX - 1)], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RADIX; d += R_THREADS) hist[(int64_t)d * nblk + blockIdx.x] = cnt[d];
}

// Radix pass, step 2: stable scatter.  Warp w owns tile positions
// [512 w, 512 w + 512), item k of lane l is position 512 w + 32 k + l, so
// (warp, item, lane) order is input order; equal digits keep that order.  The
// tile is first sorted by digit in shared memory, so that the stores to global
// memory run along each digit's consecutive destinations (one transaction per
// run instead of one per element); the destinations themselves are those of
// a direct scatter.
__global__ void __launch_bounds__(R_THREADS)
k_radix_scatter(const int32_t *__restrict__ keys_in, const int32_t *__restrict__ vals_in, int64_t N,
                int shift, int nblk, const int32_t *__restrict__ offs, int32_t *__restrict__ keys_out,
                int32_t *__restrict__ vals_out)
{
    // per-warp digit counts, then (reused) the tile's keys and values in digit order
    __shared__ union {
        int32_t wcnt[R_WARPS][RADIX + 1];
        int32_t stage[2][R_TILE];
    } sm;
    static_assert(sizeof(sm.stage) <= sizeof(sm.wcnt), "staging fits the count array");
    __shared__ int32_t base_d[RADIX];
    __shared__ int32_t tstart[RADIX];  // first tile-local slot of each digit
    __shared__ int32_t wsum[R_WARPS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = threadIdx.x; t < R_WARPS * (RADIX + 1); t += R_THREADS) (&sm.wcnt[0][0])[t] = 0;
    for (int d = threadIdx.x; d < RADIX; d += R_THREADS) base_d[d] = offs[(int64_t)d * nblk + blockIdx.x];
    __syncthreads();
    const uint32_t lt_mask = (1u << lane) - 1u;
    int64_t p0 = (int64_t)blockIdx.x * R_TILE + warp * (32 * R_ITEMS) + lane;
    int32_t key[R_ITEMS], rank[R_ITEMS];
#pragma unroll
    for (int k = 0; k < R_ITEMS; ++k) {
        int64_t i = p0 + 32 * k;
        bool valid = i < N;
        key[k] = valid ? keys_in[i] : 0;
        int d = valid ? (int)(((uint32_t)key[k] >> shift) & (RADIX - 1)) : RADIX;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        int cur = sm.wcnt[warp][d];
        __syncwarp();
        if (lane == __ffs(peers) - 1) sm.wcnt[warp][d] = cur + __popc(peers);
        __syncwarp();
        rank[k] = cur + __popc(peers & lt_mask);
    }
    __syncthreads();
    // per digit: prefix over warps, and the tile's count
    for (int d = threadIdx.x; d < RADIX; d += R_THREADS) {
        int run = 0;
#pragma unroll
        for (int w = 0; w < R_WARPS; ++w) {
            int c = sm.wcnt[w][d];
            sm.wcnt[w][d] = run;
            run += c;
        }
        tstart[d] = run;
    }
    __syncthreads();
    // exclusive scan of the tile's digit counts (four consecutive digits per thread)
    {
        constexpr int PER = RADIX / R_THREADS;
        static_assert(PER * R_THREADS == RADIX, "digits per thread");
        int v[PER], sum = 0;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            v[q] = tstart[threadIdx.x * PER + q];
            sum += v[q];
        }
        int inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int n = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += n;
        }
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        int before = 0;
        for (int w = 0; w < warp; ++w) before += wsum[w];
        int run = before + inc - sum;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            tstart[threadIdx.x * PER + q] = run;
            run += v[q];
        }
    }
    __syncthreads();
    // tile-local slots and values, before the count array is reused
    int32_t lp[R_ITEMS], val[R_ITEMS];
#pragma unroll
    for (int k = 0; k < R_ITEMS; ++k) {
        int64_t i = p0 + 32 * k;
        if (i < N) {
            int d = (int)(((uint32_t)key[k] >> shift) & (RADIX - 1));
            lp[k] = tstart[d] + sm.wcnt[warp][d] + rank[k];
            val[k] = vals_in ? vals_in[i] : (int32_t)i;
        } else {
            lp[k] = -1;
            val[k] = 0;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < R_ITEMS; ++k) {
        if (lp[k] >= 0) {
            sm.stage[0][lp[k]] = key[k];
            sm.stage[1][lp[k]] = val[k];
        }
    }
    __syncthreads();
    const int64_t tile0 = (int64_t)blockIdx.x * R_TILE;
    const int nv = (int)(N - tile0 < R_TILE ? N - tile0 : R_TILE);
    for (int j = threadIdx.x; j < nv; j += R_THREADS) {
        const int32_t kk = sm.stage[0][j];
        const int d = (int)(((uint32_t)kk >> shift) & (RADIX - 1));
        const int64_t pos = (int64_t)base_d[d] + (j - tstart[d]);
        keys_out[pos] = kk;
        vals_out[pos] = sm.stage[1][j];
    }
}

int radix_blocks(int64_t N) { return (int)((N + R_TILE - 1) / R_TILE); }

}  // namespace

size_t sort_workspace_bytes(int64_t N)
{
    const int64_t nhist = (int64_t)RADIX * radix_blocks(N);
    return round_up((size_t)N * 4, 256) * 3 + round_up((size_t)nhist * 4, 256) +
           round_up((size_t)(nhist + 1) * 4, 256) + scan_workspace_bytes(nhist);
}

int sort_index_stable(const int32_t *keys, int64_t N, int bits, int32_t *order, void *ws, cudaStream_t st,
                      const int32_t **sorted_keys)
{
    if (sorted_keys) *sorted_keys = keys;
    if (N <= 0) return HACC_OK;
    char *p = reinterpret_cast<char *>(ws);
    const int nblk = radix_blocks(N);
    const int64_t nhist = (int64_t)RADIX * nblk;
    int32_t *keys_a = reinterpret_cast<int32_t *>(p);
    p += round_up((size_t)N * 4, 256);
    int32_t *keys_b = reinterpret_cast<int32_t *>(p);
    p += round_up((size_t)N * 4, 256);
    int32_t *vals_a = reinterpret_cast<int32_t *>(p);
    p += round_up((size_t)N * 4, 256);
    int32_t *hist = reinterpret_cast<int32_t *>(p);
    p += round_up((size_t)nhist * 4, 256);
    int32_t *hist_off = reinterpret_cast<int32_t *>(p);
    p += round_up((size_t)(nhist + 1) * 4, 256);
    char *scan_ws = p;
    int passes = (bits + RADIX_BITS - 1) / RADIX_BITS;
    if (passes < 1) passes = 1;
    const int32_t *kin = keys;
    const int32_t *vin = nullptr;  // first pass: values are the indices themselves
    for (int pass = 0; pass < passes; ++pass) {
        int32_t *kout = (pass % 2 == 0) ? keys_a : keys_b;
        // values alternate so that the final pass lands in `order`
        int32_t *vout = ((passes - 1 - pass) % 2 == 0) ? order : vals_a;
        const int shift = pass * RADIX_BITS;
        k_radix_hist<<<nblk, R_THREADS, 0, st>>>(kin, N, shift, nblk, hist);
        HACC_LAUNCH_CHECK();
        int rc = scan_exclusive_i32(hist, hist_off, nhist, scan_ws, st);
        if (rc) return rc;
        k_radix_scatter<<<nblk, R_THREADS, 0, st>>>(kin, vin, N, shift, nblk, hist_off, kout, vout);
        HACC_LAUNCH_CHECK();
        kin = kout;
        vin = vout;
    }
    if (sorted_keys) *sorted_keys = kin;
    return HACC_OK;
}

}  // namespace hacc
