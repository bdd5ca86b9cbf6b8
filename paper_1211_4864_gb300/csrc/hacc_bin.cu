// Chaining-mesh binning: a stable counting sort of the particles by cell.
//
// The paper's tree build partitions structure-of-arrays particle data in three
// phases (record, apply to six arrays, apply to the rest; Sec. III) so that
// streaming hides memory latency.  The GPU analogue here is a
// least-significant-digit counting sort on the cell key that carries each
// particle's record through its passes, so that every pass reads its input
// in order and writes its output in runs of consecutive slots (no atomics
// on global memory, no random gathers):
//   1. k_bin_keys: per particle its cell key (cell_of) and its (offset, mass)
//      record, both in input order, and per tile of BIN_TILE particles the
//      counts of the key's lowest 10-bit digit, a row per tile;
//   2. a column scan of those rows (k_bin_scan_chunks, _digits, _rows): each
//      tile's first slot for each digit;
//   3. k_bin_scatter, once per digit from the lowest: each tile's keys
//      ranked stably by the digit in shared memory (warp match masks and
//      per-warp counters, so equal digits keep the tile's order), then its
//      keys, indices and records stored to their slots in digit order.
//      Before each later pass k_bin_hist counts the next digit per tile of
//      the previous pass's output.  The last pass writes perm and sorted4
//      themselves;
//   4. k_bin_cell_start: each cell's first slot by binary search of the
//      sorted keys.
// Each pass is stable, so within a cell the order is ascending input index.
#include "hacc_common.cuh"

namespace hacc {
namespace {

__device__ __forceinline__ float sanitize(float v, uint32_t *status)
{
    if (!isfinite(v)) {
        atomicOr(status, HACC_STATUS_NONFINITE);
        return 0.0f;
    }
    return v;
}

// Position x + d wrapped into [0, L) in float64, each step one
// round-to-nearest operation (used when displacements are given).
__device__ __forceinline__ double wrap64(double p, double L)
{
    double q = floor(__ddiv_rn(p, L));
    double pw = __dsub_rn(p, __dmul_rn(q, L));
    if (pw < 0.0) pw = __dadd_rn(pw, L);
    if (pw >= L) pw = __dsub_rn(pw, L);
    return pw;
}

__device__ __forceinline__ int cell64(double pw, float inv_w, int n)
{
    int c = (int)floor(__dmul_rn(pw, (double)inv_w));
    c = c > n - 1 ? n - 1 : c;
    return c < 0 ? 0 : c;
}

// One axis: cell coordinate and offset from the cell centre
// fl32((c + 1/2) w) (|o| <= w/2: half the rounding of a corner-relative
// offset).  Without a displacement every step is float32; with one, the
// position x + d is formed and wrapped in float64 and only the final offset
// is rounded to float32.
__device__ __forceinline__ int axis_cell(float x, const float *d, int64_t i, const hacc_volume &vol, float &o,
                                         uint32_t *status)
{
    const float L = vol.L, w = vol.w, iw = vol.inv_w;
    const int n = vol.n;
    if (!d) {
        const float xw = wrap32(sanitize(x, status), L);
        const int c = cell1(xw, iw, n);
        o = __fsub_rn(xw, cell_centre(c, w));
        return c;
    }
    const double pw = wrap64(__dadd_rn((double)sanitize(x, status), (double)sanitize(d[i], status)), (double)L);
    const int c = cell64(pw, iw, n);
    o = __double2float_rn(__dsub_rn(pw, (double)cell_centre(c, w)));
    return c;
}

constexpr unsigned FULL_MASK = 0xffffffffu;

constexpr int BIN_BITS = 10;  // digit of one pass: a key below 2^20 sorts in two passes
constexpr int BIN_DIGITS = 1 << BIN_BITS;
constexpr int BIN_THREADS = 512;
constexpr int BIN_ITEMS = 8;
constexpr int BIN_TILE = BIN_THREADS * BIN_ITEMS;  // 4096 particles per tile

// k_bin_scatter: two blocks of SC_THREADS per SM, SC_ITEMS items per thread.
constexpr int SC_THREADS = 512;
constexpr int SC_WARPS = SC_THREADS / 32;
constexpr int SC_ITEMS = BIN_TILE / SC_THREADS;
constexpr int SC_WORDS = BIN_DIGITS / 2 + 1;  // per-warp counters, two 16-bit digits a word; the
                                              // last word takes the items past N
// Its shared memory: the tile's keys and its first global slot per digit
// (copied in asynchronously, double-buffered, one tile ahead), the per-warp
// counters, the inverse of the tile's digit order, the tile's first local
// slot per digit and the warp totals of the scan.
constexpr size_t SM_KEY = 0;                                                  // [2][BIN_TILE]
constexpr size_t SM_BASE = SM_KEY + 2 * sizeof(int32_t) * BIN_TILE;          // [2][BIN_DIGITS]
constexpr size_t SM_CNT = SM_BASE + 2 * sizeof(int32_t) * BIN_DIGITS;
constexpr size_t SM_INV = SM_CNT + sizeof(uint32_t) * SC_WARPS * SC_WORDS;
constexpr size_t SM_TSTART = SM_INV + sizeof(uint16_t) * BIN_TILE;
constexpr size_t SM_WSUM = SM_TSTART + sizeof(int32_t) * BIN_DIGITS;
constexpr size_t SCATTER_SMEM = SM_WSUM + sizeof(int32_t) * SC_WARPS;
static_assert(SC_ITEMS * SC_THREADS == BIN_TILE && BIN_DIGITS / 2 == SC_THREADS,
              "one digit pair per thread in the prefix");
static_assert(2 * SCATTER_SMEM <= 227 * 1024, "shared memory of two blocks");
static_assert(BIN_TILE <= 65536, "16-bit tile positions");

// Asynchronous copy of 4 bytes from global to shared memory (cp.async), its
// commit and wait.
__device__ __forceinline__ void async_copy4(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(PENDING) : "memory");
}

// Asks the L2 to fetch [p, p + bytes) of global memory (a hint, no data
// returned): whole 16-byte units from the first 16-byte boundary, in
// pieces of at most 32 KB.  Called by one thread.
__device__ __forceinline__ void prefetch_l2(const void *p, int64_t bytes)
{
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    uintptr_t q = (a + 15) & ~(uintptr_t)15;
    int64_t left = (bytes - (int64_t)(q - a)) & ~(int64_t)15;
    while (left >= 16) {
        const uint32_t n = left > 32768 ? 32768u : (uint32_t)left;
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(q), "r"(n) : "memory");
        q += n;
        left -= n;
    }
}

// Elements [t BIN_TILE, (t + 1) BIN_TILE) of an array of N, clipped to N.
template <class T>
__device__ __forceinline__ void prefetch_tile(const T *a, int64_t t, int64_t N)
{
    const int64_t b = t * BIN_TILE;
    if (a && b < N) prefetch_l2(a + b, (N - b < BIN_TILE ? N - b : BIN_TILE) * (int64_t)sizeof(T));
}

// The particle arrays of a binning call (dx, dy, dz all given or all NULL).
struct ParticleIn {
    const hacc_volume *vols;
    int V;
    const float *x, *y, *z, *dx, *dy, *dz, *m;
};

__device__ __forceinline__ int key_digit(int32_t key, int shift)
{
    return (int)(((uint32_t)key >> shift) & (BIN_DIGITS - 1));
}

// Adds one digit per thread to the tile's counters (BIN_DIGITS: no item):
// a run of equal digits in consecutive lanes shares one shared-memory atomic.
__device__ __forceinline__ void count_digit(int32_t *cnt, int d)
{
    const int lane = threadIdx.x & 31;
    const int prev = __shfl_up_sync(FULL_MASK, d, 1);
    const unsigned starts = __ballot_sync(FULL_MASK, lane == 0 || prev != d);
    if (d < BIN_DIGITS && ((starts >> lane) & 1u)) {
        const unsigned after = starts & ~((2u << lane) - 1u);
        atomicAdd(&cnt[d], (after ? __ffs(after) - 1 : 32) - lane);
    }
}

// Pass 1: per particle its cell key (cell_of) and its (offset, mass) record
// (rec), both in input order; per tile (particles [t BIN_TILE, (t + 1)
// BIN_TILE)) the counts of the key's lowest digit into hist (a row per
// tile, hist[t BIN_DIGITS + d]); with mass_varies, whether any mass differs
// from the first particle's (N > 0).  Persistent blocks take tiles in turn
// and ask the L2 for their next tile's inputs while they work on the
// current one.
// DISP: displacements are given (the float64 position path).
template <bool DISP>
__global__ void __launch_bounds__(BIN_THREADS, 2)
k_bin_keys(ParticleIn P, int64_t N, int nblk, int32_t *__restrict__ cell_of, float4 *__restrict__ rec,
           int32_t *__restrict__ hist, uint32_t *status, uint32_t *mass_varies)
{
    __shared__ int32_t cnt[BIN_DIGITS];
    MassCheck mc(P.m, mass_varies);
    for (int64_t t = blockIdx.x; t < nblk; t += gridDim.x) {
        if (threadIdx.x == 0) {
            const int64_t tn = t + gridDim.x;
            prefetch_tile(P.x, tn, N);
            prefetch_tile(P.y, tn, N);
            prefetch_tile(P.z, tn, N);
            prefetch_tile(P.m, tn, N);
            if (DISP) {
                prefetch_tile(P.dx, tn, N);
                prefetch_tile(P.dy, tn, N);
                prefetch_tile(P.dz, tn, N);
            }
        }
        for (int d = threadIdx.x; d < BIN_DIGITS; d += BIN_THREADS) cnt[d] = 0;
        __syncthreads();
        const int64_t t0 = t * BIN_TILE + threadIdx.x;
        // items in groups of G, their loads in flight together (the float64
        // path takes more registers)
        constexpr int G = DISP ? 2 : 4;
#pragma unroll
        for (int g = 0; g < BIN_ITEMS; g += G) {
            float px[G], py[G], pz[G], pm[G];
#pragma unroll
            for (int k = 0; k < G; ++k) {
                const int64_t i = t0 + (int64_t)(g + k) * BIN_THREADS;
                const bool ok = i < N;
                px[k] = ok ? P.x[i] : 0.f;
                py[k] = ok ? P.y[i] : 0.f;
                pz[k] = ok ? P.z[i] : 0.f;
                pm[k] = ok ? P.m[i] : 0.f;
            }
#pragma unroll
            for (int k = 0; k < G; ++k) {
                const int64_t i = t0 + (int64_t)(g + k) * BIN_THREADS;
                int d = BIN_DIGITS;
                if (i < N) {
                    const hacc_volume &vol = P.vols[find_volume_by_particle(P.vols, P.V, i)];
                    const int n = vol.n;
                    float4 r;
                    const int cx = axis_cell(px[k], DISP ? P.dx : nullptr, i, vol, r.x, status);
                    const int cy = axis_cell(py[k], DISP ? P.dy : nullptr, i, vol, r.y, status);
                    const int cz = axis_cell(pz[k], DISP ? P.dz : nullptr, i, vol, r.z, status);
                    const int32_t key = (int32_t)(vol.cell_base + ((int64_t)cz * n + cy) * n + cx);
                    r.w = pm[k];
                    cell_of[i] = key;
                    rec[i] = r;
                    mc.check(pm[k]);
                    d = key_digit(key, 0);
                }
                count_digit(cnt, d);
            }
        }
        __syncthreads();
        for (int d = threadIdx.x; d < BIN_DIGITS; d += BIN_THREADS) hist[(int64_t)t * BIN_DIGITS + d] = cnt[d];
        __syncthreads();
    }
    mc.finish();
}

// Before a later pass: the counts of the digit at `shift` per tile of the
// previous pass's output keys, a row per tile (persistent blocks, next tile
// prefetched as in k_bin_keys).
__global__ void __launch_bounds__(BIN_THREADS)
k_bin_hist(const int32_t *__restrict__ keys, int64_t N, int shift, int nblk, int32_t *__restrict__ hist)
{
    __shared__ int32_t cnt[BIN_DIGITS];
    for (int64_t t = blockIdx.x; t < nblk; t += gridDim.x) {
        if (threadIdx.x == 0) prefetch_tile(keys, t + gridDim.x, N);
        for (int d = threadIdx.x; d < BIN_DIGITS; d += BIN_THREADS) cnt[d] = 0;
        __syncthreads();
        const int64_t t0 = t * BIN_TILE + threadIdx.x;
        int32_t kk[BIN_ITEMS];
#pragma unroll
        for (int k = 0; k < BIN_ITEMS; ++k) {
            const int64_t i = t0 + (int64_t)k * BIN_THREADS;
            kk[k] = i < N ? keys[i] : 0;
        }
#pragma unroll
        for (int k = 0; k < BIN_ITEMS; ++k)
            count_digit(cnt, t0 + (int64_t)k * BIN_THREADS < N ? key_digit(kk[k], shift) : BIN_DIGITS);
        __syncthreads();
        for (int d = threadIdx.x; d < BIN_DIGITS; d += BIN_THREADS) hist[(int64_t)t * BIN_DIGITS + d] = cnt[d];
        __syncthreads();
    }
}

// One stable counting pass by the digit at `shift`.  Persistent blocks, two
// per SM, take tiles in turn.  In tile t, warp w owns tile positions
// [w 32 SC_ITEMS, (w + 1) 32 SC_ITEMS) and item k of lane l is position
// w 32 SC_ITEMS + 32 k + l, so (warp, item, lane) order is input order and
// equal digits keep it: an item's slot is the tile's first slot for its
// digit (offs, the scanned counts) plus the number of earlier items of the
// tile with that digit (per-warp counters).  The tile's keys and first
// slots arrive in shared memory asynchronously, one tile ahead; while the
// keys are ranked the L2 fetches the tile's indices and records, which the
// store loop then gathers in digit order (through the inverse of the
// ranking), so the stores to global memory run along each digit's
// consecutive slots.  FIRST: the input is pass 1's output (keys cell_of,
// records in input order; an item's index is its position), otherwise the
// previous pass's (key, index, record) arrays.  N < 2^31.
template <bool FIRST>
__global__ void __launch_bounds__(SC_THREADS, 2)
k_bin_scatter(const int32_t *__restrict__ key_in, const int32_t *__restrict__ idx_in,
              const float4 *__restrict__ rec_in, int N, int shift, int nblk, const int32_t *__restrict__ offs,
              int32_t *__restrict__ key_out, int32_t *__restrict__ idx_out, float4 *__restrict__ rec_out,
              uint32_t *status)
{
    extern __shared__ __align__(16) unsigned char smem[];
    int32_t *skey2 = reinterpret_cast<int32_t *>(smem + SM_KEY);
    int32_t *base2 = reinterpret_cast<int32_t *>(smem + SM_BASE);
    uint32_t(*wcnt)[SC_WORDS] = reinterpret_cast<uint32_t(*)[SC_WORDS]>(smem + SM_CNT);
    uint16_t *inv = reinterpret_cast<uint16_t *>(smem + SM_INV);
    int32_t *tstart = reinterpret_cast<int32_t *>(smem + SM_TSTART);
    int32_t *wsum = reinterpret_cast<int32_t *>(smem + SM_WSUM);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const int l0 = warp * (32 * SC_ITEMS) + lane;  // tile position of item 0
    // a tile's keys and first global slots per digit, into buffer b
    auto fetch_keys = [&](int t, int b) {
        if (t < nblk) {
            const int tile0 = t * BIN_TILE;
#pragma unroll
            for (int k = 0; k < SC_ITEMS; ++k)
                if (tile0 + l0 + 32 * k < N)
                    async_copy4(skey2 + b * BIN_TILE + l0 + 32 * k, key_in + tile0 + l0 + 32 * k);
            for (int d = threadIdx.x; d < BIN_DIGITS; d += SC_THREADS)
                async_copy4(base2 + b * BIN_DIGITS + d, offs + (int64_t)t * BIN_DIGITS + d);
        }
        async_commit();
    };
    fetch_keys(blockIdx.x, 0);
    int buf = 0;
    for (int t = blockIdx.x; t < nblk; t += gridDim.x, buf ^= 1) {
        const int tile0 = t * BIN_TILE;
        const int32_t *skey = skey2 + buf * BIN_TILE;
        const int32_t *base_d = base2 + buf * BIN_DIGITS;
        async_wait<0>();  // this tile's keys and slots (fetched during the previous tile)
        for (int i = threadIdx.x; i < SC_WARPS * SC_WORDS; i += SC_THREADS) (&wcnt[0][0])[i] = 0u;
        __syncthreads();
        // the L2 fetches this tile's indices and records while its keys are
        // ranked; the next tile's keys and slots land while this one is stored
        fetch_keys(t + gridDim.x, buf ^ 1);
        if (threadIdx.x == 0) {
            prefetch_tile(rec_in, t, N);
            if (!FIRST) prefetch_tile(idx_in, t, N);
            prefetch_tile(key_in, t + 2 * gridDim.x, N);
        }
        int32_t key[SC_ITEMS];
        int slot[SC_ITEMS];
        // rank of each item among the warp's earlier items with its digit:
        // the lowest lane of each group of equal digits adds the group to the
        // warp's counter and hands the old count to the group
#pragma unroll
        for (int k = 0; k < SC_ITEMS; ++k) {
            const bool ok = tile0 + l0 + 32 * k < N;
            key[k] = ok ? skey[l0 + 32 * k] : 0;
            const int d = ok ? key_digit(key[k], shift) : BIN_DIGITS;
            const unsigned peers = __match_any_sync(FULL_MASK, d);
            const int leader = __ffs(peers) - 1;
            const int half = (d & 1) * 16;
            uint32_t old = 0u;
            if (lane == leader) old = atomicAdd(&wcnt[warp][d >> 1], (uint32_t)__popc(peers) << half);
            old = __shfl_sync(FULL_MASK, old, leader);
            slot[k] = (int)((old >> half) & 0xffffu) + __popc(peers & lt);
        }
        __syncthreads();
        // per digit pair j (thread j < 512): exclusive prefix over the warps
        // of the packed counts (both halves at once: a tile's count per digit
        // stays below 2^16), then the tile's exclusive scan of the digit
        // counts, two digits per thread: its first local slot per digit
        if (threadIdx.x < BIN_DIGITS / 2) {
            const int j = threadIdx.x;
            uint32_t run = 0u;
#pragma unroll
            for (int w = 0; w < SC_WARPS; ++w) {
                const uint32_t c = wcnt[w][j];
                wcnt[w][j] = run;
                run += c;
            }
            const int c0 = (int)(run & 0xffffu), c1 = (int)(run >> 16);
            int inc = c0 + c1;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int n = __shfl_up_sync(FULL_MASK, inc, o);
                if (lane >= o) inc += n;
            }
            if (lane == 31) wsum[warp] = inc;
            tstart[2 * j] = inc - c0 - c1;  // within the warp, completed below
            tstart[2 * j + 1] = inc - c1;
        }
        __syncthreads();
        if (threadIdx.x < BIN_DIGITS / 2) {
            int before = lane < warp ? wsum[lane] : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) before += __shfl_xor_sync(FULL_MASK, before, o);
            tstart[2 * threadIdx.x] += before;
            tstart[2 * threadIdx.x + 1] += before;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < SC_ITEMS; ++k) {
            if (tile0 + l0 + 32 * k < N) {
                const int d = key_digit(key[k], shift);
                inv[slot[k] + tstart[d] + (int)((wcnt[warp][d >> 1] >> ((d & 1) * 16)) & 0xffffu)] =
                    (uint16_t)(l0 + 32 * k);
            }
        }
        __syncthreads();
        // the tile in digit order: each item's index and record gathered from
        // the tile's range of the input (in L2), G items' loads in flight together
        const int nv = N - tile0 < BIN_TILE ? N - tile0 : BIN_TILE;
        constexpr int G = 4;
        for (int j0 = threadIdx.x; j0 < nv; j0 += G * SC_THREADS) {
            int l[G];
            int32_t ix[G];
            float4 r[G];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const int j = j0 + g * SC_THREADS;
                l[g] = j < nv ? inv[j] : 0;
                if (j < nv) {
                    ix[g] = FIRST ? tile0 + l[g] : idx_in[tile0 + l[g]];
                    r[g] = rec_in[tile0 + l[g]];
                }
            }
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const int j = j0 + g * SC_THREADS;
                if (j >= nv) break;
                const int32_t kk = skey[l[g]];
                const int d = key_digit(kk, shift);
                const int pos = base_d[d] + (j - tstart[d]);
#ifdef HACC_DEBUG_BOUNDS
                if (pos < 0 || pos >= N) {
                    atomicOr(status, HACC_STATUS_BOUNDS);
                    continue;
                }
#endif
                key_out[pos] = kk;
                idx_out[pos] = ix[g];
                rec_out[pos] = r[g];
            }
        }
        __syncthreads();  // shared memory is reused by the next tile
    }
    async_wait<0>();
}

constexpr int SCAN_TC = 32;  // tiles per chunk of the digit-count scan

// Scan of the per-tile digit counts into each tile's first slot per digit,
// offs[t][d] = (count of digits below d) + (count of digit d in tiles before
// t); rows of BIN_DIGITS per tile.  Step 1: per chunk of SCAN_TC tiles, the
// sum of each digit's counts.
__global__ void __launch_bounds__(BIN_DIGITS)
k_bin_scan_chunks(const int32_t *__restrict__ hist, int nblk, int32_t *__restrict__ csum)
{
    const int c = blockIdx.x, d = threadIdx.x;
    const int t1 = min(nblk, (c + 1) * SCAN_TC);
    int s = 0;
#pragma unroll 8
    for (int t = c * SCAN_TC; t < t1; ++t) s += hist[(int64_t)t * BIN_DIGITS + d];
    csum[(int64_t)c * BIN_DIGITS + d] = s;
}

// Step 2: per digit (one warp each, its lanes over the chunks), the
// exclusive prefix of its chunk sums in place, and its total.
__global__ void __launch_bounds__(BIN_DIGITS)
k_bin_scan_digits(int32_t *__restrict__ csum, int nchunks, int32_t *__restrict__ total)
{
    const int lane = threadIdx.x & 31;
    const int d = blockIdx.x * (BIN_DIGITS / 32) + (threadIdx.x >> 5);
    int carry = 0;
    for (int c0 = 0; c0 < nchunks; c0 += 32) {
        const int c = c0 + lane;
        const int v = c < nchunks ? csum[(int64_t)c * BIN_DIGITS + d] : 0;
        int inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int n = __shfl_up_sync(FULL_MASK, inc, o);
            if (lane >= o) inc += n;
        }
        if (c < nchunks) csum[(int64_t)c * BIN_DIGITS + d] = carry + inc - v;
        carry += __shfl_sync(FULL_MASK, inc, 31);
    }
    if (lane == 0) total[d] = carry;
}

// Step 3: each tile's row, the digit's first slot (the exclusive prefix of
// the digit totals, formed by every block) plus the chunk's prefix plus the
// counts of the chunk's earlier tiles.
__global__ void __launch_bounds__(BIN_DIGITS)
k_bin_scan_rows(const int32_t *__restrict__ hist, int nblk, const int32_t *__restrict__ csum,
                const int32_t *__restrict__ total, int32_t *__restrict__ offs)
{
    __shared__ int32_t wsum[BIN_DIGITS / 32];
    const int c = blockIdx.x, d = threadIdx.x, lane = d & 31, warp = d >> 5;
    const int v = total[d];
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int n = __shfl_up_sync(FULL_MASK, inc, o);
        if (lane >= o) inc += n;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    int before = lane < warp ? wsum[lane] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) before += __shfl_xor_sync(FULL_MASK, before, o);
    int run = before + inc - v + csum[(int64_t)c * BIN_DIGITS + d];
    const int t1 = min(nblk, (c + 1) * SCAN_TC);
#pragma unroll 8
    for (int t = c * SCAN_TC; t < t1; ++t) {
        const int64_t i = (int64_t)t * BIN_DIGITS + d;
        const int h = hist[i];
        offs[i] = run;
        run += h;
    }
}

// cell_start[c] = the first sorted slot whose key is at least c (c = 0..nc;
// cell_start[nc] = N): a binary search of the sorted keys per cell.
__global__ void __launch_bounds__(256)
k_bin_cell_start(const int32_t *__restrict__ keys, int64_t N, int64_t nc, int32_t *__restrict__ cell_start)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c <= nc; c += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = N;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int64_t)keys[mid] < c)
                lo = mid + 1;
            else
                hi = mid;
        }
        cell_start[c] = (int32_t)lo;
    }
}


// Binning workspace: one set of pass buffers (key, index, record: 24 B per
// particle), the other set's keys (its indices and records are perm and
// sorted4 themselves: 4 B per particle), the per-tile digit counts and their
// scan (4 B per digit and tile each: about 2 B per particle) and the scan's
// chunk sums and digit totals.  Nothing scales with the number of cells.
struct BinWs {
    int32_t *keyX, *idxX;
    float4 *recX;
    int32_t *keyY;
    int32_t *hist, *offs, *csum, *dtot;
    size_t total;
};

int bin_tiles(int64_t N) { return (int)((N + BIN_TILE - 1) / BIN_TILE); }
int scan_chunks(int64_t N) { return (bin_tiles(N) + SCAN_TC - 1) / SCAN_TC; }

BinWs bin_ws_layout(const hacc_mesh *mesh, void *ws)
{
    BinWs b{};
    char *p = reinterpret_cast<char *>(ws);
    size_t off = 0;
    const int64_t N = mesh->N;
    const int64_t nhist = (int64_t)BIN_DIGITS * bin_tiles(N);
    auto take = [&](size_t bytes) {
        char *q = p ? p + off : nullptr;
        off += round_up(bytes, 256);
        return q;
    };
    b.recX = reinterpret_cast<float4 *>(take((size_t)N * sizeof(float4)));
    b.keyX = reinterpret_cast<int32_t *>(take((size_t)N * 4));
    b.idxX = reinterpret_cast<int32_t *>(take((size_t)N * 4));
    b.keyY = reinterpret_cast<int32_t *>(take((size_t)N * 4));
    b.hist = reinterpret_cast<int32_t *>(take((size_t)nhist * 4));
    b.offs = reinterpret_cast<int32_t *>(take((size_t)nhist * 4));
    b.csum = reinterpret_cast<int32_t *>(take((size_t)scan_chunks(N) * BIN_DIGITS * 4));
    b.dtot = reinterpret_cast<int32_t *>(take((size_t)BIN_DIGITS * 4));
    b.total = off;
    return b;
}
int grid_for(int64_t n, int threads)
{
    int64_t g = (n + threads - 1) / threads;
    int64_t cap = (int64_t)num_sms() * 16;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace
}  // namespace hacc

using namespace hacc;

extern "C" size_t hacc_bin_workspace_size(const hacc_mesh *mesh)
{
    if (!mesh) return 0;
    return bin_ws_layout(mesh, nullptr).total;
}

extern "C" int hacc_bin(const hacc_mesh *mesh, const float *x, const float *y, const float *z,
                        const float *dx, const float *dy, const float *dz, const float *m,
                        const hacc_binned *out, void *ws, size_t ws_bytes, uint32_t *status, void *stream)
{
    if ((dx || dy || dz) && !(dx && dy && dz)) return HACC_ERR_INVALID;
    if (!mesh || !out || !mesh->vols || mesh->V < 1 || mesh->N < 0 || mesh->n_cells < 1 || !status)
        return HACC_ERR_INVALID;
    if (mesh->N >= ((int64_t)1 << 31) || mesh->n_cells >= ((int64_t)1 << 31)) return HACC_ERR_INVALID;
    if (!out->cell_start || !ws || !aligned16(ws)) return HACC_ERR_INVALID;
    const int64_t N = mesh->N, nc = mesh->n_cells;
    if (N > 0 && (!x || !y || !z || !m || !out->cell_of || !out->perm || !out->sorted4))
        return HACC_ERR_INVALID;
    if (N > 0 && !aligned16(out->sorted4)) return HACC_ERR_INVALID;
    BinWs b = bin_ws_layout(mesh, ws);
    if (ws_bytes < b.total) return HACC_ERR_CAPACITY;
    cudaStream_t st = as_stream(stream);

    if (out->mass_varies) HACC_CUDA_TRY(cudaMemsetAsync(out->mass_varies, 0, sizeof(uint32_t), st));
    if (N == 0) {
        HACC_CUDA_TRY(cudaMemsetAsync(out->cell_start, 0, (size_t)(nc + 1) * 4, st));
        return HACC_OK;
    }
    const ParticleIn P{mesh->vols, mesh->V, x, y, z, dx, dy, dz, m};
    const int nblk = bin_tiles(N);
    // digits of the largest key, nc - 1: one pass per BIN_BITS of them
    int bits = 1;
    while (bits < 31 && ((nc - 1) >> bits) != 0) ++bits;
    const int passes = (bits + BIN_BITS - 1) / BIN_BITS;
    HACC_CUDA_TRY(cudaFuncSetAttribute(k_bin_scatter<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)SCATTER_SMEM));
    HACC_CUDA_TRY(cudaFuncSetAttribute(k_bin_scatter<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)SCATTER_SMEM));
    // persistent grids: blocks per SM of each kind
    auto grid = [&](int per_sm) { return nblk < num_sms() * per_sm ? nblk : num_sms() * per_sm; };
    float4 *s4 = reinterpret_cast<float4 *>(out->sorted4);
    // the buffer sets alternate so that the last pass lands in perm and sorted4;
    // pass 1's records go to the record buffer the first counting pass does not write
    auto to_out = [&](int p) { return (passes - 1 - p) % 2 == 0; };
    float4 *rec0 = to_out(0) ? b.recX : s4;
    if (dx)
        k_bin_keys<true><<<grid(2), BIN_THREADS, 0, st>>>(P, N, nblk, out->cell_of, rec0, b.hist, status,
                                                          out->mass_varies);
    else
        k_bin_keys<false><<<grid(2), BIN_THREADS, 0, st>>>(P, N, nblk, out->cell_of, rec0, b.hist, status,
                                                           out->mass_varies);
    HACC_LAUNCH_CHECK();
    const int32_t *kin = out->cell_of, *iin = nullptr;
    const float4 *rin = rec0;
    for (int p = 0; p < passes; ++p) {
        const int shift = p * BIN_BITS;
        if (p > 0) {
            k_bin_hist<<<grid(3), BIN_THREADS, 0, st>>>(kin, N, shift, nblk, b.hist);
            HACC_LAUNCH_CHECK();
        }
        const int nch = scan_chunks(N);
        k_bin_scan_chunks<<<nch, BIN_DIGITS, 0, st>>>(b.hist, nblk, b.csum);
        HACC_LAUNCH_CHECK();
        k_bin_scan_digits<<<BIN_DIGITS / (BIN_DIGITS / 32), BIN_DIGITS, 0, st>>>(b.csum, nch, b.dtot);
        HACC_LAUNCH_CHECK();
        k_bin_scan_rows<<<nch, BIN_DIGITS, 0, st>>>(b.hist, nblk, b.csum, b.dtot, b.offs);
        HACC_LAUNCH_CHECK();
        int32_t *ko = to_out(p) ? b.keyY : b.keyX;
        int32_t *io = to_out(p) ? out->perm : b.idxX;
        float4 *ro = to_out(p) ? s4 : b.recX;
        if (p == 0)
            k_bin_scatter<true><<<grid(2), SC_THREADS, SCATTER_SMEM, st>>>(kin, nullptr, rin, (int)N, shift, nblk,
                                                                            b.offs, ko, io, ro, status);
        else
            k_bin_scatter<false><<<grid(2), SC_THREADS, SCATTER_SMEM, st>>>(kin, iin, rin, (int)N, shift, nblk,
                                                                             b.offs, ko, io, ro, status);
        HACC_LAUNCH_CHECK();
        kin = ko;
        iin = io;
        rin = ro;
    }
    k_bin_cell_start<<<grid_for(nc + 1, 256), 256, 0, st>>>(b.keyY, N, nc, out->cell_start);
    HACC_LAUNCH_CHECK();
    return HACC_OK;
}
