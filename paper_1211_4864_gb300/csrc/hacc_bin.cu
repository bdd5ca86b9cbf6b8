// Chaining-mesh binning: a stable counting sort of the particles by cell.
//
// The paper's tree build partitions structure-of-arrays particle data in three
// phases (record, apply to six arrays, apply to the rest; Sec. III) so that
// streaming hides memory latency.  The GPU analogue here streams the inputs
// once and makes every later pass touch 4- or 16-byte words only:
//   1. k_bin_keys: per particle its cell and packed (offset, mass) record in
//      input order, and the cell counts (one atomic per run of equal keys in
//      a warp);
//   2. an exclusive scan of the counts: cell_start;
//   3. k_bin_slots: each particle takes a slot in its cell's range by an
//      atomic cursor (the order inside a cell is then arbitrary);
//   4. k_bin_order: each cell's input indices sorted ascending (the stable
//      order, so the result does not depend on the atomics' order): windows
//      of small cells in one bitonic network in registers, cells of up to 256
//      particles in a warp's shared memory; larger cells go to
//      k_bin_order_big, one block per cell (LSD radix passes on the index
//      digits).  The sorted indices are perm;
//   5. k_bin_gather: the records gathered into sorted4 in perm's order.
#include "hacc_common.cuh"

namespace hacc {
namespace {

constexpr int KEY_THREADS = 256;
constexpr int RADIX_BITS = 10;  // 1024 digits: a 20-bit cell key sorts in two passes
constexpr int RADIX = 1 << RADIX_BITS;
constexpr int R_THREADS = 256;
constexpr int R_WARPS = R_THREADS / 32;
constexpr int R_ITEMS = 16;
constexpr int R_TILE = R_THREADS * R_ITEMS;  // 4096 keys per block

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

constexpr int PPL = 4;  // particles per lane in passes 1 and 2: lane l of a warp takes
                        // particles i0 + l + 32 k, k < PPL (independent loads in flight)

// Runs of equal keys in consecutive lanes (the particles of a halo are often
// consecutive): lane `start` of each run claims `len` values with one atomic,
// lane start + r takes the r-th.  Every lane of the warp calls it; inactive
// lanes (keys -1 - lane, unique) form runs of their own and claim nothing.
struct Run {
    int start, len, rank;
};

__device__ __forceinline__ Run key_run(int32_t key)
{
    const int lane = threadIdx.x & 31;
    const int32_t prev = __shfl_up_sync(FULL_MASK, key, 1);
    const unsigned starts = __ballot_sync(FULL_MASK, lane == 0 || prev != key);
    const unsigned upto = (2u << lane) - 1u;  // lanes 0..lane
    Run r;
    r.start = 31 - __clz(starts & upto);
    const unsigned after = starts & ~upto;
    r.len = (after ? __ffs(after) - 1 : 32) - r.start;
    r.rank = lane - r.start;
    return r;
}

// Pass 1: per particle, its cell key (cell_of) and its (offset, mass) record
// in input order, and the count of each cell (cnt, cleared by the host;
// one atomic per run of equal keys in a warp); with mass_varies, whether any mass
// differs from the first particle's (N > 0).  Each warp walks runs of
// 32 PPL consecutive particles, its lanes converged for the aggregation.
__global__ void __launch_bounds__(KEY_THREADS)
k_bin_keys(const hacc_volume *__restrict__ vols, int V, int64_t N, const float *__restrict__ x,
           const float *__restrict__ y, const float *__restrict__ z, const float *__restrict__ dx,
           const float *__restrict__ dy, const float *__restrict__ dz, const float *__restrict__ m,
           int32_t *__restrict__ cell_of, float4 *__restrict__ rec, int32_t *__restrict__ cnt,
           uint32_t *status, uint32_t *mass_varies)
{
    MassCheck mc(m, mass_varies);
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane) * PPL;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * PPL;
    for (int64_t i0 = warp0; i0 < N; i0 += stride) {
        float px[PPL], py[PPL], pz[PPL], pm[PPL];
#pragma unroll
        for (int k = 0; k < PPL; ++k) {
            const int64_t i = i0 + lane + 32 * k;
            const bool ok = i < N;
            px[k] = ok ? x[i] : 0.f;
            py[k] = ok ? y[i] : 0.f;
            pz[k] = ok ? z[i] : 0.f;
            pm[k] = ok ? m[i] : 0.f;
        }
#pragma unroll
        for (int k = 0; k < PPL; ++k) {
            const int64_t i = i0 + lane + 32 * k;
            const bool active = i < N;
            int32_t key = 0;
            if (active) {
                const int v = find_volume_by_particle(vols, V, i);
                const hacc_volume &vol = vols[v];
                const int n = vol.n;
                float4 r;
                const int cx = axis_cell(px[k], dx, i, vol, r.x, status);
                const int cy = axis_cell(py[k], dy, i, vol, r.y, status);
                const int cz = axis_cell(pz[k], dz, i, vol, r.z, status);
                key = (int32_t)(vol.cell_base + ((int64_t)cz * n + cy) * n + cx);
                cell_of[i] = key;
                r.w = pm[k];
                __stcs(&rec[i], r);
                mc.check(r.w);
            }
            const Run run = key_run(active ? key : -1 - lane);
            if (active && run.rank == 0) atomicAdd(&cnt[key], run.len);
        }
    }
    mc.finish();
}

// Pass 2: each particle takes a slot of its cell's range [cell_start[c],
// cell_start[c + 1]) through the per-cell cursor (initialised to cell_start)
// and leaves its input index there: a run of lanes with equal keys shares
// one atomic and takes consecutive slots in lane order.  Within a cell the order is
// whatever the atomics gave; k_bin_order restores ascending index order.
__global__ void __launch_bounds__(KEY_THREADS)
k_bin_slots(int64_t N, const int32_t *__restrict__ cell_of, int32_t *__restrict__ cursor,
            int32_t *__restrict__ unsorted, uint32_t *status)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane) * PPL;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * PPL;
    for (int64_t i0 = warp0; i0 < N; i0 += stride) {
        int32_t key[PPL], base[PPL];
        Run run[PPL];
#pragma unroll
        for (int k = 0; k < PPL; ++k) {
            const int64_t i = i0 + lane + 32 * k;
            key[k] = i < N ? __ldcs(&cell_of[i]) : -1 - lane;
        }
#pragma unroll
        for (int k = 0; k < PPL; ++k) run[k] = key_run(key[k]);
        // the atomics of the PPL rounds are independent: all in flight together
#pragma unroll
        for (int k = 0; k < PPL; ++k) {
            base[k] = 0;
            if (i0 + lane + 32 * k < N && run[k].rank == 0) base[k] = atomicAdd(&cursor[key[k]], run[k].len);
        }
#pragma unroll
        for (int k = 0; k < PPL; ++k) {
            const int32_t b = __shfl_sync(FULL_MASK, base[k], run[k].start);
            const int64_t i = i0 + lane + 32 * k;
#ifdef HACC_DEBUG_BOUNDS
            if (i < N && (b + run[k].rank < 0 || b + run[k].rank >= N)) {
                atomicOr(status, HACC_STATUS_BOUNDS);
                continue;
            }
#endif
            if (i < N) unsorted[b + run[k].rank] = (int32_t)i;
        }
    }
}

// Ascending bitonic sort of one value per lane over the first P lanes
// (P a power of two, 2..32, fixed at compile time so the network unrolls):
// lanes below P end up in ascending order.
template <int P>
__device__ __forceinline__ int32_t warp_bitonic_n(int32_t v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= P; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int32_t o = __shfl_xor_sync(FULL_MASK, v, j);
            const bool keep_min = ((lane & k) == 0) == ((lane & j) == 0);
            v = keep_min ? min(v, o) : max(v, o);
        }
    return v;
}

// The same for any count n <= 32 of valid lanes (the others hold INT32_MAX).
__device__ __forceinline__ int32_t warp_bitonic(int32_t v, int n)
{
    if (n <= 1) return v;
    if (n <= 2) return warp_bitonic_n<2>(v);
    if (n <= 4) return warp_bitonic_n<4>(v);
    if (n <= 8) return warp_bitonic_n<8>(v);
    if (n <= 16) return warp_bitonic_n<16>(v);
    return warp_bitonic_n<32>(v);
}

constexpr int ORDER_THREADS = 256;
constexpr int ORDER_WARPS = ORDER_THREADS / 32;
constexpr int WARP_SORT_MAX = 256;  // cells up to this size are sorted by one warp

constexpr int SEG_SHIFT = 26;  // packed sort key of a small-cell window: (segment << 26) | index

// Pass 3: per cell, the input indices of its slots in ascending order
// (perm).  A warp takes 32
// consecutive cells at a time (their bounds one load per lane):
//  * consecutive cells of at most 32 particles whose slots fit in 32 lanes
//    form a window sorted at once: one slot per lane, key (segment, index)
//    where the segment is the lane's cell within the window, so a single
//    bitonic network sorts every cell of the window (indices below 2^26; for
//    larger N a window holds one cell and the key is the index);
//  * a cell of up to WARP_SORT_MAX particles: the warp's shared memory
//    (bitonic network, padded with INT32_MAX);
//  * larger cells: appended to big_list for k_bin_order_big.
// The next window's slots are loaded while the current one is sorted.  The
// records follow in k_bin_gather (and k_bin_order_big).
__global__ void __launch_bounds__(ORDER_THREADS)
k_bin_order(int64_t n_cells, const int32_t *__restrict__ cell_start, const int32_t *__restrict__ unsorted,
            int32_t *__restrict__ perm, int32_t *__restrict__ big_list, int32_t *__restrict__ big_count,
            int packed)
{
    __shared__ int32_t buf[ORDER_WARPS][WARP_SORT_MAX];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t *sb = buf[warp];
    const int64_t warps = (int64_t)gridDim.x * ORDER_WARPS;
    for (int64_t c0 = ((int64_t)blockIdx.x * ORDER_WARPS + warp) * 32; c0 < n_cells; c0 += warps * 32) {
        const int nc = (int)min((int64_t)32, n_cells - c0);
        const int64_t cl = c0 + min(lane, nc - 1);
        const int32_t lo = lane < nc ? cell_start[cl] : cell_start[cl + 1];  // lanes past the group: empty cells
        const int32_t hi = cell_start[cl + 1];
        const int32_t gend = __shfl_sync(FULL_MASK, hi, 31);

        // slots from b on, speculatively 32 of them (a window never holds more)
        auto slots_from = [&](int32_t b) { return b + lane < gend ? unsorted[b + lane] : INT32_MAX; };
        int q = 0;
        int32_t next = slots_from(__shfl_sync(FULL_MASK, lo, 0));  // from the group's first slot
        while (q < nc) {
            const int32_t b = __shfl_sync(FULL_MASK, lo, q);
            const int32_t n = __shfl_sync(FULL_MASK, hi, q) - b;
            if (n == 0) {
                ++q;
                continue;
            }
            if (n <= 32) {
                // the window: cells q..ql whose slots end within b + 32 (hi is non-decreasing)
                const unsigned fit = __ballot_sync(FULL_MASK, lane >= q && lane < nc && hi - b <= 32);
                const int ql = packed ? 31 - __clz(fit) : q;
                const int32_t W = __shfl_sync(FULL_MASK, hi, ql) - b;
                // segment of each slot: boundaries at the first slots of cells q..ql
                const unsigned bit = (lane >= q && lane <= ql && lo - b < 32) ? 1u << (lo - b) : 0u;
                const unsigned bounds = __reduce_or_sync(FULL_MASK, bit);
                const int seg = __popc(bounds & ((2u << lane) - 1u)) - 1;
                const int32_t v = next;
                if (ql + 1 < nc) next = slots_from(__shfl_sync(FULL_MASK, lo, ql + 1));
                int32_t key = lane < W ? (packed ? (seg << SEG_SHIFT) | v : v) : INT32_MAX;
                key = warp_bitonic(key, W);
                if (lane < W) perm[b + lane] = packed ? key & ((1 << SEG_SHIFT) - 1) : key;
                q = ql + 1;
                continue;
            }
            if (q + 1 < nc) next = slots_from(__shfl_sync(FULL_MASK, lo, q + 1));
            if (n <= WARP_SORT_MAX) {
                int P = 64;
                while (P < n) P <<= 1;
                for (int t = lane; t < P; t += 32) sb[t] = t < n ? unsorted[b + t] : INT32_MAX;
                __syncwarp();
                for (int k = 2; k <= P; k <<= 1)
                    for (int j = k >> 1; j > 0; j >>= 1) {
                        for (int t = lane; t < P / 2; t += 32) {
                            const int e = 2 * t - (t & (j - 1));  // element whose bit j is clear
                            const int32_t u = sb[e], w = sb[e + j];
                            const bool asc = (e & k) == 0;
                            if ((u > w) == asc) {
                                sb[e] = w;
                                sb[e + j] = u;
                            }
                        }
                        __syncwarp();
                    }
                for (int t = lane; t < n; t += 32) perm[b + t] = sb[t];
                __syncwarp();
            } else if (lane == 0) {
                big_list[atomicAdd(big_count, 1)] = (int32_t)(c0 + q);
            }
            ++q;
        }
    }
}

// A 16-byte load from a random place: the L2 fetches only the 64-byte block
// that holds it, not a longer neighbourhood.
__device__ __forceinline__ float4 load_random16(const float4 *p)
{
    float4 r;
    asm volatile("ld.global.L2::64B.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
                 : "l"(p));
    return r;
}

// Pass 4: the records in sorted order, sorted4[k] = rec[perm[k]]; each lane
// gathers PPL records with all loads in flight together.
__global__ void __launch_bounds__(KEY_THREADS)
k_bin_gather(int64_t N, const int32_t *__restrict__ perm, const float4 *__restrict__ rec,
             float4 *__restrict__ sorted4)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane) * PPL;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * PPL;
    for (int64_t k0 = warp0; k0 < N; k0 += stride) {
        int32_t src[PPL];
        float4 r[PPL];
#pragma unroll
        for (int u = 0; u < PPL; ++u) {
            const int64_t k = k0 + lane + 32 * u;
            src[u] = k < N ? perm[k] : 0;
        }
#pragma unroll
        for (int u = 0; u < PPL; ++u)
            if (k0 + lane + 32 * u < N) r[u] = load_random16(&rec[src[u]]);
#pragma unroll
        for (int u = 0; u < PPL; ++u) {
            const int64_t k = k0 + lane + 32 * u;
            if (k < N) sorted4[k] = r[u];
        }
    }
}

constexpr int BIG_THREADS = 512;
constexpr int BIG_WARPS = BIG_THREADS / 32;
constexpr int DIGIT_BITS = 8;
constexpr int DIGITS = 1 << DIGIT_BITS;

// Lanes (among the valid ones) whose digit equals this lane's: one ballot per
// digit bit.
__device__ __forceinline__ unsigned same_digit_lanes(int d, bool ok)
{
    unsigned eq = __ballot_sync(FULL_MASK, ok);
#pragma unroll
    for (int b = 0; b < DIGIT_BITS; ++b) {
        const bool bit = (d >> b) & 1;
        const unsigned bal = __ballot_sync(FULL_MASK, bit);
        eq &= bit ? bal : ~bal;
    }
    return eq;
}

// Index digit at `shift` (0 beyond the 32 bits: such a pass is a stable copy).
__device__ __forceinline__ int index_digit(int32_t v, int shift)
{
    return shift < 32 ? (int)(((uint32_t)v >> shift) & (DIGITS - 1)) : 0;
}

constexpr int IPT = 16;  // indices per lane per round of a counting pass

// One stable counting pass of a block over n indices by the digit at
// `shift`: src -> dst (global memory, the cell's own ranges of the two
// buffers).  Warp w owns items [w chunk, (w + 1) chunk) and walks them in
// rounds of 32 IPT, lane l taking items r + 32 k + l (all IPT loads issued
// before any is used), so (warp, round, k, lane) order is item order; ranks
// among equal digits come from lane masks (one ballot per digit bit) and
// per-warp counters, computed once to count and again to place.
__device__ void block_digit_pass(const int32_t *src, int32_t *dst, int n, int shift, int32_t (*wcnt)[DIGITS],
                                 int32_t *dtot)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = threadIdx.x; t < BIG_WARPS * DIGITS; t += BIG_THREADS) (&wcnt[0][0])[t] = 0;
    __syncthreads();
    constexpr int ROUND = 32 * IPT;
    const int chunk = (n + BIG_WARPS * 32 - 1) / (BIG_WARPS * 32) * 32;
    const int beg = min(n, warp * chunk), end = min(n, beg + chunk);
    const uint32_t lt = (1u << lane) - 1u;
    for (int r = beg; r < end; r += ROUND) {
        int32_t v[IPT];
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            const int it = r + 32 * k + lane;
            v[k] = it < end ? src[it] : 0;
        }
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            if (r + 32 * k >= end) break;  // warp-uniform
            const bool ok = r + 32 * k + lane < end;
            const int d = ok ? index_digit(v[k], shift) : DIGITS;
            const unsigned peers = same_digit_lanes(d, ok);
            if (ok && lane == __ffs(peers) - 1) wcnt[warp][d] += __popc(peers);
            __syncwarp();
        }
    }
    __syncthreads();
    // per digit: exclusive prefix over the warps, then over the digits
    if (threadIdx.x < DIGITS) {
        const int d = threadIdx.x;
        int run = 0;
        for (int w = 0; w < BIG_WARPS; ++w) {
            const int c = wcnt[w][d];
            wcnt[w][d] = run;
            run += c;
        }
        dtot[d] = run;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        constexpr int PER = DIGITS / 32;
        int c[PER], sum = 0;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            c[q] = dtot[lane * PER + q];
            sum += c[q];
        }
        int inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(FULL_MASK, inc, o);
            if (lane >= o) inc += t;
        }
        int run = inc - sum;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            dtot[lane * PER + q] = run;
            run += c[q];
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < BIG_WARPS * DIGITS; t += BIG_THREADS) (&wcnt[0][0])[t] += dtot[t % DIGITS];
    __syncthreads();
    for (int r = beg; r < end; r += ROUND) {
        int32_t v[IPT];
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            const int it = r + 32 * k + lane;
            v[k] = it < end ? src[it] : 0;
        }
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            if (r + 32 * k >= end) break;  // warp-uniform
            const bool ok = r + 32 * k + lane < end;
            const int d = ok ? index_digit(v[k], shift) : DIGITS;
            const unsigned peers = same_digit_lanes(d, ok);
            int pos = 0;
            if (ok) pos = wcnt[warp][d] + __popc(peers & lt);
            __syncwarp();
            if (ok && lane == __ffs(peers) - 1) wcnt[warp][d] += __popc(peers);
            __syncwarp();
            if (ok) dst[pos] = v[k];
        }
    }
    __syncthreads();
}

// Pass 3 for the cells k_bin_order left (more than WARP_SORT_MAX particles):
// one block per cell, taken in turn from big_list.  LSD radix passes of
// DIGIT_BITS bits over the index bits, ping-ponging between the cell's range
// of `unsorted` and of perm so that the last pass lands in perm (an odd
// number of passes; a pass on an empty digit copies).
__global__ void __launch_bounds__(BIG_THREADS)
k_bin_order_big(const int32_t *__restrict__ cell_start, int32_t *unsorted, int32_t *perm,
                const int32_t *__restrict__ big_list,
                const int32_t *__restrict__ big_count, int32_t *big_next, int passes)
{
    __shared__ int32_t wcnt[BIG_WARPS][DIGITS];
    __shared__ int32_t dtot[DIGITS];
    __shared__ int32_t cur;
    const int nbig = *big_count;
    while (true) {
        if (threadIdx.x == 0) cur = atomicAdd(big_next, 1);
        __syncthreads();
        const int k = cur;
        __syncthreads();
        if (k >= nbig) break;
        const int c = big_list[k];
        const int32_t b = cell_start[c];
        const int n = cell_start[c + 1] - b;
        for (int p = 0; p < passes; ++p) {
            int32_t *src = (p & 1) ? perm + b : unsorted + b;
            int32_t *dst = (p & 1) ? unsorted + b : perm + b;
            block_digit_pass(src, dst, n, p * DIGIT_BITS, wcnt, dtot);
        }
    }
}

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

// Binning workspace: the records in input order (16 B per particle), the
// unsorted slot contents (4 B per particle), per-cell counts (then cursors)
// and the big-cell list (4 B per cell each), two counters and the scan's
// scratch.
struct BinWs {
    float4 *rec;
    int32_t *unsorted;
    int32_t *cnt;
    int32_t *big_list;
    int32_t *ctr;  // [0] big cells found, [1] big cells taken
    char *scan_ws;
    size_t total;
};

BinWs bin_ws_layout(const hacc_mesh *mesh, void *ws)
{
    BinWs b{};
    char *p = reinterpret_cast<char *>(ws);
    size_t off = 0;
    const int64_t N = mesh->N, nc = mesh->n_cells;
    auto take = [&](size_t bytes) {
        char *q = p ? p + off : nullptr;
        off += round_up(bytes, 256);
        return q;
    };
    b.rec = reinterpret_cast<float4 *>(take((size_t)N * sizeof(float4)));
    b.unsorted = reinterpret_cast<int32_t *>(take((size_t)N * 4));
    b.cnt = reinterpret_cast<int32_t *>(take((size_t)nc * 4));
    b.big_list = reinterpret_cast<int32_t *>(take((size_t)nc * 4));
    b.ctr = reinterpret_cast<int32_t *>(take(2 * 4));
    b.scan_ws = take(scan_workspace_bytes(nc));
    b.total = off;
    return b;
}

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

namespace {

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
    HACC_CUDA_TRY(cudaMemsetAsync(b.cnt, 0, (size_t)nc * 4, st));
    HACC_CUDA_TRY(cudaMemsetAsync(b.ctr, 0, 2 * 4, st));
    k_bin_keys<<<grid_for((N + PPL - 1) / PPL, KEY_THREADS), KEY_THREADS, 0, st>>>(mesh->vols, mesh->V, N, x, y, z, dx, dy, dz, m,
                                                                 out->cell_of, b.rec, b.cnt, status,
                                                                 out->mass_varies);
    HACC_LAUNCH_CHECK();
    int rc = scan_exclusive_i32(b.cnt, out->cell_start, nc, b.scan_ws, st);
    if (rc) return rc;
    // the counts are spent: their array becomes the per-cell cursor
    HACC_CUDA_TRY(cudaMemcpyAsync(b.cnt, out->cell_start, (size_t)nc * 4, cudaMemcpyDeviceToDevice, st));
    k_bin_slots<<<grid_for((N + PPL - 1) / PPL, KEY_THREADS), KEY_THREADS, 0, st>>>(N, out->cell_of, b.cnt, b.unsorted,
                                                                                      status);
    HACC_LAUNCH_CHECK();
    float4 *s4 = reinterpret_cast<float4 *>(out->sorted4);
    k_bin_order<<<grid_for((nc + 31) / 32 * 32, ORDER_THREADS), ORDER_THREADS, 0, st>>>(
        nc, out->cell_start, b.unsorted, out->perm, b.big_list, b.ctr, N <= ((int64_t)1 << SEG_SHIFT));
    HACC_LAUNCH_CHECK();
    // index digits of the big cells' sort: enough for N - 1, an odd number of passes
    int bits = 1;
    while (bits < 31 && ((N - 1) >> bits) != 0) ++bits;
    int passes = (bits + DIGIT_BITS - 1) / DIGIT_BITS;
    if (passes % 2 == 0) ++passes;
    k_bin_order_big<<<num_sms() * 4, BIG_THREADS, 0, st>>>(out->cell_start, b.unsorted, out->perm, b.big_list,
                                                           b.ctr, b.ctr + 1, passes);
    HACC_LAUNCH_CHECK();
    k_bin_gather<<<grid_for((N + PPL - 1) / PPL, KEY_THREADS), KEY_THREADS, 0, st>>>(N, out->perm, b.rec, s4);
    HACC_LAUNCH_CHECK();
    return HACC_OK;
}
