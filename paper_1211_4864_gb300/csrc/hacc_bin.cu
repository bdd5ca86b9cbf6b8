// Chaining-mesh binning: cell keys, stable LSD radix sort of (cell, index),
// gather of cell-relative float4 (ox, oy, oz, m) into sorted order.
//
// The paper's tree build partitions structure-of-arrays particle data in three
// phases (record, apply to six arrays, apply to the rest; Sec. III) so that
// streaming hides memory latency.  The GPU analogue is one streaming pass that
// computes each particle's cell and its packed (offset, mass) record, a stable
// radix sort that moves only 8-byte (key, index) pairs, and one gather of the
// 16-byte records.
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

// One axis: cell coordinate and cell-relative offset.  Without a
// displacement every step is float32; with one, the position x + d is formed
// and wrapped in float64 and only the final offset is rounded to float32.
__device__ __forceinline__ int axis_cell(float x, const float *d, int64_t i, const hacc_volume &vol, float &o,
                                         uint32_t *status)
{
    const float L = vol.L, w = vol.w, iw = vol.inv_w;
    const int n = vol.n;
    if (!d) {
        const float xw = wrap32(sanitize(x, status), L);
        const int c = cell1(xw, iw, n);
        o = __fsub_rn(xw, __fmul_rn((float)c, w));
        return c;
    }
    const double pw = wrap64(__dadd_rn((double)sanitize(x, status), (double)sanitize(d[i], status)), (double)L);
    const int c = cell64(pw, iw, n);
    o = __double2float_rn(__dsub_rn(pw, (double)__fmul_rn((float)c, w)));
    return c;
}

// Pass 1: per particle, its cell key and its (offset, mass) record in input
// order; with mass_varies, whether any mass differs from the first
// particle's (N > 0).
__global__ void __launch_bounds__(KEY_THREADS)
k_bin_keys(const hacc_volume *__restrict__ vols, int V, int64_t N, const float *__restrict__ x,
           const float *__restrict__ y, const float *__restrict__ z, const float *__restrict__ dx,
           const float *__restrict__ dy, const float *__restrict__ dz, const float *__restrict__ m,
           int32_t *__restrict__ cell_of, int32_t *__restrict__ keys, float4 *__restrict__ rec,
           uint32_t *status, uint32_t *mass_varies)
{
    MassCheck mc(m, mass_varies);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        int v = find_volume_by_particle(vols, V, i);
        const hacc_volume &vol = vols[v];
        const int n = vol.n;
        float4 r;
        const int cx = axis_cell(x[i], dx, i, vol, r.x, status);
        const int cy = axis_cell(y[i], dy, i, vol, r.y, status);
        const int cz = axis_cell(z[i], dz, i, vol, r.z, status);
        int32_t key = (int32_t)(vol.cell_base + ((int64_t)cz * n + cy) * n + cx);
        cell_of[i] = key;
        keys[i] = key;
        r.w = m[i];
        rec[i] = r;
        mc.check(r.w);
    }
    mc.finish();
}

// cell_start from the sorted keys: the first slot whose key is >= c (a binary
// search per cell c in [0, n_cells]; cell n_cells gets N), empty cells
// included.
__global__ void __launch_bounds__(256)
k_cell_starts(const int32_t *__restrict__ skeys, int64_t N, int64_t n_cells, int32_t *__restrict__ cell_start)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c <= n_cells;
         c += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = N;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int64_t)skeys[mid] < c) lo = mid + 1; else hi = mid;
        }
        cell_start[c] = (int32_t)lo;
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

// Gather of the (offset, mass) records into sorted order.
__global__ void __launch_bounds__(256)
k_bin_gather(int64_t N, const int32_t *__restrict__ perm, const float4 *__restrict__ rec,
             float4 *__restrict__ sorted4)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x)
        sorted4[k] = rec[perm[k]];
}

struct BinWs {
    int32_t *keys;
    float4 *rec;
    char *sort_ws;
    size_t total;
};

int radix_blocks(int64_t N) { return (int)((N + R_TILE - 1) / R_TILE); }

BinWs bin_ws_layout(const hacc_mesh *mesh, void *ws)
{
    BinWs b{};
    char *p = reinterpret_cast<char *>(ws);
    size_t off = 0;
    int64_t N = mesh->N;
    auto take = [&](size_t bytes) {
        char *q = p ? p + off : nullptr;
        off += round_up(bytes, 256);
        return q;
    };
    b.rec = reinterpret_cast<float4 *>(take((size_t)N * sizeof(float4)));
    b.keys = reinterpret_cast<int32_t *>(take((size_t)N * 4));
    b.sort_ws = take(sort_workspace_bytes(N));
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
    if (!mesh || !out || !mesh->vols || mesh->V < 1 || mesh->N < 0 || !status) return HACC_ERR_INVALID;
    if (!out->cell_start || !ws || !aligned16(ws)) return HACC_ERR_INVALID;
    const int64_t N = mesh->N;
    if (N > 0 && (!x || !y || !z || !m || !out->cell_of || !out->perm || !out->sorted4))
        return HACC_ERR_INVALID;
    if (N > 0 && !aligned16(out->sorted4)) return HACC_ERR_INVALID;
    BinWs b = bin_ws_layout(mesh, ws);
    if (ws_bytes < b.total) return HACC_ERR_CAPACITY;
    cudaStream_t st = as_stream(stream);

    if (out->mass_varies) HACC_CUDA_TRY(cudaMemsetAsync(out->mass_varies, 0, sizeof(uint32_t), st));
    if (N == 0) {
        HACC_CUDA_TRY(cudaMemsetAsync(out->cell_start, 0, (size_t)(mesh->n_cells + 1) * 4, st));
        return HACC_OK;
    }
    k_bin_keys<<<grid_for(N, KEY_THREADS), KEY_THREADS, 0, st>>>(mesh->vols, mesh->V, N, x, y, z, dx, dy, dz, m,
                                                                 out->cell_of, b.keys, b.rec, status,
                                                                 out->mass_varies);
    HACC_LAUNCH_CHECK();

    // stable sort of the particle indices by cell: perm, and the sorted keys for cell_start
    const uint32_t maxkey = (uint32_t)(mesh->n_cells - 1);
    int bits = 0;
    while (bits < 32 && (maxkey >> bits) != 0) ++bits;
    const int32_t *skeys = nullptr;
    int rc = sort_index_stable(b.keys, N, bits, out->perm, b.sort_ws, st, &skeys);
    if (rc) return rc;
    k_cell_starts<<<grid_for(mesh->n_cells + 1, 256), 256, 0, st>>>(skeys, N, mesh->n_cells, out->cell_start);
    HACC_LAUNCH_CHECK();
    k_bin_gather<<<grid_for(N, 256), 256, 0, st>>>(N, out->perm, b.rec,
                                                   reinterpret_cast<float4 *>(out->sorted4));
    HACC_LAUNCH_CHECK();
    return HACC_OK;
}
