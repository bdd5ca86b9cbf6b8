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

// Pass 1: per particle, its cell key, its (offset, mass) record in input
// order, and the cell histogram; with mass_varies, whether any mass differs
// from the first particle's (N > 0).
__global__ void __launch_bounds__(KEY_THREADS)
k_bin_keys(const hacc_volume *__restrict__ vols, int V, int64_t N, const float *__restrict__ x,
           const float *__restrict__ y, const float *__restrict__ z, const float *__restrict__ dx,
           const float *__restrict__ dy, const float *__restrict__ dz, const float *__restrict__ m,
           int32_t *__restrict__ cell_of, int32_t *__restrict__ keys, float4 *__restrict__ rec,
           int32_t *__restrict__ counts, uint32_t *status, uint32_t *mass_varies)
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
        // one atomic per distinct cell of the warp: consecutive particles of a halo share cells
        const unsigned act = __activemask();
        const unsigned peers = __match_any_sync(act, key);
        if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&counts[key], __popc(peers));
    }
    mc.finish();
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
// (warp, item, lane) order is input order; equal digits keep that order.
__global__ void __launch_bounds__(R_THREADS)
k_radix_scatter(const int32_t *__restrict__ keys_in, const int32_t *__restrict__ vals_in, int64_t N,
                int shift, int nblk, const int32_t *__restrict__ offs, int32_t *__restrict__ keys_out,
                int32_t *__restrict__ vals_out)
{
    __shared__ int32_t wcnt[R_WARPS][RADIX + 1];
    __shared__ int32_t base_d[RADIX];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = threadIdx.x; t < R_WARPS * (RADIX + 1); t += R_THREADS) (&wcnt[0][0])[t] = 0;
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
        int cur = wcnt[warp][d];
        __syncwarp();
        if (lane == __ffs(peers) - 1) wcnt[warp][d] = cur + __popc(peers);
        __syncwarp();
        rank[k] = cur + __popc(peers & lt_mask);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RADIX; d += R_THREADS) {
        int run = 0;
#pragma unroll
        for (int w = 0; w < R_WARPS; ++w) {
            int c = wcnt[w][d];
            wcnt[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < R_ITEMS; ++k) {
        int64_t i = p0 + 32 * k;
        if (i < N) {
            int d = (int)(((uint32_t)key[k] >> shift) & (RADIX - 1));
            int64_t pos = (int64_t)base_d[d] + wcnt[warp][d] + rank[k];
            keys_out[pos] = key[k];
            vals_out[pos] = vals_in ? vals_in[i] : (int32_t)i;
        }
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
    int32_t *keys, *counts;
    float4 *rec;
    char *scan_ws, *sort_ws;
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
    b.counts = reinterpret_cast<int32_t *>(take((size_t)mesh->n_cells * 4));
    b.scan_ws = take(scan_workspace_bytes(mesh->n_cells));
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

int sort_index_stable(const int32_t *keys, int64_t N, int bits, int32_t *order, void *ws, cudaStream_t st)
{
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

    HACC_CUDA_TRY(cudaMemsetAsync(b.counts, 0, (size_t)mesh->n_cells * 4, st));
    if (out->mass_varies) HACC_CUDA_TRY(cudaMemsetAsync(out->mass_varies, 0, sizeof(uint32_t), st));
    if (N > 0) {
        k_bin_keys<<<grid_for(N, KEY_THREADS), KEY_THREADS, 0, st>>>(
            mesh->vols, mesh->V, N, x, y, z, dx, dy, dz, m, out->cell_of, b.keys, b.rec, b.counts, status,
            out->mass_varies);
        HACC_LAUNCH_CHECK();
    }
    int rc = scan_exclusive_i32(b.counts, out->cell_start, mesh->n_cells, b.scan_ws, st);
    if (rc) return rc;
    if (N == 0) return HACC_OK;

    // stable sort of the particle indices by cell: perm
    const uint32_t maxkey = (uint32_t)(mesh->n_cells - 1);
    int bits = 0;
    while (bits < 32 && (maxkey >> bits) != 0) ++bits;
    rc = sort_index_stable(b.keys, N, bits, out->perm, b.sort_ws, st);
    if (rc) return rc;
    k_bin_gather<<<grid_for(N, 256), 256, 0, st>>>(N, out->perm, b.rec,
                                                   reinterpret_cast<float4 *>(out->sorted4));
    HACC_LAUNCH_CHECK();
    return HACC_OK;
}
