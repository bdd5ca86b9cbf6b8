// Per-cell neighbour-cell lists, task list and candidate-pair count.
//
// The paper's RCB tree walk builds one interaction list per leaf that every
// particle of the leaf shares (walk minimisation, Sec. III).  Here a cell
// of the chaining mesh plays the leaf: its list holds the neighbour cells
// (with their periodic image) whose boxes come closer than r_c.
#include "hacc_common.cuh"

namespace hacc {
namespace {

__device__ __forceinline__ void cell_coords(int64_t local, int n, int &cx, int &cy, int &cz)
{
    cx = (int)(local % n);
    cy = (int)((local / n) % n);
    cz = (int)(local / ((int64_t)n * n));
}

// Stencil of one reach: the box-distance predicate depends only on the
// offset and the volume, so a block evaluates it once per offset (float64 is
// slow on this GPU) for the volume of its first cell and compacts the
// offsets that pass, in stencil order, into a table; the block's cells of
// that volume then write their entries together, consecutive threads to
// consecutive entries.  A cell of another volume, or a reach beyond the
// table, evaluates the predicate itself (one thread per cell).
constexpr int STENCIL_MAX = 15 * 15 * 15;  // reach up to 7
constexpr int FILL_THREADS = 256;

// Entry of cell (cx, cy, cz) of a volume of n per side for stencil offset
// (dx, dy, dz): the neighbour cell and its periodic image code.
__device__ __forceinline__ void list_entry(const hacc_volume &vol, int cx, int cy, int cz, int dx, int dy, int dz,
                                           int32_t &cell, int8_t &shift)
{
    const int n = vol.n;
    int px = cx + dx, py = cy + dy, pz = cz + dz;
    int sx = 0, sy = 0, sz = 0;
    if (px < 0) { px += n; sx = -1; } else if (px >= n) { px -= n; sx = 1; }
    if (py < 0) { py += n; sy = -1; } else if (py >= n) { py -= n; sy = 1; }
    if (pz < 0) { pz += n; sz = -1; } else if (pz >= n) { pz -= n; sz = 1; }
    cell = (int32_t)(vol.cell_base + ((int64_t)pz * n + py) * n + px);
    shift = (int8_t)((sz + 1) * 9 + (sy + 1) * 3 + (sx + 1));
}

__global__ void __launch_bounds__(FILL_THREADS)
k_lists_fill(const hacc_volume *__restrict__ vols, int V, int64_t n_cells, int64_t n_entries,
             int64_t *__restrict__ nbr_off, int32_t *__restrict__ nbr_cell, int8_t *__restrict__ nbr_shift,
             uint32_t *status)
{
    __shared__ int table[STENCIL_MAX];  // the passing offsets, in stencil order: (dx + R) | (dy + R) << 8 | (dz + R) << 16
    __shared__ int ccoord[FILL_THREADS];  // the block's cells: cx | cy << 10 | cz << 20 (n < 1024 for the table)
    __shared__ int wsum[FILL_THREADS / 32];
    __shared__ int tcount;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t G = (int64_t)gridDim.x * FILL_THREADS;
    for (int64_t base = (int64_t)blockIdx.x * FILL_THREADS; base < n_cells; base += G) {
        __syncthreads();  // the previous round's table is no longer read
        const int vb = find_volume_by_cell(vols, V, base);
        const hacc_volume &volb = vols[vb];
        const int Rb = volb.R, Db = 2 * Rb + 1, D3 = Db * Db * Db;
        const bool tab = D3 <= STENCIL_MAX && volb.n < 1024;
        if (tab) {
            // each thread a contiguous run of offsets: count, block scan, place
            const double w = (double)volb.w, rc = (double)volb.rcut;
            const int per = (D3 + FILL_THREADS - 1) / FILL_THREADS;
            const int o0 = min(D3, (int)threadIdx.x * per), o1 = min(D3, o0 + per);
            auto pass = [&](int o) { return cells_within(o % Db - Rb, (o / Db) % Db - Rb, o / (Db * Db) - Rb, w, rc); };
            int cnt = 0;
            for (int o = o0; o < o1; ++o) cnt += pass(o) ? 1 : 0;
            int inc = cnt;
#pragma unroll
            for (int k = 1; k < 32; k <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, inc, k);
                if (lane >= k) inc += t;
            }
            if (lane == 31) wsum[warp] = inc;
            __syncthreads();
            int before = 0;
            for (int q = 0; q < warp; ++q) before += wsum[q];
            int at = before + inc - cnt;
            for (int o = o0; o < o1; ++o)
                if (pass(o)) table[at++] = (o % Db) | ((o / Db) % Db) << 8 | (o / (Db * Db)) << 16;
            if (threadIdx.x == FILL_THREADS - 1) tcount = at;
        }
        __syncthreads();
        // first entries, and the cells the table does not serve
        const int64_t c = base + threadIdx.x;
        if (c < n_cells) {
            const int v = find_volume_by_cell(vols, V, c);
            const hacc_volume &vol = vols[v];
            const int64_t local = c - vol.cell_base;
            int64_t e = vol.entry_base + local * vol.S;
            nbr_off[c] = e;
            if (c == n_cells - 1) nbr_off[n_cells] = n_entries;
            if (tab && v == vb) {
                int cx, cy, cz;
                cell_coords(local, vol.n, cx, cy, cz);
                ccoord[threadIdx.x] = cx | cy << 10 | cz << 20;
            } else {
                const int64_t e_end = e + vol.S;  // never write past this cell's planned slots
                const int R = vol.R;
                const double w = (double)vol.w, rc = (double)vol.rcut;
                int cx, cy, cz;
                cell_coords(local, vol.n, cx, cy, cz);
                for (int dz = -R; dz <= R; ++dz)
                    for (int dy = -R; dy <= R; ++dy)
                        for (int dx = -R; dx <= R; ++dx) {
                            if (!cells_within(dx, dy, dz, w, rc)) continue;
                            if (e < e_end) list_entry(vol, cx, cy, cz, dx, dy, dz, nbr_cell[e], nbr_shift[e]);
                            ++e;
                        }
                if (e != e_end) atomicOr(status, HACC_STATUS_CAPACITY);
            }
        }
        if (!tab) continue;
        __syncthreads();
        // the block's run of cells of volume vb, entry by entry
        const int S = volb.S;
        const int64_t vend = volb.cell_base + (int64_t)volb.n * volb.n * volb.n;
        const int run = (int)(min(min(base + FILL_THREADS, n_cells), vend) - base);
        const int nt = tcount;
        if (nt != S && threadIdx.x == 0) atomicOr(status, HACC_STATUS_CAPACITY);
        const int64_t e0 = volb.entry_base + (base - volb.cell_base) * S;
        for (int idx = threadIdx.x; idx < run * S; idx += FILL_THREADS) {
            const int cl = idx / S, k = idx - cl * S;
            if (k >= nt) continue;
            const int o = table[k], cc = ccoord[cl];
            list_entry(volb, cc & 1023, (cc >> 10) & 1023, cc >> 20, (o & 255) - Rb, ((o >> 8) & 255) - Rb,
                       (o >> 16) - Rb, nbr_cell[e0 + idx], nbr_shift[e0 + idx]);
        }
    }
}

__global__ void __launch_bounds__(256)
k_task_counts(const int32_t *__restrict__ cell_start, int64_t n_cells, int T, int32_t *__restrict__ nt)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_cells;
         c += (int64_t)gridDim.x * blockDim.x) {
        int cnt = cell_start[c + 1] - cell_start[c];
        nt[c] = (cnt + T - 1) / T;
    }
}

__global__ void __launch_bounds__(256)
k_task_fill(const hacc_volume *__restrict__ vols, int V, const int32_t *__restrict__ cell_start,
            int64_t n_cells, int T, const int32_t *__restrict__ task_off, int64_t cap,
            int4 *__restrict__ tasks)
{
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_cells;
         c += (int64_t)gridDim.x * blockDim.x) {
        int b = cell_start[c], e = cell_start[c + 1];
        int64_t t = task_off[c];
        int v = -1;
        for (int i = b; i < e; i += T, ++t) {
            if (t >= cap) break;
            if (v < 0) v = find_volume_by_cell(vols, V, c);
            tasks[t] = make_int4((int)c, i, (i + T < e) ? i + T : e, v);
        }
    }
}

// Per cell: the particles of its listed neighbour cells (nj, kept for the
// task costs) and, with total, the candidate ordered pairs sum_c n_c nj_c.
__global__ void __launch_bounds__(256)
k_cell_reach(const int32_t *__restrict__ cell_start, int64_t n_cells, const int64_t *__restrict__ nbr_off,
             const int32_t *__restrict__ nbr_cell, int64_t *__restrict__ nj_out, unsigned long long *__restrict__ total)
{
    unsigned long long acc = 0;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_cells;
         c += (int64_t)gridDim.x * blockDim.x) {
        int64_t nj = 0;
        for (int64_t e = nbr_off[c]; e < nbr_off[c + 1]; ++e) {
            int cp = nbr_cell[e];
            nj += cell_start[cp + 1] - cell_start[cp];
        }
        nj_out[c] = nj;
        acc += (unsigned long long)((int64_t)(cell_start[c + 1] - cell_start[c]) * nj);
    }
    if (!total) return;  // a kernel argument: uniform
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(total, acc);
}

__global__ void k_lists_finish(const int32_t *__restrict__ task_off, int64_t n_cells, int64_t cap,
                               int64_t N, int32_t *__restrict__ n_tasks, int64_t *__restrict__ n_pairs,
                               uint32_t *status)
{
    int64_t total = task_off[n_cells];
    if (total > cap) {
        atomicOr(status, HACC_STATUS_CAPACITY);
        total = cap;
    }
    *n_tasks = (int32_t)total;
    if (n_pairs) *n_pairs -= N;  // each particle meets itself once in its own cell
}

// Cost class of each task slot for the heaviest-first order: key =
// 63 - floor(log2(particles x list length)); empty slots past the task count
// get 255 and sort last.
__global__ void __launch_bounds__(256)
k_task_keys(const int4 *__restrict__ tasks, const int32_t *__restrict__ n_tasks, int64_t cap,
            const int64_t *__restrict__ nj_cell, int32_t *__restrict__ keys)
{
    const int64_t nt = *n_tasks;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < cap;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (t >= nt) {
            keys[t] = 255;
            continue;
        }
        const int4 tk = tasks[t];
        const int64_t nj = nj_cell[tk.x];
        const uint64_t cost = (uint64_t)(tk.z - tk.y) * (uint64_t)(nj > 0 ? nj : 1);
        keys[t] = 63 - (63 - __clzll((long long)cost));
    }
}

struct ListWs {
    int64_t *nj;
    int32_t *nt, *task_off, *keys;
    char *scan_ws, *sort_ws;
    size_t total;
};

ListWs lists_layout(const hacc_mesh *mesh, int64_t cap, void *ws)
{
    ListWs L{};
    char *p = reinterpret_cast<char *>(ws);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *q = p ? p + off : nullptr;
        off += round_up(bytes, 256);
        return q;
    };
    L.nj = reinterpret_cast<int64_t *>(take((size_t)mesh->n_cells * 8));
    L.nt = reinterpret_cast<int32_t *>(take((size_t)mesh->n_cells * 4));
    L.task_off = reinterpret_cast<int32_t *>(take((size_t)(mesh->n_cells + 1) * 4));
    L.scan_ws = take(scan_workspace_bytes(mesh->n_cells));
    L.keys = reinterpret_cast<int32_t *>(take((size_t)cap * 4));
    L.sort_ws = take(sort_workspace_bytes(cap));
    L.total = off;
    return L;
}

int grid_cells(int64_t n)
{
    int64_t g = (n + 255) / 256;
    int64_t cap = (int64_t)num_sms() * 16;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace
}  // namespace hacc

using namespace hacc;

extern "C" size_t hacc_lists_workspace_size(const hacc_mesh *mesh)
{
    // sized for the largest task buffer a split of one particle could need
    return mesh ? lists_layout(mesh, hacc_task_capacity(mesh, 1), nullptr).total : 0;
}

extern "C" int hacc_build_lists(const hacc_mesh *mesh, const hacc_binned *binned, const hacc_lists *lists,
                                void *ws, size_t ws_bytes, uint32_t *status, void *stream)
{
    if (!mesh || !binned || !lists || !mesh->vols || !status || !ws) return HACC_ERR_INVALID;
    if (!binned->cell_start || !lists->nbr_off || !lists->n_tasks || lists->split_T < 1 ||
        lists->task_cap < 0)
        return HACC_ERR_INVALID;
    if (mesh->n_entries > 0 && (!lists->nbr_cell || !lists->nbr_shift)) return HACC_ERR_INVALID;
    if (lists->task_cap > 0 && !lists->tasks) return HACC_ERR_INVALID;
    if (!aligned16(lists->tasks)) return HACC_ERR_INVALID;
    if (lists->task_cap > 0 && !lists->task_order) return HACC_ERR_INVALID;
    ListWs L = lists_layout(mesh, lists->task_cap, ws);
    if (ws_bytes < L.total) return HACC_ERR_CAPACITY;
    cudaStream_t st = as_stream(stream);
    const int64_t nc = mesh->n_cells;
    int g = grid_cells(nc);
    k_lists_fill<<<g, FILL_THREADS, 0, st>>>(mesh->vols, mesh->V, nc, mesh->n_entries, lists->nbr_off,
                                    lists->nbr_cell, lists->nbr_shift, status);
    HACC_LAUNCH_CHECK();
    k_task_counts<<<g, 256, 0, st>>>(binned->cell_start, nc, lists->split_T, L.nt);
    HACC_LAUNCH_CHECK();
    int rc = scan_exclusive_i32(L.nt, L.task_off, nc, L.scan_ws, st);
    if (rc) return rc;
    k_task_fill<<<g, 256, 0, st>>>(mesh->vols, mesh->V, binned->cell_start, nc, lists->split_T,
                                   L.task_off, lists->task_cap, reinterpret_cast<int4 *>(lists->tasks));
    HACC_LAUNCH_CHECK();
    if (lists->n_pairs) HACC_CUDA_TRY(cudaMemsetAsync(lists->n_pairs, 0, sizeof(int64_t), st));
    k_cell_reach<<<g, 256, 0, st>>>(binned->cell_start, nc, lists->nbr_off, lists->nbr_cell, L.nj,
                                    reinterpret_cast<unsigned long long *>(lists->n_pairs));
    HACC_LAUNCH_CHECK();
    k_lists_finish<<<1, 1, 0, st>>>(L.task_off, nc, lists->task_cap, mesh->N, lists->n_tasks,
                                    lists->n_pairs, status);
    HACC_LAUNCH_CHECK();
    if (lists->task_cap > 0) {
        int gt = grid_cells(lists->task_cap);
        k_task_keys<<<gt, 256, 0, st>>>(reinterpret_cast<const int4 *>(lists->tasks), lists->n_tasks,
                                        lists->task_cap, L.nj, L.keys);
        HACC_LAUNCH_CHECK();
        rc = sort_index_stable(L.keys, lists->task_cap, 8, lists->task_order, L.sort_ws, st);
        if (rc) return rc;
    }
    return HACC_OK;
}
