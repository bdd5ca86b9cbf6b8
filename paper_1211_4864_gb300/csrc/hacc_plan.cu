// Host-side planning of the chaining mesh and workspace queries.
#include <math.h>
#include <string.h>

#include "hacc_common.cuh"

#ifdef HACC_DEBUG_BOUNDS
extern "C" const char *hacc_version(void) { return "hacc_sr 1 sm_103a debug-bounds"; }
#else
extern "C" const char *hacc_version(void) { return "hacc_sr 1 sm_103a"; }
#endif

extern "C" int hacc_get_status(const uint32_t *status, uint32_t *value, void *stream)
{
    if (!status || !value) return HACC_ERR_INVALID;
    cudaStream_t st = hacc::as_stream(stream);
    HACC_CUDA_TRY(cudaMemcpyAsync(value, status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    HACC_CUDA_TRY(cudaStreamSynchronize(st));
    return HACC_OK;
}

extern "C" int hacc_mesh_plan(int32_t V, const float *L, const int64_t *vol_off, float cell_min,
                              float rcut, hacc_volume *table, hacc_mesh *out_mesh)
{
    if (V < 1 || !L || !vol_off || !table || !out_mesh) return HACC_ERR_INVALID;
    if (!(cell_min > 0.0f) || !isfinite(cell_min) || !(rcut > 0.0f) || !isfinite(rcut))
        return HACC_ERR_INVALID;
    if (vol_off[0] != 0) return HACC_ERR_INVALID;
    int64_t cell_base = 0, entry_base = 0;
    for (int32_t v = 0; v < V; ++v) {
        if (vol_off[v + 1] < vol_off[v]) return HACC_ERR_INVALID;
        float Lv = L[v];
        if (!(Lv > 0.0f) || !isfinite(Lv)) return HACC_ERR_INVALID;
        if ((double)Lv < 2.0 * (double)rcut) return HACC_ERR_INVALID;
        double nd = floor((double)Lv / (double)cell_min);
        if (nd < 3.0 || nd > 1290.0) return HACC_ERR_INVALID;  // n^3 must fit int32
        int32_t n = (int32_t)nd;
        float nf = (float)n;
        float w = Lv / nf;
        float inv_w = nf / Lv;
        int32_t R = (int32_t)ceil((double)rcut / (double)w);
        if (n < 2 * R + 1) return HACC_ERR_INVALID;
        int32_t S = 0;
        for (int dz = -R; dz <= R; ++dz)
            for (int dy = -R; dy <= R; ++dy)
                for (int dx = -R; dx <= R; ++dx)
                    if (hacc::cells_within(dx, dy, dz, (double)w, (double)rcut)) ++S;
        hacc_volume &t = table[v];
        memset(&t, 0, sizeof(t));
        t.p_begin = vol_off[v];
        t.p_end = vol_off[v + 1];
        t.cell_base = cell_base;
        t.entry_base = entry_base;
        t.n = n;
        t.R = R;
        t.S = S;
        t.L = Lv;
        t.w = w;
        t.inv_w = inv_w;
        t.rcut = rcut;
        int64_t nc = (int64_t)n * n * n;
        cell_base += nc;
        entry_base += nc * S;
    }
    if (vol_off[V] >= ((int64_t)1 << 31) || cell_base >= ((int64_t)1 << 31) - 1)
        return HACC_ERR_INVALID;
    memset(out_mesh, 0, sizeof(*out_mesh));
    out_mesh->vols = nullptr;
    out_mesh->V = V;
    out_mesh->N = vol_off[V];
    out_mesh->n_cells = cell_base;
    out_mesh->n_entries = entry_base;
    return HACC_OK;
}

extern "C" int64_t hacc_task_capacity(const hacc_mesh *mesh, int32_t split_T)
{
    if (!mesh || split_T < 1) return 0;
    // each non-empty cell yields ceil(count / T) <= count / T + 1 tasks
    int64_t occupied = mesh->n_cells < mesh->N ? mesh->n_cells : mesh->N;
    return mesh->N / split_T + occupied + 1;
}
