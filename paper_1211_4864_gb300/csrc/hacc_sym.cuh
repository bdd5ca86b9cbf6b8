// Device helpers shared by the Newton-III symmetric kernels (force and
// adjoint, two translation units): the empty-lane position, the list entry
// of a cell itself and the image offset of a list entry.
#pragma once

#include "hacc_pairs.cuh"

namespace hacc {
namespace {

// Position of an empty lane: every pair with it fails the cutoff test.
constexpr float FAR = 1.0e6f;

// The list entry of cell (or leaf) c itself, image 13.  A chaining-mesh list
// is symmetric under d -> -d with the cell in the middle; a tree leaf's list
// is sorted by (image code, leaf id) and symmetric too (leaf j with image s
// is listed for i iff i with image -s is listed for j), so its own entry is
// found by bisection and everything after it is the forward half.
__device__ __forceinline__ int64_t self_entry(const KArgs &a, int c, int64_t e0, int64_t e1, const hacc_volume &vol)
{
    if (!a.origin) return e0 + (vol.S - 1) / 2;
    int64_t lo = e0, hi = e1 - 1;
    while (lo < hi) {  // first entry with (code, leaf) >= (13, c)
        const int64_t mid = (lo + hi) >> 1;
        const int code = a.nbr_shift[mid], leaf = a.nbr_cell[mid];
        if (code < 13 || (code == 13 && leaf < c)) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Image offset Delta of one list entry: origin of cell (leaf) cp shifted by
// the image, minus the origin of c; float64, rounded once.
__device__ __forceinline__ void entry_delta(const KArgs &a, const hacc_volume &vol, int cp, int sh, int cx, int cy,
                                            int cz, const float4 &org_i, float &Dx, float &Dy, float &Dz)
{
    const double Ld = (double)vol.L;
    const int sx = sh % 3 - 1, sy = (sh / 3) % 3 - 1, sz = sh / 9 - 1;
    if (a.origin) {
        const float4 org_j = a.origin[cp];
        Dx = (float)((double)org_j.x - (double)org_i.x + sx * Ld);
        Dy = (float)((double)org_j.y - (double)org_i.y + sy * Ld);
        Dz = (float)((double)org_j.z - (double)org_i.z + sz * Ld);
    } else {
        const int n = vol.n;
        const float w = vol.w;
        const int64_t lp = (int64_t)cp - vol.cell_base;
        const int px = (int)(lp % n), py = (int)((lp / n) % n), pz = (int)(lp / ((int64_t)n * n));
        // exact in float64: origins are the float32 cell centres used by the binning
        Dx = (float)((double)cell_centre(px, w) - (double)cell_centre(cx, w) + sx * Ld);
        Dy = (float)((double)cell_centre(py, w) - (double)cell_centre(cy, w) + sy * Ld);
        Dz = (float)((double)cell_centre(pz, w) - (double)cell_centre(cz, w) + sz * Ld);
    }
}

}  // namespace
}  // namespace hacc
