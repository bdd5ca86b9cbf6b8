// Shared device/host helpers of the CUDA library (not of the oracle).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hacc_sr.h"

#define HACC_CUDA_TRY(expr)                                   \
    do {                                                      \
        cudaError_t err__ = (expr);                           \
        if (err__ != cudaSuccess) return HACC_ERR_CUDA;       \
    } while (0)

// After every kernel launch: count it, and turn a launch error into a code.
#define HACC_LAUNCH_CHECK()                                   \
    do {                                                      \
        hacc::count_launch();                                 \
        if (cudaPeekAtLastError() != cudaSuccess) {           \
            (void)cudaGetLastError();                         \
            return HACC_ERR_CUDA;                             \
        }                                                     \
    } while (0)

namespace hacc {

// Process-wide count of kernels this library has launched (hacc_kernel_launches).
void count_launch();

static inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

static inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

static inline size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Number of SMs of the current device (queried once per call site).
int num_sms();

// Wrap one float32 coordinate into [0, L): each step one round-to-nearest op.
__device__ __forceinline__ float wrap32(float x, float L)
{
    float q = floorf(__fdiv_rn(x, L));
    float xw = __fsub_rn(x, __fmul_rn(q, L));
    if (xw < 0.0f) xw = __fadd_rn(xw, L);
    if (xw >= L) xw = __fsub_rn(xw, L);
    return xw;
}

// Cell coordinate of a wrapped coordinate.
__device__ __forceinline__ int cell1(float xw, float inv_w, int n)
{
    int c = (int)floorf(__fmul_rn(xw, inv_w));
    c = c > n - 1 ? n - 1 : c;
    return c < 0 ? 0 : c;
}

// Centre of chaining-mesh cell c along one axis, fl32((c + 1/2) w): the
// origin of the cell's offsets.
__host__ __device__ __forceinline__ float cell_centre(int c, float w)
{
#ifdef __CUDA_ARCH__
    return __fmul_rn(__fadd_rn((float)c, 0.5f), w);
#else
    return ((float)c + 0.5f) * w;
#endif
}

// Volume owning global index `key` in a monotone array of begins (binary search).
__device__ __forceinline__ int find_volume_by_particle(const hacc_volume *vols, int V, int64_t i)
{
    int lo = 0, hi = V - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (vols[mid].p_begin <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int find_volume_by_cell(const hacc_volume *vols, int V, int64_t c)
{
    int lo = 0, hi = V - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (vols[mid].cell_base <= c) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Equal-mass detection (hacc_binned::mass_varies): every thread compares the
// masses it writes bitwise with m[0], and one barrier-OR at the end of the
// kernel lets thread 0 of a block that saw a difference set *flag.  Built at
// the top of a kernel whose threads all run to the end (finish() is a block
// barrier when flag is set); m[0] is read only with a flag (then N > 0); the
// host clears *flag beforehand.
struct MassCheck {
    uint32_t *flag;
    uint32_t m0;
    bool differs;
    __device__ __forceinline__ MassCheck(const float *m, uint32_t *f) : flag(f), m0(0u), differs(false)
    {
        if (f) m0 = __float_as_uint(m[0]);
    }
    __device__ __forceinline__ void check(float mi) { differs |= __float_as_uint(mi) != m0; }
    __device__ __forceinline__ void finish()
    {
        if (!flag) return;  // a kernel argument: every thread of the grid takes the same branch
        if (__syncthreads_or(differs) && threadIdx.x == 0) atomicOr(flag, 1u);
    }
};

// Two cells whose integer offsets are (dx, dy, dz) can hold a pair closer
// than rc iff the minimum distance of the boxes is below rc (float64).
__host__ __device__ __forceinline__ bool cells_within(int dx, int dy, int dz, double w, double rc)
{
    int ax = dx < 0 ? -dx : dx, ay = dy < 0 ? -dy : dy, az = dz < 0 ? -dz : dz;
    double gx = ax > 1 ? (double)(ax - 1) : 0.0;
    double gy = ay > 1 ? (double)(ay - 1) : 0.0;
    double gz = az > 1 ? (double)(az - 1) : 0.0;
#ifdef __CUDA_ARCH__
    // same operation order as the host, no contraction into fma
    double g2 = __dadd_rn(__dadd_rn(__dmul_rn(gx, gx), __dmul_rn(gy, gy)), __dmul_rn(gz, gz));
    return __dmul_rn(__dmul_rn(g2, w), w) < __dmul_rn(rc, rc);
#else
    return (gx * gx + gy * gy + gz * gz) * w * w < rc * rc;
#endif
}

// Exclusive scan of int32 counts into int32 offsets, out[n] = total.  Uses
// `ws` of scan_workspace_bytes(n).  Deterministic.
size_t scan_workspace_bytes(int64_t n);
int scan_exclusive_i32(const int32_t *in, int32_t *out, int64_t n, void *ws, cudaStream_t st);

// Stable sort of indices by int32 key (LSD radix, 10-bit digits, only the low
// `bits` bits significant): order[k] = index of the k-th smallest key, ties
// in index order.  ws: sort_workspace_bytes(N).  Deterministic.  If
// sorted_keys is given it receives the keys in sorted order (inside ws).
size_t sort_workspace_bytes(int64_t N);
int sort_index_stable(const int32_t *keys, int64_t N, int bits, int32_t *order, void *ws, cudaStream_t st,
                      const int32_t **sorted_keys = nullptr);

}  // namespace hacc
