// Kick / drift maps of the split-operator step (Eq. 6 of the paper) and the
// float64 global reductions (momentum, Newton-III residual, kinetic and
// short-range potential energy).
#include "hacc_common.cuh"

namespace hacc {
namespace {

__global__ void __launch_bounds__(256)
k_kick(int64_t N, float *__restrict__ vx, float *__restrict__ vy, float *__restrict__ vz,
       const float *__restrict__ ax, const float *__restrict__ ay, const float *__restrict__ az, float dtk,
       float *__restrict__ x, float *__restrict__ y, float *__restrict__ z, double dtd,
       const hacc_volume *__restrict__ vols, int V)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        float nvx = vx[i], nvy = vy[i], nvz = vz[i];
        if (ax) {  // no accelerations: the stream map alone (velocities unchanged)
            nvx = fmaf(dtk, ax[i], nvx);
            nvy = fmaf(dtk, ay[i], nvy);
            nvz = fmaf(dtk, az[i], nvz);
            vx[i] = nvx;
            vy[i] = nvy;
            vz[i] = nvz;
        }
        if (x) {
            double px = (double)x[i] + dtd * (double)nvx;
            double py = (double)y[i] + dtd * (double)nvy;
            double pz = (double)z[i] + dtd * (double)nvz;
            if (vols) {
                const double L = (double)vols[find_volume_by_particle(vols, V, i)].L;
                px -= L * floor(px / L);
                py -= L * floor(py / L);
                pz -= L * floor(pz / L);
            }
            float fx = (float)px, fy = (float)py, fz = (float)pz;
            if (vols) {
                // rounding can land exactly on L; fold it back to 0
                const float Lf = vols[find_volume_by_particle(vols, V, i)].L;
                if (fx >= Lf) fx = 0.0f;
                if (fy >= Lf) fy = 0.0f;
                if (fz >= Lf) fz = 0.0f;
            }
            x[i] = fx;
            y[i] = fy;
            z[i] = fz;
        }
    }
}

constexpr int MOM_THREADS = 256;
constexpr int MOM_BLOCKS = 1024;
constexpr int MOM_N = 9;  // sums: m v (3), m a (3), kinetic, m |a|, potential

__device__ __forceinline__ double block_sum(double v, double *sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < MOM_THREADS / 32; ++w) r += sh[w];
    __syncthreads();
    return r;
}

// Fixed grid and fixed per-thread striding: the summation order depends only
// on N, so the float64 results are reproducible run to run.
__global__ void __launch_bounds__(MOM_THREADS)
k_moments_partial(int64_t N, const float *__restrict__ m, const float *__restrict__ vx, const float *__restrict__ vy,
                  const float *__restrict__ vz, const float *__restrict__ ax, const float *__restrict__ ay,
                  const float *__restrict__ az, const float *__restrict__ phi, double *__restrict__ part)
{
    __shared__ double sh[MOM_THREADS / 32];
    double s[MOM_N] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * MOM_THREADS + threadIdx.x; i < N; i += (int64_t)MOM_BLOCKS * MOM_THREADS) {
        const double mi = m[i];
        const double v0 = vx ? vx[i] : 0.0, v1 = vy ? vy[i] : 0.0, v2 = vz ? vz[i] : 0.0;
        const double a0 = ax ? ax[i] : 0.0, a1 = ay ? ay[i] : 0.0, a2 = az ? az[i] : 0.0;
        s[0] += mi * v0;
        s[1] += mi * v1;
        s[2] += mi * v2;
        s[3] += mi * a0;
        s[4] += mi * a1;
        s[5] += mi * a2;
        s[6] += 0.5 * mi * (v0 * v0 + v1 * v1 + v2 * v2);
        s[7] += mi * sqrt(a0 * a0 + a1 * a1 + a2 * a2);
        s[8] += phi ? 0.5 * mi * (double)phi[i] : 0.0;
    }
#pragma unroll
    for (int k = 0; k < MOM_N; ++k) {
        double r = block_sum(s[k], sh);
        if (threadIdx.x == 0) part[(int64_t)k * MOM_BLOCKS + blockIdx.x] = r;
    }
}

__global__ void __launch_bounds__(MOM_THREADS) k_moments_final(const double *__restrict__ part, double *__restrict__ out)
{
    __shared__ double sh[MOM_THREADS / 32];
    for (int k = 0; k < MOM_N; ++k) {
        double s = 0.0;
        for (int b = threadIdx.x; b < MOM_BLOCKS; b += MOM_THREADS) s += part[(int64_t)k * MOM_BLOCKS + b];
        double r = block_sum(s, sh);
        if (threadIdx.x == 0) out[k] = r;
    }
}

// Stream map on sorted records: o += dt v (one float32 fma per axis); flags a
// record that leaves its cell widened by skin/2.
__global__ void __launch_bounds__(256)
k_drift_offsets(int64_t N, const hacc_volume *__restrict__ vols, int V, const int32_t *__restrict__ perm,
                const float *__restrict__ vx, const float *__restrict__ vy, const float *__restrict__ vz, float dt,
                float half_skin, float4 *__restrict__ sorted4, uint32_t *status)
{
    bool out = false;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        const int i = perm[k];
        const float w = vols[find_volume_by_particle(vols, V, k)].w;
        float4 r = sorted4[k];
        r.x = fmaf(dt, vx[i], r.x);
        r.y = fmaf(dt, vy[i], r.y);
        r.z = fmaf(dt, vz[i], r.z);
        sorted4[k] = r;
        const float lo = -half_skin, hi = w + half_skin;
        out |= !(r.x >= lo && r.x < hi && r.y >= lo && r.y < hi && r.z >= lo && r.z < hi);
    }
    if (__any_sync(0xffffffffu, out) && (threadIdx.x & 31) == 0) atomicOr(status, HACC_STATUS_SKIN);
}

}  // namespace
}  // namespace hacc

using namespace hacc;

extern "C" int hacc_drift_offsets(const hacc_mesh *mesh, const hacc_binned *binned, const float *vx, const float *vy,
                                  const float *vz, float dt, float skin, uint32_t *status, void *stream)
{
    if (!mesh || !mesh->vols || mesh->V < 1 || !binned || !status || !(skin >= 0.0f)) return HACC_ERR_INVALID;
    const int64_t N = mesh->N;
    if (N == 0) return HACC_OK;
    if (!vx || !vy || !vz || !binned->perm || !binned->sorted4 || !aligned16(binned->sorted4))
        return HACC_ERR_INVALID;
    if (binned->cell_origin) return HACC_ERR_INVALID;  // chaining-mesh cells (widths from the volumes)
    int64_t g = (N + 255) / 256;
    if (g > (int64_t)num_sms() * 16) g = (int64_t)num_sms() * 16;
    k_drift_offsets<<<(int)g, 256, 0, as_stream(stream)>>>(N, mesh->vols, mesh->V, binned->perm, vx, vy, vz, dt,
                                                           0.5f * skin, reinterpret_cast<float4 *>(binned->sorted4),
                                                           status);
    HACC_LAUNCH_CHECK();
    return HACC_OK;
}

extern "C" int hacc_kick(const hacc_mesh *mesh, int64_t N, float *vx, float *vy, float *vz, const float *ax,
                         const float *ay, const float *az, float dt_kick, float *x, float *y, float *z,
                         float dt_drift, void *stream)
{
    if (N < 0) return HACC_ERR_INVALID;
    if (N == 0) return HACC_OK;
    if (!vx || !vy || !vz) return HACC_ERR_INVALID;
    if ((ax || ay || az) && !(ax && ay && az)) return HACC_ERR_INVALID;
    if ((x || y || z) && !(x && y && z)) return HACC_ERR_INVALID;
    if (!ax && !x) return HACC_ERR_INVALID;  // neither a kick nor a drift
    if (mesh && (!mesh->vols || mesh->N != N)) return HACC_ERR_INVALID;
    int64_t g = (N + 255) / 256;
    if (g > (int64_t)num_sms() * 16) g = (int64_t)num_sms() * 16;
    k_kick<<<(int)g, 256, 0, as_stream(stream)>>>(N, vx, vy, vz, ax, ay, az, dt_kick, x, y, z, (double)dt_drift,
                                                  mesh ? mesh->vols : nullptr, mesh ? mesh->V : 0);
    HACC_LAUNCH_CHECK();
    return HACC_OK;
}

extern "C" size_t hacc_moments_workspace_size(int64_t N)
{
    (void)N;
    return (size_t)MOM_N * MOM_BLOCKS * sizeof(double);
}

extern "C" int hacc_moments(int64_t N, const float *m, const float *vx, const float *vy, const float *vz,
                            const float *ax, const float *ay, const float *az, const float *phi, double *out,
                            void *ws, size_t ws_bytes, void *stream)
{
    if (N < 0 || !out || !ws) return HACC_ERR_INVALID;
    if (N > 0 && !m) return HACC_ERR_INVALID;
    if (ws_bytes < hacc_moments_workspace_size(N)) return HACC_ERR_CAPACITY;
    cudaStream_t st = as_stream(stream);
    k_moments_partial<<<MOM_BLOCKS, MOM_THREADS, 0, st>>>(N, m, vx, vy, vz, ax, ay, az, phi,
                                                          reinterpret_cast<double *>(ws));
    HACC_LAUNCH_CHECK();
    k_moments_final<<<1, MOM_THREADS, 0, st>>>(reinterpret_cast<const double *>(ws), out);
    HACC_LAUNCH_CHECK();
    return HACC_OK;
}
