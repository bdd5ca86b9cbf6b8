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
constexpr int MOM_BLOCKS = 4096;  // 1M threads: enough loads in flight for a bandwidth-bound pass
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

// Double-float arithmetic on the float32 pipe (an unevaluated sum hi + lo of
// two float32 values, about 48 significant bits): GB300's float64 pipe is
// narrow, so the per-particle terms and each thread's partial sums are formed
// this way and only the per-thread totals are reduced in float64.
// Knuth's TwoSum: s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// TwoProduct with one fma: p + e == a * b exactly.
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e)
{
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

struct DF {
    float hi = 0.0f, lo = 0.0f;
    // += (xh + xl): TwoSum of the leading parts, the trailing parts added to
    // the error, then renormalised (Dekker's Fast2Sum)
    __device__ __forceinline__ void add(float xh, float xl)
    {
        float s, e;
        two_sum(hi, xh, s, e);
        e = __fadd_rn(e, __fadd_rn(lo, xl));
        hi = __fadd_rn(s, e);
        lo = __fsub_rn(e, __fsub_rn(hi, s));
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// (h + l) * b for a double-float h + l and a float32 b
__device__ __forceinline__ void df_mul(float h, float l, float b, float &ph, float &pl)
{
    float e;
    two_prod(h, b, ph, e);
    pl = __fmaf_rn(l, b, e);
}

// x0^2 + x1^2 + x2^2 as a double-float
__device__ __forceinline__ void df_norm2(float x0, float x1, float x2, float &h, float &l)
{
    float p0, e0, p1, e1, p2, e2, s, e;
    two_prod(x0, x0, p0, e0);
    two_prod(x1, x1, p1, e1);
    two_prod(x2, x2, p2, e2);
    two_sum(p0, p1, s, e);
    float t, f;
    two_sum(s, p2, t, f);
    const float lo = __fadd_rn(__fadd_rn(e, f), __fadd_rn(__fadd_rn(e0, e1), e2));
    h = __fadd_rn(t, lo);
    l = __fsub_rn(lo, __fsub_rn(h, t));
}

// sqrt(h + l) as a double-float: the float32 root and one Newton correction
// from the exact residual (h - r^2 formed with an fma)
__device__ __forceinline__ void df_sqrt(float h, float l, float &rh, float &rl)
{
    if (!(h > 0.0f)) {
        rh = sqrtf(h);
        rl = 0.0f;
        return;
    }
    const float r = sqrtf(h);
    const float res = __fadd_rn(__fmaf_rn(-r, r, h), l);
    rh = r;
    rl = res / __fmul_rn(2.0f, r);
}

// Four consecutive values p[i..i+3] (i a multiple of 4): one 16-byte load when
// p is 16-byte aligned, four 4-byte loads otherwise.
__device__ __forceinline__ float4 load4(const float *__restrict__ p, int64_t i, bool aligned)
{
    if (aligned) return *reinterpret_cast<const float4 *>(p + i);
    return make_float4(p[i], p[i + 1], p[i + 2], p[i + 3]);
}

__device__ __forceinline__ float lane4(const float4 &v, int k)
{
    return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w;
}

// One particle's terms added to the thread's double-float sums.
__device__ __forceinline__ void moment_terms(DF (&s)[MOM_N], float mi, bool has_v, float v0, float v1, float v2,
                                             bool has_a, float a0, float a1, float a2, bool has_phi, float ph)
{
    float p, e, h, l;
    if (has_v) {
        two_prod(mi, v0, p, e);
        s[0].add(p, e);
        two_prod(mi, v1, p, e);
        s[1].add(p, e);
        two_prod(mi, v2, p, e);
        s[2].add(p, e);
        df_norm2(v0, v1, v2, h, l);
        df_mul(h, l, mi, p, e);
        s[6].add(__fmul_rn(0.5f, p), __fmul_rn(0.5f, e));  // halving is exact
    }
    if (has_a) {
        two_prod(mi, a0, p, e);
        s[3].add(p, e);
        two_prod(mi, a1, p, e);
        s[4].add(p, e);
        two_prod(mi, a2, p, e);
        s[5].add(p, e);
        float rh, rl;
        df_norm2(a0, a1, a2, h, l);
        df_sqrt(h, l, rh, rl);
        df_mul(rh, rl, mi, p, e);
        s[7].add(p, e);
    }
    if (has_phi) {
        two_prod(mi, ph, p, e);
        s[8].add(__fmul_rn(0.5f, p), __fmul_rn(0.5f, e));
    }
}

// Fixed grid and fixed per-thread striding: the summation order depends only
// on N, so the float64 results are reproducible run to run.  Thread t takes
// the groups of four consecutive particles t, t + T, t + 2T, ... (T threads;
// each group's values by 16-byte loads where an array is aligned, all of a
// group's loads issued before its arithmetic) and then particle
// 4 floor(N / 4) + t of the last, partial group.  Per particle and per thread
// in double-float (above), across threads and blocks in float64.
__global__ void __launch_bounds__(MOM_THREADS)
k_moments_partial(int64_t N, const float *__restrict__ m, const float *__restrict__ vx, const float *__restrict__ vy,
                  const float *__restrict__ vz, const float *__restrict__ ax, const float *__restrict__ ay,
                  const float *__restrict__ az, const float *__restrict__ phi, double *__restrict__ part)
{
    __shared__ double sh[MOM_THREADS / 32];
    DF s[MOM_N];
    const bool hv = vx != nullptr, ha = ax != nullptr, hp = phi != nullptr;
    auto al = [](const float *p) { return p && (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    const bool am = al(m), avx = al(vx), avy = al(vy), avz = al(vz), aax = al(ax), aay = al(ay), aaz = al(az),
               aph = al(phi);
    const int64_t t0 = (int64_t)blockIdx.x * MOM_THREADS + threadIdx.x;
    const int64_t groups = N / 4;
    for (int64_t g = t0; g < groups; g += (int64_t)MOM_BLOCKS * MOM_THREADS) {
        const int64_t i = 4 * g;
        const float4 m4 = load4(m, i, am);
        float4 v0, v1, v2, a0, a1, a2, p4;
        if (hv) {
            v0 = load4(vx, i, avx);
            v1 = load4(vy, i, avy);
            v2 = load4(vz, i, avz);
        }
        if (ha) {
            a0 = load4(ax, i, aax);
            a1 = load4(ay, i, aay);
            a2 = load4(az, i, aaz);
        }
        if (hp) p4 = load4(phi, i, aph);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            moment_terms(s, lane4(m4, k), hv, hv ? lane4(v0, k) : 0.f, hv ? lane4(v1, k) : 0.f,
                         hv ? lane4(v2, k) : 0.f, ha, ha ? lane4(a0, k) : 0.f, ha ? lane4(a1, k) : 0.f,
                         ha ? lane4(a2, k) : 0.f, hp, hp ? lane4(p4, k) : 0.f);
    }
    const int64_t i = 4 * groups + t0;
    if (i < N)
        moment_terms(s, m[i], hv, hv ? vx[i] : 0.f, hv ? vy[i] : 0.f, hv ? vz[i] : 0.f, ha, ha ? ax[i] : 0.f,
                     ha ? ay[i] : 0.f, ha ? az[i] : 0.f, hp, hp ? phi[i] : 0.f);
#pragma unroll
    for (int k = 0; k < MOM_N; ++k) {
        double r = block_sum(s[k].value(), sh);
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
        const float hi = __fadd_rn(0.5f * w, half_skin), lo = -hi;
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
    if ((vx || vy || vz) && !(vx && vy && vz)) return HACC_ERR_INVALID;
    if ((ax || ay || az) && !(ax && ay && az)) return HACC_ERR_INVALID;
    if (ws_bytes < hacc_moments_workspace_size(N)) return HACC_ERR_CAPACITY;
    cudaStream_t st = as_stream(stream);
    k_moments_partial<<<MOM_BLOCKS, MOM_THREADS, 0, st>>>(N, m, vx, vy, vz, ax, ay, az, phi,
                                                          reinterpret_cast<double *>(ws));
    HACC_LAUNCH_CHECK();
    k_moments_final<<<1, MOM_THREADS, 0, st>>>(reinterpret_cast<const double *>(ws), out);
    HACC_LAUNCH_CHECK();
    return HACC_OK;
}
