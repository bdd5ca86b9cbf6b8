// Short-range pair force (Eq. 4 of the paper) and its adjoint.
//
// Work decomposition.  A task is a chunk of at most split_T particles of one
// mesh cell (the "i" particles); one warp owns one task at a time, one i per
// lane, and walks the cell's neighbour list.  Every neighbour cell's particle
// range (the "j" particles, contiguous in the sorted array) is staged into a
// per-warp ring of shared-memory tiles by the tensor memory accelerator
// (cp.async.bulk, completion on an mbarrier), and each staged j is broadcast to
// all 32 lanes by a 16-byte shared load.  Warps take tasks from an atomic
// counter (a persistent, work-stealing grid), so the very uneven lists of
// clustered particles balance themselves.
//
// Arithmetic per pair (float32, cutoff as a select, as in the paper's
// branch-free kernel, Sec. IV-B):
//   d  = o_j - (o_i - Delta)            cell-relative offsets, Delta = image origin difference
//   se = eps + d.d                      (three fma)
//   t  = rsqrt(se)
//   f  = t^2 t - poly~(se)              poly~(se) = poly(se - eps), coefficients shifted on the host
//   f  = se < r_c^2 + eps ? f : 0
//   a += m_j f d
// The accumulator is float32 within a tile and compensated (TwoSum into a
// hi/lo pair) across tiles.
#include <math.h>

#include "hacc_common.cuh"

namespace hacc {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr long long WAIT_LIMIT_CYCLES = 2000000000LL;  // ~1 s at 2 GHz

enum Mode { FORCE = 0, ADJOINT = 1 };

struct PairConsts {
    float eps;      // softening
    float rc2e;     // r_c^2 + eps (cut on se = s + eps)
    float nc[6];    // -(coefficients of poly~ in se), for f
    float kp[5];    // -2 (k+1) c~_{k+1}: Horner coefficients of -2 poly~'(se)
};

struct KArgs {
    const hacc_volume *vols;
    const int32_t *cell_start;
    const int64_t *nbr_off;
    const int32_t *nbr_cell;
    const int8_t *nbr_shift;
    const int4 *tasks;
    const int32_t *n_tasks;
    const float4 *pos;   // sorted (ox, oy, oz, m)
    const float4 *lam;   // sorted (lx, ly, lz, 0), adjoint only
    const int32_t *perm;
    float *out_x, *out_y, *out_z, *out_m;
    int32_t *counter;
    uint32_t *status;
    PairConsts k;
};

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ uint32_t mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok;
}

// Lane 0 only: expect `bytes` on the barrier and start the bulk copies.
__device__ __forceinline__ void tma_issue(uint32_t bar, uint32_t dst, const void *src, uint32_t bytes,
                                          uint32_t dst2, const void *src2)
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    uint32_t total = src2 ? 2 * bytes : bytes;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(total) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
    if (src2)
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                dst2),
            "l"(src2), "r"(bytes), "r"(bar)
            : "memory");
}

// All lanes wait for a barrier phase; false (uniformly) if it ran out of time.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity)
{
    long long t0 = clock64();
    while (true) {
        uint32_t ok = mbar_try_wait(bar, parity);
        if (__all_sync(FULL, ok)) return true;
        int late = (clock64() - t0) > WAIT_LIMIT_CYCLES;
        if (__shfl_sync(FULL, late, 0)) return false;
    }
}

// s = a + b exactly as s + err (Knuth's TwoSum), err added to the low word.
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float b)
{
    float s = __fadd_rn(hi, b);
    float bp = __fsub_rn(s, hi);
    float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(b, bp));
    hi = s;
    lo = __fadd_rn(lo, err);
}

// Next non-empty tile of the group at or after (k, off); entry counts live in
// lane k's `cnt`.  Warp-uniform.
template <int JT>
__device__ __forceinline__ bool next_tile(int ng, int cnt, int &k, int &off, int &n)
{
    while (k < ng) {
        int c = __shfl_sync(FULL, cnt, k);
        if (off < c) {
            n = min(JT, c - off);
            return true;
        }
        ++k;
        off = 0;
    }
    return false;
}

template <int MODE>
struct Acc;

template <>
struct Acc<FORCE> {
    float ax = 0.f, ay = 0.f, az = 0.f;
    float hx = 0.f, hy = 0.f, hz = 0.f, lx = 0.f, ly = 0.f, lz = 0.f;
    __device__ __forceinline__ void fold()
    {
        two_sum_acc(hx, lx, ax);
        two_sum_acc(hy, ly, ay);
        two_sum_acc(hz, lz, az);
        ax = ay = az = 0.f;
    }
};

template <>
struct Acc<ADJOINT> {
    float u[3] = {0.f, 0.f, 0.f}, x[3] = {0.f, 0.f, 0.f}, v = 0.f, g = 0.f;
    float hu[3] = {0.f, 0.f, 0.f}, lu[3] = {0.f, 0.f, 0.f};
    float hx[3] = {0.f, 0.f, 0.f}, lx[3] = {0.f, 0.f, 0.f};
    float hv = 0.f, lv = 0.f, hg = 0.f, lg = 0.f;
    __device__ __forceinline__ void fold()
    {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            two_sum_acc(hu[a], lu[a], u[a]);
            two_sum_acc(hx[a], lx[a], x[a]);
            u[a] = 0.f;
            x[a] = 0.f;
        }
        two_sum_acc(hv, lv, v);
        two_sum_acc(hg, lg, g);
        v = 0.f;
        g = 0.f;
    }
};

// Forward pair loop over one staged tile.
__device__ __forceinline__ void tile_force(const float4 *__restrict__ tj, int n, float oxp, float oyp,
                                           float ozp, const PairConsts &K, Acc<FORCE> &A)
{
#pragma unroll 4
    for (int j = 0; j < n; ++j) {
        float4 p = tj[j];
        float dx = p.x - oxp, dy = p.y - oyp, dz = p.z - ozp;
        float se = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, K.eps)));
        float t = rsqrtf(se);
        float t2 = t * t;
        float q = fmaf(fmaf(fmaf(fmaf(fmaf(K.nc[5], se, K.nc[4]), se, K.nc[3]), se, K.nc[2]), se, K.nc[1]), se,
                       K.nc[0]);
        float f = fmaf(t2, t, q);
        f = se < K.rc2e ? f : 0.0f;
        float g = f * p.w;
        A.ax = fmaf(g, dx, A.ax);
        A.ay = fmaf(g, dy, A.ay);
        A.az = fmaf(g, dz, A.az);
    }
}

// Adjoint pair loop over one staged tile.  Per pair, with f = f_SR(s) and
// fp2 = 2 f_SR'(s):  U += f lam_j ;  V += m_j f ;
// X += fp2 (m_i (d.lam_j) - m_j (d.lam_i)) d ;  G += f (d.lam_j).
// Then dL/dx_i = m_i U - lam_i V + X and dL/dm_i = -G.
__device__ __forceinline__ void tile_adjoint(const float4 *__restrict__ tj, const float4 *__restrict__ tl, int n,
                                             float oxp, float oyp, float ozp, float mi, float lix, float liy,
                                             float liz, const PairConsts &K, Acc<ADJOINT> &A)
{
#pragma unroll 2
    for (int j = 0; j < n; ++j) {
        float4 p = tj[j];
        float4 l = tl[j];
        float dx = p.x - oxp, dy = p.y - oyp, dz = p.z - ozp;
        float se = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, K.eps)));
        float t = rsqrtf(se);
        float t2 = t * t;
        float t3 = t2 * t;
        float q = fmaf(fmaf(fmaf(fmaf(fmaf(K.nc[5], se, K.nc[4]), se, K.nc[3]), se, K.nc[2]), se, K.nc[1]), se,
                       K.nc[0]);
        float f = t3 + q;
        float qp = fmaf(fmaf(fmaf(fmaf(K.kp[4], se, K.kp[3]), se, K.kp[2]), se, K.kp[1]), se, K.kp[0]);
        float fp2 = fmaf(-3.0f, t3 * t2, qp);
        bool in = se < K.rc2e;
        f = in ? f : 0.0f;
        fp2 = in ? fp2 : 0.0f;
        float dlj = fmaf(dz, l.z, fmaf(dy, l.y, dx * l.x));
        float dli = fmaf(dz, liz, fmaf(dy, liy, dx * lix));
        A.u[0] = fmaf(f, l.x, A.u[0]);
        A.u[1] = fmaf(f, l.y, A.u[1]);
        A.u[2] = fmaf(f, l.z, A.u[2]);
        A.v = fmaf(p.w, f, A.v);
        float r = fp2 * fmaf(mi, dlj, -(p.w * dli));
        A.x[0] = fmaf(r, dx, A.x[0]);
        A.x[1] = fmaf(r, dy, A.x[1]);
        A.x[2] = fmaf(r, dz, A.x[2]);
        A.g = fmaf(f, dlj, A.g);
    }
}

// Shared memory of one warp: STAGES tiles (two arrays in the adjoint) and
// STAGES mbarriers, padded so that every warp's tiles start 128-B aligned.
__host__ __device__ constexpr int warp_smem_bytes(int mode, int jt, int stages)
{
    return ((stages * (mode == ADJOINT ? 2 : 1) * jt * 16 + stages * 8) + 127) / 128 * 128;
}

template <int MODE, int JT, int STAGES>
__global__ void __launch_bounds__(512) k_pairs(const KArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int NBUF = MODE == ADJOINT ? 2 : 1;
    constexpr int WARP_BYTES = warp_smem_bytes(MODE, JT, STAGES);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char *wbase = smem + (size_t)warp * WARP_BYTES;
    float4 *tiles = reinterpret_cast<float4 *>(wbase);
    uint64_t *bars = reinterpret_cast<uint64_t *>(wbase + STAGES * NBUF * JT * 16);

    if (lane == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(smem_addr(&bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncwarp();

    const PairConsts &K = a.k;
    const int ntask = *a.n_tasks;
    uint32_t issued = 0, consumed = 0;  // lifetime tile counters of this warp's ring

    while (true) {
        int t = 0;
        if (lane == 0) t = atomicAdd(a.counter, 1);
        t = __shfl_sync(FULL, t, 0);
        if (t >= ntask) break;
        const int4 task = a.tasks[t];
        const int c = task.x, ib = task.y, ie = task.z;
        const hacc_volume &vol = a.vols[task.w];
        const int n = vol.n;
        const float w = vol.w;
        const double Ld = (double)vol.L;
        const int64_t lc = (int64_t)c - vol.cell_base;
        const int cx = (int)(lc % n), cy = (int)((lc / n) % n), cz = (int)(lc / ((int64_t)n * n));

        const int i = ib + lane;
        const bool active = i < ie;
        float4 oi = active ? a.pos[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        float4 li = make_float4(0.f, 0.f, 0.f, 0.f);
        if (MODE == ADJOINT && active) li = a.lam[i];
        Acc<MODE> A;

        const int64_t e0 = a.nbr_off[c], e1 = a.nbr_off[c + 1];
        bool failed = false;
        for (int64_t g0 = e0; g0 < e1 && !failed; g0 += 32) {
            const int ng = (int)min((int64_t)32, e1 - g0);
            // lane l describes entry g0 + l: its j range and image offset Delta
            int jb = 0, cnt = 0;
            float Dx = 0.f, Dy = 0.f, Dz = 0.f;
            if (lane < ng) {
                const int cp = a.nbr_cell[g0 + lane];
                const int sh = a.nbr_shift[g0 + lane];
                jb = a.cell_start[cp];
                cnt = a.cell_start[cp + 1] - jb;
                const int64_t lp = (int64_t)cp - vol.cell_base;
                const int px = (int)(lp % n), py = (int)((lp / n) % n), pz = (int)(lp / ((int64_t)n * n));
                const int sx = sh % 3 - 1, sy = (sh / 3) % 3 - 1, sz = sh / 9 - 1;
                // exact in float64: origins are the float32 products used by the binning
                Dx = (float)((double)__fmul_rn((float)px, w) - (double)__fmul_rn((float)cx, w) + sx * Ld);
                Dy = (float)((double)__fmul_rn((float)py, w) - (double)__fmul_rn((float)cy, w) + sy * Ld);
                Dz = (float)((double)__fmul_rn((float)pz, w) - (double)__fmul_rn((float)cz, w) + sz * Ld);
            }
            int pk = 0, poff = 0, pn = 0;  // producer cursor
            int ck = 0, coff = 0, cn = 0;  // consumer cursor
            // prologue: fill the ring
            for (int s = 0; s < STAGES; ++s) {
                if (!next_tile<JT>(ng, cnt, pk, poff, pn)) break;
                const int pjb = __shfl_sync(FULL, jb, pk);
                if (lane == 0) {
                    const uint32_t st = issued % STAGES;
                    tma_issue(smem_addr(&bars[st]), smem_addr(tiles + (size_t)st * NBUF * JT), a.pos + pjb + poff,
                              pn * 16, smem_addr(tiles + (size_t)st * NBUF * JT + JT),
                              MODE == ADJOINT ? (const void *)(a.lam + pjb + poff) : nullptr);
                }
                poff += pn;
                ++issued;
            }
            int cur = -1;
            float oxp = 0.f, oyp = 0.f, ozp = 0.f;
            while (consumed < issued) {
                next_tile<JT>(ng, cnt, ck, coff, cn);
                const uint32_t st = consumed % STAGES;
                if (!warp_wait(smem_addr(&bars[st]), (consumed / STAGES) & 1u)) {
                    failed = true;
                    break;
                }
                if (ck != cur) {
                    cur = ck;
                    oxp = oi.x - __shfl_sync(FULL, Dx, ck);
                    oyp = oi.y - __shfl_sync(FULL, Dy, ck);
                    ozp = oi.z - __shfl_sync(FULL, Dz, ck);
                }
                const float4 *tj = tiles + (size_t)st * NBUF * JT;
                if constexpr (MODE == FORCE)
                    tile_force(tj, cn, oxp, oyp, ozp, K, A);
                else
                    tile_adjoint(tj, tj + JT, cn, oxp, oyp, ozp, oi.w, li.x, li.y, li.z, K, A);
                A.fold();
                coff += cn;
                ++consumed;
                __syncwarp();
                if (next_tile<JT>(ng, cnt, pk, poff, pn)) {
                    const int pjb = __shfl_sync(FULL, jb, pk);
                    if (lane == 0) {
                        const uint32_t s2 = issued % STAGES;
                        tma_issue(smem_addr(&bars[s2]), smem_addr(tiles + (size_t)s2 * NBUF * JT),
                                  a.pos + pjb + poff, pn * 16, smem_addr(tiles + (size_t)s2 * NBUF * JT + JT),
                                  MODE == ADJOINT ? (const void *)(a.lam + pjb + poff) : nullptr);
                    }
                    poff += pn;
                    ++issued;
                }
            }
        }
        if (failed) {
            if (lane == 0) atomicOr(a.status, HACC_STATUS_TIMEOUT);
            // let the copies still in flight land (bounded) before leaving
            while (consumed < issued) {
                const uint32_t st = consumed % STAGES;
                warp_wait(smem_addr(&bars[st]), (consumed / STAGES) & 1u);
                ++consumed;
            }
            return;
        }
        if (active) {
            const int o = a.perm[i];
            if constexpr (MODE == FORCE) {
                a.out_x[o] = A.hx + A.lx;
                a.out_y[o] = A.hy + A.ly;
                a.out_z[o] = A.hz + A.lz;
            } else {
                const Acc<ADJOINT> &J = A;
                const float U0 = J.hu[0] + J.lu[0], U1 = J.hu[1] + J.lu[1], U2 = J.hu[2] + J.lu[2];
                const float X0 = J.hx[0] + J.lx[0], X1 = J.hx[1] + J.lx[1], X2 = J.hx[2] + J.lx[2];
                const float Vs = J.hv + J.lv;
                a.out_x[o] = fmaf(oi.w, U0, fmaf(-li.x, Vs, X0));
                a.out_y[o] = fmaf(oi.w, U1, fmaf(-li.y, Vs, X1));
                a.out_z[o] = fmaf(oi.w, U2, fmaf(-li.z, Vs, X2));
                if (a.out_m) a.out_m[o] = -(J.hg + J.lg);
            }
        }
    }
}

// Sorted cotangent records (lx, ly, lz, 0) for the adjoint.
__global__ void __launch_bounds__(256)
k_gather_lam(int64_t N, const int32_t *__restrict__ perm, const float *__restrict__ gx,
             const float *__restrict__ gy, const float *__restrict__ gz, float4 *__restrict__ lam)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x) {
        int i = perm[k];
        lam[k] = make_float4(gx[i], gy[i], gz[i], 0.f);
    }
}

// poly~(se) = poly(se - eps): c~_m = sum_{k>=m} c_k C(k, m) (-eps)^(k-m), in float64.
void pair_consts(const hacc_sr_params *p, PairConsts &K)
{
    double c[6], ct[6];
    for (int k = 0; k < 6; ++k) c[k] = (double)p->c[k];
    const double e = -(double)p->eps;
    const double binom[6][6] = {{1, 0, 0, 0, 0, 0},  {1, 1, 0, 0, 0, 0},   {1, 2, 1, 0, 0, 0},
                                {1, 3, 3, 1, 0, 0},  {1, 4, 6, 4, 1, 0},   {1, 5, 10, 10, 5, 1}};
    for (int mdeg = 0; mdeg < 6; ++mdeg) {
        double s = 0.0;
        for (int k = mdeg; k < 6; ++k) s += c[k] * binom[k][mdeg] * pow(e, (double)(k - mdeg));
        ct[mdeg] = s;
    }
    K.eps = p->eps;
    K.rc2e = (float)((double)p->rcut * (double)p->rcut + (double)p->eps);
    for (int k = 0; k < 6; ++k) K.nc[k] = (float)(-ct[k]);
    for (int k = 0; k < 5; ++k) K.kp[k] = (float)(-2.0 * (k + 1) * ct[k + 1]);
}

struct ForceWs {
    int32_t *counter;
    float4 *lam;
    size_t total;
};

ForceWs force_layout(const hacc_mesh *mesh, void *ws)
{
    ForceWs F{};
    char *p = reinterpret_cast<char *>(ws);
    F.counter = reinterpret_cast<int32_t *>(p);
    F.lam = reinterpret_cast<float4 *>(p ? p + 256 : nullptr);
    F.total = 256 + round_up((size_t)mesh->N * 16, 256);
    return F;
}

template <int MODE, int JT, int STAGES>
int launch_t(const KArgs &a, int warps, int ctas_per_sm, cudaStream_t st)
{
    const size_t smem = (size_t)warps * warp_smem_bytes(MODE, JT, STAGES);
    auto kern = k_pairs<MODE, JT, STAGES>;
    if (smem > 48 * 1024)
        HACC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    HACC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, warps * 32, smem));
    if (occ < 1) return HACC_ERR_INVALID;
    int per_sm = ctas_per_sm < occ ? ctas_per_sm : occ;
    kern<<<num_sms() * per_sm, warps * 32, smem, st>>>(a);
    HACC_LAUNCH_CHECK();
    return HACC_OK;
}

template <int MODE>
int launch_mode(const KArgs &a, const hacc_launch &L, cudaStream_t st)
{
    const int wp = L.warps_per_cta, cps = L.ctas_per_sm;
#define HACC_CASE(JT, S) \
    if (L.jtile == JT && L.stages == S) return launch_t<MODE, JT, S>(a, wp, cps, st);
    HACC_CASE(32, 2) HACC_CASE(32, 4) HACC_CASE(64, 2) HACC_CASE(64, 3) HACC_CASE(64, 4)
    HACC_CASE(128, 2) HACC_CASE(128, 3) HACC_CASE(128, 4) HACC_CASE(256, 2)
#undef HACC_CASE
    return HACC_ERR_INVALID;
}

hacc_launch default_launch(int mode)
{
    hacc_launch L;
    L.warps_per_cta = 8;
    L.ctas_per_sm = 2;
    L.jtile = mode == FORCE ? 64 : 64;
    L.stages = 4;
    return L;
}

int check_common(const hacc_mesh *mesh, const hacc_binned *b, const hacc_lists *l, const hacc_sr_params *p,
                 const hacc_launch *launch, void *ws, size_t ws_bytes, uint32_t *status)
{
    if (!mesh || !b || !l || !p || !mesh->vols || !status || !ws || !aligned16(ws)) return HACC_ERR_INVALID;
    if (!(p->eps > 0.0f) || !isfinite(p->eps) || !(p->rcut > 0.0f) || !isfinite(p->rcut)) return HACC_ERR_INVALID;
    for (int k = 0; k < 6; ++k)
        if (!isfinite(p->c[k])) return HACC_ERR_INVALID;
    if (!b->cell_start || !b->perm || !b->sorted4 || !aligned16(b->sorted4)) return HACC_ERR_INVALID;
    if (!l->nbr_off || !l->n_tasks || (mesh->n_entries > 0 && (!l->nbr_cell || !l->nbr_shift)))
        return HACC_ERR_INVALID;
    if (!l->tasks || !aligned16(l->tasks)) return HACC_ERR_INVALID;
    if (l->split_T < 1 || l->split_T > 32) return HACC_ERR_INVALID;  // one i particle per lane
    if (launch) {
        if (launch->warps_per_cta < 1 || launch->warps_per_cta > 16 || launch->ctas_per_sm < 1 ||
            launch->ctas_per_sm > 8)
            return HACC_ERR_INVALID;
    }
    if (ws_bytes < force_layout(mesh, nullptr).total) return HACC_ERR_CAPACITY;
    return HACC_OK;
}

}  // namespace
}  // namespace hacc

using namespace hacc;

extern "C" size_t hacc_force_workspace_size(const hacc_mesh *mesh)
{
    return mesh ? force_layout(mesh, nullptr).total : 0;
}

extern "C" int hacc_sr_force(const hacc_mesh *mesh, const hacc_binned *binned, const hacc_lists *lists,
                             const hacc_sr_params *p, float *ax, float *ay, float *az, const hacc_launch *launch,
                             void *ws, size_t ws_bytes, uint32_t *status, void *stream)
{
    int rc = check_common(mesh, binned, lists, p, launch, ws, ws_bytes, status);
    if (rc) return rc;
    if (mesh->N > 0 && (!ax || !ay || !az)) return HACC_ERR_INVALID;
    if (mesh->N == 0) return HACC_OK;
    cudaStream_t st = as_stream(stream);
    ForceWs F = force_layout(mesh, ws);
    KArgs a{};
    a.vols = mesh->vols;
    a.cell_start = binned->cell_start;
    a.nbr_off = lists->nbr_off;
    a.nbr_cell = lists->nbr_cell;
    a.nbr_shift = lists->nbr_shift;
    a.tasks = reinterpret_cast<const int4 *>(lists->tasks);
    a.n_tasks = lists->n_tasks;
    a.pos = reinterpret_cast<const float4 *>(binned->sorted4);
    a.lam = nullptr;
    a.perm = binned->perm;
    a.out_x = ax;
    a.out_y = ay;
    a.out_z = az;
    a.out_m = nullptr;
    a.counter = F.counter;
    a.status = status;
    pair_consts(p, a.k);
    HACC_CUDA_TRY(cudaMemsetAsync(F.counter, 0, sizeof(int32_t), st));
    hacc_launch L = launch ? *launch : default_launch(FORCE);
    return launch_mode<FORCE>(a, L, st);
}

extern "C" int hacc_sr_force_adjoint(const hacc_mesh *mesh, const hacc_binned *binned, const hacc_lists *lists,
                                     const hacc_sr_params *p, const float *gax, const float *gay,
                                     const float *gaz, float *gx, float *gy, float *gz, float *gm,
                                     const hacc_launch *launch, void *ws, size_t ws_bytes, uint32_t *status,
                                     void *stream)
{
    int rc = check_common(mesh, binned, lists, p, launch, ws, ws_bytes, status);
    if (rc) return rc;
    if (mesh->N > 0 && (!gax || !gay || !gaz || !gx || !gy || !gz)) return HACC_ERR_INVALID;
    if (mesh->N == 0) return HACC_OK;
    cudaStream_t st = as_stream(stream);
    ForceWs F = force_layout(mesh, ws);
    int g = (int)((mesh->N + 255) / 256);
    if (g > num_sms() * 16) g = num_sms() * 16;
    k_gather_lam<<<g, 256, 0, st>>>(mesh->N, binned->perm, gax, gay, gaz, F.lam);
    HACC_LAUNCH_CHECK();
    KArgs a{};
    a.vols = mesh->vols;
    a.cell_start = binned->cell_start;
    a.nbr_off = lists->nbr_off;
    a.nbr_cell = lists->nbr_cell;
    a.nbr_shift = lists->nbr_shift;
    a.tasks = reinterpret_cast<const int4 *>(lists->tasks);
    a.n_tasks = lists->n_tasks;
    a.pos = reinterpret_cast<const float4 *>(binned->sorted4);
    a.lam = F.lam;
    a.perm = binned->perm;
    a.out_x = gx;
    a.out_y = gy;
    a.out_z = gz;
    a.out_m = gm;
    a.counter = F.counter;
    a.status = status;
    pair_consts(p, a.k);
    HACC_CUDA_TRY(cudaMemsetAsync(F.counter, 0, sizeof(int32_t), st));
    hacc_launch L = launch ? *launch : default_launch(ADJOINT);
    return launch_mode<ADJOINT>(a, L, st);
}
