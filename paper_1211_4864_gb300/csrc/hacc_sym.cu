// Newton-III symmetric short-range force (Eq. 7): every pair inside the
// cutoff is evaluated once and its force applied to both particles, +m_j f d
// to i and -m_i f d to j.
//
// Work decomposition.  The same tasks, lists and staging ring as the gather
// kernel, but each task walks half of its cell's stencil: the cell itself and
// the entries after it in the canonical list (the stencil is symmetric, so
// every other neighbour pair is met from the other cell).  Inside the cell a
// task meets its own chunk (pairs j > i) and the particles after the chunk.
//
// Warp rotation.  A block of 32 j records sits one per lane, each with its
// own force partial sums; for 32 steps every lane pairs its i particles
// (one or two) with the j it holds, then passes the j and its partial sums to
// the next lane by shuffles, so each of the 32 x 32 IPL pairs is evaluated
// exactly once and no lane ever waits on another's sum.  After the block the
// j sums are added to float64 per-particle totals (atomics, skipped when a j
// met nothing); the i sums stay in registers for the whole task (float32 per
// staged tile, compensated across tiles) and are added at its end.  A last pass
// converts the totals to float32 in input order.  The sums are formed in a
// run-dependent order, so results agree with the gather kernel to rounding
// but are not bitwise reproducible.
#include "hacc_pairs.cuh"

namespace hacc {
namespace {

// Position of an empty lane: every pair with it fails the cutoff test.
constexpr float FAR = 1.0e6f;

// One j of a rotation block: its record shifted into the i frame, its
// sorted slot (-1: empty lane) and its force partial sums.
struct JRec {
    float x, y, z, m;
    float fx, fy, fz;
    int slot;
};

__device__ __forceinline__ void rotate_one(JRec &J, int src)
{
    J.x = __shfl_sync(FULL, J.x, src);
    J.y = __shfl_sync(FULL, J.y, src);
    J.z = __shfl_sync(FULL, J.z, src);
    J.m = __shfl_sync(FULL, J.m, src);
    J.fx = __shfl_sync(FULL, J.fx, src);
    J.fy = __shfl_sync(FULL, J.fy, src);
    J.fz = __shfl_sync(FULL, J.fz, src);
}

// One pair, both sides: a_i += m_j f d, f_j -= m_i f d, predicated on the
// cutoff (and on `ok`, the upper-triangle test of a diagonal block).
template <bool MASKED>
__device__ __forceinline__ void pair_sym(JRec &J, const float4 &oi, const PairConsts &K, float (&ai)[3], bool ok)
{
    const float dx = J.x - oi.x, dy = J.y - oi.y, dz = J.z - oi.z;
    const float se = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, K.eps)));
    const float t = rsqrt_hw(se);
    const float t2 = t * t;
    const float q = fmaf(fmaf(fmaf(fmaf(fmaf(K.nc[5], se, K.nc[4]), se, K.nc[3]), se, K.nc[2]), se, K.nc[1]), se,
                         K.nc[0]);
    const float f = fmaf(t2, t, q);
    const float gi = f * J.m, gj = -f * oi.w;
    if constexpr (MASKED) {
        asm("{\n\t.reg .pred p, q;\n\tsetp.lt.f32 p, %6, %7;\n\tsetp.ne.s32 q, %13, 0;\n\tand.pred p, p, q;\n\t"
            "@p fma.rn.f32 %0, %8, %10, %0;\n\t@p fma.rn.f32 %1, %8, %11, %1;\n\t@p fma.rn.f32 %2, %8, %12, %2;\n\t"
            "@p fma.rn.f32 %3, %9, %10, %3;\n\t@p fma.rn.f32 %4, %9, %11, %4;\n\t@p fma.rn.f32 %5, %9, %12, %5;\n\t}"
            : "+f"(ai[0]), "+f"(ai[1]), "+f"(ai[2]), "+f"(J.fx), "+f"(J.fy), "+f"(J.fz)
            : "f"(se), "f"(K.rc2e), "f"(gi), "f"(gj), "f"(dx), "f"(dy), "f"(dz), "r"((int)ok));
    } else {
        asm("{\n\t.reg .pred p;\n\tsetp.lt.f32 p, %6, %7;\n\t"
            "@p fma.rn.f32 %0, %8, %10, %0;\n\t@p fma.rn.f32 %1, %8, %11, %1;\n\t@p fma.rn.f32 %2, %8, %12, %2;\n\t"
            "@p fma.rn.f32 %3, %9, %10, %3;\n\t@p fma.rn.f32 %4, %9, %11, %4;\n\t@p fma.rn.f32 %5, %9, %12, %5;\n\t}"
            : "+f"(ai[0]), "+f"(ai[1]), "+f"(ai[2]), "+f"(J.fx), "+f"(J.fy), "+f"(J.fz)
            : "f"(se), "f"(K.rc2e), "f"(gi), "f"(gj), "f"(dx), "f"(dy), "f"(dz));
    }
}

// 32 rotation steps: at step k lane l holds the j that started in lane
// (l + k) mod 32.  UPPER bit u: i set u meets only j with a larger in-block
// index (k >= 1 and l + k <= 31: the block of a chunk meeting itself); SKIP
// bit u: i set u meets none of this block (j < i for all of them).
template <int IPL, unsigned UPPER, unsigned SKIP>
__device__ __forceinline__ void rotate_block(JRec &J, const float4 (&oi)[IPL], const PairConsts &K,
                                             float (&ai)[IPL][3], int lane)
{
    const int src = (lane + 1) & 31;
#pragma unroll 4
    for (int k = 0; k < 32; ++k) {
        // k >= 1 and lane + k <= 31, without short-circuit branches
        const bool upper_ok = (k != 0) & (lane + k < 32);
#pragma unroll
        for (int u = 0; u < IPL; ++u) {
            if ((SKIP >> u) & 1u) continue;
            if ((UPPER >> u) & 1u)
                pair_sym<true>(J, oi[u], K, ai[u], upper_ok);
            else
                pair_sym<false>(J, oi[u], K, ai[u], true);
        }
        rotate_one(J, src);
    }
}

// After a block: add the j partial sums to the float64 totals (skipped for
// a j that met no i inside the cutoff).
__device__ __forceinline__ void flush_j(const JRec &J, double *acc, int64_t N)
{
    if (J.slot < 0 || (J.fx == 0.0f && J.fy == 0.0f && J.fz == 0.0f)) return;
    atomicAdd(acc + J.slot, (double)J.fx);
    atomicAdd(acc + N + J.slot, (double)J.fy);
    atomicAdd(acc + 2 * N + J.slot, (double)J.fz);
}

template <int IPL>
struct AccI {
    float a[IPL][3], h[IPL][3], l[IPL][3];
    __device__ __forceinline__ AccI()
    {
#pragma unroll
        for (int u = 0; u < IPL; ++u)
#pragma unroll
            for (int k = 0; k < 3; ++k) a[u][k] = h[u][k] = l[u][k] = 0.f;
    }
    __device__ __forceinline__ void fold()
    {
#pragma unroll
        for (int u = 0; u < IPL; ++u)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                two_sum_acc(h[u][k], l[u][k], a[u][k]);
                a[u][k] = 0.f;
            }
    }
};

// One task: i particles [ib, ie) of cell c against their own chunk (j > i),
// the rest of the cell, and the forward half of the cell's list.
template <int JT, int STAGES, int IPL>
__device__ __forceinline__ bool run_task_sym(const KArgs &a, Ring<FORCE, JT, STAGES> &ring, double *acc, int64_t N,
                                             int lane, int c, int ib, int ie, const hacc_volume &vol)
{
    const PairConsts &K = a.k;
    const int n = vol.n;
    const float w = vol.w;
    const double Ld = (double)vol.L;
    const int64_t lc = (int64_t)c - vol.cell_base;
    const int cx = (int)(lc % n), cy = (int)((lc / n) % n), cz = (int)(lc / ((int64_t)n * n));

    float4 oi[IPL];
    bool active[IPL];
#pragma unroll
    for (int u = 0; u < IPL; ++u) {
        const int i = ib + lane + 32 * u;
        active[u] = i < ie;
        oi[u] = active[u] ? a.pos[i] : make_float4(FAR, FAR, FAR, 0.f);
    }
    AccI<IPL> A;

    // the chunk against itself: block u holds the chunk's i set u as j
    {
        JRec J{oi[0].x, oi[0].y, oi[0].z, oi[0].w, 0.f, 0.f, 0.f, active[0] ? ib + lane : -1};
        rotate_block<IPL, 1u, (IPL == 2 ? 2u : 0u)>(J, oi, K, A.a, lane);
        flush_j(J, acc, N);
        if constexpr (IPL == 2) {
            JRec J1{oi[1].x, oi[1].y, oi[1].z, oi[1].w, 0.f, 0.f, 0.f, active[1] ? ib + 32 + lane : -1};
            rotate_block<IPL, 2u, 0u>(J1, oi, K, A.a, lane);
            flush_j(J1, acc, N);
        }
        A.fold();
    }

    // the cell after the chunk, then the forward entries (staged)
    const int64_t e0 = a.nbr_off[c], e1 = a.nbr_off[c + 1];
    const int64_t mid = e0 + (vol.S - 1) / 2;  // the cell itself (image 13) sits in the middle of its list
    const int ce = a.cell_start[c + 1];
    for (int64_t g0 = mid; g0 < e1; g0 += 32) {
        const int ng = (int)min((int64_t)32, e1 - g0);
        int jb = 0, cnt = 0;
        float Dx = 0.f, Dy = 0.f, Dz = 0.f;
        if (lane < ng) {
            if (g0 + lane == mid) {
                jb = ie;
                cnt = ce - ie;
            } else {
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
        }
        int pk = 0, poff = 0;  // producer cursor
        int ck = 0, coff = 0;  // consumer cursor
        for (int s = 0; s < STAGES; ++s)
            if (!ring.produce(a, lane, ng, cnt, jb, pk, poff)) break;
        while (ring.consumed < ring.issued) {
            if (!ring.wait_next()) return false;
            const float4 *tj = ring.tile(ring.consumed % STAGES);
            // the producer's pieces again: piece start in the tile, source slot, image offset
            int filled = 0;
            const int k_first = ck, off_first = coff;
            while (ck < ng && filled < JT) {
                const int cc = __shfl_sync(FULL, cnt, ck);
                if (coff >= cc) {
                    ++ck;
                    coff = 0;
                    continue;
                }
                const int take = min(JT - filled, cc - coff);
                filled += take;
                coff += take;
            }
            // blocks of 32 records; the piece cursor carries over from block to block
            int kk = k_first, oo = off_first, at = 0;  // the piece that starts at tile record `at`
            for (int b0 = 0; b0 < filled; b0 += 32) {
                const int r = b0 + lane;
                const int bend = min(filled, b0 + 32);
                JRec J{FAR, FAR, FAR, 0.f, 0.f, 0.f, 0.f, -1};
                while (kk < ng && at < bend) {
                    const int cc = __shfl_sync(FULL, cnt, kk);
                    if (oo >= cc) {
                        ++kk;
                        oo = 0;
                        continue;
                    }
                    const int take = min(JT - at, cc - oo);
                    const int src = __shfl_sync(FULL, jb, kk) + oo;
                    const float dx = __shfl_sync(FULL, Dx, kk), dy = __shfl_sync(FULL, Dy, kk),
                                dz = __shfl_sync(FULL, Dz, kk);
                    if (r >= at && r < at + take) {
                        const float4 p = tj[r];
                        J.x = p.x + dx;
                        J.y = p.y + dy;
                        J.z = p.z + dz;
                        J.m = p.w;
                        J.slot = src + (r - at);
                    }
                    if (at + take > bend) break;  // the piece goes on into the next block
                    at += take;
                    oo += take;
                }
                rotate_block<IPL, 0u, 0u>(J, oi, K, A.a, lane);
                flush_j(J, acc, N);
            }
            A.fold();
            ++ring.consumed;
            __syncwarp();
            ring.produce(a, lane, ng, cnt, jb, pk, poff);
        }
    }
#pragma unroll
    for (int u = 0; u < IPL; ++u) {
        if (!active[u]) continue;
        const int i = ib + lane + 32 * u;
        atomicAdd(acc + i, (double)A.h[u][0] + (double)A.l[u][0]);
        atomicAdd(acc + N + i, (double)A.h[u][1] + (double)A.l[u][1]);
        atomicAdd(acc + 2 * N + i, (double)A.h[u][2] + (double)A.l[u][2]);
    }
    return true;
}

template <int JT, int STAGES>
__global__ void __launch_bounds__(256, 3) k_pairs_sym(const KArgs a, double *acc, int64_t N)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int WARP_BYTES = warp_smem_bytes(FORCE, JT, STAGES);
    constexpr int TILE_BYTES = warp_tiles_bytes(FORCE, JT, STAGES);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char *wbase = smem + (size_t)warp * WARP_BYTES;
    Ring<FORCE, JT, STAGES> ring;
    ring.tiles = reinterpret_cast<float4 *>(wbase);
    ring.bars = reinterpret_cast<uint64_t *>(wbase + TILE_BYTES);
    if (lane == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(smem_addr(&ring.bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncwarp();
    const int ntask = *a.n_tasks;
    while (true) {
        int t = 0;
        if (lane == 0) t = atomicAdd(a.counter, 1);
        t = __shfl_sync(FULL, t, 0);
        if (t >= ntask) break;
        const int4 task = a.tasks[a.order[t]];
        const hacc_volume &vol = a.vols[task.w];
        bool ok;
        if (task.z - task.y > 32)
            ok = run_task_sym<JT, STAGES, 2>(a, ring, acc, N, lane, task.x, task.y, task.z, vol);
        else
            ok = run_task_sym<JT, STAGES, 1>(a, ring, acc, N, lane, task.x, task.y, task.z, vol);
        if (!ok) {
            if (lane == 0) atomicOr(a.status, HACC_STATUS_TIMEOUT);
            ring.drain();
            return;
        }
    }
}

// float64 totals (sorted slots) to float32 accelerations in input order.
__global__ void __launch_bounds__(256)
k_sym_finish(int64_t N, const double *__restrict__ acc, const int32_t *__restrict__ perm, float *__restrict__ ax,
             float *__restrict__ ay, float *__restrict__ az)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        const int i = perm[k];
        ax[i] = (float)acc[k];
        ay[i] = (float)acc[N + k];
        az[i] = (float)acc[2 * N + k];
    }
}

template <int JT, int STAGES>
int launch_sym_t(const KArgs &a, double *acc, int64_t N, int warps, int ctas_per_sm, cudaStream_t st)
{
    const size_t smem = (size_t)warps * warp_smem_bytes(FORCE, JT, STAGES);
    auto kern = k_pairs_sym<JT, STAGES>;
    if (smem > 48 * 1024)
        HACC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    HACC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, warps * 32, smem));
    if (occ < 1) return HACC_ERR_INVALID;
    const int per_sm = ctas_per_sm < occ ? ctas_per_sm : occ;
    kern<<<num_sms() * per_sm, warps * 32, smem, st>>>(a, acc, N);
    HACC_LAUNCH_CHECK();
    return HACC_OK;
}

int launch_sym(const KArgs &a, double *acc, int64_t N, const hacc_launch &L, cudaStream_t st)
{
    const int wp = L.warps_per_cta, cps = L.ctas_per_sm;
#define HACC_CASE(JT, S) \
    if (L.jtile == JT && L.stages == S) return launch_sym_t<JT, S>(a, acc, N, wp, cps, st);
    HACC_CASE(32, 2) HACC_CASE(32, 4) HACC_CASE(64, 2) HACC_CASE(64, 3) HACC_CASE(64, 4)
    HACC_CASE(128, 2) HACC_CASE(128, 3) HACC_CASE(128, 4) HACC_CASE(256, 2)
#undef HACC_CASE
    return HACC_ERR_INVALID;
}

}  // namespace
}  // namespace hacc

using namespace hacc;

extern "C" int hacc_sr_force_symmetric(const hacc_mesh *mesh, const hacc_binned *binned, const hacc_lists *lists,
                                       const hacc_sr_params *p, float *ax, float *ay, float *az,
                                       const hacc_launch *launch, void *ws, size_t ws_bytes, uint32_t *status,
                                       void *stream)
{
    int rc = check_common(mesh, binned, lists, p, launch, ws, ws_bytes, status);
    if (rc) return rc;
    if (binned->cell_origin) return HACC_ERR_INVALID;  // the half stencil needs the chaining mesh's lists
    if (mesh->N > 0 && (!ax || !ay || !az)) return HACC_ERR_INVALID;
    if (mesh->N == 0) return HACC_OK;
    cudaStream_t st = as_stream(stream);
    ForceWs F = force_layout(mesh, ws);
    KArgs a = base_args(mesh, binned, lists, p, status);
    a.counter = F.counter;
    HACC_CUDA_TRY(cudaMemsetAsync(F.counter, 0, sizeof(int32_t), st));
    HACC_CUDA_TRY(cudaMemsetAsync(F.acc, 0, (size_t)mesh->N * 3 * sizeof(double), st));
    hacc_launch L;
    if (launch) {
        L = *launch;
    } else {
        L.warps_per_cta = 8;
        L.ctas_per_sm = 3;
        L.jtile = 128;
        L.stages = 2;
    }
    rc = launch_sym(a, F.acc, mesh->N, L, st);
    if (rc) return rc;
    int g = (int)((mesh->N + 255) / 256);
    if (g > num_sms() * 16) g = num_sms() * 16;
    k_sym_finish<<<g, 256, 0, st>>>(mesh->N, F.acc, binned->perm, ax, ay, az);
    HACC_LAUNCH_CHECK();
    return HACC_OK;
}
