// Newton-III symmetric adjoint of the short-range force (the vector-Jacobian
// product of Eq. 7's forces, not in the paper), on the symmetric force
// kernel's tasks, half-stencil walk, staging ring and warp rotation
// (hacc_sym.cu, hacc_sym.cuh).
#include "hacc_sym.cuh"

namespace hacc {
namespace {

// ---------------------------------------------------------------------------
// Symmetric adjoint.  The pair (i, j)'s terms of the vector-Jacobian product
// are antisymmetric in dL/dx (J(d) = f I + 2 f' d d^T is even in d):
//   dL/dx_i += m_i J lam_j - m_j J lam_i,   dL/dx_j gets the same with minus,
// so each pair is evaluated once.  Both sides keep the gather adjoint's
// factored sums, U = sum f lam_p, V = sum m_p f, X = sum r d_k (r = 2 f'
// (m_k d_k.lam_p - m_p d_k.lam_k)), G = sum f d_k.lam_p, over partners p with
// d_k = x_p - x_k, so that dL/dx_k = m_k U - lam_k V + X and dL/dm_k = -G.
// For the pair seen from j every term flips sign or swaps: U_j += f lam_i,
// V_j += m_i f, X_j -= r d, G_j -= f d.lam_i.
// Without dL/dm (the W form): with mu = m_i lam_j - m_j lam_i the pair's
// whole term w = f mu + fp2 (d.mu) d is antisymmetric, like a force, so i
// adds w and j subtracts it; each side carries three sums (u0, u1, u2) and
// dL/dx_k = W_k (equal masses: mu / m summed, dL/dx_k = m W_k).
// ---------------------------------------------------------------------------

// One j of an adjoint rotation block: record shifted into the i frame, its
// cotangent, its partial sums and sorted slot (-1: empty lane).
struct JAdj {
    float x, y, z, m, lx, ly, lz;
    float u0, u1, u2, v, x0, x1, x2, g;
    int slot;
};

template <bool GM, bool EQ>
__device__ __forceinline__ void rotate_adj(JAdj &J, int src)
{
    constexpr bool WF = adj_wform(GM ? ADJOINT_GM : ADJOINT);
    J.x = __shfl_sync(FULL, J.x, src);
    J.y = __shfl_sync(FULL, J.y, src);
    J.z = __shfl_sync(FULL, J.z, src);
    if constexpr (!EQ) J.m = __shfl_sync(FULL, J.m, src);
    J.lx = __shfl_sync(FULL, J.lx, src);
    J.ly = __shfl_sync(FULL, J.ly, src);
    J.lz = __shfl_sync(FULL, J.lz, src);
    J.u0 = __shfl_sync(FULL, J.u0, src);
    J.u1 = __shfl_sync(FULL, J.u1, src);
    J.u2 = __shfl_sync(FULL, J.u2, src);
    if constexpr (WF) return;
    J.v = __shfl_sync(FULL, J.v, src);
    J.x0 = __shfl_sync(FULL, J.x0, src);
    J.x1 = __shfl_sync(FULL, J.x1, src);
    J.x2 = __shfl_sync(FULL, J.x2, src);
    if constexpr (GM) J.g = __shfl_sync(FULL, J.g, src);
}

// One pair of the adjoint, both sides; outside the cutoff (or outside the
// upper triangle of a diagonal block) f and r are zero, so every sum is
// unchanged.  Equal masses (EQ): V sums f on both sides and r = fp2
// d.(lam_j - lam_i) (the W form: mu / m), the common mass applied by the
// finishing pass.
template <bool GM, bool EQ>
__device__ __forceinline__ void pair_adj_sym(JAdj &J, const float4 &oi, const float4 &li, const PairConsts &K,
                                             float (&acc)[ADJ_NACC], bool ok)
{
    const float dx = J.x - oi.x, dy = J.y - oi.y, dz = J.z - oi.z;
    const float se = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, K.eps)));
    const float t = rsqrt_hw(se);
    const float t2 = t * t;
    const float t3 = t2 * t;
    const float q = fmaf(fmaf(fmaf(fmaf(fmaf(K.nc[5], se, K.nc[4]), se, K.nc[3]), se, K.nc[2]), se, K.nc[1]), se,
                         K.nc[0]);
    const float qp = fmaf(fmaf(fmaf(fmaf(K.kp[4], se, K.kp[3]), se, K.kp[2]), se, K.kp[1]), se, K.kp[0]);
    const float fp2 = fmaf(-3.0f, t3 * t2, qp);
    const bool in = ok & (se < K.rc2e);
    const float f = in ? t3 + q : 0.0f;
    if constexpr (!GM) {  // the W form
        float ex, ey, ez;  // mu (equal masses: mu / m)
        if constexpr (EQ) {
            ex = J.lx - li.x;
            ey = J.ly - li.y;
            ez = J.lz - li.z;
        } else {
            ex = fmaf(oi.w, J.lx, -(J.m * li.x));
            ey = fmaf(oi.w, J.ly, -(J.m * li.y));
            ez = fmaf(oi.w, J.lz, -(J.m * li.z));
        }
        const float r = in ? fp2 * fmaf(dz, ez, fmaf(dy, ey, dx * ex)) : 0.0f;
        const float wx = fmaf(f, ex, r * dx), wy = fmaf(f, ey, r * dy), wz = fmaf(f, ez, r * dz);
        acc[0] += wx;
        acc[1] += wy;
        acc[2] += wz;
        J.u0 -= wx;
        J.u1 -= wy;
        J.u2 -= wz;
        return;
    }
    const float dlj = fmaf(dz, J.lz, fmaf(dy, J.ly, dx * J.lx));
    const float dli = fmaf(dz, li.z, fmaf(dy, li.y, dx * li.x));
    float rr;
    if constexpr (EQ)
        rr = fp2 * (dlj - dli);
    else
        rr = fp2 * fmaf(oi.w, dlj, -(J.m * dli));
    const float r = in ? rr : 0.0f;
    const float mj = EQ ? 1.0f : J.m, mi = EQ ? 1.0f : oi.w;
    // i side
    acc[0] = fmaf(f, J.lx, acc[0]);
    acc[1] = fmaf(f, J.ly, acc[1]);
    acc[2] = fmaf(f, J.lz, acc[2]);
    acc[3] = fmaf(mj, f, acc[3]);
    acc[4] = fmaf(r, dx, acc[4]);
    acc[5] = fmaf(r, dy, acc[5]);
    acc[6] = fmaf(r, dz, acc[6]);
    if constexpr (GM) acc[7] = fmaf(f, dlj, acc[7]);
    // j side
    J.u0 = fmaf(f, li.x, J.u0);
    J.u1 = fmaf(f, li.y, J.u1);
    J.u2 = fmaf(f, li.z, J.u2);
    J.v = fmaf(mi, f, J.v);
    J.x0 = fmaf(-r, dx, J.x0);
    J.x1 = fmaf(-r, dy, J.x1);
    J.x2 = fmaf(-r, dz, J.x2);
    if constexpr (GM) J.g = fmaf(-f, dli, J.g);
}

// W rotation steps within groups of W lanes, as the force kernel's
// rotate_block; a half-warp block with an UPPER set (the chunk's own block of
// a half-warp task) pairs on the low half only.
template <int IPL, bool GM, bool EQ, unsigned UPPER, unsigned SKIP, int W = 32>
__device__ __forceinline__ void rotate_block_adj(JAdj &J, const float4 (&oi)[IPL], const float4 (&li)[IPL],
                                                 const PairConsts &K, float (&p)[IPL][ADJ_NACC], int lane)
{
    static_assert(W == 32 || W == 16, "rotation width");
    const int src = (lane & (32 - W)) | ((lane + 1) & (W - 1));
    const int lg = lane & (W - 1);
    const bool rows = W == 32 || UPPER == 0u || lane < 16;
#pragma unroll 2
    for (int k = 0; k < W; ++k) {
        const bool upper_ok = (k != 0) & (lg + k < W) & rows;
#pragma unroll
        for (int u = 0; u < IPL; ++u) {
            if ((SKIP >> u) & 1u) continue;
            pair_adj_sym<GM, EQ>(J, oi[u], li[u], K, p[u], ((UPPER >> u) & 1u) ? upper_ok : true);
        }
        rotate_adj<GM, EQ>(J, src);
    }
}

// j sums of a block to the float64 totals acc[c N + slot], c = U0 U1 U2 V X0 X1 X2 G
// (the W form: W0 W1 W2).
template <bool GM, bool EQ>
__device__ __forceinline__ void flush_adj(const JAdj &J, double *acc, int64_t N)
{
    constexpr int NC = adj_nacc(GM ? ADJOINT_GM : ADJOINT);
    if (J.slot < 0) return;
    if (J.u0 == 0.f && J.u1 == 0.f && J.u2 == 0.f &&
        (NC == 3 || (J.v == 0.f && J.x0 == 0.f && J.x1 == 0.f && J.x2 == 0.f)) && (!GM || J.g == 0.f))
        return;
    const float c[8] = {J.u0, J.u1, J.u2, J.v, J.x0, J.x1, J.x2, J.g};
#pragma unroll
    for (int k = 0; k < NC; ++k) atomicAdd(acc + k * N + J.slot, (double)c[k]);
}

// The chunk's own block B (its i set B as the j): sets below B meet every j,
// set B the upper triangle, the sets above none (they meet set B's records
// when their own block comes round).
template <int B, int IPL, bool GM, bool EQ>
__device__ __forceinline__ void own_block_adj(const float4 (&oi)[IPL], const float4 (&li)[IPL],
                                              const bool (&active)[IPL], int ib, int lane, const PairConsts &K,
                                              float (&p)[IPL][ADJ_NACC], double *acc, int64_t N)
{
    constexpr unsigned SKIP = (0xFu << (B + 1)) & ((1u << IPL) - 1u);
    JAdj J{oi[B].x, oi[B].y, oi[B].z, oi[B].w, li[B].x, li[B].y, li[B].z,
           0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, active[B] ? ib + 32 * B + lane : -1};
    rotate_block_adj<IPL, GM, EQ, 1u << B, SKIP>(J, oi, li, K, p, lane);
    flush_adj<GM, EQ>(J, acc, N);
}

// One task (sub-chunk): i particles [ib, ie) against their own chunk, the
// rest of the cell and the forward half of the list.  HALF (at most 16
// particles): each i in lanes l and l + 16, the half-warps rotate the two
// halves of each block of 32 j (as the force kernel).
template <int JT, int STAGES, int IPL, bool GM, bool EQ, bool HALF = false>
__device__ __forceinline__ bool run_task_adj_sym(const KArgs &a, Ring<ADJOINT, JT, STAGES> &ring, float *comp,
                                                 double *acc, int64_t N, int lane, int c, int ib, int ie,
                                                 const hacc_volume &vol)
{
    static_assert(!HALF || IPL == 1, "half-warp tasks hold one i set");
    constexpr int W = HALF ? 16 : 32;
    const int il = HALF ? (lane & 15) : lane;
    constexpr int MODE = GM ? ADJOINT_GM : ADJOINT;
    const PairConsts &K = a.k;
    const int n = vol.n;
    const int64_t lc = (int64_t)c - vol.cell_base;
    const int cx = (int)(lc % n), cy = (int)((lc / n) % n), cz = (int)(lc / ((int64_t)n * n));
    const float4 org_i = a.origin ? a.origin[c] : make_float4(0.f, 0.f, 0.f, 0.f);

    float4 oi[IPL], li[IPL];
    bool active[IPL];
#pragma unroll
    for (int u = 0; u < IPL; ++u) {
        const int i = ib + il + 32 * u;
        active[u] = i < ie;
        oi[u] = active[u] ? a.pos[i] : make_float4(FAR, FAR, FAR, 0.f);
        li[u] = active[u] ? a.lam[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    AccAdj<MODE, IPL, adj_nacc(MODE)> A(comp, lane);

    if constexpr (HALF) {  // the chunk against itself on the low half-warp, 16 steps
        const bool lo = lane < 16;
        JAdj J{oi[0].x, oi[0].y, oi[0].z, oi[0].w, li[0].x, li[0].y, li[0].z,
               0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, (lo && active[0]) ? ib + lane : -1};
        if (!lo) {
            J.x = J.y = J.z = FAR;
            J.m = J.lx = J.ly = J.lz = 0.f;
        }
        rotate_block_adj<1, GM, EQ, 1u, 0u, 16>(J, oi, li, K, A.p, lane);
        flush_adj<GM, EQ>(J, acc, N);
        A.fold();
    } else {  // the chunk against itself
        own_block_adj<0, IPL, GM, EQ>(oi, li, active, ib, lane, K, A.p, acc, N);
        if constexpr (IPL >= 2) own_block_adj<1, IPL, GM, EQ>(oi, li, active, ib, lane, K, A.p, acc, N);
        if constexpr (IPL >= 4) {
            own_block_adj<2, IPL, GM, EQ>(oi, li, active, ib, lane, K, A.p, acc, N);
            own_block_adj<3, IPL, GM, EQ>(oi, li, active, ib, lane, K, A.p, acc, N);
        }
        A.fold();
    }

    const int64_t e0 = a.nbr_off[c], e1 = a.nbr_off[c + 1];
    const int64_t mid = self_entry(a, c, e0, e1, vol);
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
                jb = a.cell_start[cp];
                cnt = a.cell_start[cp + 1] - jb;
                entry_delta(a, vol, cp, a.nbr_shift[g0 + lane], cx, cy, cz, org_i, Dx, Dy, Dz);
            }
        }
        int pk = 0, poff = 0;
        int ck = 0, coff = 0;
        for (int s = 0; s < STAGES; ++s)
            if (!ring.produce(a, lane, ng, cnt, jb, pk, poff)) break;
        while (ring.consumed < ring.issued) {
            if (!ring.wait_next(a.wait_limit)) return false;
            const float4 *tj = ring.tile(ring.consumed % STAGES);
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
            int kk = k_first, oo = off_first, at = 0;
            for (int b0 = 0; b0 < filled; b0 += 32) {
                const int r = b0 + lane;
                const int bend = min(filled, b0 + 32);
                JAdj J{FAR, FAR, FAR, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, -1};
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
                        const float4 pp = tj[r], ll = tj[JT + r];
                        J.x = pp.x + dx;
                        J.y = pp.y + dy;
                        J.z = pp.z + dz;
                        J.m = pp.w;
                        J.lx = ll.x;
                        J.ly = ll.y;
                        J.lz = ll.z;
                        J.slot = src + (r - at);
                    }
                    if (at + take > bend) break;
                    at += take;
                    oo += take;
                }
                rotate_block_adj<IPL, GM, EQ, 0u, 0u, W>(J, oi, li, K, A.p, lane);
                flush_adj<GM, EQ>(J, acc, N);
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
        const int i = ib + il + 32 * u;  // HALF: both lanes of i add their part
#pragma unroll
        for (int k = 0; k < A.NACC; ++k)
            atomicAdd(acc + k * N + i, (double)A.hi(u, k) + (double)A.lo(u, k));
    }
    return true;
}

template <int JT, int STAGES, bool GM, bool EQ>
__global__ void __launch_bounds__(256, 2) k_adj_sym(const KArgs a, double *acc, int64_t N)
{
    const bool eq = a.mass_varies && *a.mass_varies == 0u;
    if (eq != EQ) return;  // the other instantiation does the work
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int WARP_BYTES = warp_smem_bytes(ADJOINT, JT, STAGES);
    constexpr int TILE_BYTES = warp_tiles_bytes(ADJOINT, JT, STAGES);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char *wbase = smem + (size_t)warp * WARP_BYTES;
    Ring<ADJOINT, JT, STAGES> ring;
    ring.tiles = reinterpret_cast<float4 *>(wbase);
    float *comp = reinterpret_cast<float *>(wbase + TILE_BYTES);
    ring.bars = reinterpret_cast<uint64_t *>(wbase + TILE_BYTES + ADJ_COMP_BYTES);
    if (lane == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(smem_addr(&ring.bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncwarp();
    const int ntask = task_count(a);
    while (true) {
        int t = 0;
        if (lane == 0) t = atomicAdd(a.counter, 1);
        t = __shfl_sync(FULL, t, 0);
        if (t >= ntask) break;
        int4 task;
        if (!take_task(a, t, lane, task, a.order)) continue;
        const hacc_volume &vol = a.vols[task.w];
        bool ok = true;
        // sub-chunks of larger tasks: 128 particles (four i per lane) in the W form,
        // whose three sums leave the registers for it, else 64
        constexpr int CHUNK = adj_wform(GM ? ADJOINT_GM : ADJOINT) ? 128 : 64;
        for (int sb = task.y; ok && sb < task.z; sb += CHUNK) {
            const int se = min(sb + CHUNK, task.z);
            if (CHUNK == 128 && se - sb > 64)
                ok = run_task_adj_sym<JT, STAGES, (CHUNK == 128 ? 4 : 2), GM, EQ>(a, ring, comp, acc, N, lane,
                                                                                  task.x, sb, se, vol);
            else if (se - sb > 32)
                ok = run_task_adj_sym<JT, STAGES, 2, GM, EQ>(a, ring, comp, acc, N, lane, task.x, sb, se, vol);
            else if (se - sb > 16)
                ok = run_task_adj_sym<JT, STAGES, 1, GM, EQ>(a, ring, comp, acc, N, lane, task.x, sb, se, vol);
            else
                ok = run_task_adj_sym<JT, STAGES, 1, GM, EQ, true>(a, ring, comp, acc, N, lane, task.x, sb, se,
                                                                   vol);
        }
        if (!ok) {
            if (lane == 0) atomicOr(a.status, HACC_STATUS_TIMEOUT);
            ring.drain();
            return;
        }
    }
}

// The W form: one component of dL/dx = W (equal masses: m W, m the common
// mass) from the float64 totals, in input order; one component per launch
// for the reason given at k_sym_finish.
__global__ void __launch_bounds__(256)
k_adj_sym_finish_w(int64_t N, const double *__restrict__ acc, const int32_t *__restrict__ perm,
                   const float4 *__restrict__ pos, const uint32_t *mass_varies, float *__restrict__ out)
{
    const bool eq = mass_varies && *mass_varies == 0u;
    const double sc = eq ? (double)pos[0].w : 1.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x)
        out[__ldcs(perm + k)] = (float)(sc * __ldcs(acc + k));
}

// With dL/dm: dL/dx_k = m_k U - lam_k V + X (equal masses: m_k (U - lam_k V +
// X)) and dL/dm_k = -G from the float64 totals, in input order.
__global__ void __launch_bounds__(256)
k_adj_sym_finish(int64_t N, const double *__restrict__ acc, const int32_t *__restrict__ perm,
                 const float4 *__restrict__ pos, const float4 *__restrict__ lam, const uint32_t *mass_varies,
                 float *__restrict__ gx, float *__restrict__ gy, float *__restrict__ gz, float *__restrict__ gm)
{
    const bool eq = mass_varies && *mass_varies == 0u;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        const int i = perm[k];
        const double m = (double)pos[k].w;
        const float4 l = lam[k];
        const double V = acc[3 * N + k];
        if (eq) {
            gx[i] = (float)(m * (acc[k] - (double)l.x * V + acc[4 * N + k]));
            gy[i] = (float)(m * (acc[N + k] - (double)l.y * V + acc[5 * N + k]));
            gz[i] = (float)(m * (acc[2 * N + k] - (double)l.z * V + acc[6 * N + k]));
        } else {
            gx[i] = (float)(m * acc[k] - (double)l.x * V + acc[4 * N + k]);
            gy[i] = (float)(m * acc[N + k] - (double)l.y * V + acc[5 * N + k]);
            gz[i] = (float)(m * acc[2 * N + k] - (double)l.z * V + acc[6 * N + k]);
        }
        gm[i] = (float)(-acc[7 * N + k]);
    }
}

template <int JT, int STAGES, bool GM, bool EQ>
int launch_adj_sym_one(const KArgs &a, double *acc, int64_t N, int warps, int ctas_per_sm, cudaStream_t st)
{
    const size_t smem = (size_t)warps * warp_smem_bytes(ADJOINT, JT, STAGES);
    auto kern = k_adj_sym<JT, STAGES, GM, EQ>;
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

template <int JT, int STAGES, bool GM>
int launch_adj_sym_t(const KArgs &a, double *acc, int64_t N, int warps, int ctas_per_sm, cudaStream_t st)
{
    if (a.mass_varies) {
        const int rc = launch_adj_sym_one<JT, STAGES, GM, true>(a, acc, N, warps, ctas_per_sm, st);
        if (rc) return rc;
    }
    return launch_adj_sym_one<JT, STAGES, GM, false>(a, acc, N, warps, ctas_per_sm, st);
}

template <bool GM>
int launch_adj_sym(const KArgs &a, double *acc, int64_t N, const hacc_launch &L, cudaStream_t st)
{
    const int wp = L.warps_per_cta, cps = L.ctas_per_sm;
#define HACC_CASE(JT, S) \
    if (L.jtile == JT && L.stages == S) return launch_adj_sym_t<JT, S, GM>(a, acc, N, wp, cps, st);
    HACC_CASE(32, 2) HACC_CASE(32, 4) HACC_CASE(64, 2) HACC_CASE(64, 3) HACC_CASE(64, 4)
    HACC_CASE(128, 2) HACC_CASE(128, 3) HACC_CASE(128, 4) HACC_CASE(256, 2)
#undef HACC_CASE
    return HACC_ERR_INVALID;
}

}  // namespace
}  // namespace hacc

using namespace hacc;

extern "C" int hacc_sr_force_adjoint_symmetric(const hacc_mesh *mesh, const hacc_binned *binned,
                                               const hacc_lists *lists, const hacc_sr_params *p, const float *gax,
                                               const float *gay, const float *gaz, float *gx, float *gy, float *gz,
                                               float *gm, const hacc_launch *launch, void *ws, size_t ws_bytes,
                                               uint32_t *status, void *stream)
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
    KArgs a = base_args(mesh, binned, lists, p, status);
    a.lam = F.lam;
    a.counter = F.counter;
    HACC_CUDA_TRY(cudaMemsetAsync(F.counter, 0, sizeof(int32_t), st));
    HACC_CUDA_TRY(cudaMemsetAsync(F.acc, 0, (size_t)mesh->N * (gm ? 8 : 3) * sizeof(double), st));
    hacc_launch L;
    if (launch) {
        L = *launch;
    } else {
        L.warps_per_cta = 8;
        L.ctas_per_sm = 2;
        L.jtile = 128;
        L.stages = 2;
        L.wait_cycles = 0;
    }
    a.wait_limit = wait_limit_of(L);
    rc = gm ? launch_adj_sym<true>(a, F.acc, mesh->N, L, st) : launch_adj_sym<false>(a, F.acc, mesh->N, L, st);
    if (rc) return rc;
    const float4 *pos = reinterpret_cast<const float4 *>(binned->sorted4);
    if (gm) {
        k_adj_sym_finish<<<g, 256, 0, st>>>(mesh->N, F.acc, binned->perm, pos, F.lam, binned->mass_varies, gx, gy,
                                            gz, gm);
        HACC_LAUNCH_CHECK();
        return HACC_OK;
    }
    float *out[3] = {gx, gy, gz};
    for (int c = 0; c < 3; ++c) {
        k_adj_sym_finish_w<<<g, 256, 0, st>>>(mesh->N, F.acc + c * mesh->N, binned->perm, pos, binned->mass_varies,
                                              out[c]);
        HACC_LAUNCH_CHECK();
    }
    return HACC_OK;
}
