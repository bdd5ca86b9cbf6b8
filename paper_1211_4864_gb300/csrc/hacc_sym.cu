// Newton-III symmetric short-range force (Eq. 7): every pair inside the
// cutoff is evaluated once and its force applied to both particles, +m_j f d
// to i and -m_i f d to j (the adjoint's pair terms are antisymmetric the same
// way: hacc_sym_adj.cu).
//
// Work decomposition.  The same tasks, lists and staging ring as the gather
// kernel, but each task walks half of its cell's list: the cell itself and
// the entries after it (lists are symmetric, so every other neighbour pair is
// met from the other cell); chaining-mesh cells and tree leaves alike.
// Inside the cell a task meets its own chunk (pairs j > i) and the particles
// after the chunk.
//
// Warp rotation.  A block of 32 j records sits one per lane, each with its
// own force partial sums; for 32 steps every lane pairs its i particles
// (one, two or four) with the j it holds, then passes the j and its partial
// sums to the next lane by shuffles, so each of the 32 x 32 IPL pairs is
// evaluated exactly once and no lane ever waits on another's sum.  A task of
// at most 16 particles puts each i in two lanes and rotates the two halves
// of the block separately (16 steps).  After the block the
// j sums are added to float64 per-particle totals (atomics, skipped when a j
// met nothing); the i sums stay in registers for the whole task (float32 per
// staged tile, compensated across tiles) and are added at its end.  A last pass
// converts the totals to float32 in input order.  The sums are formed in a
// run-dependent order, so results agree with the gather kernel to rounding
// but are not bitwise reproducible.
//
// Equal masses (the binning found every mass equal): both sides accumulate
// f d, the j masses no longer rotate, and each total is scaled by the
// particle's own mass when it is added (a_i = m sum_j f d, a_j = -m sum_i f d),
// which takes the two mass products out of every pair.
#include "hacc_sym.cuh"

namespace hacc {
namespace {

// One j of a rotation block: its record shifted into the i frame, its
// sorted slot (-1: empty lane) and its force partial sums.
struct JRec {
    float x, y, z, m;
    float fx, fy, fz;
    int slot;
};

template <bool EQ>
__device__ __forceinline__ void rotate_one(JRec &J, int src)
{
    J.x = __shfl_sync(FULL, J.x, src);
    J.y = __shfl_sync(FULL, J.y, src);
    J.z = __shfl_sync(FULL, J.z, src);
    if constexpr (!EQ) J.m = __shfl_sync(FULL, J.m, src);  // equal masses: the lane keeps its own
    J.fx = __shfl_sync(FULL, J.fx, src);
    J.fy = __shfl_sync(FULL, J.fy, src);
    J.fz = __shfl_sync(FULL, J.fz, src);
}

// One pair, both sides: a_i += m_j f d, f_j -= m_i f d (equal masses: both
// += f d), predicated on the cutoff (and on `ok`, a diagonal block's test that
// meets each pair of a set once).
template <bool MASKED, bool EQ>
__device__ __forceinline__ void pair_sym(JRec &J, const float4 &oi, const PairConsts &K, float (&ai)[3], bool ok)
{
    const float dx = J.x - oi.x, dy = J.y - oi.y, dz = J.z - oi.z;
    const float se = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, K.eps)));
    const float t = rsqrt_hw(se);
    const float t2 = t * t;
    const float q = fmaf(fmaf(fmaf(fmaf(fmaf(K.nc[5], se, K.nc[4]), se, K.nc[3]), se, K.nc[2]), se, K.nc[1]), se,
                         K.nc[0]);
    const float f = fmaf(t2, t, q);
    const float gi = EQ ? f : f * J.m, gj = EQ ? f : -f * oi.w;
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

// W rotation steps within groups of W lanes (W = 32: the whole warp; W = 16:
// each half-warp rotates its own 16 records): at step k lane l holds the j
// that started in lane g + (l - g + k) mod W of its group g.  UPPER bit u: i
// set u meets only j with a larger in-group index (k >= 1 and (l - g) + k <=
// W - 1: the block of a chunk meeting itself); SKIP bit u: i set u meets none
// of this block (j < i for all of them).
template <int IPL, unsigned UPPER, unsigned SKIP, bool EQ, int W = 32>
__device__ __forceinline__ void rotate_block(JRec &J, const float4 (&oi)[IPL], const PairConsts &K,
                                             float (&ai)[IPL][3], int lane)
{
    static_assert(W == 32 || W == 16, "rotation width");
    const int src = (lane & (32 - W)) | ((lane + 1) & (W - 1));
    const int lg = lane & (W - 1);
    const bool rows = W == 32 || UPPER == 0u || lane < 16;  // a half-warp task's own block: low half only
#pragma unroll 4
    for (int k = 0; k < W; ++k) {
        // k >= 1 and lg + k <= W - 1, without short-circuit branches
        const bool upper_ok = (k != 0) & (lg + k < W) & rows;
#pragma unroll
        for (int u = 0; u < IPL; ++u) {
            if ((SKIP >> u) & 1u) continue;
            if ((UPPER >> u) & 1u)
                pair_sym<true, EQ>(J, oi[u], K, ai[u], upper_ok);
            else
                pair_sym<false, EQ>(J, oi[u], K, ai[u], true);
        }
        rotate_one<EQ>(J, src);
    }
}

// After a block: add the j partial sums to the float64 totals (skipped for
// a j that met no i inside the cutoff); equal masses: times -m_j.
template <bool EQ>
__device__ __forceinline__ void flush_j(const JRec &J, double *acc, int64_t N)
{
    if (J.slot < 0 || (J.fx == 0.0f && J.fy == 0.0f && J.fz == 0.0f)) return;
    if constexpr (EQ) {
        atomicAdd(acc + J.slot, (double)(-J.m * J.fx));
        atomicAdd(acc + N + J.slot, (double)(-J.m * J.fy));
        atomicAdd(acc + 2 * N + J.slot, (double)(-J.m * J.fz));
    } else {
        atomicAdd(acc + J.slot, (double)J.fx);
        atomicAdd(acc + N + J.slot, (double)J.fy);
        atomicAdd(acc + 2 * N + J.slot, (double)J.fz);
    }
}

// i sums of a task: float32 within a staged tile, folded into a compensated
// (hi, lo) pair per component across tiles.  One or two i per lane keep the
// pairs in registers; four i per lane keep them in shared memory
// (comp[((u * 3 + k) * 2 + {0, 1}) * 32 + lane]) to stay within 80 registers.
constexpr int SYM_IPL_MAX = 4;
constexpr int SYM_COMP_BYTES = SYM_IPL_MAX * 3 * 2 * 32 * 4;

template <int IPL>
struct AccI {
    static constexpr bool SMEM = IPL > 2;
    float a[IPL][3];
    float h[SMEM ? 1 : IPL][3], l[SMEM ? 1 : IPL][3];
    float *comp;
    int lane;
    __device__ __forceinline__ float &chi(int u, int k) const { return comp[((u * 3 + k) * 2 + 0) * 32 + lane]; }
    __device__ __forceinline__ float &clo(int u, int k) const { return comp[((u * 3 + k) * 2 + 1) * 32 + lane]; }
    __device__ __forceinline__ AccI(float *c, int ln) : comp(c), lane(ln)
    {
#pragma unroll
        for (int u = 0; u < IPL; ++u)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                a[u][k] = 0.f;
                if constexpr (SMEM) {
                    chi(u, k) = 0.f;
                    clo(u, k) = 0.f;
                } else {
                    h[u][k] = 0.f;
                    l[u][k] = 0.f;
                }
            }
    }
    __device__ __forceinline__ void fold()
    {
#pragma unroll
        for (int u = 0; u < IPL; ++u)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                if constexpr (SMEM) {
                    float hh = chi(u, k), ll = clo(u, k);
                    two_sum_acc(hh, ll, a[u][k]);
                    chi(u, k) = hh;
                    clo(u, k) = ll;
                } else {
                    two_sum_acc(h[u][k], l[u][k], a[u][k]);
                }
                a[u][k] = 0.f;
            }
    }
    // the compensated total as a float64
    __device__ __forceinline__ double total(int u, int k) const
    {
        if constexpr (SMEM)
            return (double)chi(u, k) + (double)clo(u, k);
        else
            return (double)h[u][k] + (double)l[u][k];
    }
};

// The chunk against itself, block B: its i set B held as j.  Sets below B
// meet all of it (32 steps); set B meets its own records only at steps 1..15,
// and at step 16 on the low half-warp: the pair of lanes a and b comes round
// at step (b - a) mod 32 in lane a and at the complementary step in lane b,
// so this meets each pair of the set once, in 16 of the 32 steps.  Block 0
// (no set below it) stops after 17 steps and flushes each j from the lane it
// has reached.
template <int IPL, int B, bool EQ>
__device__ __forceinline__ void diag_block(const float4 (&oi)[IPL], int ib, int ie, const PairConsts &K,
                                           AccI<IPL> &A, double *acc, int64_t N, int lane)
{
    constexpr unsigned BELOW = (1u << B) - 1u;
    const int src = (lane + 1) & 31;
    const int i_own = ib + 32 * B + lane;
    JRec J{oi[B].x, oi[B].y, oi[B].z, oi[B].w, 0.f, 0.f, 0.f, i_own < ie ? i_own : -1};
    auto below = [&]() {
#pragma unroll
        for (int u = 0; u < B; ++u)
            if ((BELOW >> u) & 1u) pair_sym<false, EQ>(J, oi[u], K, A.a[u], true);
    };
    below();  // step 0: the set's own records meet themselves (d = 0): nothing
    rotate_one<EQ>(J, src);
#pragma unroll 4
    for (int k = 1; k <= 16; ++k) {
        below();
        pair_sym<true, EQ>(J, oi[B], K, A.a[B], (k < 16) | (lane < 16));
        rotate_one<EQ>(J, src);
    }
    if constexpr (B > 0) {
#pragma unroll 3
        for (int k = 17; k < 32; ++k) {
            below();
            rotate_one<EQ>(J, src);
        }
    } else {
        const int h = (lane + 17) & 31;  // the record this lane holds after 17 steps
        const int i_h = ib + 32 * B + h;
        J.slot = i_h < ie ? i_h : -1;
        // equal masses do not rotate: the lane's own may be an empty lane's 0, so take the
        // common mass from lane 0 (always a particle of the task)
        if constexpr (EQ) J.m = __shfl_sync(FULL, J.m, 0);
    }
    flush_j<EQ>(J, acc, N);
}

// Half-warp tasks (at most 16 particles, i = lane mod 16 in both halves):
// the chunk against itself on the low half only (16 steps, upper triangle);
// the high half holds no i and no j for this block.
template <bool EQ>
__device__ __forceinline__ void diag_block_half(const float4 (&oi)[1], bool active, int ib, const PairConsts &K,
                                                AccI<1> &A, double *acc, int64_t N, int lane)
{
    const float4 od[1] = {lane < 16 ? oi[0] : make_float4(FAR, FAR, FAR, 0.f)};
    JRec J{od[0].x, od[0].y, od[0].z, od[0].w, 0.f, 0.f, 0.f, (lane < 16 && active) ? ib + lane : -1};
    rotate_block<1, 1u, 0u, EQ, 16>(J, od, K, A.a, lane);
    flush_j<EQ>(J, acc, N);
}

// One task: i particles [ib, ie) of cell c against their own chunk (j > i),
// the rest of the cell, and the forward half of the cell's list.  HALF (one
// i set of at most 16): every i sits in lane l and lane l + 16, and the two
// half-warps rotate the two halves of each block of 32 j, so that all 32
// lanes work and each pair is still met once.
template <int JT, int STAGES, int IPL, bool EQ, bool HALF = false>
__device__ __forceinline__ bool run_task_sym(const KArgs &a, Ring<FORCE, JT, STAGES> &ring, float *comp, double *acc,
                                             int64_t N, int lane, int c, int ib, int ie, const hacc_volume &vol)
{
    static_assert(!HALF || IPL == 1, "half-warp tasks hold one i set");
    constexpr int W = HALF ? 16 : 32;
    const int il = HALF ? (lane & 15) : lane;  // this lane's i within its set
    const PairConsts &K = a.k;
    const int n = vol.n;
    const int64_t lc = (int64_t)c - vol.cell_base;
    const int cx = (int)(lc % n), cy = (int)((lc / n) % n), cz = (int)(lc / ((int64_t)n * n));
    const float4 org_i = a.origin ? a.origin[c] : make_float4(0.f, 0.f, 0.f, 0.f);

    float4 oi[IPL];
    bool active[IPL];
#pragma unroll
    for (int u = 0; u < IPL; ++u) {
        const int i = ib + il + 32 * u;
        active[u] = i < ie;
        oi[u] = active[u] ? a.pos[i] : make_float4(FAR, FAR, FAR, 0.f);
    }
    AccI<IPL> A(comp, lane);

    // the chunk against itself: block B holds the chunk's i set B as j
    if constexpr (HALF) {
        diag_block_half<EQ>(oi, active[0], ib, K, A, acc, N, lane);
    } else {
        diag_block<IPL, 0, EQ>(oi, ib, ie, K, A, acc, N, lane);
    }
    if constexpr (IPL > 1) diag_block<IPL, 1, EQ>(oi, ib, ie, K, A, acc, N, lane);
    if constexpr (IPL > 2) {
        diag_block<IPL, 2, EQ>(oi, ib, ie, K, A, acc, N, lane);
        diag_block<IPL, 3, EQ>(oi, ib, ie, K, A, acc, N, lane);
    }
    A.fold();

    // the cell after the chunk, then the forward entries (staged)
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
        int pk = 0, poff = 0;  // producer cursor
        int ck = 0, coff = 0;  // consumer cursor
        for (int s = 0; s < STAGES; ++s)
            if (!ring.produce(a, lane, ng, cnt, jb, pk, poff)) break;
        while (ring.consumed < ring.issued) {
            if (!ring.wait_next(a.wait_limit)) return false;
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
                rotate_block<IPL, 0u, 0u, EQ, W>(J, oi, K, A.a, lane);
                flush_j<EQ>(J, acc, N);
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
        if constexpr (EQ) {
            const double m = (double)oi[u].w;
            atomicAdd(acc + i, m * A.total(u, 0));
            atomicAdd(acc + N + i, m * A.total(u, 1));
            atomicAdd(acc + 2 * N + i, m * A.total(u, 2));
        } else {
            atomicAdd(acc + i, A.total(u, 0));
            atomicAdd(acc + N + i, A.total(u, 1));
            atomicAdd(acc + 2 * N + i, A.total(u, 2));
        }
    }
    return true;
}

// Shared memory of one warp of the symmetric force kernel: the staged tiles,
// the compensated i sums of four-i tasks, the mbarriers; 128-B aligned.
__host__ __device__ constexpr int sym_warp_smem_bytes(int jt, int stages)
{
    return (warp_tiles_bytes(FORCE, jt, stages) + SYM_COMP_BYTES + stages * 8 + 127) / 128 * 128;
}

// EQ: the equal-mass instantiation.  Both are launched when the binning
// checked the masses, and the one that does not match the flag returns at
// once; each keeps its own register allocation.
template <int JT, int STAGES, bool EQ>
__global__ void __launch_bounds__(256, 3) k_pairs_sym(const KArgs a, double *acc, int64_t N)
{
    const bool eq = a.mass_varies && *a.mass_varies == 0u;
    if (eq != EQ) return;
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int WARP_BYTES = sym_warp_smem_bytes(JT, STAGES);
    constexpr int TILE_BYTES = warp_tiles_bytes(FORCE, JT, STAGES);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char *wbase = smem + (size_t)warp * WARP_BYTES;
    Ring<FORCE, JT, STAGES> ring;
    ring.tiles = reinterpret_cast<float4 *>(wbase);
    float *comp = reinterpret_cast<float *>(wbase + TILE_BYTES);
    ring.bars = reinterpret_cast<uint64_t *>(wbase + TILE_BYTES + SYM_COMP_BYTES);
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
        bool ok;
        const int size = task.z - task.y;
        if (size > 64)
            ok = run_task_sym<JT, STAGES, 4, EQ>(a, ring, comp, acc, N, lane, task.x, task.y, task.z, vol);
        else if (size > 32)
            ok = run_task_sym<JT, STAGES, 2, EQ>(a, ring, comp, acc, N, lane, task.x, task.y, task.z, vol);
        else if (size > 16)
            ok = run_task_sym<JT, STAGES, 1, EQ>(a, ring, comp, acc, N, lane, task.x, task.y, task.z, vol);
        else
            ok = run_task_sym<JT, STAGES, 1, EQ, true>(a, ring, comp, acc, N, lane, task.x, task.y, task.z, vol);
        if (!ok) {
            if (lane == 0) atomicOr(a.status, HACC_STATUS_TIMEOUT);
            ring.drain();
            return;
        }
    }
}

// One component of the float64 totals (sorted slots) to float32 in input
// order.  The stores scatter through the permutation, 4 bytes each; they merge
// into whole sectors in L2 only while the target array stays resident there,
// which one 67 MB component per launch does and three at once do not (each
// partial sector is then read and written back in DRAM).  The streamed totals
// and perm are loaded evict-first for the same reason.
__global__ void __launch_bounds__(256)
k_sym_finish(int64_t N, const double *__restrict__ acc, const int32_t *__restrict__ perm, float *__restrict__ out)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x)
        out[__ldcs(perm + k)] = (float)__ldcs(acc + k);
}

template <int JT, int STAGES, bool EQ>
int launch_sym_one(const KArgs &a, double *acc, int64_t N, int warps, int ctas_per_sm, cudaStream_t st)
{
    const size_t smem = (size_t)warps * sym_warp_smem_bytes(JT, STAGES);
    auto kern = k_pairs_sym<JT, STAGES, EQ>;
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

template <int JT, int STAGES>
int launch_sym_t(const KArgs &a, double *acc, int64_t N, int warps, int ctas_per_sm, cudaStream_t st)
{
    if (a.mass_varies) {
        const int rc = launch_sym_one<JT, STAGES, true>(a, acc, N, warps, ctas_per_sm, st);
        if (rc) return rc;
    }
    return launch_sym_one<JT, STAGES, false>(a, acc, N, warps, ctas_per_sm, st);
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
        L.wait_cycles = 0;
    }
    a.wait_limit = wait_limit_of(L);
    rc = launch_sym(a, F.acc, mesh->N, L, st);
    if (rc) return rc;
    int g = (int)((mesh->N + 255) / 256);
    if (g > num_sms() * 16) g = num_sms() * 16;
    float *out[3] = {ax, ay, az};
    for (int c = 0; c < 3; ++c) {
        k_sym_finish<<<g, 256, 0, st>>>(mesh->N, F.acc + c * mesh->N, binned->perm, out[c]);
        HACC_LAUNCH_CHECK();
    }
    return HACC_OK;
}
