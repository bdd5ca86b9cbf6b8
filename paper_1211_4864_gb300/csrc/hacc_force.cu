// Short-range pair force (Eq. 7 of the paper) and its adjoint.
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
// branch-free kernel, Sec. III):
//   d  = o_j - (o_i - Delta)            cell-relative offsets, Delta = image origin difference
//   se = eps + d.d                      (three fma)
//   t  = rsqrt(se)
//   f  = t^2 t - poly~(se)              poly~(se) = poly(se - eps), coefficients shifted on the host
//   f  = se < r_c^2 + eps ? f : 0
//   a += m_j f d
// The accumulator is float32 within a tile and compensated (TwoSum into a
// hi/lo pair) across tiles.
#include "hacc_pairs.cuh"

namespace hacc {
namespace {

// Per-lane accumulators of IPL i particles: float32 within a tile, then
// folded into a compensated (hi, lo) pair.
template <int MODE, int IPL>
struct Acc;

template <int IPL, int NC>
struct AccN {
    float a[IPL][NC], h[IPL][NC], l[IPL][NC];
    __device__ __forceinline__ AccN()
    {
#pragma unroll
        for (int u = 0; u < IPL; ++u)
#pragma unroll
            for (int k = 0; k < NC; ++k) a[u][k] = h[u][k] = l[u][k] = 0.f;
    }
    __device__ __forceinline__ void fold()
    {
#pragma unroll
        for (int u = 0; u < IPL; ++u)
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                two_sum_acc(h[u][k], l[u][k], a[u][k]);
                a[u][k] = 0.f;
            }
    }
};

template <int IPL>
struct Acc<FORCE, IPL> : AccN<IPL, 3> {};

template <int IPL>
struct Acc<POTENTIAL, IPL> : AccN<IPL, 1> {};

// One pair of the forward law, accumulated into acc[3] (EQ, equal masses:
// f d, the mass applied to the total).  The cutoff test is a compare whose
// predicate guards the three accumulating fma (no branch, no select): the
// paper folds the same test into the loop with fsel (Sec. III).
template <bool EQ>
__device__ __forceinline__ void pair_force(const float4 p, float oxp, float oyp, float ozp, const PairConsts &K,
                                           float *acc)
{
    float dx = p.x - oxp, dy = p.y - oyp, dz = p.z - ozp;
    float se = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, K.eps)));
    float t = rsqrt_hw(se);
    float t2 = t * t;
    float q = fmaf(fmaf(fmaf(fmaf(fmaf(K.nc[5], se, K.nc[4]), se, K.nc[3]), se, K.nc[2]), se, K.nc[1]), se,
                   K.nc[0]);
    float g = EQ ? fmaf(t2, t, q) : fmaf(t2, t, q) * p.w;
    asm("{\n\t.reg .pred p;\n\tsetp.lt.f32 p, %3, %4;\n\t"
        "@p fma.rn.f32 %0, %5, %6, %0;\n\t@p fma.rn.f32 %1, %5, %7, %1;\n\t@p fma.rn.f32 %2, %5, %8, %2;\n\t}"
        : "+f"(acc[0]), "+f"(acc[1]), "+f"(acc[2])
        : "f"(se), "f"(K.rc2e), "f"(g), "f"(dx), "f"(dy), "f"(dz));
}

// Forward pair loop over one staged tile: every staged j meets the IPL i
// particles of this lane.  Unrolled by hand, four j per trip.
template <int IPL, bool EQ>
__device__ __forceinline__ void tile_force(const float4 *__restrict__ tj, int n, const float (&op)[IPL][3],
                                           const PairConsts &K, Acc<FORCE, IPL> &A)
{
    int j = 0;
    for (; j + 4 <= n; j += 4) {
        const float4 p0 = tj[j], p1 = tj[j + 1], p2 = tj[j + 2], p3 = tj[j + 3];
#pragma unroll
        for (int u = 0; u < IPL; ++u) {
            pair_force<EQ>(p0, op[u][0], op[u][1], op[u][2], K, A.a[u]);
            pair_force<EQ>(p1, op[u][0], op[u][1], op[u][2], K, A.a[u]);
            pair_force<EQ>(p2, op[u][0], op[u][1], op[u][2], K, A.a[u]);
            pair_force<EQ>(p3, op[u][0], op[u][1], op[u][2], K, A.a[u]);
        }
    }
    for (; j < n; ++j) {
        const float4 p = tj[j];
#pragma unroll
        for (int u = 0; u < IPL; ++u) pair_force<EQ>(p, op[u][0], op[u][1], op[u][2], K, A.a[u]);
    }
}

// The short-range pair potential V(s) = pv(se) - (s + eps)^-1/2 (se = s + eps):
// the integral of the force law, zero at the cutoff (F = -grad V).
__device__ __forceinline__ float pair_potential_of(float se, const PairConsts &K)
{
    const float h = fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(K.pv[6], se, K.pv[5]), se, K.pv[4]), se, K.pv[3]), se, K.pv[2]),
                              se, K.pv[1]),
                         se, K.pv[0]);
    return h - rsqrt_hw(se);
}

__device__ __forceinline__ void pair_potential(const float4 p, float oxp, float oyp, float ozp, const PairConsts &K,
                                               float *acc)
{
    float dx = p.x - oxp, dy = p.y - oyp, dz = p.z - ozp;
    float se = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, K.eps)));
    float v = pair_potential_of(se, K);
    asm("{\n\t.reg .pred p;\n\tsetp.lt.f32 p, %1, %2;\n\t@p fma.rn.f32 %0, %3, %4, %0;\n\t}"
        : "+f"(acc[0])
        : "f"(se), "f"(K.rc2e), "f"(p.w), "f"(v));
}

template <int IPL>
__device__ __forceinline__ void tile_potential(const float4 *__restrict__ tj, int n, const float (&op)[IPL][3],
                                               const PairConsts &K, Acc<POTENTIAL, IPL> &A)
{
    int j = 0;
    for (; j + 4 <= n; j += 4) {
        const float4 p0 = tj[j], p1 = tj[j + 1], p2 = tj[j + 2], p3 = tj[j + 3];
#pragma unroll
        for (int u = 0; u < IPL; ++u) {
            pair_potential(p0, op[u][0], op[u][1], op[u][2], K, A.a[u]);
            pair_potential(p1, op[u][0], op[u][1], op[u][2], K, A.a[u]);
            pair_potential(p2, op[u][0], op[u][1], op[u][2], K, A.a[u]);
            pair_potential(p3, op[u][0], op[u][1], op[u][2], K, A.a[u]);
        }
    }
    for (; j < n; ++j) {
        const float4 p = tj[j];
#pragma unroll
        for (int u = 0; u < IPL; ++u) pair_potential(p, op[u][0], op[u][1], op[u][2], K, A.a[u]);
    }
}

// Adjoint pair loop over one staged tile.  Per pair, with f = f_SR(s) and
// fp2 = 2 f_SR'(s):  U += f lam_j ;  V += m_j f ;
// X += fp2 (m_i (d.lam_j) - m_j (d.lam_i)) d ;  G += f (d.lam_j).
// Then dL/dx_i = m_i U - lam_i V + X and dL/dm_i = -G.
// Equal masses (EQ): V += f and X += fp2 (d.(lam_j - lam_i)) d, so that
// dL/dx_i = m (U - lam_i V + X).
// Without G (the W form) the three sums fold into one: with mu = m_i lam_j -
// m_j lam_i, W += f mu + fp2 (d.mu) d and dL/dx_i = W (equal masses: mu / m
// summed, dL/dx_i = m W).
// One pair of the adjoint, accumulated into acc[8] = (U, V, X, G) of one i
// (the W form: acc[3] = W).
template <bool GM, bool EQ>
__device__ __forceinline__ void pair_adjoint(const float4 p, const float4 l, float oxp, float oyp, float ozp,
                                             float mi, float lix, float liy, float liz, const PairConsts &K,
                                             float (&acc)[ADJ_NACC])
{
    float dx = p.x - oxp, dy = p.y - oyp, dz = p.z - ozp;
    float se = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, K.eps)));
    float t = rsqrt_hw(se);
    float t2 = t * t;
    float t3 = t2 * t;
    float q = fmaf(fmaf(fmaf(fmaf(fmaf(K.nc[5], se, K.nc[4]), se, K.nc[3]), se, K.nc[2]), se, K.nc[1]), se,
                   K.nc[0]);
    float f = t3 + q;
    float qp = fmaf(fmaf(fmaf(fmaf(K.kp[4], se, K.kp[3]), se, K.kp[2]), se, K.kp[1]), se, K.kp[0]);
    float fp2 = fmaf(-3.0f, t3 * t2, qp);
    if constexpr (!GM) {
        float ex, ey, ez;  // mu (equal masses: mu / m)
        if constexpr (EQ) {
            ex = l.x - lix;
            ey = l.y - liy;
            ez = l.z - liz;
        } else {
            ex = fmaf(mi, l.x, -(p.w * lix));
            ey = fmaf(mi, l.y, -(p.w * liy));
            ez = fmaf(mi, l.z, -(p.w * liz));
        }
        const float r = fp2 * fmaf(dz, ez, fmaf(dy, ey, dx * ex));
        asm("{\n\t.reg .pred p;\n\tsetp.lt.f32 p, %3, %4;\n\t"
            "@p fma.rn.f32 %0, %5, %6, %0;\n\t@p fma.rn.f32 %1, %5, %7, %1;\n\t@p fma.rn.f32 %2, %5, %8, %2;\n\t"
            "@p fma.rn.f32 %0, %9, %10, %0;\n\t@p fma.rn.f32 %1, %9, %11, %1;\n\t@p fma.rn.f32 %2, %9, %12, %2;\n\t}"
            : "+f"(acc[0]), "+f"(acc[1]), "+f"(acc[2])
            : "f"(se), "f"(K.rc2e), "f"(f), "f"(ex), "f"(ey), "f"(ez), "f"(r), "f"(dx), "f"(dy), "f"(dz));
        return;
    }
    float dlj = fmaf(dz, l.z, fmaf(dy, l.y, dx * l.x));
    float r;
    if constexpr (EQ) {
        r = fp2 * (dlj - fmaf(dz, liz, fmaf(dy, liy, dx * lix)));
    } else {
        const float dli = fmaf(dz, liz, fmaf(dy, liy, dx * lix));
        r = fp2 * fmaf(mi, dlj, -(p.w * dli));
    }
    const float mj = EQ ? 1.0f : p.w;
    // the accumulations of this pair happen only inside the cutoff
    asm("{\n\t.reg .pred p;\n\tsetp.lt.f32 p, %8, %9;\n\t"
        "@p fma.rn.f32 %0, %10, %11, %0;\n\t@p fma.rn.f32 %1, %10, %12, %1;\n\t@p fma.rn.f32 %2, %10, %13, %2;\n\t"
        "@p fma.rn.f32 %3, %14, %10, %3;\n\t"
        "@p fma.rn.f32 %4, %15, %16, %4;\n\t@p fma.rn.f32 %5, %15, %17, %5;\n\t@p fma.rn.f32 %6, %15, %18, %6;\n\t"
        "@p fma.rn.f32 %7, %10, %19, %7;\n\t}"
        : "+f"(acc[0]), "+f"(acc[1]), "+f"(acc[2]), "+f"(acc[3]), "+f"(acc[4]), "+f"(acc[5]), "+f"(acc[6]),
          "+f"(acc[7])
        : "f"(se), "f"(K.rc2e), "f"(f), "f"(l.x), "f"(l.y), "f"(l.z), "f"(mj), "f"(r), "f"(dx), "f"(dy),
          "f"(dz), "f"(dlj));
}

// Adjoint pair loop over one staged tile (positions tj, cotangents tl).
template <int MODE, int IPL, bool EQ>
__device__ __forceinline__ void tile_adjoint(const float4 *__restrict__ tj, const float4 *__restrict__ tl, int n,
                                             const float (&op)[IPL][3], const float4 (&oi)[IPL],
                                             const float4 (&li)[IPL], const PairConsts &K,
                                             AccAdj<MODE, IPL, adj_nacc(MODE)> &A)
{
    constexpr bool GM = MODE == ADJOINT_GM;
    int j = 0;
    if constexpr (IPL == 1) {
        // one i per lane: two j per trip for independent work
        for (; j + 2 <= n; j += 2) {
            const float4 p0 = tj[j], p1 = tj[j + 1], l0 = tl[j], l1 = tl[j + 1];
            pair_adjoint<GM, EQ>(p0, l0, op[0][0], op[0][1], op[0][2], oi[0].w, li[0].x, li[0].y, li[0].z, K,
                                 A.p[0]);
            pair_adjoint<GM, EQ>(p1, l1, op[0][0], op[0][1], op[0][2], oi[0].w, li[0].x, li[0].y, li[0].z, K,
                                 A.p[0]);
        }
    }
    for (; j < n; ++j) {
        const float4 p0 = tj[j], l0 = tl[j];
#pragma unroll
        for (int u = 0; u < IPL; ++u)
            pair_adjoint<GM, EQ>(p0, l0, op[u][0], op[u][1], op[u][2], oi[u].w, li[u].x, li[u].y, li[u].z, K,
                                 A.p[u]);
    }
}



template <int MODE, int IPL>
__device__ __forceinline__ auto make_acc(float *comp, int lane)
{
    if constexpr (MODE == FORCE || MODE == POTENTIAL)
        return Acc<MODE, IPL>();
    else
        return AccAdj<MODE, IPL, adj_nacc(MODE)>(comp, lane);
}

// One task: i particles [ib, ie) of cell c (at most 32 IPL of them), every
// entry of the cell's neighbour list.  Returns false if a wait ran out.
// With one i per lane and at most 16 i (half, decided per task), lanes l and
// l + 16 hold the same i and each takes half of every staged piece of j
// records; the two compensated partial sums are added in a fixed order at the
// end, so the result stays deterministic.
template <int MODE, int JT, int STAGES, int IPL, bool EQ>
__device__ __forceinline__ bool run_task(const KArgs &a, Ring<MODE, JT, STAGES> &ring, float *comp, int lane,
                                         int c, int ib, int ie, const hacc_volume &vol)
{
    const bool half = IPL == 1 && ie - ib <= 16;
    const int il = half ? (lane & 15) : lane;  // this lane's i within the task
    const PairConsts &K = a.k;
    const int n = vol.n;
    const float w = vol.w;
    const double Ld = (double)vol.L;
    const int64_t lc = (int64_t)c - vol.cell_base;
    const int cx = (int)(lc % n), cy = (int)((lc / n) % n), cz = (int)(lc / ((int64_t)n * n));
    const float4 org_i = a.origin ? a.origin[c] : make_float4(0.f, 0.f, 0.f, 0.f);

    float4 oi[IPL];
    bool active[IPL];
#pragma unroll
    for (int u = 0; u < IPL; ++u) {
        const int i = ib + il + 32 * u;
        active[u] = i < ie;
        oi[u] = active[u] ? a.pos[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float4 li[IPL];
#pragma unroll
    for (int u = 0; u < IPL; ++u) {
        li[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if constexpr (is_adjoint(MODE)) {
            if (active[u]) li[u] = a.lam[ib + il + 32 * u];
        }
    }
    auto A = make_acc<MODE, IPL>(comp, lane);

    const int64_t e0 = a.nbr_off[c], e1 = a.nbr_off[c + 1];
    for (int64_t g0 = e0; g0 < e1; g0 += 32) {
        const int ng = (int)min((int64_t)32, e1 - g0);
        // lane l describes entry g0 + l: its j range and image offset Delta
        int jb = 0, cnt = 0;
        float Dx = 0.f, Dy = 0.f, Dz = 0.f;
        if (lane < ng) {
            const int cp = a.nbr_cell[g0 + lane];
            const int sh = a.nbr_shift[g0 + lane];
            jb = a.cell_start[cp];
            cnt = a.cell_start[cp + 1] - jb;
            const int sx = sh % 3 - 1, sy = (sh / 3) % 3 - 1, sz = sh / 9 - 1;
            if (a.origin) {
                // tree leaves: float32 origins, difference and image exact in float64
                const float4 org_j = a.origin[cp];
                Dx = (float)((double)org_j.x - (double)org_i.x + sx * Ld);
                Dy = (float)((double)org_j.y - (double)org_i.y + sy * Ld);
                Dz = (float)((double)org_j.z - (double)org_i.z + sz * Ld);
            } else {
                const int64_t lp = (int64_t)cp - vol.cell_base;
                const int px = (int)(lp % n), py = (int)((lp / n) % n), pz = (int)(lp / ((int64_t)n * n));
                // exact in float64: origins are the float32 cell centres used by the binning
                Dx = (float)((double)cell_centre(px, w) - (double)cell_centre(cx, w) + sx * Ld);
                Dy = (float)((double)cell_centre(py, w) - (double)cell_centre(cy, w) + sy * Ld);
                Dz = (float)((double)cell_centre(pz, w) - (double)cell_centre(cz, w) + sz * Ld);
            }
        }
        int pk = 0, poff = 0;  // producer cursor (entry, record within it)
        int ck = 0, coff = 0;  // consumer cursor
        for (int s = 0; s < STAGES; ++s)  // prologue: fill the ring
            if (!ring.produce(a, lane, ng, cnt, jb, pk, poff)) break;
        int cur = -1;
        float op[IPL][3];
        while (ring.consumed < ring.issued) {
            if (!ring.wait_next(a.wait_limit)) return false;
            const float4 *tj = ring.tile(ring.consumed % STAGES);
            // replay the producer's pieces: each piece is one entry's records
            int filled = 0;
            while (ck < ng && filled < JT) {
                const int c = __shfl_sync(FULL, cnt, ck);
                if (coff >= c) {
                    ++ck;
                    coff = 0;
                    continue;
                }
                const int n = min(JT - filled, c - coff);
                if (ck != cur) {
                    cur = ck;
                    const float dx = __shfl_sync(FULL, Dx, ck), dy = __shfl_sync(FULL, Dy, ck),
                                dz = __shfl_sync(FULL, Dz, ck);
#pragma unroll
                    for (int u = 0; u < IPL; ++u) {
                        op[u][0] = oi[u].x - dx;
                        op[u][1] = oi[u].y - dy;
                        op[u][2] = oi[u].z - dz;
                    }
                }
                // the pair loop over records [o, o + m) of the staged tile
                auto tile = [&](int o, int m) {
                    if constexpr (MODE == FORCE)
                        tile_force<IPL, EQ>(tj + o, m, op, K, A);
                    else if constexpr (MODE == POTENTIAL)
                        tile_potential<IPL>(tj + o, m, op, K, A);
                    else
                        tile_adjoint<MODE, IPL, EQ>(tj + o, tj + JT + o, m, op, oi, li, K, A);
                };
                if constexpr (IPL == 1) {
                    // half: lanes < 16 take records [0, n/2) and, for odd n, record
                    // n/2 alone; lanes >= 16 the rest.  Equal trip counts keep the
                    // loop converged.
                    const int hn = n >> 1;
                    tile(filled + (half && (lane & 16) ? hn + (n & 1) : 0), half ? hn : n);
                    if (half && (n & 1) && lane < 16) tile(filled + hn, 1);
                } else {
                    tile(filled, n);
                }
                filled += n;
                coff += n;
            }
            A.fold();
            ++ring.consumed;
            __syncwarp();
            ring.produce(a, lane, ng, cnt, jb, pk, poff);
        }
    }
    if (half) {
        // lane l (< 16) adds lane l + 16's compensated sums to its own
        if constexpr (MODE == FORCE || MODE == POTENTIAL) {
#pragma unroll
            for (int k = 0; k < (MODE == FORCE ? 3 : 1); ++k) {
                const float h2 = __shfl_down_sync(FULL, A.h[0][k], 16), l2 = __shfl_down_sync(FULL, A.l[0][k], 16);
                two_sum_acc(A.h[0][k], A.l[0][k], h2);
                A.l[0][k] = __fadd_rn(A.l[0][k], l2);
            }
        } else {
#pragma unroll
            for (int k = 0; k < decltype(A)::NACC; ++k) {
                float h = A.hi(0, k), l = A.lo(0, k);
                const float h2 = __shfl_down_sync(FULL, h, 16), l2 = __shfl_down_sync(FULL, l, 16);
                two_sum_acc(h, l, h2);
                A.hi(0, k) = h;
                A.lo(0, k) = __fadd_rn(l, l2);
            }
        }
    }
#pragma unroll
    for (int u = 0; u < IPL; ++u) {
        if (!active[u] || (half && lane >= 16)) continue;
        const int o = a.perm[ib + il + 32 * u];
        if constexpr (MODE == FORCE && EQ) {
            a.out_x[o] = oi[u].w * (A.h[u][0] + A.l[u][0]);
            a.out_y[o] = oi[u].w * (A.h[u][1] + A.l[u][1]);
            a.out_z[o] = oi[u].w * (A.h[u][2] + A.l[u][2]);
        } else if constexpr (MODE == FORCE) {
            a.out_x[o] = A.h[u][0] + A.l[u][0];
            a.out_y[o] = A.h[u][1] + A.l[u][1];
            a.out_z[o] = A.h[u][2] + A.l[u][2];
        } else if constexpr (MODE == POTENTIAL) {
            // the sum met particle i itself once (d = 0, se = eps exactly): take that term out
            const float self = pair_potential_of(K.eps, K);
            a.out_x[o] = (A.h[u][0] + A.l[u][0]) - oi[u].w * self;
        } else if constexpr (adj_wform(MODE)) {
            // dL/dx_i = W (equal masses: m W)
            const float sc = EQ ? oi[u].w : 1.0f;
            a.out_x[o] = sc * A.total(u, 0);
            a.out_y[o] = sc * A.total(u, 1);
            a.out_z[o] = sc * A.total(u, 2);
        } else {
            // dL/dx_i = m_i U - lam_i V + X (equal masses: m (U - lam_i V + X)) ;  dL/dm_i = -G
            const float Vs = A.total(u, 3);
            if constexpr (EQ) {
                a.out_x[o] = oi[u].w * (A.total(u, 0) + fmaf(-li[u].x, Vs, A.total(u, 4)));
                a.out_y[o] = oi[u].w * (A.total(u, 1) + fmaf(-li[u].y, Vs, A.total(u, 5)));
                a.out_z[o] = oi[u].w * (A.total(u, 2) + fmaf(-li[u].z, Vs, A.total(u, 6)));
            } else {
                a.out_x[o] = fmaf(oi[u].w, A.total(u, 0), fmaf(-li[u].x, Vs, A.total(u, 4)));
                a.out_y[o] = fmaf(oi[u].w, A.total(u, 1), fmaf(-li[u].y, Vs, A.total(u, 5)));
                a.out_z[o] = fmaf(oi[u].w, A.total(u, 2), fmaf(-li[u].z, Vs, A.total(u, 6)));
            }
            if constexpr (MODE == ADJOINT_GM) a.out_m[o] = -A.total(u, 7);
        }
    }
    return true;
}

// Persistent work-stealing kernel: each warp takes tasks from a global
// counter until none is left.  A task of more than 32 particles runs two i
// particles per lane (four, above 64, in the adjoint's W form), one of at most
// 16 runs each i on two lanes.
// Register budgets: the forward and potential kernels keep 80 registers so that
// 3 CTAs (24 warps) fit an SM; the adjoint's staging needs twice the shared
// memory, which caps it at 2 CTAs, so it may use up to 128 registers.
__host__ __device__ constexpr int min_ctas(int mode) { return is_adjoint(mode) ? 2 : 3; }

// EQ (force and adjoint): the equal-mass instantiation; as for the
// symmetric kernel both are launched and the one that does not match the
// flag returns.
template <int MODE, int JT, int STAGES, bool EQ>
__global__ void __launch_bounds__(256, min_ctas(MODE)) k_pairs(const KArgs a)
{
    if constexpr (MODE != POTENTIAL) {
        const bool eq = a.mass_varies && *a.mass_varies == 0u;
        if (eq != EQ) return;
    }
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int WARP_BYTES = warp_smem_bytes(MODE, JT, STAGES);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char *wbase = smem + (size_t)warp * WARP_BYTES;
    constexpr int TILE_BYTES = warp_tiles_bytes(MODE, JT, STAGES);
    constexpr int COMP_BYTES = is_adjoint(MODE) ? ADJ_COMP_BYTES : 0;
    Ring<MODE, JT, STAGES> ring;
    ring.tiles = reinterpret_cast<float4 *>(wbase);
    float *comp = reinterpret_cast<float *>(wbase + TILE_BYTES);
    ring.bars = reinterpret_cast<uint64_t *>(wbase + TILE_BYTES + COMP_BYTES);

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
        // sub-chunks of larger tasks: 128 particles (four i per lane) for the adjoint's W form,
        // whose three sums leave the registers for it, else 64
        constexpr int CHUNK = adj_wform(MODE) ? 128 : 64;
        for (int sb = task.y; ok && sb < task.z; sb += CHUNK) {
            const int se = min(sb + CHUNK, task.z);
            if (CHUNK == 128 && se - sb > 64)
                ok = run_task<MODE, JT, STAGES, (CHUNK == 128 ? 4 : 2), EQ>(a, ring, comp, lane, task.x, sb, se,
                                                                             vol);
            else if (se - sb > 32)
                ok = run_task<MODE, JT, STAGES, 2, EQ>(a, ring, comp, lane, task.x, sb, se, vol);
            else
                ok = run_task<MODE, JT, STAGES, 1, EQ>(a, ring, comp, lane, task.x, sb, se, vol);
        }
        if (!ok) {
            if (lane == 0) atomicOr(a.status, HACC_STATUS_TIMEOUT);
            ring.drain();
            return;
        }
    }
}

// Ordered pairs (j != i) inside the cutoff, decided exactly as the pair
// kernels decide it (same offsets, same float32 s + eps, same compare).  One
// warp per task, one i per lane, j read straight from global memory: a
// reporting tool, not a hot path.
__global__ void __launch_bounds__(256)
k_count_pairs(const KArgs a, unsigned long long *__restrict__ total)
{
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    const int ntask = task_count(a);
    unsigned long long cnt = 0;
    for (int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < ntask; t += warps) {
        int4 task;
        if (!take_task(a, t, lane, task, nullptr)) continue;
        const hacc_volume &vol = a.vols[task.w];
        const int n = vol.n;
        const float w = vol.w;
        const double Ld = (double)vol.L;
        const int64_t lc = (int64_t)task.x - vol.cell_base;
        const int cx = (int)(lc % n), cy = (int)((lc / n) % n), cz = (int)(lc / ((int64_t)n * n));
        const float4 org_i = a.origin ? a.origin[task.x] : make_float4(0.f, 0.f, 0.f, 0.f);
        for (int i = task.y + lane; i - lane < task.z; i += 32) {
            const bool active = i < task.z;
            const float4 oi = active ? a.pos[i] : make_float4(0.f, 0.f, 0.f, 0.f);
            for (int64_t e = a.nbr_off[task.x]; e < a.nbr_off[task.x + 1]; ++e) {
                const int cp = a.nbr_cell[e];
                const int sh = a.nbr_shift[e];
                const int sx = sh % 3 - 1, sy = (sh / 3) % 3 - 1, sz = sh / 9 - 1;
                float Dx, Dy, Dz;
                if (a.origin) {
                    const float4 org_j = a.origin[cp];
                    Dx = (float)((double)org_j.x - (double)org_i.x + sx * Ld);
                    Dy = (float)((double)org_j.y - (double)org_i.y + sy * Ld);
                    Dz = (float)((double)org_j.z - (double)org_i.z + sz * Ld);
                } else {
                    const int64_t lp = (int64_t)cp - vol.cell_base;
                    const int px = (int)(lp % n), py = (int)((lp / n) % n), pz = (int)(lp / ((int64_t)n * n));
                    Dx = (float)((double)cell_centre(px, w) - (double)cell_centre(cx, w) + sx * Ld);
                    Dy = (float)((double)cell_centre(py, w) - (double)cell_centre(cy, w) + sy * Ld);
                    Dz = (float)((double)cell_centre(pz, w) - (double)cell_centre(cz, w) + sz * Ld);
                }
                const float oxp = oi.x - Dx, oyp = oi.y - Dy, ozp = oi.z - Dz;
                for (int j = a.cell_start[cp]; j < a.cell_start[cp + 1]; ++j) {
                    const float4 p = a.pos[j];
                    const float dx = p.x - oxp, dy = p.y - oyp, dz = p.z - ozp;
                    const float se = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, a.k.eps)));
                    cnt += (active && j != i && se < a.k.rc2e) ? 1ull : 0ull;
                }
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(FULL, cnt, o);
    if (lane == 0 && cnt) atomicAdd(total, cnt);
}


template <int MODE, int JT, int STAGES, bool EQ>
int launch_one(const KArgs &a, int warps, int ctas_per_sm, cudaStream_t st)
{
    const size_t smem = (size_t)warps * warp_smem_bytes(MODE, JT, STAGES);
    auto kern = k_pairs<MODE, JT, STAGES, EQ>;
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

template <int MODE, int JT, int STAGES>
int launch_t(const KArgs &a, int warps, int ctas_per_sm, cudaStream_t st)
{
    if constexpr (MODE != POTENTIAL) {
        if (a.mass_varies) {
            const int rc = launch_one<MODE, JT, STAGES, true>(a, warps, ctas_per_sm, st);
            if (rc) return rc;
        }
    }
    return launch_one<MODE, JT, STAGES, false>(a, warps, ctas_per_sm, st);
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
    L.ctas_per_sm = 3;
    L.jtile = mode == FORCE ? 64 : 64;
    L.stages = 4;
    L.wait_cycles = 0;
    return L;
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
    KArgs a = base_args(mesh, binned, lists, p, status);
    a.out_x = ax;
    a.out_y = ay;
    a.out_z = az;
    a.counter = F.counter;
    HACC_CUDA_TRY(cudaMemsetAsync(F.counter, 0, sizeof(int32_t), st));
    hacc_launch L = launch ? *launch : default_launch(FORCE);
    a.wait_limit = wait_limit_of(L);
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
    KArgs a = base_args(mesh, binned, lists, p, status);
    a.lam = F.lam;
    a.out_x = gx;
    a.out_y = gy;
    a.out_z = gz;
    a.out_m = gm;
    a.counter = F.counter;
    HACC_CUDA_TRY(cudaMemsetAsync(F.counter, 0, sizeof(int32_t), st));
    hacc_launch L = launch ? *launch : default_launch(ADJOINT);
    a.wait_limit = wait_limit_of(L);
    if (gm) return launch_mode<ADJOINT_GM>(a, L, st);
    return launch_mode<ADJOINT>(a, L, st);
}

extern "C" int hacc_sr_potential(const hacc_mesh *mesh, const hacc_binned *binned, const hacc_lists *lists,
                                 const hacc_sr_params *p, float *phi, const hacc_launch *launch, void *ws,
                                 size_t ws_bytes, uint32_t *status, void *stream)
{
    int rc = check_common(mesh, binned, lists, p, launch, ws, ws_bytes, status);
    if (rc) return rc;
    if (mesh->N > 0 && !phi) return HACC_ERR_INVALID;
    if (mesh->N == 0) return HACC_OK;
    cudaStream_t st = as_stream(stream);
    ForceWs F = force_layout(mesh, ws);
    KArgs a = base_args(mesh, binned, lists, p, status);
    a.out_x = phi;
    a.counter = F.counter;
    HACC_CUDA_TRY(cudaMemsetAsync(F.counter, 0, sizeof(int32_t), st));
    hacc_launch L = launch ? *launch : default_launch(FORCE);
    a.wait_limit = wait_limit_of(L);
    return launch_mode<POTENTIAL>(a, L, st);
}

extern "C" int hacc_count_pairs(const hacc_mesh *mesh, const hacc_binned *binned, const hacc_lists *lists,
                                const hacc_sr_params *p, int64_t *out, void *stream)
{
    if (!mesh || !binned || !lists || !p || !out || !mesh->vols) return HACC_ERR_INVALID;
    if (!(p->eps > 0.0f) || !(p->rcut > 0.0f)) return HACC_ERR_INVALID;
    if (!binned->cell_start || !lists->nbr_off || !lists->tasks || !lists->n_tasks) return HACC_ERR_INVALID;
    if (mesh->N > 0 && !binned->sorted4) return HACC_ERR_INVALID;
    cudaStream_t st = as_stream(stream);
    HACC_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int64_t), st));
    if (mesh->N == 0) return HACC_OK;
    KArgs a = base_args(mesh, binned, lists, p, nullptr);
    k_count_pairs<<<num_sms() * 8, 256, 0, st>>>(a, reinterpret_cast<unsigned long long *>(out));
    HACC_LAUNCH_CHECK();
    return HACC_OK;
}
